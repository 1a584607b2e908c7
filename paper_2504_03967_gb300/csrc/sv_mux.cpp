// Multiplexor recognition (host).
//
// QCrank (App. D.3) writes every data qubit with a uniformly controlled RY
// over the address qubits, which the circuit spells out as 2^a alternating
// RY / CX steps (the Mottonen et al. decomposition the paper cites).  Played
// gate by gate that is 2 * 2^a full passes over the state per data qubit;
// collapsed back, it is one block-diagonal operator per data qubit, and five
// of them share one pass.
//
// Algebra of a run on target t.  Let the run's gates be rotations G_i about
// one axis (RY: family Y; RZ, P, Z: family D) and X-type gates (CX from a
// control c, or X on t).  For a fixed value j of the control bits every CX is
// X or I, and X R(theta) X = R(-theta) for RY and RZ (for a diagonal,
// X diag(a, b) X = diag(b, a)).  Moving all X's to the end of the run gives
//     U_j = X^(p_L(j)) * prod_i R_i(j),  p_i(j) = popcount(j & m_i) ^ k_i,
// where m_i is the mask of controls whose CX count before G_i is odd and k_i
// the parity of X gates on t before it.  With chi_m(j) = (-1)^popcount(j & m):
//   Y: phi_j = sum_i (-1)^k_i theta_i chi_{m_i}(j)   -> one Walsh-Hadamard
//      transform of w[m] = sum over rotations with m_i = m;
//   D: a rotation diag(e^{i a_i}, e^{i b_i}) contributes (a_i, b_i) when
//      p_i = 0 and (b_i, a_i) when p_i = 1, so with S = sum (a_i + b_i) and
//      W = WHT of sum (-1)^k_i (a_i - b_i) at m_i:
//      phi0_j = (S + W_j) / 2, phi1_j = (S - W_j) / 2.
//
// A run stays open while the gates in between commute with it: they must not
// touch t, and must act diagonally on every control the run has so far.  The
// collapsed gate then sits where the run's last gate was.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "sv_internal.h"

namespace sv {
namespace {

bool family_y(uint32_t t) { return t == SV_RY; }
bool family_d(uint32_t t) { return t == SV_RZ || t == SV_P || t == SV_Z; }

// Whether gate g acts diagonally (in the computational basis) on qubit q it touches.
bool diagonal_on(const CGate& g, int q) {
    if (g.kind == GK_DIAG) return true;
    if (g.type == SV_CX) return g.q[0] == q;  // the control side
    return false;
}

struct Run {
    int target = -1;
    int family = -1;  // -1: no rotation yet
    uint64_t cmask = 0;  // controls (qubit bitmask)
    std::vector<int> idx;  // gate indices in order
    int ncx = 0;
};

}  // namespace

bool recognise_mux(int n, const std::vector<CGate>& g, std::vector<CGate>* rewritten, std::vector<Mux>* muxes,
                   int mode) {
    muxes->clear();
    if (mode < 0 || n < 2) return false;
    const size_t G = g.size();
    const size_t min_gates = mode == 1 ? 4 : (size_t)kMuxMinGates;
    std::vector<int> owner(G, -1);       // converted run owning the gate
    std::vector<int> emit_at;            // per converted run: index of its last gate
    std::vector<Run> open(n);            // open run per target (target < 0: none)
    std::vector<Mux> made;

    auto close = [&](int t) {
        Run& r = open[t];
        if (r.target < 0) return;
        int nc = 0;
        int ctl[64];
        for (int q = 0; q < n; ++q)
            if (r.cmask >> q & 1) ctl[nc++] = q;
        const bool ok = r.idx.size() >= min_gates && nc >= 1 && nc <= kMuxMaxControls && r.family >= 0;
        if (ok) {
            Mux M;
            M.target = t;
            M.controls.assign(ctl, ctl + nc);
            M.family = r.family;
            int bit[64];
            for (int b = 0; b < nc; ++b) bit[ctl[b]] = b;
            const size_t J = (size_t)1 << nc;
            std::vector<double> w(J, 0.0);
            double S = 0.0;
            uint32_t m = 0;
            int k = 0;
            for (int gi : r.idx) {
                const CGate& x = g[gi];
                M.ngates++;
                M.type_count[x.type < 14 ? x.type : 13]++;
                if (x.type == SV_CX) {
                    m ^= 1u << bit[x.q[0]];
                } else if (x.type == SV_X) {
                    k ^= 1;
                } else if (r.family == MUX_Y) {
                    w[m] += (k ? -1.0 : 1.0) * x.p[0];
                } else {
                    const double a = x.ph[0], b = x.ph[1];
                    S += a + b;
                    w[m] += (k ? -1.0 : 1.0) * (a - b);
                }
            }
            for (size_t h = 1; h < J; h <<= 1)  // in-place fast Walsh-Hadamard transform
                for (size_t i = 0; i < J; i += 2 * h)
                    for (size_t e = i; e < i + h; ++e) {
                        const double u = w[e], v = w[e + h];
                        w[e] = u + v;
                        w[e + h] = u - v;
                    }
            M.flip = m;
            M.flip_c = k;
            if (r.family == MUX_Y) {
                M.phi0.swap(w);
            } else {
                M.phi0.resize(J);
                M.phi1.resize(J);
                for (size_t j = 0; j < J; ++j) {
                    M.phi0[j] = 0.5 * (S + w[j]);
                    M.phi1[j] = 0.5 * (S - w[j]);
                }
            }
            const int id = (int)made.size();
            for (int gi : r.idx) owner[gi] = id;
            emit_at.push_back(r.idx.back());
            made.push_back(std::move(M));
        }
        r = Run();
    };
    // close every run that has q as a control
    auto close_controlled_by = [&](int q) {
        for (int t = 0; t < n; ++t)
            if (open[t].target >= 0 && (open[t].cmask >> q & 1)) close(t);
    };

    for (size_t i = 0; i < G; ++i) {
        const CGate& x = g[i];
        int t = -1, c = -1, fam = -1;
        if (x.nq == 1 && (family_y(x.type) || family_d(x.type) || x.type == SV_X)) {
            t = x.q[0];
            fam = family_y(x.type) ? MUX_Y : (family_d(x.type) ? MUX_D : -1);
        } else if (x.type == SV_CX) {
            c = x.q[0];
            t = x.q[1];
        }
        if (t >= 0) {
            Run& r = open[t];
            const bool fits = r.target < 0 || fam < 0 || r.family < 0 || r.family == fam;
            if (!fits) close(t);
            if (c >= 0) close(c);  // c is about to be used as a control: no run may have it as target
            // the gate is not diagonal on t (X, RY, CX target) unless it is in family D
            if (fam != MUX_D) close_controlled_by(t);
            Run& R = open[t];
            if (R.target < 0) R.target = t;
            if (fam >= 0 && R.family < 0) R.family = fam;
            if (c >= 0) {
                R.cmask |= 1ull << c;
                R.ncx++;
            }
            R.idx.push_back((int)i);
            continue;
        }
        // any other gate: close runs on the qubits it touches, and runs
        // controlled by a qubit it acts on non-diagonally
        for (int a = 0; a < x.nq; ++a) {
            const int q = x.q[a];
            close(q);
            if (!diagonal_on(x, q)) close_controlled_by(q);
        }
    }
    for (int t = 0; t < n; ++t) close(t);
    if (made.empty()) return false;

    std::vector<CGate>& out = *rewritten;
    out.clear();
    out.reserve(G);
    for (size_t i = 0; i < G; ++i) {
        const int id = owner[i];
        if (id < 0) {
            out.push_back(g[i]);
            continue;
        }
        if ((size_t)emit_at[id] != i) continue;
        CGate x;
        memset(&x, 0, sizeof(x));
        x.kind = GK_MUX;
        x.nq = 1;
        x.q[0] = made[id].target;
        x.q[1] = -1;
        x.type = made[id].family == MUX_Y ? SV_RY : SV_RZ;
        x.mux = id;
        out.push_back(x);
    }
    muxes->swap(made);
    return true;
}

}  // namespace sv

namespace sv {

void mux_region(const Plan& p, const HostPass& hp, PassDev* P, std::vector<unsigned char>* out) {
    const double kTwoPi = 6.28318530717958647692;
    MuxDev D;
    memset(&D, 0, sizeof(D));
    std::vector<const Mux*> ms;
    for (int id : hp.mux) ms.push_back(&p.muxes[id]);
    std::sort(ms.begin(), ms.end(), [](const Mux* a, const Mux* b) { return a->target < b->target; });
    D.K = (int)ms.size();
    // union of the controls, ascending; runs of consecutive qubits
    uint64_t cu = 0;
    for (const Mux* M : ms)
        for (int c : M->controls) cu |= 1ull << c;
    int U[64], nu = 0, ubit[64];
    for (int q = 0; q < p.n; ++q)
        if (cu >> q & 1) ubit[q] = nu, U[nu++] = q;
    D.nc = nu;
    for (int b = 0; b < nu;) {
        int e = b + 1;
        while (e < nu && U[e] == U[e - 1] + 1) ++e;
        D.rs[D.nruns] = U[b];
        D.rw[D.nruns] = e - b;
        D.ro[D.nruns] = b;
        D.nruns++;
        b = e;
    }
    const size_t J = (size_t)1 << nu;
    const size_t esz = p.dtype == SV_C64 ? sizeof(float) : sizeof(double);
    size_t off = sizeof(MuxDev);
    std::vector<size_t> toff(D.K);
    for (int k = 0; k < D.K; ++k) {
        toff[k] = off;
        off += (J * esz * (ms[k]->family == MUX_Y ? 1 : 2) + 15) & ~(size_t)15;
    }
    out->assign(off, 0);
    for (int k = 0; k < D.K; ++k) {
        const Mux& M = *ms[k];
        D.t[k] = M.target;
        D.family[k] = M.family;
        D.flip_c[k] = M.flip_c;
        D.tab_off[k] = (int)toff[k];
        int pos[kMuxMaxControls];  // bit b of the multiplexor's own index <-> union bit pos[b]
        const int nc = (int)M.controls.size();
        for (int b = 0; b < nc; ++b) pos[b] = ubit[M.controls[b]];
        uint32_t fl = 0;
        for (int b = 0; b < nc; ++b)
            if (M.flip >> b & 1) fl |= 1u << pos[b];
        D.flip[k] = fl;
        // RY(phi) has period 4 pi, a phase 2 pi
        const double period = M.family == MUX_Y ? 2.0 * kTwoPi : kTwoPi;
        unsigned char* tab = out->data() + toff[k];
        for (size_t j = 0; j < J; ++j) {
            size_t sub = 0;
            for (int b = 0; b < nc; ++b) sub |= ((j >> pos[b]) & 1) << b;
            const int per = M.family == MUX_Y ? 1 : 2;
            for (int e = 0; e < per; ++e) {
                const double v = std::remainder(e ? M.phi1[sub] : M.phi0[sub], period);
                if (p.dtype == SV_C64) ((float*)tab)[j * per + e] = (float)v;
                else ((double*)tab)[j * per + e] = v;
            }
        }
    }
    memcpy(out->data(), &D, sizeof(D));
    P->rmode = kRmodeMux;
    P->m = 0;
    P->nops = 0;
    P->ops_bytes = 0;
    P->region_bytes = (int)out->size();
}

}  // namespace sv
