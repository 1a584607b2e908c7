// Host side of the simulator: gate canonicalisation (FP64) and planning.
//
// A plan turns the gate list into passes over the state.  Fusion is exact in
// exact arithmetic: consecutive gates are multiplied into dense blocks of at
// most k_max qubits (App. D.2, "gate fusion = 5"; a k-qubit block is a
// 2^k x 2^k unitary, stored row-major as in App. B Lemma 1), and diagonal
// gates (RZ, P, Z, CZ, CP = cr1 of App. D.2 Eq. "cr1") are collected into
// phase runs phase(x) = c + sum a_q x_q + sum b_pq x_p x_q that can be applied
// to any amplitude from its index alone.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "sv_internal.h"

namespace sv {

namespace {

const double kPi = 3.14159265358979323846;

int arity(uint32_t t) {
    switch (t) {
    case SV_H: case SV_X: case SV_Y: case SV_Z: case SV_RX: case SV_RY: case SV_RZ:
    case SV_P: case SV_U3: case SV_MEASURE:
        return 1;
    case SV_CX: case SV_CZ: case SV_CP: case SV_SWAP:
        return 2;
    default:
        return -1;
    }
}

// Gate -> canonical form.  Local index j = sum_i bit(q[i]) << i (LSB first).
void make_canonical(const sv_gate& g, CGate* c) {
    memset(c, 0, sizeof(*c));
    c->type = g.type;
    c->nq = (int)g.nq;
    c->q[0] = (int)g.q[0];
    c->q[1] = g.nq > 1 ? (int)g.q[1] : -1;
    for (int i = 0; i < 3; ++i) c->p[i] = g.p[i];
    const cd I(0.0, 1.0);
    const double h = 0.5 * g.p[0];
    // the half-angle cosine and sine only for the gates that use them
    const bool rot = g.type == SV_RX || g.type == SV_RY || g.type == SV_U3;
    const double cs = rot ? cos(h) : 0.0, sn = rot ? sin(h) : 0.0;
    cd* m = c->m;
    c->kind = GK_DENSE;
    switch (g.type) {
    case SV_H: {
        const double r = 1.0 / sqrt(2.0);
        m[0] = r; m[1] = r; m[2] = r; m[3] = -r;
        break;
    }
    case SV_X: m[1] = 1.0; m[2] = 1.0; break;
    case SV_Y: m[1] = -I; m[2] = I; break;
    case SV_RX: m[0] = cs; m[1] = -I * sn; m[2] = -I * sn; m[3] = cs; break;
    case SV_RY: m[0] = cs; m[1] = -sn; m[2] = sn; m[3] = cs; break;
    case SV_U3: {
        const double ph = g.p[1], la = g.p[2];
        m[0] = cs;
        m[1] = -std::polar(1.0, la) * sn;
        m[2] = std::polar(1.0, ph) * sn;
        m[3] = std::polar(1.0, ph + la) * cs;
        break;
    }
    case SV_Z: c->kind = GK_DIAG; c->ph[0] = 0.0; c->ph[1] = kPi; break;
    case SV_RZ: c->kind = GK_DIAG; c->ph[0] = -h; c->ph[1] = h; break;
    case SV_P: c->kind = GK_DIAG; c->ph[0] = 0.0; c->ph[1] = g.p[0]; break;
    case SV_CZ: c->kind = GK_DIAG; c->ph[3] = kPi; break;
    case SV_CP: c->kind = GK_DIAG; c->ph[3] = g.p[0]; break;
    case SV_CX:
        // control = local bit 0, target = local bit 1: |1,t> -> |1,1-t>
        m[0 * 4 + 0] = 1.0; m[2 * 4 + 2] = 1.0; m[3 * 4 + 1] = 1.0; m[1 * 4 + 3] = 1.0;
        break;
    case SV_SWAP:
        m[0 * 4 + 0] = 1.0; m[3 * 4 + 3] = 1.0; m[1 * 4 + 2] = 1.0; m[2 * 4 + 1] = 1.0;
        break;
    default:
        break;
    }
}

// Dense block under construction.
struct Block {
    std::vector<int> qubits;  // sorted
    std::vector<cd> mat;
    std::vector<CGate> seq;   // the gates multiplied into mat, in order
    int ngates = 0;
    bool active() const { return !qubits.empty(); }
    int pos(int q) const {
        for (size_t i = 0; i < qubits.size(); ++i)
            if (qubits[i] == q) return (int)i;
        return -1;
    }
};

// Re-express the block on the sorted qubit set nq (a superset), identity on
// the added qubits.
void expand_block(Block* b, const std::vector<int>& nq) {
    const int k = (int)nq.size();
    const int d = 1 << k;
    std::vector<cd> out((size_t)d * d, cd(0.0, 0.0));
    std::vector<int> old_pos;  // position in nq of each old qubit
    int oldmask = 0;
    for (int q : b->qubits) {
        int p = (int)(std::find(nq.begin(), nq.end(), q) - nq.begin());
        old_pos.push_back(p);
        oldmask |= 1 << p;
    }
    const int ko = (int)b->qubits.size();
    const int dold = 1 << ko;
    for (int r = 0; r < d; ++r) {
        int ro = 0;
        for (int i = 0; i < ko; ++i) ro |= ((r >> old_pos[i]) & 1) << i;
        for (int cc = 0; cc < d; ++cc) {
            if ((r & ~oldmask) != (cc & ~oldmask)) continue;
            int co = 0;
            for (int i = 0; i < ko; ++i) co |= ((cc >> old_pos[i]) & 1) << i;
            out[(size_t)r * d + cc] = ko ? b->mat[(size_t)ro * dold + co] : cd(r == cc ? 1.0 : 0.0);
        }
    }
    b->qubits = nq;
    b->mat.swap(out);
}

// Left-multiply the block by a dense gate whose qubits are in the block.
void block_apply_dense(Block* b, const CGate& g) {
    const int k = (int)b->qubits.size();
    const int d = 1 << k;
    const int gd = 1 << g.nq;
    int gp[2] = {b->pos(g.q[0]), g.nq > 1 ? b->pos(g.q[1]) : -1};
    int gmask = 0;
    for (int i = 0; i < g.nq; ++i) gmask |= 1 << gp[i];
    std::vector<cd> col(d), nc(d);
    for (int c = 0; c < d; ++c) {
        for (int r = 0; r < d; ++r) col[r] = b->mat[(size_t)r * d + c];
        for (int r = 0; r < d; ++r) {
            if (r & gmask) continue;  // r = group base (gate bits zero)
            cd v[4], w[4];
            int idx[4];
            for (int j = 0; j < gd; ++j) {
                int x = r;
                for (int i = 0; i < g.nq; ++i)
                    if ((j >> i) & 1) x |= 1 << gp[i];
                idx[j] = x;
                v[j] = col[x];
            }
            for (int a = 0; a < gd; ++a) {
                cd acc(0.0, 0.0);
                for (int bb = 0; bb < gd; ++bb) acc += g.m[a * gd + bb] * v[bb];
                w[a] = acc;
            }
            for (int j = 0; j < gd; ++j) nc[idx[j]] = w[j];
        }
        for (int r = 0; r < d; ++r) b->mat[(size_t)r * d + c] = nc[r];
    }
}

// Left-multiply the block by a diagonal gate whose qubits are in the block.
void block_apply_diag(Block* b, const CGate& g) {
    const int k = (int)b->qubits.size();
    const int d = 1 << k;
    int gp[2] = {b->pos(g.q[0]), g.nq > 1 ? b->pos(g.q[1]) : -1};
    for (int r = 0; r < d; ++r) {
        int j = 0;
        for (int i = 0; i < g.nq; ++i) j |= ((r >> gp[i]) & 1) << i;
        const cd f = std::polar(1.0, g.ph[j]);
        for (int c = 0; c < d; ++c) b->mat[(size_t)r * d + c] *= f;
    }
}

// The 2^k x 2^k matrix of gates on the sorted qubit set qubits.
std::vector<cd> block_matrix(const std::vector<int>& qubits, const std::vector<CGate>& seq) {
    Block b;
    expand_block(&b, qubits);
    for (const CGate& g : seq) {
        if (g.kind == GK_DIAG) block_apply_diag(&b, g);
        else block_apply_dense(&b, g);
    }
    return b.mat;
}

void diag_add(DiagForm* D, int n, const CGate& g) {
    if (g.nq == 1) {
        const int q = g.q[0];
        D->c += g.ph[0];
        D->a[q] += g.ph[1] - g.ph[0];
        D->support[q] = 1;
    } else {
        const int q0 = g.q[0], q1 = g.q[1];
        const double* t = g.ph;  // local j = b0 + 2 b1
        D->c += t[0];
        D->a[q0] += t[1] - t[0];
        D->a[q1] += t[2] - t[0];
        const int lo = std::min(q0, q1), hi = std::max(q0, q1);
        D->b[(size_t)lo * n + hi] += t[3] - t[2] - t[1] + t[0];
        D->support[q0] = 1;
        D->support[q1] = 1;
    }
}

bool touches(const DiagForm& D, const CGate& g) {
    for (int i = 0; i < g.nq; ++i)
        if (D.support[g.q[i]]) return true;
    return false;
}

// Estimated CUDA-core instructions per amplitude of a block of k qubits as a
// dense 2^k x 2^k product, and as a gate sequence applied in registers.
double dense_cost(int k) { return 4.0 * (double)(1 << k) + 2.0; }
// A real rotation [[c, -s], [s, c]] costs 2 in a register pass (its factor is
// deferred to the write-back), another real 2x2 4.
double gate_sequence_cost(const std::vector<GateRec>& recs, const std::vector<cd>* data = nullptr) {
    double c = 2.0;
    const double hs = 1.0 / std::sqrt(2.0);
    for (const GateRec& r : recs) {
        if (r.kind == GR_UR && data) {
            const cd* m = data->data() + r.off;
            // a Hadamard becomes a butterfly (its factor deferred), a rotation
            // a two-FMA form; other real 2x2 products cost 4
            const bool had = m[0] == cd(hs, 0.0) && m[1] == cd(hs, 0.0) && m[2] == cd(hs, 0.0) && m[3] == cd(-hs, 0.0);
            c += had ? 1.0 : (m[0] == m[3] && m[1] == -m[2] ? 2.0 : 4.0);
        } else {
            c += r.kind == GR_U ? 8.0 : r.kind == GR_UR ? 4.0 : r.kind == GR_DT ? 5.0 : 1.0;
        }
    }
    return c;
}

// A 4- or 5-qubit block on the tensor cores (register passes), in the same
// units: the FP16 split of the registers (about 11 instructions per
// amplitude), the TMEM traffic and the exposed latency of the products
// (measured: random U3+CX blocks of about 45 run faster on the tensor cores,
// QFT blocks of about 27 slower).
double tc_cost(int k) { return k >= 5 ? 32.0 : 28.0; }

bool is_real(const cd* m, int cnt) {
    for (int i = 0; i < cnt; ++i)
        if (m[i].imag() != 0.0) return false;
    return true;
}

// The block as a sequence on block-local positions: consecutive one-qubit
// gates on one position multiplied together, diagonal gates gathered into
// one 2^k-entry phase table, CX and SWAP kept as permutations.  The pending
// table is applied only before a one-qubit gate on a position it depends on:
// it commutes with one-qubit gates elsewhere, and it moves past a
// permutation P as D'[j] = D[P(j)] (CX and SWAP are involutions).  Before
// such a flush, later diagonal gates that commute with every gate between
// join the table.  With split_u3, U3(t, f, l) enters as P(l) RY(t) P(f), an
// exact factorisation whose phases join the tables and whose RY is a real
// 2x2 (half the arithmetic of a complex one).  False when the block holds a
// gate this form does not cover or exceeds the record limits.
bool gate_sequence(const Block& B, std::vector<GateRec>* recs, std::vector<cd>* data, bool split_u3 = false) {
    recs->clear();
    data->clear();
    const int k = (int)B.qubits.size(), D = 1 << k;
    std::vector<CGate> seq;
    seq.reserve(B.seq.size() * 3);
    for (const CGate& g : B.seq) {
        if (split_u3 && g.type == SV_U3) {
            sv_gate e;
            memset(&e, 0, sizeof(e));
            e.nq = 1;
            e.q[0] = (uint32_t)g.q[0];
            CGate c;
            e.type = SV_P;
            e.p[0] = g.p[2];
            make_canonical(e, &c);
            seq.push_back(c);
            e.type = SV_RY;
            e.p[0] = g.p[0];
            make_canonical(e, &c);
            seq.push_back(c);
            e.type = SV_P;
            e.p[0] = g.p[1];
            make_canonical(e, &c);
            seq.push_back(c);
        } else {
            seq.push_back(g);
        }
    }
    auto posmask = [&](const CGate& g) {
        int m = 1 << B.pos(g.q[0]);
        if (g.nq > 1) m |= 1 << B.pos(g.q[1]);
        return m;
    };
    std::vector<double> ph(D, 0.0);
    bool dpend = false;
    int dep = 0;  // positions the pending table depends on
    auto add_diag = [&](const CGate& g) {
        const int p0 = B.pos(g.q[0]), p1 = g.nq > 1 ? B.pos(g.q[1]) : 0;
        for (int j = 0; j < D; ++j) {
            int li = (j >> p0) & 1;
            if (g.nq > 1) li |= ((j >> p1) & 1) << 1;
            ph[j] += g.ph[li];
        }
        dpend = true;
        dep |= posmask(g);
    };
    auto flush_diag = [&]() {
        if (!dpend) return;
        // a = the positions the table depends on: entry j equals entry j & a
        recs->push_back(GateRec{GR_DT, dep, 0, (int)data->size()});
        for (int j = 0; j < D; ++j) data->push_back(std::polar(1.0, ph[j]));
        std::fill(ph.begin(), ph.end(), 0.0);
        dpend = false;
        dep = 0;
    };
    const int N = (int)seq.size();
    std::vector<char> used(N, 0);
    for (int i = 0; i < N; ++i) {
        if (used[i]) continue;
        const CGate& g = seq[i];
        if (g.kind == GK_DIAG) {
            add_diag(g);
            continue;
        }
        if (g.type == SV_CX || g.type == SV_SWAP) {
            const int pa = B.pos(g.q[0]), pb = B.pos(g.q[1]);
            if (dpend) {
                std::vector<double> moved(D);
                for (int j = 0; j < D; ++j) {
                    const int ba = (j >> pa) & 1, bb = (j >> pb) & 1;
                    const int pj = g.type == SV_CX ? j ^ (ba << pb)
                                                   : (j & ~((1 << pa) | (1 << pb))) | (bb << pa) | (ba << pb);
                    moved[j] = ph[pj];
                }
                ph.swap(moved);
                const int da = (dep >> pa) & 1, db = (dep >> pb) & 1;
                if (g.type == SV_CX) dep |= db << pa;  // the target's phase now reads the control too
                else dep = (dep & ~((1 << pa) | (1 << pb))) | (db << pa) | (da << pb);
            }
            recs->push_back(GateRec{g.type == SV_CX ? GR_CX : GR_SWAP, pa, pb, 0});
            continue;
        }
        if (g.nq != 1) return false;
        const int p = B.pos(g.q[0]);
        if (dpend && ((dep >> p) & 1)) {
            // take in later diagonal gates that commute with everything
            // between, then apply the table
            int blocked = 1 << p;
            for (int j = i + 1; j < N && blocked != D - 1; ++j) {
                if (used[j]) continue;
                const int pm = posmask(seq[j]);
                if (seq[j].kind == GK_DIAG) {
                    if (!(pm & blocked)) {
                        add_diag(seq[j]);
                        used[j] = 1;
                    }
                } else {
                    blocked |= pm;
                }
            }
            flush_diag();
        }
        // merge with the previous record when it is a one-qubit gate on the
        // same position (a pending table here does not depend on p)
        if (!recs->empty() && (recs->back().kind == GR_U || recs->back().kind == GR_UR) && recs->back().a == p) {
            cd* Mp = data->data() + recs->back().off;  // merge: M = G * M_prev
            const cd M[4] = {g.m[0] * Mp[0] + g.m[1] * Mp[2], g.m[0] * Mp[1] + g.m[1] * Mp[3],
                             g.m[2] * Mp[0] + g.m[3] * Mp[2], g.m[2] * Mp[1] + g.m[3] * Mp[3]};
            for (int t = 0; t < 4; ++t) Mp[t] = M[t];
            recs->back().kind = is_real(Mp, 4) ? GR_UR : GR_U;
        } else {
            recs->push_back(GateRec{is_real(g.m, 4) ? GR_UR : GR_U, p, 0, (int)data->size()});
            for (int t = 0; t < 4; ++t) data->push_back(g.m[t]);
        }
    }
    flush_diag();
    return (int)recs->size() <= kMaxGateRecs && (int)data->size() <= kMaxGateData;
}

// A block's gate sequence: the cheaper of the plain form and, when the block
// holds U3 gates, the form with each U3 split into P RY P.
bool best_gate_sequence(const Block& B, std::vector<GateRec>* recs, std::vector<cd>* data) {
    const bool ok = gate_sequence(B, recs, data, false);
    bool u3 = false;
    for (const CGate& g : B.seq) u3 |= g.type == SV_U3;
    if (!u3) return ok;
    std::vector<GateRec> r2;
    std::vector<cd> d2;
    if (gate_sequence(B, &r2, &d2, true) && (!ok || gate_sequence_cost(r2, &d2) < gate_sequence_cost(*recs, data))) {
        recs->swap(r2);
        data->swap(d2);
        return true;
    }
    return ok;
}

constexpr int kMaxBlockGates = 40;  // 20 one-qubit gates and 20 phase tables fit kMaxGateData
constexpr int kMaxTcBlockGates = 4096;  // a tensor-core block is a dense matrix: any gate count
// Tensor-core matrices (hi and lo operands) one register pass may stage when
// the planner chooses them itself: two 5-qubit blocks, which keeps a 13-qubit
// complex64 pass at two CTAs per SM (measured: a pass staging three ran on one
// CTA per SM at less than half the speed).
constexpr int kTcStageBudget = 2 * 2 * (8 << 10);

// Estimated instructions per amplitude of a pass's ops: each block pays its
// own cost plus a register remap (a shared-memory round trip of the tile),
// each diagonal run one table product.
double ops_cost(const std::vector<HostOp>& ops) {
    constexpr double kRemap = 16.0, kDiagRun = 6.0;
    double c = 0.0;
    for (const HostOp& o : ops) {
        if (o.kind == OP_DIAG) c += kDiagRun;
        else if (o.kind == OP_GATES) c += gate_sequence_cost(o.recs, &o.gdata) + kRemap;
        else if (o.tc) c += tc_cost((int)o.qubits.size()) + kRemap;
        else c += dense_cost((int)o.qubits.size()) + kRemap;
    }
    return c;
}

// Reorder a pass's gates so that they come in groups of at most kmax qubits:
// each group starts from the earliest gate that can run next and grows its
// qubit set S one gate at a time, taking the gate whose qubits let the most
// further gates join, and every gate that can run next with qubits inside S
// joins.  A gate can run next once all earlier gates on its qubits have; so
// each qubit sees its gates in the original order and the product of the
// reordered list is the same operator.
std::vector<int> cluster_order(const std::vector<CGate>& gates, const std::vector<int>& order, int kmax) {
    const int G = (int)order.size();
    int nq = 0;
    for (int gi : order)
        for (int i = 0; i < gates[gi].nq; ++i) nq = std::max(nq, gates[gi].q[i] + 1);
    if (nq > 64) return order;
    std::vector<std::vector<int>> seq(nq);  // positions in `order` per qubit
    for (int i = 0; i < G; ++i)
        for (int j = 0; j < gates[order[i]].nq; ++j) seq[gates[order[i]].q[j]].push_back(i);
    auto qmask = [&](int i) {
        uint64_t m = 0;
        for (int j = 0; j < gates[order[i]].nq; ++j) m |= 1ull << gates[order[i]].q[j];
        return m;
    };
    std::vector<uint64_t> masks(G);
    for (int i = 0; i < G; ++i) masks[i] = qmask(i);
    auto is_ready = [&](const std::vector<int>& head, int i) {
        for (int j = 0; j < gates[order[i]].nq; ++j) {
            const int q = gates[order[i]].q[j];
            if (head[q] >= (int)seq[q].size() || seq[q][head[q]] != i) return false;
        }
        return true;
    };
    // take every gate that can run next with qubits inside S; returns the count
    auto closure = [&](uint64_t S, std::vector<int>& head, std::vector<int>* emit) {
        int cnt = 0;
        for (bool progress = true; progress;) {
            progress = false;
            for (uint64_t r = S; r; r &= r - 1) {
                const int q = __builtin_ctzll(r);
                while (head[q] < (int)seq[q].size()) {
                    const int i = seq[q][head[q]];
                    if ((masks[i] & ~S) || !is_ready(head, i)) break;
                    for (int j = 0; j < gates[order[i]].nq; ++j) ++head[gates[order[i]].q[j]];
                    if (emit) emit->push_back(i);
                    ++cnt;
                    progress = true;
                }
            }
        }
        return cnt;
    };
    std::vector<int> head(nq, 0), out;  // out: positions in `order`
    std::vector<char> taken(G, 0);
    out.reserve(G);
    auto take = [&](uint64_t S) {
        const size_t b = out.size();
        closure(S, head, &out);
        for (size_t t = b; t < out.size(); ++t) taken[out[t]] = 1;
    };
    while ((int)out.size() < G) {
        // a gate that can run next is at the head of each of its qubits'
        // queues: the candidates, in list order
        std::vector<int> cand;
        for (int q = 0; q < nq; ++q)
            if (head[q] < (int)seq[q].size() && is_ready(head, seq[q][head[q]])) cand.push_back(seq[q][head[q]]);
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        // seed: the earliest of them, dense before diagonal
        int seed = -1;
        for (int pass = 0; pass < 2 && seed < 0; ++pass)
            for (int i : cand)
                if ((pass == 0) == (gates[order[i]].kind == GK_DENSE)) {
                    seed = i;
                    break;
                }
        if (seed < 0) return order;  // cannot happen for a valid order
        uint64_t S = masks[seed];
        take(S);
        for (;;) {
            int best = -1, best_gain = 0, best_pop = 0;
            for (uint64_t r = S; r; r &= r - 1) {
                const int q = __builtin_ctzll(r);
                if (head[q] >= (int)seq[q].size()) continue;
                const int i = seq[q][head[q]];
                const uint64_t S2 = S | masks[i];
                if (S2 == S || __builtin_popcountll(S2) > kmax || !is_ready(head, i)) continue;
                std::vector<int> h2 = head;
                const int gain = closure(S2, h2, nullptr);
                const int pop = __builtin_popcountll(S2);
                if (gain > best_gain || (gain == best_gain && best >= 0 && (pop < best_pop || (pop == best_pop && i < best)))) {
                    best = i;
                    best_gain = gain;
                    best_pop = pop;
                }
            }
            // also grow into a qubit outside S through any gate that can run next
            if (best < 0) {
                cand.clear();
                for (int q = 0; q < nq; ++q)
                    if (head[q] < (int)seq[q].size() && is_ready(head, seq[q][head[q]])) cand.push_back(seq[q][head[q]]);
                std::sort(cand.begin(), cand.end());
                cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
                for (int i : cand) {
                    const uint64_t S2 = S | masks[i];
                    if (S2 == S || __builtin_popcountll(S2) > kmax) continue;
                    std::vector<int> h2 = head;
                    const int gain = closure(S2, h2, nullptr);
                    const int pop = __builtin_popcountll(S2);
                    if (gain > best_gain || (gain == best_gain && best >= 0 && pop < best_pop)) {
                        best = i;
                        best_gain = gain;
                        best_pop = pop;
                    }
                }
            }
            if (best < 0) break;
            S |= masks[best];
            take(S);
        }
    }
    for (int& i : out) i = order[i];
    return out;
}

}  // namespace

int canonicalise(int n, const sv_gate* g, size_t count, std::vector<CGate>* out, size_t* bad) {
    out->clear();
    out->reserve(count);
    for (size_t i = 0; i < count; ++i) {
        const int k = arity(g[i].type);
        bool ok = k > 0 && (int)g[i].nq == k;
        for (int a = 0; ok && a < k; ++a) {
            if (g[i].q[a] >= (uint32_t)n) ok = false;
            for (int b = 0; ok && b < a; ++b)
                if (g[i].q[a] == g[i].q[b]) ok = false;
        }
        const uint32_t t = g[i].type;
        const int np = t == SV_U3 ? 3 : ((t == SV_RX || t == SV_RY || t == SV_RZ || t == SV_P || t == SV_CP) ? 1 : 0);
        for (int a = 0; ok && a < np; ++a)
            if (!std::isfinite(g[i].p[a])) ok = false;
        if (!ok) {
            *bad = i;
            return SV_EINVAL;
        }
        if (g[i].type == SV_MEASURE) continue;
        out->emplace_back();
        make_canonical(g[i], &out->back());
    }
    return SV_OK;
}

void drop_small_phases(std::vector<CGate>* g, double eps) {
    if (!(eps > 0.0)) return;
    std::vector<CGate> kept;
    kept.reserve(g->size());
    for (const CGate& x : *g) {
        if (x.type == SV_P || x.type == SV_RZ || x.type == SV_CP) {
            // reduced modulo the gate's period: 2 pi for P and CP, 4 pi for RZ
            // (RZ(2 pi) = -I is not the identity)
            const double a = std::remainder(x.p[0], (x.type == SV_RZ ? 4.0 : 2.0) * kPi);
            if (std::fabs(a) < eps) continue;
        }
        kept.push_back(x);
    }
    g->swap(kept);
}

PlanOptions resolve_options(int n, int dtype, const sv_options* opt) {
    PlanOptions po;
    po.tile_m = dtype == SV_C64 ? 13 : 12;
    // complex128 keeps 2^4 amplitudes per thread in registers: 4-qubit blocks
    // keep its passes on the register kernel (measured 2.4-3.9x faster than
    // 5-qubit blocks on the shared-memory kernel)
    if (dtype != SV_C64) po.k_max = 4;
    if (opt) {
        if (opt->k_max > 0) po.k_max = opt->k_max;
        if (opt->tile_m > 0) po.tile_m = opt->tile_m;
        po.planner = opt->planner;
        po.tensor = opt->tensor > 0 ? 0 : -1;
        po.pass_kernel = opt->pass_kernel == 1 || opt->pass_kernel == 2 ? opt->pass_kernel : 0;
        po.relabel = opt->relabel == 1 ? 1 : 0;
        po.drop_phase_below = opt->drop_phase_below > 0.0 && std::isfinite(opt->drop_phase_below) ? opt->drop_phase_below : 0.0;
        po.mux = opt->mux < 0 ? -1 : (opt->mux > 0 ? 1 : 0);
        po.jit = opt->jit < 0 ? -1 : (opt->jit > 0 ? 1 : 0);
        po.tc_auto = opt->tensor == 0 ? kTcAutoDefault : 0;
    } else {
        po.tc_auto = kTcAutoDefault;
    }
    if (dtype != SV_C64) po.tensor = -1, po.tc_auto = 0;
    po.k_max = std::max(2, std::min(kMaxK, po.k_max));
    const int mmax = dtype == SV_C64 ? 14 : 13;
    po.tile_m = std::max(1, std::min(mmax, po.tile_m));
    po.tile_m = std::min(po.tile_m, n);
    return po;
}

// One pass of the greedy planner from the front of `remaining` (gate
// indices in circuit order): the pass, and in *deferred_out the gates left
// for later passes, in order.  form_matrices = false leaves the dense blocks'
// matrices unformed (their gates in HostOp::seq; see form_dense_matrices).
void greedy_pass(int n, int dtype, const std::vector<CGate>& gates, const std::vector<Mux>& muxes,
                 const PlanOptions& po, const std::vector<int>& remaining, HostPass* pass_out,
                 std::vector<int>* deferred_out, bool form_matrices) {
    const int L = std::min(row_bits(dtype, po.pass_kernel), n);
    // the tile holds the row bits plus room for any two-qubit gate
    const int m = std::max(std::min(n, L + 2), std::min(po.tile_m, n));
    const int kmax = std::min(po.k_max, m);
    // tensor-core blocks run in register passes of at least 128 threads
    const bool tc_auto_ok = po.tc_auto && dtype == SV_C64 && po.pass_kernel == 0 && m - reg_bits(dtype) >= 7;
    std::vector<char> inT(n), blocked(n);
    std::vector<int> executed, deferred;
    int nblocked = 0;
    auto block = [&](const CGate& g) {
        for (int i = 0; i < g.nq; ++i)
            if (!blocked[g.q[i]]) blocked[g.q[i]] = 1, ++nblocked;
        if (g.kind == GK_MUX)
            for (int c : muxes[g.mux].controls)
                if (!blocked[c]) blocked[c] = 1, ++nblocked;
    };
    // A multiplexor at the front opens a multiplexor pass: it takes every
    // later multiplexor that the gates skipped over commute with (no
    // shared qubit), up to kMuxMaxTargets targets whose controls stay off
    // the targets and number at most kMuxMaxControls together.
    if (gates[remaining[0]].kind == GK_MUX) {
        HostPass pass;
        std::fill(blocked.begin(), blocked.end(), 0);
        nblocked = 0;
        uint64_t tmask = 0, cunion = 0;
        deferred.clear();
        for (size_t r = 0; r < remaining.size(); ++r) {
            const int gi = remaining[r];
            const CGate& g = gates[gi];
            bool take = false;
            uint64_t tm = 0, cm = 0;
            if (g.kind == GK_MUX && (int)pass.mux.size() < kMuxMaxTargets && nblocked < n) {
                const Mux& M = muxes[g.mux];
                tm = 1ull << M.target;
                bool fr = !blocked[M.target];
                for (int c : M.controls) {
                    cm |= 1ull << c;
                    fr &= !blocked[c];
                }
                const uint64_t nu = cunion | cm;
                take = fr && !(tmask & (tm | cm)) && !(nu & (tmask | tm)) &&
                       __builtin_popcountll(nu) <= kMuxMaxControls;
                if (take) cunion = nu;
            }
            if (take) {
                const Mux& M = muxes[g.mux];
                pass.mux.push_back(g.mux);
                tmask |= tm;
                pass.ngates += M.ngates;
                for (int t = 0; t < 14; ++t) pass.type_count[t] += M.type_count[t];
            } else {
                deferred.push_back(gi);
                block(g);
            }
        }
        *pass_out = std::move(pass);
        deferred_out->swap(deferred);
        return;
    }
    // Scan 1: grow the tile set T from the front of the remaining list.
    std::fill(inT.begin(), inT.end(), 0);
    std::fill(blocked.begin(), blocked.end(), 0);
    int cnt = 0;
    nblocked = 0;
    for (int q = 0; q < L; ++q) inT[q] = 1, ++cnt;
    for (int gi : remaining) {
        const CGate& g = gates[gi];
        bool tb = false;
        for (int i = 0; i < g.nq; ++i) tb |= blocked[g.q[i]] != 0;
        if (tb || g.kind == GK_MUX) { block(g); }
        else if (g.kind == GK_DENSE) {
            int need = 0;
            for (int i = 0; i < g.nq; ++i) need += !inT[g.q[i]];
            if (cnt + need <= m) {
                for (int i = 0; i < g.nq; ++i)
                    if (!inT[g.q[i]]) inT[g.q[i]] = 1, ++cnt;
            } else {
                block(g);
            }
        }
        if (nblocked == n) break;
    }
    // Fill the tile up to m qubits (lowest unused qubits first): a wider
    // tile costs nothing extra and keeps all passes the same shape.
    for (int q = 0; q < n && cnt < m; ++q)
        if (!inT[q]) inT[q] = 1, ++cnt;

    // Scan 2: partition with the final T.
    std::fill(blocked.begin(), blocked.end(), 0);
    nblocked = 0;
    executed.clear();
    deferred.clear();
    for (int gi : remaining) {
        const CGate& g = gates[gi];
        if (nblocked == n) { deferred.push_back(gi); continue; }
        bool tb = false, fits = true;
        for (int i = 0; i < g.nq; ++i) {
            tb |= blocked[g.q[i]] != 0;
            fits &= inT[g.q[i]] != 0;
        }
        if (!tb && g.kind != GK_MUX && (g.kind == GK_DIAG || fits)) executed.push_back(gi);
        else { deferred.push_back(gi); block(g); }
    }

    HostPass pass;
    for (int q = 0; q < n; ++q)
        if (inT[q]) pass.tile.push_back(q);
    pass.L = L;
    pass.ngates = (int)executed.size();
    for (int gi : executed) pass.type_count[gates[gi].type < 14 ? gates[gi].type : 13]++;

    // Fuse the executed gates into dense blocks and diagonal runs, in the
    // given order (any order that keeps each qubit's gates in sequence).
    // Blocks keep their qubits and gates; a dense op's matrix is formed
    // when it is emitted, a gate sequence's only if a kernel needs it.
    auto fuse = [&](const std::vector<int>& order, std::vector<HostOp>* ops_out) {
        Block B;
        DiagForm D;
        D.init(n);
        bool dpend = false;
        int tc_bytes = 0;  // tensor-core matrices the pass stages so far
        auto flushB = [&]() {
            if (!B.active()) return;
            HostOp op;
            op.qubits = B.qubits;
            op.ngates = B.ngates;
            const int kb = (int)B.qubits.size();
            // tensor-core blocks: forced (tensor = 1) or where their cost
            // is below the gate sequence's (the default)
            const bool tc_forced = po.tensor == 0 && dtype == SV_C64 && kb >= 4;
            // (the automatic choice keeps the pass's staged matrices within
            // kTcStageBudget: beyond it the pass would hold one CTA per SM)
            const bool tc_auto = tc_auto_ok && (kb == 4 || kb == 5) && tc_bytes + 2 * tc16_bytes(kb) <= kTcStageBudget;
            const bool seq = !tc_forced && kb <= max_gates_k(dtype) && best_gate_sequence(B, &op.recs, &op.gdata);
            const double seq_cost = seq ? gate_sequence_cost(op.recs, &op.gdata) : 1e30;
            if (tc_forced || (tc_auto && seq_cost > tc_cost(kb))) {
                op.kind = OP_DENSE;
                op.tc = true;
                tc_bytes += 2 * tc16_bytes(kb);
                if (form_matrices) op.mat = block_matrix(B.qubits, B.seq);
                else op.seq = B.seq;
                op.recs.clear();
                op.gdata.clear();
            } else if (seq && (seq_cost <= dense_cost(kb) || (kb > kRegDenseMaxK && po.pass_kernel != 1))) {
                // the cheaper representation: the dense 2^k matrix, or the
                // gate sequence applied in registers (blocks wider than the
                // register kernel's dense limit stay gate sequences, which
                // keeps the pass on the register kernel)
                op.kind = OP_GATES;
                op.seq = B.seq;
            } else {
                op.kind = OP_DENSE;
                // (the shared-memory kernel's 3xTF32 path also takes 3-qubit blocks)
                op.tc = po.tensor == 0 && dtype == SV_C64 && kb >= kMinTcK && po.pass_kernel == 1;
                if (form_matrices) op.mat = block_matrix(B.qubits, B.seq);
                else op.seq = B.seq;
                op.recs.clear();
                op.gdata.clear();
            }
            ops_out->push_back(std::move(op));
            B = Block();
        };
        int dgates = 0;
        auto flushD = [&]() {
            if (!dpend) return;
            HostOp op;
            op.kind = OP_DIAG;
            op.diag = D;
            op.ngates = dgates;
            ops_out->push_back(std::move(op));
            D.init(n);
            dpend = false;
            dgates = 0;
        };
        for (int gi : order) {
            const CGate& g = gates[gi];
            if (g.kind == GK_DIAG) {
                bool inB = B.active();
                for (int i = 0; inB && i < g.nq; ++i) inB = B.pos(g.q[i]) >= 0;
                // A diagonal gate on tile qubits may also widen the current
                // block (diagonals commute with the pending run D, so moving
                // it into the block is exact).
                bool widen = false;
                std::vector<int> u;
                if (!inB && B.active()) {
                    bool inT_all = true;
                    u = B.qubits;
                    for (int i = 0; i < g.nq; ++i) {
                        inT_all &= inT[g.q[i]] != 0;
                        if (B.pos(g.q[i]) < 0) u.push_back(g.q[i]);
                    }
                    widen = inT_all && (int)u.size() <= kmax;
                }
                if (widen) {
                    std::sort(u.begin(), u.end());
                    B.qubits = u;
                }
                if (inB || widen) {
                    B.seq.push_back(g);
                    B.ngates++;
                } else {
                    diag_add(&D, n, g);
                    dpend = true;
                    dgates++;
                }
                continue;
            }
            if (dpend && touches(D, g)) {
                flushB();
                flushD();
            }
            std::vector<int> u = B.qubits;
            for (int i = 0; i < g.nq; ++i)
                if (std::find(u.begin(), u.end(), g.q[i]) == u.end()) u.push_back(g.q[i]);
            std::sort(u.begin(), u.end());
            // a block holds at most kMaxBlockGates gates, so that its gate
            // sequence stays within the record and data limits
            // (with tensor-core blocks available, 4- and 5-qubit blocks
            // take any number of gates: their cost does not grow with it)
            const int cap = (tc_auto_ok || (po.tensor == 0 && dtype == SV_C64)) && (int)B.qubits.size() >= 4
                                ? kMaxTcBlockGates : kMaxBlockGates;
            if (B.active() && ((int)u.size() > kmax || B.ngates >= cap)) {
                flushB();
                u.assign(g.q, g.q + g.nq);
                std::sort(u.begin(), u.end());
            }
            B.qubits = u;
            B.seq.push_back(g);
            B.ngates++;
        }
        flushB();
        flushD();
    };
    fuse(executed, &pass.ops);
    // A reordering that groups gates by qubit set (each qubit's gates
    // kept in sequence, so the circuit is the same) often needs fewer
    // blocks; keep it when its estimated cost is lower.
    if (kmax >= 2) {
        const std::vector<int> reord = cluster_order(gates, executed, kmax);
        if (reord != executed) {
            std::vector<HostOp> alt;
            fuse(reord, &alt);
            if (ops_cost(alt) < ops_cost(pass.ops)) pass.ops.swap(alt);
        }
    }
    *pass_out = std::move(pass);
    deferred_out->swap(deferred);
}

// Dense blocks planned without their matrix get it now.
void form_dense_matrices(HostPass* hp) {
    for (HostOp& op : hp->ops)
        if (op.kind == OP_DENSE && op.mat.empty() && !op.seq.empty()) {
            op.mat = block_matrix(op.qubits, op.seq);
            op.seq.clear();
        }
}

void plan_greedy(int n, int dtype, const std::vector<CGate>& gates, const PlanOptions& po, Plan* out,
                 const std::vector<Mux>* muxes) {
    out->muxes.clear();
    if (muxes) out->muxes = *muxes;
    out->n = n;
    out->dtype = dtype;
    out->plain = false;
    out->passes.clear();
    out->gates = (int64_t)gates.size();
    out->tensor = po.tensor;
    out->no_register_passes = po.pass_kernel == 1;
    out->use_tma = po.pass_kernel == 2;
    out->jit = po.jit;
    std::vector<int> remaining(gates.size()), deferred;
    for (size_t i = 0; i < gates.size(); ++i) remaining[i] = (int)i;
    while (!remaining.empty()) {
        HostPass pass;
        greedy_pass(n, dtype, gates, out->muxes, po, remaining, &pass, &deferred, true);
        out->passes.push_back(std::move(pass));
        remaining.swap(deferred);
        deferred.clear();
    }
}

void plan_plain(int n, int dtype, const std::vector<CGate>& gates, Plan* out) {
    out->n = n;
    out->dtype = dtype;
    out->plain = true;
    out->passes.clear();
    out->plain_ops.clear();
    out->gates = (int64_t)gates.size();
    for (const CGate& g : gates) {
        PlainOp op;
        memset(&op, 0, sizeof(op));
        op.q0 = g.q[0];
        op.q1 = g.q[1];
        if (g.kind == GK_DENSE && g.nq == 1) {
            op.kind = PK_1Q;
            for (int i = 0; i < 4; ++i) op.m[i] = g.m[i];
        } else if (g.kind == GK_DIAG && g.nq == 1) {
            if (g.ph[0] == 0.0) {
                op.kind = PK_PHASE1;
                op.m[0] = std::polar(1.0, g.ph[1]);
            } else {
                op.kind = PK_DIAG1;
                op.m[0] = std::polar(1.0, g.ph[0]);
                op.m[1] = std::polar(1.0, g.ph[1]);
            }
        } else if (g.type == SV_CX) {
            op.kind = PK_CX;
        } else if (g.type == SV_SWAP) {
            op.kind = PK_SWAP;
        } else {  // CZ, CP: phase on |11>
            op.kind = PK_CPHASE;
            op.m[0] = std::polar(1.0, g.ph[3]);
        }
        out->plain_ops.push_back(op);
    }
}

void plan_summary(const Plan& p, sv_plan_info* info) {
    memset(info, 0, sizeof(*info));
    info->gates = p.gates;
    const double N = ldexp(1.0, p.n);
    const double s = p.dtype == SV_C64 ? 8.0 : 16.0;
    double bytes = 0.0;
    if (p.plain) {
        info->passes = (int64_t)p.plain_ops.size();
        for (const PlainOp& o : p.plain_ops) {
            switch (o.kind) {
            case PK_1Q: case PK_DIAG1: bytes += 2.0 * N * s; break;
            case PK_CX: case PK_SWAP: case PK_PHASE1: bytes += N * s; break;
            case PK_CPHASE: bytes += 0.5 * N * s; break;
            }
            info->dense_ops += (o.kind == PK_1Q || o.kind == PK_CX || o.kind == PK_SWAP);
            info->diag_ops += !(o.kind == PK_1Q || o.kind == PK_CX || o.kind == PK_SWAP);
        }
        info->max_k = p.plain_ops.empty() ? 0 : 2;
    } else {
        info->passes = (int64_t)p.passes.size();
        for (const HostPass& hp : p.passes) {
            bytes += 2.0 * N * s;
            info->mux_ops += (int64_t)hp.mux.size();
            info->mux_passes += !hp.mux.empty();
            for (const HostOp& o : hp.ops) {
                if (o.kind == OP_DENSE || o.kind == OP_GATES) {
                    info->dense_ops++;
                    info->gate_ops += o.kind == OP_GATES;
                    info->tc_ops += o.tc;
                    info->max_k = std::max<int64_t>(info->max_k, (int64_t)o.qubits.size());
                } else {
                    info->diag_ops++;
                }
            }
        }
    }
    info->bytes_moved = (int64_t)bytes;
}

std::vector<float> pass_features(int n, int dtype, const HostPass& p, bool tensor_cores, bool register_pass) {
    std::vector<float> f(kFeatures, 0.0f);
    const int m = (int)p.tile.size();
    f[0] = n / 34.0f;
    f[1] = (float)dtype;
    f[2] = m / 14.0f;
    f[3] = p.L / 4.0f;
    double flops = 0.0, msize = 0.0;
    int ndiag = 0, ntc = 0;
    for (const HostOp& o : p.ops) {
        if (o.kind == OP_DENSE || o.kind == OP_GATES) {
            const int k = (int)o.qubits.size();
            f[3 + k] += 1.0f / 8.0f;  // f[4..8]: dense blocks of width 1..5
            flops += (o.kind == OP_GATES ? gate_sequence_cost(o.recs, &o.gdata)
                                         : o.tc ? tc_cost(k) : dense_cost(k)) / 4.0;
            msize += ldexp(1.0, 2 * k);
            ntc += o.tc;
        } else {
            ++ndiag;
        }
    }
    f[9] = ndiag / 8.0f;
    f[10] = p.ngates / 64.0f;
    f[11] = (float)(flops / 64.0);
    f[12] = (float)(msize / 1024.0);
    f[13] = (float)p.ops.size() / 16.0f;
    for (int t = 0; t < 14; ++t) f[14 + t] = p.type_count[t] / 16.0f;  // f[14..27]
    f[28] = (float)(ldexp(1.0, n) * (dtype == SV_C64 ? 16.0 : 32.0) / ldexp(1.0, 36));
    f[29] = register_pass ? 1.0f : 0.0f;  // kernel: register-resident or shared-memory
    f[30] = tensor_cores ? ntc / 4.0f : 0.0f;  // blocks on the tensor cores
    f[31] = 1.0f;
    return f;
}

// ---------------------------------------------------------------------------
// Device blob: [PassDev x P][OpDev x O][mats (float2 or double2)][diag doubles]
// ---------------------------------------------------------------------------
namespace {
size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// IEEE 754 binary32 -> binary16, round to nearest, ties to even (subnormal
// results included; overflow to infinity).
uint16_t f32_to_f16(float f) {
    uint32_t x;
    memcpy(&x, &f, 4);
    const uint32_t sign = (x >> 16) & 0x8000u, e8 = (x >> 23) & 0xffu;
    uint32_t mant = x & 0x7fffffu;
    if (e8 == 0xffu) return (uint16_t)(sign | 0x7c00u | (mant ? 0x200u : 0u));
    const int e = (int)e8 - 127 + 15;
    if (e >= 31) return (uint16_t)(sign | 0x7c00u);
    if (e <= 0) {
        if (e < -10) return (uint16_t)sign;
        mant |= 0x800000u;  // the implicit bit
        const int shift = 14 - e;
        uint32_t h = mant >> shift;
        const uint32_t rem = mant & ((1u << shift) - 1u), half = 1u << (shift - 1);
        if (rem > half || (rem == half && (h & 1u))) ++h;
        return (uint16_t)(sign | h);
    }
    uint32_t h = ((uint32_t)e << 10) | (mant >> 13);
    const uint32_t rem = mant & 0x1fffu;
    if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;  // a carry moves into the exponent
    return (uint16_t)(sign | h);
}
float f16_to_f32(uint16_t h) {
    const uint32_t sign = (uint32_t)(h & 0x8000u) << 16, e = (h >> 10) & 0x1fu, mant = h & 0x3ffu;
    float f;
    if (e == 0) {
        f = (float)mant * 0x1p-24f;  // zero or subnormal, exact
        return sign ? -f : f;
    }
    const uint32_t x = sign | (e == 31 ? 0x7f800000u | (mant << 13) : ((e - 15 + 127) << 23) | (mant << 13));
    memcpy(&f, &x, 4);
    return f;
}

// FP32 -> TF32 value (10-bit mantissa) rounded to nearest, ties away from
// zero: add half of the dropped 13-bit field to the magnitude, then clear it.
float tf32_round(float v) {
    uint32_t bits;
    memcpy(&bits, &v, 4);
    bits = (bits + 0x1000u) & 0xFFFFE000u;
    float r;
    memcpy(&r, &bits, 4);
    return r;
}

// Phase (radians) as fixed-point turns: the fraction of a turn in units of
// 2^-64, so that sums of coefficients wrap exactly modulo one turn.  The
// FP64 phase carries 53 significant bits; the fraction is rounded to 2^-53.
uint64_t fx_turns(double rad) {
    double t = rad / (2.0 * kPi);
    t -= floor(t);  // [0, 1)
    const uint64_t q = (uint64_t)llround(ldexp(t, 53)) & ((1ull << 53) - 1ull);
    return q << 11;
}

// A diagonal run, split for pass P (layout in DiagLayout).  Everything that
// does not depend on the tile's non-tile bits is precomputed here: the
// tile-internal quadratic tables over the lo (h bits) and hi (m-h bits)
// halves of the tile index and the lo-hi coupling table, each entry the
// exact (modulo one turn) sum of its fixed-point terms.
void write_diag(const DiagForm& D, int n, const HostPass& hp, const PassDev& P, uint64_t* d) {
    const int m = P.m, no = P.nother;
    const DiagLayout Lo(m, no);
    auto B = [&](int qa, int qb) {
        if (qa == qb) return (uint64_t)0;
        const int lo = qa < qb ? qa : qb, hi = qa < qb ? qb : qa;
        return fx_turns(D.b[(size_t)lo * n + hi]);
    };
    d[Lo.c] = fx_turns(D.c);
    for (int t = 0; t < m; ++t) d[Lo.at + t] = fx_turns(D.a[P.tq[t]]);
    for (int o = 0; o < no; ++o) d[Lo.ao + o] = fx_turns(D.a[P.oq[o]]);
    for (int t = 0; t < m; ++t)
        for (int o = 0; o < no; ++o) d[Lo.bo + t * no + o] = B(P.tq[t], P.oq[o]);
    for (int o = 0; o < no; ++o)
        for (int o2 = 0; o2 < no; ++o2) d[Lo.boo + o * no + o2] = B(P.oq[o], P.oq[o2]);
    const int h = Lo.h, mh = Lo.mh;
    for (int e = 0; e < (1 << h); ++e) {
        uint64_t v = 0;
        for (int b = 0; b < h; ++b)
            for (int b2 = 0; b2 < b; ++b2)
                if (((e >> b) & 1) && ((e >> b2) & 1)) v += B(P.tq[b], P.tq[b2]);
        d[Lo.qlo + e] = v;
    }
    for (int e = 0; e < (1 << mh); ++e) {
        uint64_t v = 0;
        for (int b = 0; b < mh; ++b)
            for (int b2 = 0; b2 < b; ++b2)
                if (((e >> b) & 1) && ((e >> b2) & 1)) v += B(P.tq[h + b], P.tq[h + b2]);
        d[Lo.qhi + e] = v;
    }
    for (int t = 0; t < mh; ++t)
        for (int e = 0; e < (1 << h); ++e) {
            uint64_t v = 0;
            for (int b = 0; b < h; ++b)
                if ((e >> b) & 1) v += B(P.tq[b], P.tq[h + t]);
            d[Lo.rt + (t << h) + e] = v;
        }
    (void)hp;
}
}  // namespace

namespace {

// Payload bytes of one region, 16-byte aligned pieces; offsets are bytes
// from the start of the payload until the OpDev array is put in front.
struct Payload {
    std::vector<unsigned char> b;
    size_t put(const void* p, size_t n) {
        const size_t off = b.size();
        b.resize(off + align16(n), 0);
        if (n) memcpy(b.data() + off, p, n);
        return off;
    }
    size_t put_cplx(const std::vector<cd>& v, int dtype) {
        if (dtype == SV_C64) {
            std::vector<float> f(2 * v.size());
            for (size_t e = 0; e < v.size(); ++e) {
                f[2 * e] = (float)v[e].real();
                f[2 * e + 1] = (float)v[e].imag();
            }
            return put(f.data(), sizeof(float) * f.size());
        }
        std::vector<double> f(2 * v.size());
        for (size_t e = 0; e < v.size(); ++e) {
            f[2 * e] = v[e].real();
            f[2 * e + 1] = v[e].imag();
        }
        return put(f.data(), sizeof(double) * f.size());
    }
};

void assemble(std::vector<OpDev>& ops, const Payload& pay, PassDev* P, std::vector<unsigned char>* out) {
    const size_t ob = align16(sizeof(OpDev) * ops.size());
    for (OpDev& O : ops) {
        if (O.kind == OP_DENSE || O.kind == OP_DENSE_TC || O.kind == OP_GATES || O.kind == OP_REMAP)
            O.mat_off += (int)ob;
        if (O.kind == OP_GATES) O.rec_off += (int)ob;
        if (O.kind == OP_DIAG) O.diag_off += (int)ob;
    }
    out->assign(ob + pay.b.size(), 0);
    if (!ops.empty()) memcpy(out->data(), ops.data(), sizeof(OpDev) * ops.size());
    if (!pay.b.empty()) memcpy(out->data() + ob, pay.b.data(), pay.b.size());
    P->nops = (int)ops.size();
    P->ops_bytes = (int)ob;
    P->region_bytes = (int)out->size();
}

// Tensor-core block of the shared-memory pass kernel (3xTF32): a block marked
// for the tensor cores in a pass the register kernel does not take.
bool use_tc(const Plan& p, const HostOp& o) {
    return o.tc && p.dtype == SV_C64 && o.kind == OP_DENSE && (int)o.qubits.size() >= kMinTcK;
}
// Tensor-core block of a register pass (OP_DENSE_TC).
bool reg_tc(const Plan& p, const HostOp& o, int tb) {
    const int k = (int)o.qubits.size();
    return o.tc && o.kind == OP_DENSE && p.dtype == SV_C64 && !p.use_tma && (k == 4 || k == 5) && tb >= 7;
}

uint16_t f32_to_f16(float f);
float f16_to_f32(uint16_t h);
// B operand of an OP_DENSE_TC block: the real form of the 2^k x 2^k matrix
// (times kTcMatScale), B[2r + c'][2j + c] = Re / Im parts of U[r][j] as
// [[Re, -Im], [Im, Re]] per entry, FP16 hi = fp16(b) and lo = fp16(b - hi),
// K-major no-swizzle core matrices (8 rows x 8 values; 128 bytes along K,
// 16 N bytes between 8-row groups), hi then lo.
std::vector<uint16_t> tc16_operand(const std::vector<cd>& mat, int k) {
    const int D = 1 << k, N = 2 * D;
    std::vector<uint16_t> b((size_t)2 * N * N);
    for (int n = 0; n < N; ++n)
        for (int kk = 0; kk < N; ++kk) {
            const cd u = mat[(size_t)(n >> 1) * D + (kk >> 1)];
            const double re = u.real(), im = u.imag();
            const double val = ((n & 1) == 0 ? ((kk & 1) == 0 ? re : -im) : ((kk & 1) == 0 ? im : re)) * kTcMatScale;
            const uint16_t hi = f32_to_f16((float)val);
            const uint16_t lo = f32_to_f16((float)(val - (double)f16_to_f32(hi)));
            const size_t off = ((size_t)(n >> 3) * (N / 8) + (kk >> 3)) * 64 + (n & 7) * 8 + (kk & 7);
            b[off] = hi;
            b[(size_t)N * N + off] = lo;
        }
    return b;
}

// Region for the shared-memory pass kernel: dense blocks, gate sequences of
// at most smem_gates_max_k qubits (wider ones as their dense matrix) and
// diagonal runs in the DiagLayout form.
void smem_region(const Plan& p, const HostPass& hp, PassDev* P, const int* loc, float* tcf, size_t* ti,
                 std::vector<unsigned char>* out) {
    std::vector<OpDev> ops;
    Payload pay;
    for (const HostOp& o : hp.ops) {
        OpDev O;
        memset(&O, 0, sizeof(O));
        O.ngates = o.ngates;
        if (o.kind == OP_DENSE || o.kind == OP_GATES) {
            O.k = (int)o.qubits.size();
            for (int i = 0; i < O.k; ++i) O.lq[i] = loc[o.qubits[i]];
            const bool gates = o.kind == OP_GATES && O.k <= smem_gates_max_k(p.dtype);
            O.kind = gates ? OP_GATES : OP_DENSE;
            if (gates) {
                O.mat_off = (int)pay.put_cplx(o.gdata, p.dtype);
                O.ndata = (int)o.gdata.size();
                O.nrec = (int)o.recs.size();
                O.rec_off = (int)pay.put(o.recs.data(), sizeof(GateRec) * o.recs.size());
            } else {
                O.mat_off = (int)pay.put_cplx(o.kind == OP_DENSE ? o.mat : block_matrix(o.qubits, o.seq), p.dtype);
            }
            if (use_tc(p, o)) {
                // B = [Ur; Ui]: row n < D holds Re U[n][j], row D + n holds Im U[n][j]
                const int k = O.k, Dm = 1 << k, N = 2 * Dm, K = Dm;
                O.tc = 1;
                O.tc_off = (int)*ti;
                float* hi = tcf + *ti;
                float* lo = hi + N * K;
                for (int r = 0; r < N; ++r)
                    for (int j = 0; j < K; ++j) {
                        const cd u = o.mat[(size_t)(r % Dm) * Dm + j];
                        const float v = (float)(r < Dm ? u.real() : u.imag());
                        const float vh = tf32_round(v);
                        const int idx = tc_kmajor_index(r, j, K);
                        hi[idx] = vh;
                        lo[idx] = tf32_round(v - vh);
                    }
                if (!P->tc_k) P->tc_base = (int)*ti;
                *ti += (size_t)tc_floats(k);
                if (k > P->tc_k) P->tc_k = k;
                P->tc_res = (int)*ti - P->tc_base;  // all of the pass's B operands so far
            }
        } else {
            O.kind = OP_DIAG;
            std::vector<uint64_t> w(diag_doubles(P->m, P->nother));
            write_diag(o.diag, p.n, hp, *P, w.data());
            O.diag_off = (int)pay.put(w.data(), sizeof(uint64_t) * w.size());
        }
        ops.push_back(O);
    }
    if (P->tc_res > kTcResidentFloats) P->tc_res = 0;  // too large: staged per op and tile
    assemble(ops, pay, P, out);
}

// Region for the register-resident pass kernel, or false when the pass
// needs the shared-memory kernel (tensor-core blocks, dense blocks wider than
// kRegDenseMaxK, a thread count outside 32..512, or a region too large to
// stage).  Register layouts are chosen here: before a block whose qubits are
// not all in registers, a remap brings them in (for dense blocks, in block
// order at register bits 0..k-1) and fills the other register bits with the
// tile positions the following blocks use soonest.
bool reg_region(const Plan& p, const HostPass& hp, PassDev* P, const int* loc, std::vector<unsigned char>* out) {
    const int r = reg_bits(p.dtype), m = P->m, tb = m - r, nops = (int)hp.ops.size();
    if (tb < 5 || tb > 9) return false;
    std::vector<std::vector<int>> used(nops);
    for (int i = 0; i < nops; ++i) {
        const HostOp& o = hp.ops[i];
        if (o.kind == OP_DIAG) continue;
        if (o.tc && !reg_tc(p, o, tb) && (int)o.qubits.size() > kRegDenseMaxK) return false;
        if (o.kind == OP_DENSE && !reg_tc(p, o, tb) && (int)o.qubits.size() > kRegDenseMaxK) return false;
        if ((int)o.qubits.size() > r) return false;
        for (int q : o.qubits) used[i].push_back(loc[q]);
    }
    auto next_use = [&](int pos, int from) {
        for (int j = from; j < nops; ++j)
            if (std::find(used[j].begin(), used[j].end(), pos) != used[j].end()) return j;
        return nops + 1;
    };
    std::vector<OpDev> ops;
    Payload pay;
    std::vector<int> rpos, tpos;
    // Thread bits 0..4 are the lane bits, the others the warp bits.  A remap
    // whose incoming register positions all sit at lane bits can hand each
    // lane bit it frees to an outgoing register position: every warp's
    // amplitudes then stay within the warp, and the kernels order the remap
    // with a warp barrier instead of a block barrier.  Other remaps lay the
    // thread bits out afresh: lane bits for the positions used soonest (so
    // that later remaps stay within warps), subject to the lanes' shared-
    // memory offsets reaching as many bank groups as the candidates allow.
    const bool c64 = p.dtype == SV_C64;
    auto bank_vec = [&](int pos, bool wide) {
        int s = 1 << pos;
        s = c64 ? (s ^ (((s >> 4) & 7) << 1)) : (s ^ ((s >> 3) & 7));  // the tile swizzle
        return c64 ? (wide ? (s >> 1) & 7 : s & 15) : s & 7;
    };
    auto reduce = [](int* basis, int v) {  // GF(2) elimination: true when v is independent
        for (int b = 3; b >= 0; --b)
            if ((v >> b) & 1) {
                if (!basis[b]) {
                    basis[b] = v;
                    return true;
                }
                v ^= basis[b];
            }
        return false;
    };
    auto lane_rank = [&](const std::vector<int>& lanes, bool wide) {
        int basis[4] = {0, 0, 0, 0}, rank = 0;
        for (int q : lanes) rank += reduce(basis, bank_vec(q, wide));
        return rank;
    };
    // A layout whose lanes hold tile positions 0 and 1 (complex64 with
    // position 0 at register bit 0: position 1; complex128: position 0) moves
    // runs of at least 32 bytes per warp access, so the compiled kernels load
    // a pass's first layout and store its last straight between registers and
    // global memory.  The first and the last remap of a pass (edge) take the
    // row positions 0..L-1 into the lanes first.
    auto coalesced = [&](const std::vector<int>& rp, const std::vector<int>& tp) {
        const int nl = std::min(5, tb);
        auto lane = [&](int q) { return std::find(tp.begin(), tp.begin() + nl, q) != tp.begin() + nl; };
        if (!c64) return lane(0);
        return rp[0] == 0 ? lane(1) : lane(0) && lane(1);
    };
    auto fresh_threads = [&](int i, const std::vector<int>& regs, bool wide, bool edge) {
        std::vector<int> cand;
        for (int q = 0; q < m; ++q)
            if (std::find(regs.begin(), regs.end(), q) == regs.end()) cand.push_back(q);
        std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) {
            const int na = edge && a < P->L ? -1 : next_use(a, i + 1);
            const int nb = edge && b < P->L ? -1 : next_use(b, i + 1);
            return na < nb;
        });
        const int nl = std::min(5, tb);
        const int target = std::min(lane_rank(cand, wide), c64 ? (wide ? 3 : 4) : 3);
        int basis[4] = {0, 0, 0, 0}, rank = 0;
        std::vector<int> lanes, rest;
        for (int q : cand) {
            int trial[4] = {basis[0], basis[1], basis[2], basis[3]};
            const bool indep = reduce(trial, bank_vec(q, wide));
            const int left = nl - (int)lanes.size();
            if (left > 0 && (indep || left > target - rank)) {
                lanes.push_back(q);
                if (indep) std::copy(trial, trial + 4, basis), ++rank;
            } else {
                rest.push_back(q);
            }
        }
        std::sort(lanes.begin(), lanes.end());
        lanes.insert(lanes.end(), rest.begin(), rest.end());
        return lanes;
    };
    auto remap = [&](int i, const std::vector<int>& PQ) {
        std::vector<int> cand;
        for (int q = 0; q < m; ++q)
            if (std::find(PQ.begin(), PQ.end(), q) == PQ.end()) cand.push_back(q);
        // when the block's own qubits can come in from lane bits, the other
        // register slots are filled from registers and lanes only, so that a
        // filler at a warp bit does not turn the remap into a block-wide one
        const int nl0 = std::min(5, tb);
        auto at_warp = [&](int q) {
            const auto it = std::find(tpos.begin(), tpos.end(), q);
            return it != tpos.end() && it - tpos.begin() >= nl0;
        };
        bool pq_local = !rpos.empty();
        for (int q : PQ) pq_local = pq_local && !at_warp(q);
        std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) {
            if (pq_local && at_warp(a) != at_warp(b)) return !at_warp(a);
            const int na = next_use(a, i + 1), nb = next_use(b, i + 1);
            if (na != nb) return na < nb;
            const bool ia = std::find(rpos.begin(), rpos.end(), a) != rpos.end();
            const bool ib = std::find(rpos.begin(), rpos.end(), b) != rpos.end();
            return ia && !ib;
        });
        std::vector<int> slots = PQ;
        for (size_t c = 0; c < cand.size() && (int)slots.size() < r; ++c) slots.push_back(cand[c]);
        std::sort(slots.begin() + PQ.size(), slots.end());
        // before a gate sequence (any register order serves it), tile position
        // 0 goes to register bit 0: compiled complex64 passes then move
        // register pairs with 16-byte shared-memory accesses
        if (hp.ops[i].kind == OP_GATES) {
            const auto z = std::find(slots.begin(), slots.end(), 0);
            if (z != slots.end()) std::iter_swap(slots.begin(), z);
        }
        const bool wide = c64 && slots[0] == 0;
        // the last remap when every later block finds its qubits in registers
        bool last = true;
        for (int j = i + 1; last && j < nops; ++j)
            for (int q : used[j])
                if (std::find(slots.begin(), slots.end(), q) == slots.end()) last = false;
        std::vector<int> fresh = fresh_threads(i, slots, wide, rpos.empty() || last);
        bool local = false;
        if (!rpos.empty()) {
            std::vector<int> in, out, tp = tpos;
            for (int q : slots)
                if (std::find(rpos.begin(), rpos.end(), q) == rpos.end()) in.push_back(q);
            for (int q : rpos)
                if (std::find(slots.begin(), slots.end(), q) == slots.end()) out.push_back(q);
            local = true;
            for (size_t j = 0; local && j < in.size(); ++j) {
                const int t = (int)(std::find(tpos.begin(), tpos.end(), in[j]) - tpos.begin());
                if (t >= 5) local = false;
                else tp[t] = out[j];
            }
            const int nl = std::min(5, tb);
            const std::vector<int> lanes_l(tp.begin(), tp.begin() + nl), lanes_f(fresh.begin(), fresh.begin() + nl);
            if (local && lane_rank(lanes_l, wide) >= lane_rank(lanes_f, wide) &&
                (!last || coalesced(slots, tp) || !coalesced(slots, fresh)))
                fresh = tp;
            else
                local = false;
        }
        // Shared-memory accesses are served a quarter warp (16-byte: lanes
        // 0..7) or a half warp (8-byte: lanes 0..15) at a time: the first
        // three / four lane bits take positions whose bank vectors are
        // independent where the lanes hold such a set (lane bits may be
        // permuted freely: the remap stays within warps either way)
        {
            const int nl = std::min(5, tb), q = c64 && !wide ? 4 : 3;
            std::vector<int> lanes(fresh.begin(), fresh.begin() + nl), first, later;
            std::sort(lanes.begin(), lanes.end());
            int basis[4] = {0, 0, 0, 0};
            for (int pos : lanes) {
                if ((int)first.size() < q && reduce(basis, bank_vec(pos, wide))) first.push_back(pos);
                else later.push_back(pos);
            }
            first.insert(first.end(), later.begin(), later.end());
            std::copy(first.begin(), first.end(), fresh.begin());
        }
        rpos = slots;
        tpos = fresh;
        OpDev O;
        memset(&O, 0, sizeof(O));
        O.kind = OP_REMAP;
        O.k = r;
        O.nrec = local ? 1 : 0;
        for (int b = 0; b < r; ++b) O.lq[b] = rpos[b];
        int tp[16];
        for (int t = 0; t < 16; ++t) tp[t] = t < (int)tpos.size() ? tpos[t] : -1;
        O.mat_off = (int)pay.put(tp, sizeof(tp));
        ops.push_back(O);
    };
    auto slot = [&](int pos) { return (int)(std::find(rpos.begin(), rpos.end(), pos) - rpos.begin()); };
    int nd = 0;
    for (int i = 0; i < nops; ++i) {
        const HostOp& o = hp.ops[i];
        if (o.kind == OP_DIAG) {
            if (rpos.empty()) {
                std::vector<int> PQ;
                for (int j = i + 1; j < nops; ++j)
                    if (!used[j].empty()) {
                        PQ = used[j];
                        break;
                    }
                remap(i, PQ);
            }
            OpDev O;
            memset(&O, 0, sizeof(O));
            O.kind = OP_DIAG;
            O.ngates = o.ngates;
            O.ord = nd++;
            const RDiagLayout Lr(m, P->nother);
            std::vector<uint64_t> w(Lr.total, 0);
            std::vector<uint64_t> full(diag_doubles(m, P->nother));
            write_diag(o.diag, p.n, hp, *P, full.data());  // c, a_t, a_o, Bo, Boo come first in both layouts
            for (int e = 0; e < Lr.tqlo; ++e) w[e] = full[e];
            auto B = [&](int pa, int pb) {
                if (pa == pb) return (uint64_t)0;
                const int qa = P->tq[pa], qb = P->tq[pb];
                return fx_turns(o.diag.b[(size_t)std::min(qa, qb) * p.n + std::max(qa, qb)]);
            };
            const int nlo = std::min(4, tb);
            for (int e = 0; e < 16; ++e) {
                uint64_t v = 0;
                for (int t = 0; t < nlo; ++t)
                    for (int t2 = 0; t2 < t; ++t2)
                        if (((e >> t) & 1) && ((e >> t2) & 1)) v += B(tpos[t], tpos[t2]);
                w[Lr.tqlo + e] = v;
            }
            for (int e = 0; e < 32; ++e) {
                uint64_t v = 0;
                for (int t = 4; t < tb; ++t)
                    for (int t2 = 4; t2 < t; ++t2)
                        if (((e >> (t - 4)) & 1) && ((e >> (t2 - 4)) & 1)) v += B(tpos[t], tpos[t2]);
                w[Lr.tqhi + e] = v;
            }
            for (int t = 4; t < tb; ++t)
                for (int e = 0; e < 16; ++e) {
                    uint64_t v = 0;
                    for (int t2 = 0; t2 < nlo; ++t2)
                        if ((e >> t2) & 1) v += B(tpos[t], tpos[t2]);
                    w[Lr.tr + (t - 4) * 16 + e] = v;
                }
            for (int b = 0; b < r; ++b) {
                for (int e = 0; e < 16; ++e) {
                    uint64_t v = 0;
                    for (int t = 0; t < nlo; ++t)
                        if ((e >> t) & 1) v += B(rpos[b], tpos[t]);
                    w[Lr.talo + b * 16 + e] = v;
                }
                for (int e = 0; e < 32; ++e) {
                    uint64_t v = 0;
                    for (int t = 4; t < tb; ++t)
                        if ((e >> (t - 4)) & 1) v += B(rpos[b], tpos[t]);
                    w[Lr.tahi + b * 32 + e] = v;
                }
                for (int b2 = 0; b2 < r; ++b2) w[Lr.beta + b * 5 + b2] = B(rpos[b], rpos[b2]);
            }
            O.diag_off = (int)pay.put(w.data(), sizeof(uint64_t) * w.size());
            ops.push_back(O);
            continue;
        }
        const std::vector<int>& PQ = used[i];
        bool ok = !rpos.empty();
        for (size_t j = 0; ok && j < PQ.size(); ++j)
            ok = o.kind == OP_DENSE ? rpos[j] == PQ[j] : slot(PQ[j]) < r;
        if (!ok) remap(i, PQ);
        OpDev O;
        memset(&O, 0, sizeof(O));
        O.kind = o.kind;
        O.ngates = o.ngates;
        O.k = (int)PQ.size();
        for (int j = 0; j < O.k; ++j) O.lq[j] = slot(PQ[j]);
        if (o.kind == OP_DENSE && reg_tc(p, o, tb)) {
            // the registers enter at the true amplitudes times kTcInScale and
            // leave at kTcInScale * kTcMatScale times them (the pass's
            // write-back scale undoes it)
            O.kind = OP_DENSE_TC;
            const std::vector<uint16_t> b = tc16_operand(o.mat, O.k);
            O.mat_off = (int)pay.put(b.data(), sizeof(uint16_t) * b.size());
            O.tc_scale = (float)((double)kTcInScale * P->scale);
            P->scale = 1.0 / ((double)kTcInScale * (double)kTcMatScale);
            if (O.k > P->tc_k) P->tc_k = O.k;
        } else if (o.kind == OP_DENSE) {
            O.mat_off = (int)pay.put_cplx(o.mat, p.dtype);
        } else {
            std::vector<GateRec> recs;
            std::vector<cd> data;
            for (const GateRec& g : o.recs) {
                GateRec t = g;
                if (g.kind == GR_DT) {
                    // the table over all 2^r register values; b = mask of the
                    // entries that are not exactly 1 (the others are skipped),
                    // a = the register bits the entries depend on
                    t.off = (int)data.size();
                    t.b = 0;
                    t.a = 0;
                    for (int j = 0; j < O.k; ++j)
                        if ((g.a >> j) & 1) t.a |= 1 << O.lq[j];
                    for (int v = 0; v < (1 << r); ++v) {
                        int idx = 0;
                        for (int j = 0; j < O.k; ++j) idx |= ((v >> O.lq[j]) & 1) << j;
                        const cd e = o.gdata[(size_t)g.off + idx];
                        data.push_back(e);
                        if (e != cd(1.0, 0.0)) t.b |= 1 << v;
                    }
                } else {
                    t.a = O.lq[g.a];
                    if (g.kind == GR_CX || g.kind == GR_SWAP) t.b = O.lq[g.b];
                    const cd* gm = g.kind == GR_U || g.kind == GR_UR ? &o.gdata[(size_t)g.off] : nullptr;
                    const double hs = 1.0 / std::sqrt(2.0);
                    // (factors deferred only while the growth they leave in the
                    // registers stays below 2^40)
                    if (g.kind == GR_UR && gm[0] == cd(hs, 0.0) && gm[1] == cd(hs, 0.0) && gm[2] == cd(hs, 0.0) &&
                        gm[3] == cd(-hs, 0.0) && std::fabs(P->scale) > 0x1p-40) {
                        t.kind = GR_H;  // butterfly; the factor goes to the pass's write-back scale
                        t.off = 0;
                        P->scale *= hs;
                    } else if (g.kind == GR_UR && gm[0] == gm[3] && gm[1] == -gm[2] && std::fabs(P->scale) > 0x1p-40) {
                        // rotation [[c, -s], [s, c]]: the larger of c, s goes to the
                        // write-back scale (each factor is at least 1/sqrt(2) in
                        // magnitude, so the deferred growth stays below 2^40)
                        const double c = gm[0].real(), sn = gm[2].real();
                        const bool cform = std::fabs(c) >= std::fabs(sn);
                        t.kind = GR_URS;
                        t.b = cform ? 0 : 1;
                        t.off = (int)data.size();
                        data.push_back(cd(cform ? sn / c : c / sn, 0.0));
                        P->scale *= cform ? c : sn;
                    } else if (gm) {
                        t.off = (int)data.size();
                        for (int e = 0; e < 4; ++e) data.push_back(gm[e]);
                    }
                }
                recs.push_back(t);
            }
            // a butterfly followed by a phase table: one record
            std::vector<GateRec> fused;
            for (size_t r = 0; r < recs.size(); ++r) {
                if (recs[r].kind == GR_H && r + 1 < recs.size() && recs[r + 1].kind == GR_DT) {
                    fused.push_back(GateRec{GR_HD, recs[r].a, recs[r + 1].b, recs[r + 1].off});
                    ++r;
                } else {
                    fused.push_back(recs[r]);
                }
            }
            recs.swap(fused);
            O.mat_off = (int)pay.put_cplx(data, p.dtype);
            O.ndata = (int)data.size();
            O.nrec = (int)recs.size();
            O.rec_off = (int)pay.put(recs.data(), sizeof(GateRec) * recs.size());
        }
        ops.push_back(O);
    }
    if (rpos.empty()) remap(0, {});
    assemble(ops, pay, P, out);
    P->rmode = p.use_tma ? 2 : 1;
    P->ndiag = nd;
    // passes with tensor-core blocks stage their matrices (16 KiB per 5-qubit
    // block) in a larger region
    return P->region_bytes <= (P->tc_k ? kStageCapTc : kStageCap);
}

}  // namespace

bool register_pass_eligible(const Plan& p, const HostPass& hp) {
    if (p.no_register_passes) return false;
    const int r = reg_bits(p.dtype), tb = (int)hp.tile.size() - r;
    if (tb < 5 || tb > 9) return false;
    for (const HostOp& o : hp.ops) {
        if (o.kind == OP_DIAG) continue;
        if (o.kind == OP_DENSE && !reg_tc(p, o, tb) && (int)o.qubits.size() > kRegDenseMaxK) return false;
        if ((int)o.qubits.size() > r) return false;
    }
    return true;
}

void serialise_plans(const std::vector<const Plan*>& plans, PlanBlob* blob) {
    const int dtype = plans.empty() ? SV_C64 : plans[0]->dtype;
    size_t ntc = 0, npass = 0;
    for (const Plan* pp : plans) {
        npass += pp->passes.size();
        for (const HostPass& hp : pp->passes)
            for (const HostOp& o : hp.ops)
                if (use_tc(*pp, o)) ntc += (size_t)tc_floats((int)o.qubits.size());
    }
    (void)dtype;
    blob->npasses = (int)npass;
    blob->pass_off = 0;
    blob->tc_off = align16(sizeof(PassDev) * npass);
    const size_t roff0 = align16(blob->tc_off + sizeof(float) * ntc);
    std::vector<PassDev> pds(npass);
    std::vector<std::vector<unsigned char>> regions(npass);
    std::vector<float> tcf(ntc);
    size_t ti = 0, gpi = 0;
    for (const Plan* pp : plans) {
        const Plan& p = *pp;
        const int n = p.n;
        for (size_t pi = 0; pi < p.passes.size(); ++pi, ++gpi) {
            const HostPass& hp = p.passes[pi];
            PassDev& P = pds[gpi];
            memset(&P, 0, sizeof(P));
            P.scale = 1.0;
            P.basis = -1;
            P.n = n;
            P.m = (int)hp.tile.size();
            P.L = hp.L;
            int loc[64];
            for (int i = 0; i < 64; ++i) loc[i] = -1;
            for (int i = 0; i < P.m; ++i) {
                P.tq[i] = hp.tile[i];
                loc[hp.tile[i]] = i;
            }
            P.nother = 0;
            for (int q = 0; q < n; ++q)
                if (loc[q] < 0) P.oq[P.nother++] = q;
            if (!hp.mux.empty()) {
                mux_region(p, hp, &P, &regions[gpi]);
                continue;
            }
            if (!p.no_register_passes) {
                PassDev R = P;
                if (reg_region(p, hp, &R, loc, &regions[gpi])) {
                    P = R;
                    continue;
                }
            }
            smem_region(p, hp, &P, loc, tcf.data(), &ti, &regions[gpi]);
        }
    }
    size_t roff = roff0;
    blob->max_region = 0;
    for (size_t i = 0; i < npass; ++i) {
        pds[i].region_off = (int)roff;
        roff += regions[i].size();
        if (pds[i].rmode != kRmodeMux) blob->max_region = std::max(blob->max_region, pds[i].region_bytes);
    }
    blob->bytes.assign(roff, 0);
    unsigned char* base = blob->bytes.data();
    if (npass) memcpy(base + blob->pass_off, pds.data(), sizeof(PassDev) * npass);
    if (ntc) memcpy(base + blob->tc_off, tcf.data(), sizeof(float) * ntc);
    for (size_t i = 0; i < npass; ++i)
        if (!regions[i].empty()) memcpy(base + pds[i].region_off, regions[i].data(), regions[i].size());
}

void serialise_plan(const Plan& p, PlanBlob* blob) { serialise_plans({&p}, blob); }

}  // namespace sv
