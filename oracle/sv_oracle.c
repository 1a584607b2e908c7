/*
 * FP64 CPU oracle for the state-vector simulator.  TEST INFRASTRUCTURE ONLY:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference arm may load this library.  It shares no code, header, table or
 * constant generator with the CUDA library; it reads the same 48-byte gate
 * records (workloads/ defines that input format) and nothing else.
 *
 * What it computes, one plain definition per function:
 *   - state vector: 2^n complex128 amplitudes, sum |a_i|^2 = 1
 *     (App. A, Eq. "hilbert");
 *   - gate application one gate at a time: a k-qubit gate with matrix U acts
 *     on every group of 2^k amplitudes whose indices differ only in the
 *     gate's qubit bits, i.e. U_k = I (x) .. (x) U (x) .. (x) I (App. A,
 *     Eq. "tp"), CX flips the target where the control is 1 (App. A, Eq. "cx"
 *     and the 3-qubit worked example), CR1 = diag(1,1,1,e^{i lambda})
 *     (App. D.2, Eq. "cr1");
 *   - probabilities p_x = |a_x|^2, the sequential inclusive CDF, shot
 *     sampling outcome = min{x : C_x > u * C_{N-1}} (Sec. 3, QCrank shots);
 *   - <Z_i> = sum_x p_x (1 - 2 x_i);
 *   - Philox4x64-10 (Salmon et al., SC'11) for seeded uniforms.
 *
 * Conventions (readings of the paper, where it is silent or garbled):
 *   - qubit q is bit q of the amplitude index (LSB = q0);
 *   - a k-qubit gate on qubits (q[0], .., q[k-1]) uses the local index
 *     j = sum_i bit(q[i]) * 2^(k-1-i): q[0] is the most significant, so the
 *     CX matrix is the textbook one with the control first;
 *   - gate matrices: H, X, Y, Z; RX(t) = [[c,-is],[-is,c]];
 *     RY(t) = [[c,-s],[s,c]] (c = cos t/2, s = sin t/2);
 *     RZ(f) = diag(e^{-if/2}, e^{if/2}); P(l) = diag(1, e^{il});
 *     U3(t,f,l) = [[c, -e^{il} s], [e^{if} s, e^{i(f+l)} c]];
 *     CX; CZ = diag(1,1,1,-1); CP(l) = CR1(l); SWAP.  Global phases kept.
 *   - MEASURE records are terminal and leave the state untouched.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    uint32_t type;
    uint32_t nq;
    uint32_t q[3];
    double p[3];
} or_gate; /* 48 bytes: 4 + 4 + 12 + 4 (pad) + 24 */

enum { G_H, G_X, G_Y, G_Z, G_RX, G_RY, G_RZ, G_P, G_U3, G_CX, G_CZ, G_CP,
       G_SWAP, G_MEASURE, G_COUNT };

static int g_threads = 1;

void or_set_threads(int t) { g_threads = t > 0 ? t : 1; }

int or_get_threads(void) { return g_threads; }

int or_gate_struct_size(void) { return (int)sizeof(or_gate); }

/* Number of qubits a gate type acts on; -1 for an unknown type. */
int or_gate_arity(uint32_t type) {
    switch (type) {
    case G_H: case G_X: case G_Y: case G_Z: case G_RX: case G_RY: case G_RZ:
    case G_P: case G_U3: case G_MEASURE:
        return 1;
    case G_CX: case G_CZ: case G_CP: case G_SWAP:
        return 2;
    default:
        return -1;
    }
}

/* Dense gate matrix, row-major, 2^k x 2^k complex128 written as interleaved
 * (re, im) doubles into out (room for 16 complex).  Returns k, 0 for MEASURE
 * (no matrix) or -1 for an unknown type. */
static int gate_matrix(uint32_t type, const double *p, cplx *m) {
    const double r2 = 1.0 / sqrt(2.0);
    double c, s;
    switch (type) {
    case G_H:
        m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2;
        return 1;
    case G_X:
        m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0;
        return 1;
    case G_Y:
        m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0;
        return 1;
    case G_Z:
        m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1;
        return 1;
    case G_RX:
        c = cos(0.5 * p[0]); s = sin(0.5 * p[0]);
        m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c;
        return 1;
    case G_RY:
        c = cos(0.5 * p[0]); s = sin(0.5 * p[0]);
        m[0] = c; m[1] = -s; m[2] = s; m[3] = c;
        return 1;
    case G_RZ:
        m[0] = cexp(-0.5 * I * p[0]); m[1] = 0; m[2] = 0;
        m[3] = cexp(0.5 * I * p[0]);
        return 1;
    case G_P:
        m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * p[0]);
        return 1;
    case G_U3:
        c = cos(0.5 * p[0]); s = sin(0.5 * p[0]);
        m[0] = c;
        m[1] = -cexp(I * p[2]) * s;
        m[2] = cexp(I * p[1]) * s;
        m[3] = cexp(I * (p[1] + p[2])) * c;
        return 1;
    case G_CX: case G_CZ: case G_CP: case G_SWAP:
        for (int i = 0; i < 16; ++i) m[i] = 0;
        if (type == G_CX) {
            m[0 * 4 + 0] = 1; m[1 * 4 + 1] = 1; m[2 * 4 + 3] = 1; m[3 * 4 + 2] = 1;
        } else if (type == G_SWAP) {
            m[0 * 4 + 0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[3 * 4 + 3] = 1;
        } else {
            m[0] = 1; m[5] = 1; m[10] = 1;
            m[15] = (type == G_CZ) ? -1.0 : cexp(I * p[0]);
        }
        return 2;
    case G_MEASURE:
        return 0;
    default:
        return -1;
    }
}

int or_gate_matrix(uint32_t type, const double *p, double *out) {
    cplx m[16];
    int k = gate_matrix(type, p, m);
    if (k > 0) {
        int d = 1 << k;
        for (int i = 0; i < d * d; ++i) {
            out[2 * i] = creal(m[i]);
            out[2 * i + 1] = cimag(m[i]);
        }
    }
    return k;
}

/* Insert a zero bit at position pos into v. */
static inline uint64_t insert_zero(uint64_t v, int pos) {
    uint64_t lo = v & ((1ull << pos) - 1ull);
    return ((v >> pos) << (pos + 1)) | lo;
}

/* Apply a dense k-qubit matrix (k <= 3) on qubits q[0..k-1] to every group of
 * 2^k amplitudes that differ only in those bits (App. A, Eq. "tp"). */
static void apply_dense(int n, cplx *psi, int k, const uint32_t *q, const cplx *m) {
    const int d = 1 << k;
    uint32_t sorted[3];
    for (int i = 0; i < k; ++i) sorted[i] = q[i];
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j)
            if (sorted[j] < sorted[i]) { uint32_t t = sorted[i]; sorted[i] = sorted[j]; sorted[j] = t; }
    uint64_t off[8];
    for (int j = 0; j < d; ++j) {
        uint64_t o = 0;
        for (int i = 0; i < k; ++i)
            if ((j >> (k - 1 - i)) & 1) o |= 1ull << q[i];
        off[j] = o;
    }
    const int64_t groups = (int64_t)1 << (n - k);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t r = 0; r < groups; ++r) {
        uint64_t base = (uint64_t)r;
        for (int i = 0; i < k; ++i) base = insert_zero(base, (int)sorted[i]);
        cplx v[8], w[8];
        for (int j = 0; j < d; ++j) v[j] = psi[base | off[j]];
        for (int a = 0; a < d; ++a) {
            cplx acc = 0;
            for (int b = 0; b < d; ++b) acc += m[a * d + b] * v[b];
            w[a] = acc;
        }
        for (int j = 0; j < d; ++j) psi[base | off[j]] = w[j];
    }
}

/* Validate one gate record against n qubits; 0 if fine, -1 otherwise. */
static int check_gate(int n, const or_gate *g) {
    int k = or_gate_arity(g->type);
    if (k < 0 || (int)g->nq != k) return -1;
    for (int i = 0; i < k; ++i) {
        if ((int)g->q[i] >= n) return -1;
        for (int j = 0; j < i; ++j)
            if (g->q[i] == g->q[j]) return -1;
    }
    return 0;
}

/* Apply the circuit one gate at a time, in list order.  psi holds 2^n
 * complex128 as interleaved (re, im).  Returns 0, or -(1 + index) of the
 * first invalid gate record (the state is untouched in that case). */
int64_t or_apply_circuit(int n, double *psi_ri, const or_gate *g, int64_t count) {
    for (int64_t i = 0; i < count; ++i)
        if (check_gate(n, &g[i]) != 0) return -(1 + i);
    cplx *psi = (cplx *)psi_ri;
    for (int64_t i = 0; i < count; ++i) {
        cplx m[16];
        int k = gate_matrix(g[i].type, g[i].p, m);
        if (k == 0) continue; /* measure: terminal, no state change */
        apply_dense(n, psi, k, g[i].q, m);
    }
    return 0;
}

/* |x> (App. A: state initialisation). */
void or_init_basis(int n, double *psi_ri, uint64_t x) {
    const int64_t N = (int64_t)1 << n;
    memset(psi_ri, 0, sizeof(double) * 2 * (size_t)N);
    psi_ri[2 * x] = 1.0;
}

/* p_x = |a_x|^2. */
void or_probs(int n, const double *psi_ri, double *p) {
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t x = 0; x < N; ++x)
        p[x] = psi_ri[2 * x] * psi_ri[2 * x] + psi_ri[2 * x + 1] * psi_ri[2 * x + 1];
}

/* Sequential FP64 inclusive CDF C_x = p_0 + ... + p_x. */
void or_cdf(int n, const double *p, double *c) {
    const int64_t N = (int64_t)1 << n;
    double acc = 0.0;
    for (int64_t x = 0; x < N; ++x) {
        acc += p[x];
        c[x] = acc;
    }
}

/* outcome = min{x : C_x > u * C_{N-1}} for each uniform u in [0,1).  C is
 * non-decreasing, so a binary search returns the same x as a linear scan. */
void or_sample_cdf(int n, const double *c, const double *u, int64_t shots, uint64_t *out) {
    const int64_t N = (int64_t)1 << n;
    const double S = c[N - 1];
    for (int64_t s = 0; s < shots; ++s) {
        const double t = u[s] * S;
        int64_t lo = 0, hi = N - 1; /* C[hi] = S > t always holds as u < 1 */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (c[mid] > t) hi = mid; else lo = mid + 1;
        }
        out[s] = (uint64_t)lo;
    }
}

/* <Z_i> = sum_x p_x (1 - 2 x_i), summed sequentially in x. */
void or_expect_z(int n, const double *psi_ri, double *ez) {
    const int64_t N = (int64_t)1 << n;
    for (int i = 0; i < n; ++i) ez[i] = 0.0;
    for (int64_t x = 0; x < N; ++x) {
        double p = psi_ri[2 * x] * psi_ri[2 * x] + psi_ri[2 * x + 1] * psi_ri[2 * x + 1];
        for (int i = 0; i < n; ++i) ez[i] += ((x >> i) & 1) ? -p : p;
    }
}

/* ---------------- Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) -------
 * Round: (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1,
 * lo(M0*c0)); the key is bumped by the Weyl constants between rounds. */
static inline void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 pr = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(pr >> 64);
    *lo = (uint64_t)pr;
}

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Shot s draws word (s mod 4) of block Philox(ctr = (s div 4, 0, 0, 0),
 * key = (seed, 0)) and maps it to u = (w >> 11) * 2^-53 in [0,1). */
void or_uniforms(uint64_t seed, int64_t shots, double *u) {
    const uint64_t key[2] = {seed, 0};
    uint64_t blk[4];
    for (int64_t s = 0; s < shots; ++s) {
        if ((s & 3) == 0 || s == 0) {
            uint64_t ctr[4] = {(uint64_t)(s >> 2), 0, 0, 0};
            or_philox4x64_10(ctr, key, blk);
        }
        u[s] = (double)(blk[s & 3] >> 11) * 0x1.0p-53;
    }
}
