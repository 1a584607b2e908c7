// Register-resident tile pass: device code shared by the library's
// interpreting kernel (k_rpass, which walks a pass's op list at run time) and
// the pass kernels compiled at run time for one pass structure (the same
// code with every op, position, mask and layout fixed at compile time).
//
// A pass covers every tile of 2^m amplitudes whose index varies only in the
// tile qubits; one HBM read and one write of the state per pass (App. A,
// App. D.2 "gate fusion = 5").  Nothing here may need a host header: the
// run-time compiler sees only this file and sv_dev.h.
#pragma once

#ifdef __CUDACC_RTC__
typedef unsigned long long uint64_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef int int32_t;
#else
#include <stdint.h>
#endif

#include "sv_dev.h"
#include "sv_tc.cuh"

// Loops whose trip counts are compile-time constants in the run-time
// compiled kernels (layout sizes) are unrolled there.
#ifdef SV_JIT
#define SV_UNROLL _Pragma("unroll")
#else
#define SV_UNROLL
#endif

namespace sv {

template <typename R> struct CT;
template <> struct CT<float> { using V = float2; };
template <> struct CT<double> { using V = double2; };

template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename V> __device__ __forceinline__ V cfma(V a, V b, V c) {  // a*b + c
    V r;
    r.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
    r.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
    return r;
}
template <typename V> __device__ __forceinline__ V czero() {
    V r;
    r.x = 0;
    r.y = 0;
    return r;
}


// ---------------------------------------------------------------------------
// Asynchronous 16-byte copies and the shared-memory swizzle.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Shared-memory position of tile amplitude i: the 16-byte chunks of each
// 128-byte row are XOR-permuted by the row number (mod 8), so that a warp
// reading one amplitude from each of 8 consecutive rows (slices of a block on
// the low tile qubits) hits 8 different bank groups.  The map is linear over
// XOR: swz(a ^ b) = swz(a) ^ swz(b), so slice offsets can be swizzled once.
template <typename V> __device__ __forceinline__ int swz(int i) {
    if constexpr (sizeof(V) == 8) return i ^ (((i >> 4) & 7) << 1);  // 2 amplitudes per chunk
    else return i ^ ((i >> 3) & 7);                                   // 1 amplitude per chunk
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}


// ---------------------------------------------------------------------------
// Gate-sequence block: one thread holds a whole 2^K-amplitude slice in
// registers and applies the block's gates one after the other, each with
// code unrolled for its (compile-time) position inside the block:
//   GR_U   2x2 complex matrix on position a        8 FMA per amplitude
//   GR_UR  2x2 real matrix on position a           4
//   GR_URS rotation with its factor deferred       2
//   GR_DT  2^K-entry diagonal (phase) table        one complex product
//   GR_CX  controlled-NOT (control a, target b)    register moves
//   GR_SWAP                                        register moves
// ---------------------------------------------------------------------------
template <typename V, int K, int P>
__device__ __forceinline__ void reg_u(V* v, V u00, V u01, V u10, V u11) {
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
        if (!((j >> P) & 1)) {
            const V a = v[j], b = v[j | (1 << P)];
            v[j] = cfma(u00, a, cmul(u01, b));
            v[j | (1 << P)] = cfma(u10, a, cmul(u11, b));
        }
}
template <typename V, int K, int P, typename R>
__device__ __forceinline__ void reg_ur(V* v, R u00, R u01, R u10, R u11) {
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
        if (!((j >> P) & 1)) {
            const V a = v[j], b = v[j | (1 << P)];
            V x, y;
            x.x = fma(u00, a.x, u01 * b.x);
            x.y = fma(u00, a.y, u01 * b.y);
            y.x = fma(u10, a.x, u11 * b.x);
            y.y = fma(u10, a.y, u11 * b.y);
            v[j] = x;
            v[j | (1 << P)] = y;
        }
}
// Rotation without its factor: FORM 0 [[1, -t], [t, 1]], FORM 1 [[t, -1], [1, t]].
template <typename V, int K, int P, int FORM, typename R>
__device__ __forceinline__ void reg_urs(V* v, R t) {
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
        if (!((j >> P) & 1)) {
            const V a = v[j], b = v[j | (1 << P)];
            V x, y;
            if (FORM == 0) {
                x.x = fma(-t, b.x, a.x);
                x.y = fma(-t, b.y, a.y);
                y.x = fma(t, a.x, b.x);
                y.y = fma(t, a.y, b.y);
            } else {
                x.x = fma(t, a.x, -b.x);
                x.y = fma(t, a.y, -b.y);
                y.x = fma(t, b.x, a.x);
                y.y = fma(t, b.y, a.y);
            }
            v[j] = x;
            v[j | (1 << P)] = y;
        }
}
template <typename V, int K, int P>
__device__ __forceinline__ void reg_h(V* v) {  // unscaled butterfly (a + b, a - b)
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
        if (!((j >> P) & 1)) {
            const V a = v[j], b = v[j | (1 << P)];
            V x, y;
            x.x = a.x + b.x;
            x.y = a.y + b.y;
            y.x = a.x - b.x;
            y.y = a.y - b.y;
            v[j] = x;
            v[j | (1 << P)] = y;
        }
}
template <typename V, int K, int C, int T>
__device__ __forceinline__ void reg_cx(V* v) {
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
        if (((j >> C) & 1) && !((j >> T) & 1)) {
            const V a = v[j];
            v[j] = v[j | (1 << T)];
            v[j | (1 << T)] = a;
        }
}
template <typename V, int K, int A, int B>
__device__ __forceinline__ void reg_swap(V* v) {
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
        if (((j >> A) & 1) && !((j >> B) & 1)) {
            const V a = v[j];
            v[j] = v[j ^ (1 << A) ^ (1 << B)];
            v[j ^ (1 << A) ^ (1 << B)] = a;
        }
}

// Phase table on the registers whose bit is set in MASK (a compile-time
// GR_DT / the table half of GR_HD).
template <typename V, int K, unsigned MASK>
__device__ __forceinline__ void reg_dt(V* v, const V* __restrict__ t) {
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
        if ((MASK >> j) & 1u) v[j] = cmul(t[j], v[j]);
}

// The same when the table depends only on the register bits in DEP (entry j
// equals entry j & DEP): each distinct entry is read once.
template <typename V, int K, unsigned MASK, unsigned DEP>
__device__ __forceinline__ void reg_dt_dep(V* v, const V* __restrict__ t) {
    V e[1 << K];
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
        if ((j & ~DEP) == 0 && ((MASK >> j) & 1u)) e[j] = t[j];
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
        if ((MASK >> j) & 1u) v[j] = cmul(e[j & DEP], v[j]);
}

template <typename V, int K>
__device__ __forceinline__ void reg_u_any(V* v, int p, V u00, V u01, V u10, V u11) {
    switch (p) {
    case 0: reg_u<V, K, 0>(v, u00, u01, u10, u11); break;
    case 1: if constexpr (K > 1) reg_u<V, K, 1>(v, u00, u01, u10, u11); break;
    case 2: if constexpr (K > 2) reg_u<V, K, 2>(v, u00, u01, u10, u11); break;
    case 3: if constexpr (K > 3) reg_u<V, K, 3>(v, u00, u01, u10, u11); break;
    default: if constexpr (K > 4) reg_u<V, K, 4>(v, u00, u01, u10, u11); break;
    }
}
template <typename V, int K, typename R>
__device__ __forceinline__ void reg_ur_any(V* v, int p, R u00, R u01, R u10, R u11) {
    switch (p) {
    case 0: reg_ur<V, K, 0>(v, u00, u01, u10, u11); break;
    case 1: if constexpr (K > 1) reg_ur<V, K, 1>(v, u00, u01, u10, u11); break;
    case 2: if constexpr (K > 2) reg_ur<V, K, 2>(v, u00, u01, u10, u11); break;
    case 3: if constexpr (K > 3) reg_ur<V, K, 3>(v, u00, u01, u10, u11); break;
    default: if constexpr (K > 4) reg_ur<V, K, 4>(v, u00, u01, u10, u11); break;
    }
}
template <typename V, int K, int FORM, typename R>
__device__ __forceinline__ void reg_urs_p(V* v, int p, R t) {
    switch (p) {
    case 0: reg_urs<V, K, 0, FORM, R>(v, t); break;
    case 1: if constexpr (K > 1) reg_urs<V, K, 1, FORM, R>(v, t); break;
    case 2: if constexpr (K > 2) reg_urs<V, K, 2, FORM, R>(v, t); break;
    case 3: if constexpr (K > 3) reg_urs<V, K, 3, FORM, R>(v, t); break;
    default: if constexpr (K > 4) reg_urs<V, K, 4, FORM, R>(v, t); break;
    }
}
template <typename V, int K, typename R>
__device__ __forceinline__ void reg_urs_any(V* v, int p, int form, R t) {
    if (form == 0) reg_urs_p<V, K, 0, R>(v, p, t);
    else reg_urs_p<V, K, 1, R>(v, p, t);
}
template <typename V, int K>
__device__ __forceinline__ void reg_h_any(V* v, int p) {
    switch (p) {
    case 0: reg_h<V, K, 0>(v); break;
    case 1: if constexpr (K > 1) reg_h<V, K, 1>(v); break;
    case 2: if constexpr (K > 2) reg_h<V, K, 2>(v); break;
    case 3: if constexpr (K > 3) reg_h<V, K, 3>(v); break;
    default: if constexpr (K > 4) reg_h<V, K, 4>(v); break;
    }
}
// (a, b) -> compile-time pair; a != b, both < K
template <typename V, int K, int A>
__device__ __forceinline__ void reg_cx_b(V* v, int b) {
    switch (b) {
    case 0: if constexpr (A != 0) reg_cx<V, K, A, 0>(v); break;
    case 1: if constexpr (A != 1 && K > 1) reg_cx<V, K, A, 1>(v); break;
    case 2: if constexpr (A != 2 && K > 2) reg_cx<V, K, A, 2>(v); break;
    case 3: if constexpr (A != 3 && K > 3) reg_cx<V, K, A, 3>(v); break;
    default: if constexpr (A != 4 && K > 4) reg_cx<V, K, A, 4>(v); break;
    }
}
template <typename V, int K>
__device__ __forceinline__ void reg_cx_any(V* v, int a, int b) {
    switch (a) {
    case 0: reg_cx_b<V, K, 0>(v, b); break;
    case 1: if constexpr (K > 1) reg_cx_b<V, K, 1>(v, b); break;
    case 2: if constexpr (K > 2) reg_cx_b<V, K, 2>(v, b); break;
    case 3: if constexpr (K > 3) reg_cx_b<V, K, 3>(v, b); break;
    default: if constexpr (K > 4) reg_cx_b<V, K, 4>(v, b); break;
    }
}
template <typename V, int K, int A>
__device__ __forceinline__ void reg_swap_b(V* v, int b) {
    switch (b) {
    case 0: if constexpr (A != 0) reg_swap<V, K, A, 0>(v); break;
    case 1: if constexpr (A != 1 && K > 1) reg_swap<V, K, A, 1>(v); break;
    case 2: if constexpr (A != 2 && K > 2) reg_swap<V, K, A, 2>(v); break;
    case 3: if constexpr (A != 3 && K > 3) reg_swap<V, K, A, 3>(v); break;
    default: if constexpr (A != 4 && K > 4) reg_swap<V, K, A, 4>(v); break;
    }
}
template <typename V, int K>
__device__ __forceinline__ void reg_swap_any(V* v, int a, int b) {
    switch (a) {
    case 0: reg_swap_b<V, K, 0>(v, b); break;
    case 1: if constexpr (K > 1) reg_swap_b<V, K, 1>(v, b); break;
    case 2: if constexpr (K > 2) reg_swap_b<V, K, 2>(v, b); break;
    case 3: if constexpr (K > 3) reg_swap_b<V, K, 3>(v, b); break;
    default: if constexpr (K > 4) reg_swap_b<V, K, 4>(v, b); break;
    }
}


// Phases as fixed-point turns (2^-64 turn units, so integer addition is
// addition modulo one turn); the complex64 path uses the top 32 bits.
template <typename R> struct Turns;
template <> struct Turns<float> {
    using U = uint32_t;
    static __device__ __forceinline__ U coef(uint64_t x) { return (U)((x + 0x80000000ull) >> 32); }
    static __device__ __forceinline__ void sincos(U ph, float* s, float* c) {
        __sincosf((float)(int32_t)ph * 1.46291807926715968e-09f, s, c);  // 2 pi / 2^32
    }
    static __device__ __forceinline__ void sincos_t(U ph, const double2*, float* s, float* c) { sincos(ph, s, c); }
};
template <> struct Turns<double> {
    using U = uint64_t;
    static __device__ __forceinline__ U coef(uint64_t x) { return x; }
    static __device__ __forceinline__ void sincos(U ph, double* s, double* c) {
        sincospi((double)(int64_t)ph * 1.08420217248550443e-19, s, c);  // 2 / 2^64
    }
    // Table-driven (Tang's method): the top 8 bits of the phase pick
    // (cos, sin)(2 pi k / 256) from tab, the remaining fraction of a turn
    // (an angle below 2 pi / 256) goes through its Taylor series to the
    // x^9 / x^8 terms (truncation below 1e-18), and the angle-sum formulas
    // combine the two: about half the FP64 work of a general sincos.
    static __device__ __forceinline__ void sincos_t(U ph, const double2* tab, double* s, double* c) {
        if (!tab) {
            sincos(ph, s, c);
            return;
        }
        const double2 e = tab[ph >> 56];
        const double th = (double)(ph & 0x00ffffffffffffffull) * 3.4061215800865545e-19;  // 2 pi / 2^64
        const double t = th * th;
        const double sn = th * fma(t, fma(t, fma(t, fma(t, 2.7557319223985893e-06, -1.984126984126984e-04),
                                                  8.333333333333333e-03), -1.6666666666666666e-01), 1.0);
        const double cs = fma(t, fma(t, fma(t, fma(t, 2.48015873015873e-05, -1.388888888888889e-03),
                                             4.1666666666666664e-02), -0.5), 1.0);
        *c = fma(e.x, cs, -e.y * sn);
        *s = fma(e.y, cs, e.x * sn);
    }
};
// (cos, sin)(2 pi k / 256), k < 256, into a CTA's table (complex128 phases).
__device__ __forceinline__ void build_turn_table(double2* tab) {
    for (int k = threadIdx.x; k < 256; k += blockDim.x) {
        double sn, cs;
        sincospi((double)k / 128.0, &sn, &cs);
        tab[k] = make_double2(cs, sn);
    }
}

// ---------------------------------------------------------------------------
// Register-resident tile pass.  Thread t of a CTA of 2^(m-RB) threads holds
// the 2^RB amplitudes of the tile whose register bits (tile positions
// rpos[0..RB-1]) vary and whose other bits are the bits of t (tile positions
// tpos[]).  Gate records, dense blocks (on register bits 0..k-1) and diagonal
// runs act on the registers directly; shared memory is used only to load and
// store the tile and to exchange amplitudes when the plan changes the
// register layout (remap).  The layouts are chosen on the host.
// ---------------------------------------------------------------------------
template <typename V, int RB> struct RegLayout {
    int sbase;     // swizzled tile offset of this thread's register 0
    int sbit[RB];  // swizzled offset of register bit b
};

template <typename V, int RB>
__device__ __forceinline__ void reg_layout(RegLayout<V, RB>& L, const int* rpos, const int* tpos, int tb) {
    int base = 0;
    SV_UNROLL
    for (int t = 0; t < tb; ++t) base |= ((int)(threadIdx.x >> t) & 1) << tpos[t];
    L.sbase = swz<V>(base);
#pragma unroll
    for (int b = 0; b < RB; ++b) L.sbit[b] = swz<V>(1 << rpos[b]);
}

template <typename V, int RB>
__device__ __forceinline__ void reg_read(V* v, const V* tile, const RegLayout<V, RB>& L) {
#pragma unroll
    for (int k = 0; k < (1 << RB); ++k) {
        int o = L.sbase;
#pragma unroll
        for (int b = 0; b < RB; ++b)
            if ((k >> b) & 1) o ^= L.sbit[b];
        v[k] = tile[o];
    }
}

template <typename V, int RB>
__device__ __forceinline__ void reg_write(const V* v, V* tile, const RegLayout<V, RB>& L) {
#pragma unroll
    for (int k = 0; k < (1 << RB); ++k) {
        int o = L.sbase;
#pragma unroll
        for (int b = 0; b < RB; ++b)
            if ((k >> b) & 1) o ^= L.sbit[b];
        tile[o] = v[k];
    }
}

// Dense 2^K x 2^K block on register bits 0..K-1.
template <typename V, int RB, int K>
__device__ __forceinline__ void reg_dense(V* v, const V* __restrict__ U) {
    constexpr int D = 1 << K;
#pragma unroll
    for (int hi = 0; hi < (1 << (RB - K)); ++hi) {
        V x[D];
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = v[hi * D + j];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            V a = czero<V>();
#pragma unroll
            for (int j = 0; j < D; ++j) a = cfma(U[r * D + j], x[j], a);
            v[hi * D + r] = a;
        }
    }
}

// ---------------------------------------------------------------------------
// Dense block on the tensor cores (OP_DENSE_TC; complex64, register bits
// 0..K-1, K = 4 or 5).  The CTA's threads form groups of 128 (four warps:
// TMEM lanes 0..127 of columns [128 g, 128 g + 128) of the CTA's
// allocation).  Each thread's 32 amplitudes are 32 / 2^K slices of the block,
// one row of the A operand each: the slice's 2^(K+1) reals, (re, im)
// interleaved, as FP16 pairs (one TMEM column per amplitude), split into
// hi = fp16(x s) at columns [0, 32) and lo = fp16(x s - hi) at [32, 64).  B is
// the real form of the block's matrix, B[2r + c'][2j + c] (c, c' = 0 real, 1
// imaginary part), staged (times kTcMatScale) in shared memory, K-major
// no-swizzle, hi then lo.  One thread issues D = A_hi B_hi + A_hi B_lo +
// A_lo B_hi with FP32 accumulation into columns [64, 128); every thread reads
// its row back: the slice's outputs, (re, im) interleaved, which is again one
// register per amplitude.  The dropped A_lo B_lo term is below 2^-22 of the
// result, about FP32 rounding.
// ---------------------------------------------------------------------------
struct TcCtx {
    uint32_t tmem;   // TMEM base address of the CTA's allocation (128 columns per group)
    uint64_t* mbar;  // one mbarrier per group (shared memory)
    int* abort;      // per group: a bounded wait gave up, skip the remaining products
    int* err;        // device error word: set to 1 when a wait gives up
    uint32_t phase;  // waits this thread has completed (parity of the next)
    float* nin;      // per warp: sum of |a|^2 of the tile as loaded (passes with tensor-core blocks)
    float* nout;     // per warp: the same after the pass's ops
};

// Sum of |a|^2 over this thread's registers (four partial sums), then over
// the warp; lane 0 writes it to slot[warp].  Passes with tensor-core blocks
// use it to restore each tile's norm: every op of a pass acts on the tile
// alone and is unitary, so the tile's norm is preserved exactly, while the
// tensor cores' accumulation rounds toward zero (a systematic shrink of a few
// 10^-7 per block that would add up over a circuit).
template <int RB>
__device__ __forceinline__ void warp_norm_to(const float2* v, float* slot) {
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < (1 << RB); ++k) {
        s[k & 3] = fmaf(v[k].x, v[k].x, s[k & 3]);
        s[k & 3] = fmaf(v[k].y, v[k].y, s[k & 3]);
    }
    float t = (s[0] + s[1]) + (s[2] + s[3]);
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) t += __shfl_xor_sync(0xffffffffu, t, sh);
    if ((threadIdx.x & 31) == 0) slot[threadIdx.x >> 5] = t;
}
// sqrt(sum nin / sum nout) over the CTA's warps (read after a barrier that
// follows both writes); 1 for a tile that is zero.  The write-back factor is
// this with the sign of the pass's deferred factors (PassDev::scale), whose
// magnitude it replaces.
__device__ __forceinline__ float tile_norm_fix(const float* nin, const float* nout) {
    const int nw = (int)(blockDim.x >> 5);
    float a = 0.f, b = 0.f;
    for (int w = 0; w < nw; ++w) {
        a += nin[w];
        b += nout[w];
    }
    return b > 0.f ? sqrtf(a / b) : 1.0f;
}

__device__ __forceinline__ uint32_t f16x2_pack(float lo, float hi) {  // round to nearest even
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;\n" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ float2 f16x2_unpack(uint32_t p) {
    float2 r;
    asm("{\n.reg .f16 l, h;\nmov.b32 {l, h}, %2;\ncvt.f32.f16 %0, l;\ncvt.f32.f16 %1, h;\n}\n"
        : "=f"(r.x), "=f"(r.y)
        : "r"(p));
    return r;
}

template <int RB, int K>
__device__ __forceinline__ void reg_dense_tc(float2* v, const unsigned char* bmat, float s_in, TcCtx& T) {
    static_assert(RB == 5 && (K == 4 || K == 5), "tensor-core blocks: 32 amplitudes per thread, 4 or 5 qubits");
    constexpr int D = 1 << K;            // amplitudes of a slice
    constexpr int NS = 32 / D;           // slices per thread
    constexpr uint32_t N = 2 * D;        // reals of a slice (the MMA's N and K)
    constexpr uint32_t IDESC = tc::idesc_f16(128, N);
    constexpr uint32_t SBO = 16 * N;     // bytes between 8-row groups of B
    constexpr uint32_t OPB = 2 * N * N;  // bytes of one B operand (hi or lo)
    const int tid = threadIdx.x, grp = tid >> 7;
    const uint32_t cols = T.tmem + (uint32_t)grp * 128u;
    const uint32_t lane = cols + (((uint32_t)((tid >> 5) & 3) * 32u) << 16);
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 8) {  // (eight at a time: fewer live registers)
        uint32_t h[8], l[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float xr = v[c0 + j].x * s_in, xi = v[c0 + j].y * s_in;
            h[j] = f16x2_pack(xr, xi);
            const float2 hf = f16x2_unpack(h[j]);
            l[j] = f16x2_pack(xr - hf.x, xi - hf.y);
        }
        tc::tmem_st8(lane + c0, h);
        tc::tmem_st8(lane + 32 + c0, l);
    }
    tc::tmem_wait_st();
    tc::fence_before();
    tc::named_barrier(1 + grp, 128);
    tc::fence_after();
    if (T.abort[grp]) return;  // an earlier wait of the group gave up (read after the barrier: uniform)
    if ((tid & 127) == 0) {
        const uint32_t bh = tc::smem_u32(bmat), bl = bh + OPB;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const uint32_t d = cols + 64 + s * N, ah = cols + s * D, al = cols + 32 + s * D;
#pragma unroll
            for (int kk = 0; kk < (int)N / 16; ++kk)
                tc::mma_f16_ts(d, ah + 8 * kk, tc::sdesc_noswz(bh + 256 * kk, 128, SBO), IDESC, kk > 0);
#pragma unroll
            for (int kk = 0; kk < (int)N / 16; ++kk)
                tc::mma_f16_ts(d, ah + 8 * kk, tc::sdesc_noswz(bl + 256 * kk, 128, SBO), IDESC, 1);
#pragma unroll
            for (int kk = 0; kk < (int)N / 16; ++kk)
                tc::mma_f16_ts(d, al + 8 * kk, tc::sdesc_noswz(bh + 256 * kk, 128, SBO), IDESC, 1);
        }
        tc::mma_commit(&T.mbar[grp]);
    }
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait_bounded(&T.mbar[grp], T.phase & 1u, 1u << 22));
    T.phase += 1;
    tc::fence_after();
    if (!ok) {  // warp-uniform: the whole warp skips the TMEM reads
        T.abort[grp] = 1;
        atomicExch(T.err, 1);
        return;
    }
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
        uint32_t d[32];
        tc::tmem_ld32(lane + 64 + c0, d);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            v[c0 / 2 + j].x = __uint_as_float(d[2 * j]);
            v[c0 / 2 + j].y = __uint_as_float(d[2 * j + 1]);
        }
    }
}

template <typename V, int RB>
__device__ __forceinline__ void reg_gates(V* v, const GateRec* __restrict__ recs, int nrec, const V* __restrict__ sd) {
    using R = decltype(V().x);
    for (int r = 0; r < nrec; ++r) {
        const GateRec g = recs[r];
        switch (g.kind) {
        case GR_U: reg_u_any<V, RB>(v, g.a, sd[g.off], sd[g.off + 1], sd[g.off + 2], sd[g.off + 3]); break;
        case GR_UR:
            reg_ur_any<V, RB, R>(v, g.a, sd[g.off].x, sd[g.off + 1].x, sd[g.off + 2].x, sd[g.off + 3].x);
            break;
        case GR_DT:  // b: entries that differ from 1
#pragma unroll
            for (int j = 0; j < (1 << RB); ++j)
                if ((g.b >> j) & 1) v[j] = cmul(sd[g.off + j], v[j]);
            break;
        case GR_URS: reg_urs_any<V, RB, R>(v, g.a, g.b, sd[g.off].x); break;
        case GR_CX: reg_cx_any<V, RB>(v, g.a, g.b); break;
        case GR_H: reg_h_any<V, RB>(v, g.a); break;
        case GR_HD:
            reg_h_any<V, RB>(v, g.a);
#pragma unroll
            for (int j = 0; j < (1 << RB); ++j)
                if ((g.b >> j) & 1) v[j] = cmul(sd[g.off + j], v[j]);
            break;
        default: reg_swap_any<V, RB>(v, g.a, g.b); break;
        }
    }
}

// Tile copies of a register pass: every thread moves exactly 16 chunks of 16
// bytes (2^RB amplitudes), chunk k of thread t being tile chunk t + k * blockDim,
// so the row and in-row offsets advance by compile-time multiples.
template <typename V>
__device__ __forceinline__ void rissue_tile(V* tile, const V* __restrict__ psi, uint64_t base, const uint32_t* rowoff,
                                            int L) {
    constexpr int PER = 16 / sizeof(V);
    const int i0 = PER * (int)threadIdx.x, istep = PER * (int)blockDim.x;
    const int ioff = i0 & ((1 << L) - 1);
    const V* src = psi + base + ioff;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
        const int i = i0 + k * istep;
        cp_async16(tile + swz<V>(i), src + ((uint64_t)rowoff[i >> L] << L));
    }
}
template <typename V>
__device__ __forceinline__ void rstore_tile(const V* tile, V* __restrict__ psi, uint64_t base, const uint32_t* rowoff,
                                            int L) {
    constexpr int PER = 16 / sizeof(V);
    const int i0 = PER * (int)threadIdx.x, istep = PER * (int)blockDim.x;
    const int ioff = i0 & ((1 << L) - 1);
    V* dst = psi + base + ioff;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
        const int i = i0 + k * istep;
        *(float4*)(dst + ((uint64_t)rowoff[i >> L] << L)) = *(const float4*)(tile + swz<V>(i));
    }
}

// Global index of a tile's first amplitude from its number t: the bits of t
// scattered to the non-tile qubits, via per-byte tables (entries in units of
// 2^L amplitudes; at most 24 non-tile qubits here).
__device__ __forceinline__ void build_base_tables(uint32_t (*tb)[256], const PassDev& P) {
    for (int e = threadIdx.x; e < 3 * 256; e += blockDim.x) {
        const int b = e >> 8, v = e & 255;
        uint32_t o = 0;
        for (int i = 0; i < 8; ++i) {
            const int q = 8 * b + i;
            if (q < P.nother && ((v >> i) & 1)) o |= 1u << (P.oq[q] - P.L);
        }
        tb[b][v] = o;
    }
}
__device__ __forceinline__ uint64_t table_base(const uint32_t (*tb)[256], uint64_t t, int L) {
    return (uint64_t)(tb[0][t & 255] | tb[1][(t >> 8) & 255] | tb[2][(t >> 16) & 255]) << L;
}

// Diagonal run on the registers.  fold = the run's per-tile linear
// coefficients a'_j (tile positions j < m) and constant C (at m); dw = the
// run's RDiagLayout words for the current layout.
template <typename V, typename R, int RB>
__device__ __forceinline__ void reg_diag(V* v, const uint64_t* __restrict__ dw, const uint64_t* fold, int m, int no,
                                         const int* rpos, const int* tpos, int tb, const double2* ttab = nullptr) {
    using T = Turns<R>;
    using U = typename T::U;
    const RDiagLayout Lr(m, no);
    const int tid = threadIdx.x, lo = tid & 15, hi = tid >> 4;
    U phT = (U)fold[m] + T::coef(dw[Lr.tqlo + lo]) + T::coef(dw[Lr.tqhi + hi]);
    SV_UNROLL
    for (int t = 0; t < tb; ++t)
        if ((tid >> t) & 1) phT += (U)fold[tpos[t]];
    SV_UNROLL
    for (int t = 4; t < tb; ++t)
        if ((tid >> t) & 1) phT += T::coef(dw[Lr.tr + (t - 4) * 16 + lo]);
    U al[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b)
        al[b] = (U)fold[rpos[b]] + T::coef(dw[Lr.talo + b * 16 + lo]) + T::coef(dw[Lr.tahi + b * 32 + hi]);
    U be[RB][RB];
#pragma unroll
    for (int b = 0; b < RB; ++b)
#pragma unroll
        for (int b2 = b + 1; b2 < RB; ++b2) be[b][b2] = T::coef(dw[Lr.beta + b * 5 + b2]);
    constexpr int LB = (RB + 1) / 2, HB = RB - LB;
    U PL[1 << LB];
#pragma unroll
    for (int u = 0; u < (1 << LB); ++u) {
        U s = 0;
#pragma unroll
        for (int b = 0; b < LB; ++b)
            if ((u >> b) & 1) {
                s += al[b];
#pragma unroll
                for (int b2 = b + 1; b2 < LB; ++b2)
                    if ((u >> b2) & 1) s += be[b][b2];
            }
        PL[u] = s;
    }
#pragma unroll
    for (int w = 0; w < (1 << HB); ++w) {
        U PH = phT;
        U cb[LB];
#pragma unroll
        for (int b = 0; b < LB; ++b) cb[b] = 0;
#pragma unroll
        for (int c = 0; c < HB; ++c)
            if ((w >> c) & 1) {
                PH += al[LB + c];
#pragma unroll
                for (int c2 = c + 1; c2 < HB; ++c2)
                    if ((w >> c2) & 1) PH += be[LB + c][LB + c2];
#pragma unroll
                for (int b = 0; b < LB; ++b) cb[b] += be[b][LB + c];
            }
#pragma unroll
        for (int u = 0; u < (1 << LB); ++u) {
            U ph = PH + PL[u];
#pragma unroll
            for (int b = 0; b < LB; ++b)
                if ((u >> b) & 1) ph += cb[b];
            R sn, cs;
            T::sincos_t(ph, ttab, &sn, &cs);
            V f;
            f.x = cs;
            f.y = sn;
            const int k = (w << LB) | u;
            v[k] = cmul(f, v[k]);
        }
    }
}

// ---- helpers for the run-time compiled kernels (compile-time geometry) ----
// Swizzled tile offset of this thread's register 0 for thread-bit positions
// tp[0..TB-1].
template <typename V, int TB>
__device__ __forceinline__ int thread_sbase(const int* tp) {
    int base = 0;
#pragma unroll
    for (int t = 0; t < TB; ++t) base |= ((int)(threadIdx.x >> t) & 1) << tp[t];
    return swz<V>(base);
}
// Registers from / to the tile: register k sits at sb ^ C[k] (sb + C[k]
// when no bit of sb can meet a bit of C, so the offset is an immediate).
template <typename V, int RB, bool ADD>
__device__ __forceinline__ void reg_read_ct(V* v, const V* tile, int sb, const int* C) {
#pragma unroll
    for (int k = 0; k < (1 << RB); ++k) v[k] = tile[ADD ? sb + C[k] : sb ^ C[k]];
}
template <typename V, int RB, bool ADD>
__device__ __forceinline__ void reg_write_ct(const V* v, V* tile, int sb, const int* C) {
#pragma unroll
    for (int k = 0; k < (1 << RB); ++k) tile[ADD ? sb + C[k] : sb ^ C[k]] = v[k];
}
// The same for complex64 when register bit 0 is tile position 0: registers
// 2j and 2j + 1 share one 16-byte chunk (sb and C[2j] are even), moved with
// one 16-byte access.
template <typename V, int RB, bool ADD>
__device__ __forceinline__ void reg_read_ct2(V* v, const V* tile, int sb, const int* C) {
#pragma unroll
    for (int k = 0; k < (1 << RB); k += 2) {
        const float4 q = *reinterpret_cast<const float4*>(tile + (ADD ? sb + C[k] : sb ^ C[k]));
        v[k].x = q.x;
        v[k].y = q.y;
        v[k + 1].x = q.z;
        v[k + 1].y = q.w;
    }
}
template <typename V, int RB, bool ADD>
__device__ __forceinline__ void reg_write_ct2(const V* v, V* tile, int sb, const int* C) {
#pragma unroll
    for (int k = 0; k < (1 << RB); k += 2)
        *reinterpret_cast<float4*>(tile + (ADD ? sb + C[k] : sb ^ C[k])) =
            make_float4(v[k].x, v[k].y, v[k + 1].x, v[k + 1].y);
}
// Tile copies: chunk k of this thread is 16 bytes at psi[g + KO[k]] and at
// tile[s0 ^ SW[k]] (s0 + SW[k] under ADD).
template <typename V, int NCH, bool ADD>
__device__ __forceinline__ void issue_ct(V* tile, const V* __restrict__ psi, uint64_t g, int s0, const uint64_t* KO,
                                         const int* SW) {
#pragma unroll
    for (int k = 0; k < NCH; ++k) cp_async16(tile + (ADD ? s0 + SW[k] : s0 ^ SW[k]), psi + g + KO[k]);
}
template <typename V, int NCH, bool ADD>
__device__ __forceinline__ void store_ct(const V* tile, V* __restrict__ psi, uint64_t g, int s0, const uint64_t* KO,
                                         const int* SW) {
#pragma unroll
    for (int k = 0; k < NCH; ++k)
        *(float4*)(psi + g + KO[k]) = *(const float4*)(tile + (ADD ? s0 + SW[k] : s0 ^ SW[k]));
}
// Tile of |x> (the deferred basis state) instead of loading it: this
// thread's chunks are written with zeros, and the one holding tile position
// ix (-1: x is not in this tile) gets the 1.
template <typename V, int NCH, bool ADD>
__device__ __forceinline__ void fill_basis_ct(V* tile, int ix, int i0, int istep, int s0, const int* SW) {
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const int i = i0 + k * istep;
        V* dst = tile + (ADD ? s0 + SW[k] : s0 ^ SW[k]);
        if constexpr (sizeof(V) == 8) {  // two amplitudes per 16-byte chunk
            *(float4*)dst = make_float4(ix == i ? 1.f : 0.f, 0.f, ix == i + 1 ? 1.f : 0.f, 0.f);
        } else {
            V a;
            a.x = ix == i ? 1.0 : 0.0;
            a.y = 0.0;
            *dst = a;
        }
    }
}

template <typename V, int RB>
__device__ __forceinline__ void scale_regs(V* v, decltype(V().x) sc) {
#pragma unroll
    for (int k = 0; k < (1 << RB); ++k) {
        v[k].x *= sc;
        v[k].y *= sc;
    }
}

// Per-tile fold of every diagonal run of the pass for tile t.
template <typename R>
__device__ __forceinline__ void fold_diags(const PassDev& P, const unsigned char* stage, uint64_t* fold,
                                           const int* dofs, uint64_t t) {
    using T = Turns<R>;
    const int m = P.m, no = P.nother, nd = P.ndiag;
    // per-tile fold of every diagonal run: a'_j = a_j + sum_o b_jo x_o (one
    // thread per run and tile position) and C = c + sum_o x_o (a_o +
    // sum_{o2<o} b_oo2 x_o2) (one warp per run, one non-tile bit per lane),
    // with x_o = bit o of t
    {
        const RDiagLayout Lr(m, no);
        for (int idx = threadIdx.x; idx < nd * m; idx += blockDim.x) {
            const int d = idx / m, j = idx - d * m;
            const uint64_t* dw = (const uint64_t*)(stage + dofs[d]);
            uint64_t a = dw[Lr.at + j];
            for (int o = 0; o < no; ++o)
                if ((t >> o) & 1) a += dw[Lr.bo + j * no + o];
            fold[d * (m + 1) + j] = T::coef(a);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        for (int d = warp; d < nd; d += nwarps) {
            const uint64_t* dw = (const uint64_t*)(stage + dofs[d]);
            uint64_t a = 0;
            if (lane < no && ((t >> lane) & 1)) {
                a = dw[Lr.ao + lane];
                for (int o2 = 0; o2 < lane; ++o2)
                    if ((t >> o2) & 1) a += dw[Lr.boo + lane * no + o2];
            }
#pragma unroll
            for (int sh = 16; sh > 0; sh >>= 1) a += __shfl_xor_sync(0xffffffffu, a, sh);
            if (lane == 0) fold[d * (m + 1) + m] = T::coef(a + dw[Lr.c]);
        }
    }
}

// The op list of a pass, walked at run time (the library's kernel).  On
// return the amplitudes are in registers in the last layout (Lg).  issue /
// store move a tile between the state and shared memory; finish applies the
// pass's write-back scale and puts the registers back into the tile.
template <bool TC>
struct InterpOps {
    // tiles move through shared memory (the compiled passes may load their
    // first layout and store their last straight to and from registers)
    static constexpr bool kDirectLoad = false, kDirectStore = false;
    template <typename V>
    static __device__ __forceinline__ void issue(V* tile, const V* __restrict__ psi, uint64_t base,
                                                 const uint32_t* rowoff, int L, const PassDev&) {
        rissue_tile(tile, psi, base, rowoff, L);
    }
    template <typename V>
    static __device__ __forceinline__ void store(const V* tile, V* __restrict__ psi, uint64_t base,
                                                 const uint32_t* rowoff, int L) {
        rstore_tile(tile, psi, base, rowoff, L);
    }
    template <typename V, typename R, int RB>
    static __device__ __forceinline__ void finish(V* v, V* tile, const PassDev& P, const RegLayout<V, RB>& Lg,
                                                  TcCtx& T) {
        if constexpr (TC && sizeof(R) == 4 && RB == 5) {
            if (P.tc_k) {  // the tile's norm as loaded: scale = sqrt(in / out)
                warp_norm_to<RB>((const float2*)v, T.nout);
                __syncthreads();
                scale_regs<V, RB>(v, copysignf(tile_norm_fix(T.nin, T.nout), (float)P.scale));
                reg_write<V, RB>(v, tile, Lg);
                return;
            }
        }
        if (P.scale != 1.0) {
            const R sc = (R)P.scale;
#pragma unroll
            for (int k = 0; k < (1 << RB); ++k) {
                v[k].x *= sc;
                v[k].y *= sc;
            }
        }
        // each warp writes back the positions it read last, which no other
        // warp reads: the caller's barrier before the store orders the rest
        reg_write<V, RB>(v, tile, Lg);
    }
    template <typename V, typename R, int RB>
    static __device__ __forceinline__ void tile(V* v, V* tile, const PassDev& P, const unsigned char* stage,
                                                const uint64_t* fold, RegLayout<V, RB>& Lg, const double2* ttab,
                                                TcCtx& T) {
    const int m = P.m, tb = m - RB, no = P.nother;
    const OpDev* ops = (const OpDev*)stage;
    const int* rpos = nullptr;
    const int* tpos = nullptr;
    bool in_regs = false;
    for (int oi = 0; oi < P.nops; ++oi) {
        const OpDev& op = ops[oi];
        switch (op.kind) {
        case OP_REMAP:
            // the write needs no barrier before it (a warp writes exactly the
            // positions it read last); the read after it needs the other
            // writers: the warp's own lanes when the remap keeps every warp's
            // amplitudes within the warp (nrec = 1), else the whole block
            if (in_regs) {
                reg_write<V, RB>(v, tile, Lg);
                if (op.nrec == 1) __syncwarp();
                else __syncthreads();
            } else {
                __syncthreads();
            }
            rpos = op.lq;
            tpos = (const int*)(stage + op.mat_off);
            reg_layout<V, RB>(Lg, rpos, tpos, tb);
            reg_read<V, RB>(v, tile, Lg);
            if constexpr (TC && sizeof(R) == 4 && RB == 5)
                if (!in_regs && P.tc_k) warp_norm_to<RB>((const float2*)v, T.nin);
            in_regs = true;
            break;
        case OP_GATES:
            reg_gates<V, RB>(v, (const GateRec*)(stage + op.rec_off), op.nrec, (const V*)(stage + op.mat_off));
            break;
        case OP_DENSE: {
            const V* U = (const V*)(stage + op.mat_off);
            switch (op.k) {
            case 1: reg_dense<V, RB, 1>(v, U); break;
            case 2: reg_dense<V, RB, 2>(v, U); break;
            default: reg_dense<V, RB, 3>(v, U); break;
            }
            break;
        }
        case OP_DENSE_TC:
            if constexpr (TC && sizeof(R) == 4 && RB == 5) {
                if (op.k == 5) reg_dense_tc<RB, 5>((float2*)v, stage + op.mat_off, op.tc_scale, T);
                else reg_dense_tc<RB, 4>((float2*)v, stage + op.mat_off, op.tc_scale, T);
            }
            break;
        default:
            reg_diag<V, R, RB>(v, (const uint64_t*)(stage + op.diag_off), fold + (size_t)op.ord * (m + 1), m, no,
                               rpos, tpos, tb, ttab);
            break;
        }
    }
    }
};

// One register-resident pass: each CTA walks tiles t = blockIdx.x, +gridDim.x,
// ...  Per tile: the tile arrives (16-byte cp.async copies into shared memory,
// double-buffered when the layout allows; or, for Ops::kDirectLoad, straight
// into registers in the first layout), the op list runs on the registers with
// remaps through shared memory, and the tile leaves (through shared memory,
// or for Ops::kDirectStore straight from registers in the last layout).
// MAXT/MINB: launch bounds of the instance (up to 128 threads: registers are
// not capped below 255, so the 2^RB amplitudes and the op state never spill;
// 256 and 512 threads: 128 registers).
// Passes with tensor-core blocks (P.tc_k > 0, complex64) hold 128 TMEM
// columns per group of 128 threads for the whole kernel; every wait on the
// tensor cores is bounded (expiry: *err = 1, the group skips its remaining
// products, the TMEM is still freed).
template <typename R, int RB, class Ops, bool TC = false>
__device__ __forceinline__ void rpass_body(typename CT<R>::V* __restrict__ psi, int n,
                                           const PassDev* __restrict__ pdp, const unsigned char* __restrict__ blob,
                                           const PassLayout& lay, int* __restrict__ err) {
    using V = typename CT<R>::V;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ PassDev P;
    __shared__ uint32_t tbase[3][256];
    __shared__ double2 ttab[sizeof(R) == 8 ? 256 : 1];  // complex128: the phase table of Turns::sincos_t
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[4];
    __shared__ int s_abort[4];
    __shared__ float s_norm[2][16];  // per warp: tile norm in / out (passes with tensor-core blocks)
    {
        const int* src = (const int*)pdp;
        int* dst = (int*)&P;
        for (int i = threadIdx.x; i < (int)(sizeof(PassDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int ngroups = (int)(blockDim.x >> 7);
    const uint32_t tmem_cols = 128u * (uint32_t)ngroups;  // 128, 256 or 512
    // (TC: the instance for passes with tensor-core blocks; the others carry
    // none of the TMEM code)
    const bool tcp = TC && sizeof(R) == 4 && RB == 5 && P.tc_k > 0 && ngroups >= 1;
    if (tcp) {
        if (threadIdx.x < 32) {
            tc::tmem_alloc(&s_tmem, tmem_cols);
            tc::tmem_relinquish();
        }
        if (threadIdx.x == 0) {
            for (int g = 0; g < ngroups; ++g) {
                tc::mbar_init(&s_mbar[g], 1);
                s_abort[g] = 0;
            }
            tc::fence_mbar_init();
        }
    }
    const int m = P.m, L = P.L, nd = P.ndiag;
    V* tiles[2] = {(V*)smem, (V*)(smem + (lay.nbuf == 2 ? lay.tile_bytes : 0))};
    uint32_t* rowoff = (uint32_t*)(smem + lay.rowoff_off);
    unsigned char* stage = smem + lay.stage_off;
    uint64_t* fold = (uint64_t*)(smem + lay.work_off);  // nd x (m + 1)
    int* dofs = (int*)(fold + (size_t)nd * (m + 1));   // diag word offsets by ordinal
    const unsigned char* greg = blob + P.region_off;
    for (int e = threadIdx.x; e < lay.stage_bytes / 16; e += blockDim.x) cp_async16(stage + 16 * e, greg + 16 * e);
    cp_async_commit();
    const int nrows = 1 << (m - L);
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        uint32_t o = 0;
        for (int b = 0; b < m - L; ++b)
            if ((r >> b) & 1) o |= 1u << (P.tq[L + b] - L);
        rowoff[r] = o;
    }
    build_base_tables(tbase, P);
    if constexpr (sizeof(R) == 8) build_turn_table(ttab);
    cp_async_wait_group<0>();
    if (tcp) {
        tc::fence_proxy_async();  // the staged matrices are read by the tensor cores
        tc::fence_before();
    }
    __syncthreads();
    if (tcp) tc::fence_after();
    TcCtx T{tcp ? s_tmem : 0u, s_mbar, s_abort, err, 0u, s_norm[0], s_norm[1]};
    const OpDev* ops = (const OpDev*)stage;
    if (threadIdx.x == 0)
        for (int i = 0; i < P.nops; ++i)
            if (ops[i].kind == OP_DIAG) dofs[ops[i].ord] = ops[i].diag_off;
    const uint64_t ntiles = 1ull << (n - m);
    auto tile_base = [&](uint64_t t) { return table_base(tbase, t, L); };
    int cur = 0;
    if constexpr (!Ops::kDirectLoad) {
        if (lay.nbuf == 2 && (uint64_t)blockIdx.x < ntiles) {
            Ops::template issue<V>(tiles[0], psi, tile_base(blockIdx.x), rowoff, L, P);
            cp_async_commit();
        }
    }
    V v[1 << RB];
    RegLayout<V, RB> Lg;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t base = tile_base(t);
        if constexpr (Ops::kDirectLoad) {
            // the first layout straight from global memory into registers;
            // the barrier keeps this tile's shared-memory writes behind the
            // previous tile's reads
            Ops::template load<V>(v, psi, base, P);
            __syncthreads();
        } else {
            const uint64_t tn = t + gridDim.x;
            if (lay.nbuf == 2) {
                if (tn < ntiles) {
                    Ops::template issue<V>(tiles[cur ^ 1], psi, tile_base(tn), rowoff, L, P);
                    cp_async_commit();
                    cp_async_wait_group<1>();
                } else {
                    cp_async_wait_group<0>();
                }
            } else {
                Ops::template issue<V>(tiles[0], psi, base, rowoff, L, P);
                cp_async_commit();
                cp_async_wait_group<0>();
            }
            __syncthreads();
        }
        V* tile = tiles[cur];
        if (nd) {
            fold_diags<R>(P, stage, fold, dofs, t);
            if constexpr (Ops::kDirectLoad) __syncthreads();
        }
        Ops::template tile<V, R, RB>(v, tile, P, stage, fold, Lg, sizeof(R) == 8 ? ttab : nullptr, T);
        Ops::template finish<V, R, RB>(v, tile, P, Lg, T);
        if constexpr (Ops::kDirectStore) {
            // the last layout straight from registers to global memory
            Ops::template store_regs<V>(v, psi, base);
            if constexpr (!Ops::kDirectLoad) __syncthreads();  // this tile's reads before the next copies land
        } else {
            __syncthreads();
            Ops::template store<V>(tile, psi, base, rowoff, L);
            __syncthreads();
        }
        if (lay.nbuf == 2) cur ^= 1;
    }
    if (tcp) {
        tc::fence_before();
        __syncthreads();
        if (threadIdx.x < 32) tc::tmem_dealloc(s_tmem, tmem_cols);
    }
}

#ifndef __CUDACC_RTC__
template <typename R, int RB, int MAXT, int MINB, bool TC>
__global__ void __launch_bounds__(MAXT, MINB) k_rpass(typename CT<R>::V* __restrict__ psi, int n,
                                                  const PassDev* __restrict__ pdp,
                                                  const unsigned char* __restrict__ blob, const PassLayout lay,
                                                  int* __restrict__ err) {
    rpass_body<R, RB, InterpOps<TC>, TC>(psi, n, pdp, blob, lay, err);
}
#endif

}  // namespace sv
