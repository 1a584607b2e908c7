// Gate-application kernels for sm_103a.
//
//  * Plain path: one kernel per gate over the whole state (App. A: a gate
//    U_k = I (x) .. (x) U (x) .. (x) I acts on every amplitude pair that
//    differs only in bit k; CX exchanges the target pair where the control is
//    1, touching 2^(n-1) amplitudes; CR1 multiplies the |11> quarter).
//  * Tile pass: one HBM read + one write of the state applies a whole list of
//    fused dense blocks (<= 5 qubits, App. D.2 "gate fusion = 5") and
//    diagonal-phase runs to each 2^m-amplitude tile held in shared memory.
//    Tiles are gathered with 16-byte cp.async copies of contiguous rows of
//    2^L amplitudes (128 bytes), so every HBM access is a full line.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sv_internal.h"
#include "sv_philox.cuh"
#include "sv_rpass.cuh"
#include "sv_tc.cuh"
#include "sv_mux.cuh"

namespace sv {

__device__ __forceinline__ uint64_t insert_zero(uint64_t v, int pos) {
    const uint64_t lo = v & ((1ull << pos) - 1ull);
    return ((v >> pos) << (pos + 1)) | lo;
}

template <typename V> V to_dev(const cd& c) {
    V r;
    r.x = (decltype(r.x))c.real();
    r.y = (decltype(r.y))c.imag();
    return r;
}

// ---------------------------------------------------------------------------
// |x>
// ---------------------------------------------------------------------------
template <typename V>
__global__ void k_init_basis(V* __restrict__ psi, uint64_t N, uint64_t x) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        V v = czero<V>();
        if (i == x) v.x = 1;
        psi[i] = v;
    }
}

// ---------------------------------------------------------------------------
// Plain per-gate kernels.  Each thread handles UNR independent items per
// loop trip with all loads issued before any store (memory-level
// parallelism); items never overlap, so this is safe in place.
// ---------------------------------------------------------------------------
constexpr int UNR = 4;

template <typename V>
__global__ void __launch_bounds__(256) k_plain_1q(V* __restrict__ psi, uint64_t npairs, int q, V u00, V u01,
                                                  V u10, V u11) {
    const uint64_t lom = (1ull << q) - 1ull;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < npairs; r0 += stride * UNR) {
        V a[UNR], b[UNR];
        uint64_t i0[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const uint64_t r = r0 + u * stride;
            i0[u] = ((r & ~lom) << 1) | (r & lom);
            if (r < npairs) {
                a[u] = psi[i0[u]];
                b[u] = psi[i0[u] | (lom + 1)];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (r0 + u * stride < npairs) {
                psi[i0[u]] = cfma(u00, a[u], cmul(u01, b[u]));
                psi[i0[u] | (lom + 1)] = cfma(u10, a[u], cmul(u11, b[u]));
            }
        }
    }
}

// Exchange psi[i | A] and psi[i | B] for every i with bits lo, hi clear
// (CX: A = 1<<c, B = 1<<c | 1<<t; SWAP: A = 1<<q0, B = 1<<q1).
template <typename V>
__global__ void __launch_bounds__(256) k_plain_swap(V* __restrict__ psi, uint64_t nquads, int lo, int hi,
                                                    uint64_t A, uint64_t B) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < nquads; r0 += stride * UNR) {
        V a[UNR], b[UNR];
        uint64_t i[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const uint64_t r = r0 + u * stride;
            i[u] = insert_zero(insert_zero(r, lo), hi);
            if (r < nquads) {
                a[u] = psi[i[u] | A];
                b[u] = psi[i[u] | B];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (r0 + u * stride < nquads) {
                psi[i[u] | A] = b[u];
                psi[i[u] | B] = a[u];
            }
        }
    }
}

// Multiply psi[i | M] by f for every i with bits lo, hi clear (CP/CZ: M =
// both bits); with lo == hi a single bit (P, Z: the bit-1 half).
template <typename V>
__global__ void __launch_bounds__(256) k_plain_phase(V* __restrict__ psi, uint64_t nitems, int lo, int hi,
                                                     uint64_t M, V f) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < nitems; r0 += stride * UNR) {
        V a[UNR];
        uint64_t i[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const uint64_t r = r0 + u * stride;
            uint64_t x = insert_zero(r, lo);
            if (hi != lo) x = insert_zero(x, hi);
            i[u] = x | M;
            if (r < nitems) a[u] = psi[i[u]];
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            if (r0 + u * stride < nitems) psi[i[u]] = cmul(f, a[u]);
    }
}

// Diagonal single-qubit gate on every amplitude: psi[x] *= d[bit q of x].
template <typename V>
__global__ void __launch_bounds__(256) k_plain_diag1(V* __restrict__ psi, uint64_t N, int q, V d0, V d1) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x0 < N; x0 += stride * UNR) {
        V a[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            if (x0 + u * stride < N) a[u] = psi[x0 + u * stride];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const uint64_t x = x0 + u * stride;
            if (x < N) psi[x] = cmul(((x >> q) & 1) ? d1 : d0, a[u]);
        }
    }
}

// ---------------------------------------------------------------------------
// Tile pass.
// ---------------------------------------------------------------------------
// Dense k-qubit block on tile positions lq[0..K-1] (ascending).  A round
// covers blockDim/G whole slices; thread t takes row group g = t / (blockDim/G)
// (uniform across each warp, so matrix reads are shared-memory broadcasts)
// and slice t mod (blockDim/G).  With more than one group per slice all
// inputs of the round are read before any output is written (block barrier).
template <typename V, int K>
__device__ __forceinline__ void tile_dense(V* __restrict__ tile, int m, const OpDev& op, const V* __restrict__ sU) {
    constexpr int D = 1 << K;
    constexpr int RG = D < 8 ? D : 8;
    constexpr int G = D / RG;
    int bitv[K];  // swizzled offsets of the block's bits
#pragma unroll
    for (int i = 0; i < K; ++i) bitv[i] = swz<V>(1 << op.lq[i]);
    const int nslices = 1 << (m - K);
    const int per_round = blockDim.x / G;
    const int g = threadIdx.x / per_round;
    const int sl = threadIdx.x - g * per_round;
    for (int s0 = 0; s0 < nslices; s0 += per_round) {
        const int s = s0 + sl;
        const bool act = s < nslices;
        int base = s;
#pragma unroll
        for (int i = 0; i < K; ++i) base = (int)insert_zero((uint64_t)base, op.lq[i]);
        base = swz<V>(base);
        V acc[RG];
#pragma unroll
        for (int r = 0; r < RG; ++r) acc[r] = czero<V>();
        if (act) {
#pragma unroll
            for (int j = 0; j < D; ++j) {
                int o = 0;
#pragma unroll
                for (int i = 0; i < K; ++i)
                    if ((j >> i) & 1) o ^= bitv[i];
                const V x = tile[base ^ o];
#pragma unroll
                for (int r = 0; r < RG; ++r) acc[r] = cfma(sU[(g * RG + r) * D + j], x, acc[r]);
            }
        }
        if (G > 1) __syncthreads();
        if (act) {
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                const int row = g * RG + r;
                int o = 0;
#pragma unroll
                for (int i = 0; i < K; ++i)
                    if ((row >> i) & 1) o ^= bitv[i];
                tile[base ^ o] = acc[r];
            }
        }
        if (G > 1) __syncthreads();
    }
}

// recs/sdata: the op's gate records and matrices/tables (shared memory).
template <typename V, int K>
__device__ __forceinline__ void tile_gates(V* __restrict__ tile, int m, const OpDev& op, const GateRec* recs,
                                           const V* __restrict__ sdata) {
    constexpr int D = 1 << K;
    using R = decltype(V().x);
    int bitv[K];  // swizzled offsets of the block's bits
#pragma unroll
    for (int i = 0; i < K; ++i) bitv[i] = swz<V>(1 << op.lq[i]);
    const int nslices = 1 << (m - K);
    const int nrec = op.nrec;
    for (int s = threadIdx.x; s < nslices; s += blockDim.x) {
        int base = s;
#pragma unroll
        for (int i = 0; i < K; ++i) base = (int)insert_zero((uint64_t)base, op.lq[i]);
        base = swz<V>(base);
        V v[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            int o = 0;
#pragma unroll
            for (int i = 0; i < K; ++i)
                if ((j >> i) & 1) o ^= bitv[i];
            v[j] = tile[base ^ o];
        }
        for (int r = 0; r < nrec; ++r) {
            const GateRec g = recs[r];
            switch (g.kind) {
            case GR_U:
                reg_u_any<V, K>(v, g.a, sdata[g.off], sdata[g.off + 1], sdata[g.off + 2], sdata[g.off + 3]);
                break;
            case GR_UR:
                reg_ur_any<V, K, R>(v, g.a, sdata[g.off].x, sdata[g.off + 1].x, sdata[g.off + 2].x,
                                    sdata[g.off + 3].x);
                break;
            case GR_DT:
#pragma unroll
                for (int j = 0; j < D; ++j) v[j] = cmul(sdata[g.off + j], v[j]);
                break;
            case GR_CX: reg_cx_any<V, K>(v, g.a, g.b); break;
            default: reg_swap_any<V, K>(v, g.a, g.b); break;
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            int o = 0;
#pragma unroll
            for (int i = 0; i < K; ++i)
                if ((j >> i) & 1) o ^= bitv[i];
            tile[base ^ o] = v[j];
        }
    }
}

// Diagonal-phase run: psi_x *= exp(2 pi i phase(x)), phase(x) = c + sum_q a_q
// x_q + sum_{p<q} b_pq x_p x_q (turns).  Coefficients arrive as fixed-point
// turns (2^-64 turn units, so integer addition is addition modulo one turn);
// the complex64 path uses the top 32 bits.  For the tile with non-tile bits
// "base" the non-tile part folds into a constant C and per-tile linear
// coefficients a'_t, all in integer arithmetic; the tile-internal quadratic
// part comes precomputed per pass (Qlo, Qhi over the lo/hi halves of the tile
// index, Rt coupling them), so each amplitude costs two integer adds, one
// table lookup, one conversion and one sincos.
template <typename V, typename R>
__device__ __forceinline__ void tile_diag(V* __restrict__ tile, const PassDev& P, uint64_t base,
                                          const uint64_t* __restrict__ dd, R* tabs, uint64_t* s_ap,
                                          uint64_t* s_c) {
    using T = Turns<R>;
    using U = typename T::U;
    const int m = P.m, no = P.nother;
    const DiagLayout Lo(m, no);
    const int h = Lo.h, mh = Lo.mh;
    const int tid = threadIdx.x;
    // a'_t = a_t + sum_o b_to x_o for the tile bits (thread t), and the
    // non-tile constant C = c + sum_o a_o x_o + sum_{o2<o} b_oo2 x_o x_o2
    // (warp 1, one non-tile bit per lane).  Loads are unrolled to the 32-bit
    // bound and predicated so that they are all in flight together.
    if (tid < m) {
        const uint64_t* row = dd + Lo.bo + tid * no;
        U r[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) r[o] = (o < no && ((base >> P.oq[o]) & 1)) ? T::coef(row[o]) : (U)0;
        U v = T::coef(dd[Lo.at + tid]);
#pragma unroll
        for (int o = 0; o < 32; ++o) v += r[o];
        s_ap[tid] = v;
    }
    if (tid >= 32 && tid < 64) {
        const int o = tid - 32;
        const bool set = o < no && ((base >> P.oq[o < no ? o : 0]) & 1);
        U v = 0;
        if (set) {
            const uint64_t* row = dd + Lo.boo + o * no;
            U r[32];
#pragma unroll
            for (int o2 = 0; o2 < 32; ++o2) r[o2] = (o2 < o && ((base >> P.oq[o2]) & 1)) ? T::coef(row[o2]) : (U)0;
            v = T::coef(dd[Lo.ao + o]);
#pragma unroll
            for (int o2 = 0; o2 < 32; ++o2) v += r[o2];
        }
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
        if (o == 0) *s_c = v + T::coef(dd[Lo.c]);
    }
    __syncthreads();
    U* Lhi = reinterpret_cast<U*>(tabs);
    const U cc = (U)*s_c;
    for (int e = tid; e < (1 << mh); e += blockDim.x) {
        U v = T::coef(dd[Lo.qhi + e]) + cc;
        for (int b = 0; b < mh; ++b)
            if ((e >> b) & 1) v += (U)s_ap[h + b];
        Lhi[e] = v;
    }
    // Amplitude i = tid + 256 k: its lo half (tid mod 2^h) is fixed per thread
    // because 2^h divides the 256-thread block, and its hi half is
    // hi0 + k * 2^(8-h).  The lo-hi coupling terms for this lo therefore sit
    // in registers, and the coupling of the k bits is two table entries.
    static_assert(kPassThreads == 256, "diagonal runs assume 256 threads");
    const int lo = tid & ((1 << h) - 1);
    const int sb = 8 - h;  // hi bits fixed per thread
    const int hi0 = tid >> h;
    U ph0 = T::coef(dd[Lo.qlo + lo]);
    for (int b = 0; b < h; ++b)
        if ((lo >> b) & 1) ph0 += (U)s_ap[b];
    for (int t = 0; t < sb && t < mh; ++t)
        if ((hi0 >> t) & 1) ph0 += T::coef(dd[Lo.rt + (t << h) + lo]);
    U Rk[7];  // coupling of bit b of k (hi bit sb + b) with this lo
#pragma unroll
    for (int b = 0; b < 7; ++b) Rk[b] = (sb + b < mh) ? T::coef(dd[Lo.rt + ((sb + b) << h) + lo]) : (U)0;
    U C3[8];  // coupling of the three low bits of k
#pragma unroll
    for (int j = 0; j < 8; ++j)
        C3[j] = ((j & 1) ? Rk[0] : (U)0) + ((j & 2) ? Rk[1] : (U)0) + ((j & 4) ? Rk[2] : (U)0);
    __syncthreads();
    const int K = m >= 8 ? (1 << (m - 8)) : (tid < (1 << m) ? 1 : 0);
    const int stid = swz<V>(tid);  // swz(tid + (k << 8)) = swz(tid) + (k << 8)
    for (int kh = 0; kh < K; kh += 8) {
        U chi = ph0;
#pragma unroll
        for (int b = 3; b < 7; ++b)
            if ((kh >> b) & 1) chi += Rk[b];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = kh + j;
            if (k < K) {
                const int i = stid + (k << 8);
                R sn, cs;
                T::sincos(chi + C3[j] + Lhi[hi0 + (k << sb)], &sn, &cs);
                V f;
                f.x = cs;
                f.y = sn;
                tile[i] = cmul(f, tile[i]);
            }
        }
    }
}

template <typename V>
__device__ __forceinline__ void store_tile(const V* tile, V* __restrict__ psi, uint64_t base, const uint32_t* rowoff,
                                           int m, int L) {
    constexpr int PER = 16 / sizeof(V);
    const int nch = (1 << m) / PER;
    const int rmask = (1 << L) - 1;
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
        const int i = c * PER;
        const uint64_t g = base + ((uint64_t)rowoff[i >> L] << L) + (uint64_t)(i & rmask);
        *(float4*)(psi + g) = *(const float4*)(tile + swz<V>(i));
    }
}

// Shared-memory words (8 bytes) of a diagonal run's per-tile table Lhi.
__host__ __device__ inline int diag_table_elems(int m) {
    const int h = m < 7 ? m : 7;
    return 1 << (m - h);
}

// Tensor-core dense block of K qubits (complex64 only).  The CTA's 256
// threads form two groups of four warps; each group owns 128 TMEM lanes and
// 4*2^K columns (A_hi, A_lo: 2^K each; accumulator: 2^(K+1)).  Lane 2s+c of a
// group holds component c (0 = real, 1 = imaginary) of slice s, so one MMA
// round covers 64 slices per group:
//   acc[(s,c)][n] = sum_j X_c[s][j] B[n][j],  B = [Ur; Ui]  (N = 2^(K+1))
// with 3xTF32 products (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulate),
// and the complex result y_r = (Ur Xr - Ui Xi) + i (Ui Xr + Ur Xi) is formed
// by exchanging accumulator halves between the two lanes of each slice.
template <int K>
__device__ __forceinline__ void tile_dense_tc(float2* __restrict__ tile, int m, const OpDev& op,
                                              const float* __restrict__ sB, uint32_t tmem_base, uint64_t* mbar,
                                              uint32_t* phase, int* s_abort, int* __restrict__ err) {
    constexpr int D = 1 << K;
    constexpr int N = 2 * D;
    constexpr uint32_t IDESC = tc::idesc_tf32(128, N);
    constexpr uint32_t SBO = (uint32_t)(D / 4) * 128u;
    constexpr int CH = D < 16 ? D : 16;  // TMEM columns per load/store
    const int tid = threadIdx.x;
    const int grp = tid >> 7;
    const int row = tid & 127;
    const int c = row & 1;
    const uint32_t col0 = (uint32_t)grp * 4u * D;
    const uint32_t lane_addr = tmem_base + ((uint32_t)(row & ~31) << 16);
    int bitv[K];  // swizzled offsets of the block's bits
#pragma unroll
    for (int i = 0; i < K; ++i) bitv[i] = swz<float2>(1 << op.lq[i]);
    const int nslices = 1 << (m - K);
    float* tw = reinterpret_cast<float*>(tile);
    const uint32_t sb_hi = tc::smem_u32(sB), sb_lo = sb_hi + (uint32_t)(N * D * 4);
    for (int s0 = 0; s0 < nslices; s0 += 128) {
        const int s = s0 + grp * 64 + (row >> 1);
        const bool act = s < nslices;
        int base = s;
#pragma unroll
        for (int i = 0; i < K; ++i) base = (int)insert_zero((uint64_t)base, op.lq[i]);
        base = swz<float2>(base);
#pragma unroll
        for (int j0 = 0; j0 < D; j0 += CH) {
            uint32_t vh[CH], vl[CH];
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) {
                const int j = j0 + jj;
                int o = 0;
#pragma unroll
                for (int i = 0; i < K; ++i)
                    if ((j >> i) & 1) o ^= bitv[i];
                // 3xTF32 split with rounding to nearest, so the products are
                // not biased toward zero (the tensor core itself truncates)
                const float a = act ? tw[2 * (base ^ o) + c] : 0.0f;
                const uint32_t ah = tc::to_tf32(a);
                vh[jj] = ah;
                vl[jj] = tc::to_tf32(a - __uint_as_float(ah));
            }
            if (CH == 16) {
                tc::tmem_st16(lane_addr + col0 + j0, vh);
                tc::tmem_st16(lane_addr + col0 + D + j0, vl);
            } else {
                tc::tmem_st8(lane_addr + col0 + j0, vh);
                tc::tmem_st8(lane_addr + col0 + D + j0, vl);
            }
        }
        tc::tmem_wait_st();
        tc::fence_before();
        tc::named_barrier(1 + grp, 128);
        tc::fence_after();
        if (s_abort[grp]) break;  // uniform across the group (read after the barrier)
        if (row == 0) {
            const uint32_t dcol = tmem_base + col0 + 2 * D, ah = tmem_base + col0, al = tmem_base + col0 + D;
#pragma unroll
            for (int kk = 0; kk < D / 8; ++kk)
                tc::mma_tf32_ts(dcol, ah + 8 * kk, tc::sdesc_noswz(sb_hi + kk * 256, 128, SBO), IDESC, kk > 0);
#pragma unroll
            for (int kk = 0; kk < D / 8; ++kk)
                tc::mma_tf32_ts(dcol, ah + 8 * kk, tc::sdesc_noswz(sb_lo + kk * 256, 128, SBO), IDESC, 1);
#pragma unroll
            for (int kk = 0; kk < D / 8; ++kk)
                tc::mma_tf32_ts(dcol, al + 8 * kk, tc::sdesc_noswz(sb_hi + kk * 256, 128, SBO), IDESC, 1);
            tc::mma_commit(&mbar[grp]);
        }
        const bool ok = tc::mbar_wait_bounded(&mbar[grp], *phase & 1u, 1u << 22);
        *phase += 1;
        tc::fence_after();
        if (!ok) {
            s_abort[grp] = 1;
            atomicExch(err, 1);
            continue;
        }
#pragma unroll
        for (int r0 = 0; r0 < D; r0 += CH) {
            uint32_t own[CH], oth[CH];
            if (CH == 16) {
                tc::tmem_ld16(lane_addr + col0 + 2 * D + r0, own);
                tc::tmem_ld16(lane_addr + col0 + 3 * D + r0, oth);
            } else {
                tc::tmem_ld8(lane_addr + col0 + 2 * D + r0, own);
                tc::tmem_ld8(lane_addr + col0 + 3 * D + r0, oth);
            }
            tc::tmem_wait_ld();
#pragma unroll
            for (int rr = 0; rr < CH; ++rr) {
                const float partner = __shfl_xor_sync(0xffffffffu, __uint_as_float(oth[rr]), 1);
                const float y = __uint_as_float(own[rr]) + (c ? partner : -partner);
                const int r = r0 + rr;
                int o = 0;
#pragma unroll
                for (int i = 0; i < K; ++i)
                    if ((r >> i) & 1) o ^= bitv[i];
                if (act) tw[2 * (base ^ o) + c] = y;
            }
        }
    }
}

// Start the 16-byte copies of a tile (no wait).
template <typename V>
__device__ __forceinline__ void issue_tile(V* tile, const V* __restrict__ psi, uint64_t base, const uint32_t* rowoff,
                                           int m, int L) {
    constexpr int PER = 16 / sizeof(V);
    const int nch = (1 << m) / PER;
    const int rmask = (1 << L) - 1;
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
        const int i = c * PER;
        const uint64_t g = base + ((uint64_t)rowoff[i >> L] << L) + (uint64_t)(i & rmask);
        cp_async16(tile + swz<V>(i), psi + g);
    }
}

template <typename R, bool TC>
__global__ void __launch_bounds__(kPassThreads, 2) k_pass(typename CT<R>::V* __restrict__ psi, int n,
                                                      const PassDev* __restrict__ pdp,
                                                      const unsigned char* __restrict__ blob,
                                                      const float* __restrict__ tcmats, int* __restrict__ err,
                                                      const PassLayout lay) {
    using V = typename CT<R>::V;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ PassDev P;
    __shared__ uint64_t s_ap[kMaxTileM];
    __shared__ uint64_t s_c;
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ int s_abort[2];
    {
        const int* src = (const int*)pdp;
        int* dst = (int*)&P;
        for (int i = threadIdx.x; i < (int)(sizeof(PassDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int m = P.m, L = P.L;
    const int tc_k = TC ? P.tc_k : 0;
    const uint32_t tc_cols = tc_k ? (8u << tc_k) : 0u;  // two groups x 4 * 2^k columns
    if (tc_k) {
        if (threadIdx.x < 32) {
            tc::tmem_alloc(&s_taddr, tc_cols);
            tc::tmem_relinquish();
        }
        if (threadIdx.x == 0) {
            tc::mbar_init(&s_mbar[0], 1);
            tc::mbar_init(&s_mbar[1], 1);
            tc::fence_mbar_init();
            s_abort[0] = s_abort[1] = 0;
        }
        tc::fence_before();
    }
    V* tiles[2] = {(V*)smem, (V*)(smem + (lay.nbuf == 2 ? lay.tile_bytes : 0))};
    uint32_t* rowoff = (uint32_t*)(smem + lay.rowoff_off);
    float* bres = (float*)(smem + lay.bres_off);
    unsigned char* stage = smem + lay.stage_off;
    R* work = (R*)(smem + lay.work_off);
    const unsigned char* greg = blob + P.region_off;
    const int nrows = 1 << (m - L);
    // the pass region (or its OpDev array) and the resident B operands
    for (int e = threadIdx.x; e < lay.stage_bytes / 16; e += blockDim.x) cp_async16(stage + 16 * e, greg + 16 * e);
    const int tc_res = TC ? lay.tc_res : 0;
    if (tc_res) {
        const float* src = tcmats + P.tc_base;
        for (int e = threadIdx.x; e < tc_res / 4; e += blockDim.x) cp_async16(bres + 4 * e, src + 4 * e);
    }
    cp_async_commit();
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        uint32_t o = 0;
        for (int b = 0; b < m - L; ++b)
            if ((r >> b) & 1) o |= 1u << (P.tq[L + b] - L);
        rowoff[r] = o;
    }
    cp_async_wait_group<0>();
    if (tc_res) tc::fence_proxy_async();
    __syncthreads();
    if (tc_k) tc::fence_after();
    const OpDev* opsp = (const OpDev*)(lay.stage_bytes >= P.ops_bytes ? (const unsigned char*)stage : greg);
    const unsigned char* reg = lay.staged ? (const unsigned char*)stage : greg;
    const uint32_t tmem_base = tc_k ? s_taddr : 0u;
    uint32_t phase = 0;
    const uint64_t ntiles = 1ull << (n - m);
    auto tile_base = [&](uint64_t t) {
        uint64_t b = 0;
        for (int i = 0; i < P.nother; ++i) b |= ((t >> i) & 1ull) << P.oq[i];
        return b;
    };
    int cur = 0;
    if (lay.nbuf == 2 && (uint64_t)blockIdx.x < ntiles) {
        issue_tile(tiles[0], psi, tile_base(blockIdx.x), rowoff, m, L);
        cp_async_commit();
    }
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t base = tile_base(t);
        const uint64_t tn = t + gridDim.x;
        if (lay.nbuf == 2) {
            if (tn < ntiles) {
                issue_tile(tiles[cur ^ 1], psi, tile_base(tn), rowoff, m, L);
                cp_async_commit();
                cp_async_wait_group<1>();
            } else {
                cp_async_wait_group<0>();
            }
        } else {
            issue_tile(tiles[0], psi, base, rowoff, m, L);
            cp_async_commit();
            cp_async_wait_group<0>();
        }
        __syncthreads();
        V* tile = tiles[cur];
        for (int oi = 0; oi < P.nops; ++oi) {
            const OpDev& op = opsp[oi];
            const int kind = op.kind;
            if (kind == OP_DENSE && op.tc) {
                if constexpr (TC && sizeof(R) == 4) {
                    const float* sB = bres + (op.tc_off - P.tc_base);
                    if (!tc_res) {  // B operands [hi | lo] of this block into shared memory
                        const int nch = tc_floats(op.k) / 4;
                        const float* src = tcmats + op.tc_off;
                        for (int e = threadIdx.x; e < nch; e += blockDim.x)
                            *(float4*)((float*)work + 4 * e) = *(const float4*)(src + 4 * e);
                        tc::fence_proxy_async();
                        __syncthreads();
                        sB = (const float*)work;
                    }
                    switch (op.k) {
                    case 3: tile_dense_tc<3>(tile, m, op, sB, tmem_base, s_mbar, &phase, s_abort, err); break;
                    case 4: tile_dense_tc<4>(tile, m, op, sB, tmem_base, s_mbar, &phase, s_abort, err); break;
                    default: tile_dense_tc<5>(tile, m, op, sB, tmem_base, s_mbar, &phase, s_abort, err); break;
                    }
                }
            } else if (kind == OP_GATES) {
                const V* sd = (const V*)(reg + op.mat_off);
                const GateRec* sr = (const GateRec*)(reg + op.rec_off);
                if (!lay.staged) {
                    V* wd = (V*)work;
                    GateRec* wr = (GateRec*)(wd + kMaxGateData);
                    for (int e = threadIdx.x; e < op.ndata; e += blockDim.x) wd[e] = sd[e];
                    for (int e = threadIdx.x; e < op.nrec; e += blockDim.x) wr[e] = sr[e];
                    __syncthreads();
                    sd = wd;
                    sr = wr;
                }
                switch (op.k) {  // k <= smem_gates_max_k: 4 (complex64), 3 (complex128)
                case 1: tile_gates<V, 1>(tile, m, op, sr, sd); break;
                case 2: tile_gates<V, 2>(tile, m, op, sr, sd); break;
                case 3: tile_gates<V, 3>(tile, m, op, sr, sd); break;
                default: if constexpr (sizeof(V) == 8) tile_gates<V, 4>(tile, m, op, sr, sd); break;
                }
            } else if (kind == OP_DENSE) {
                const V* sU = (const V*)(reg + op.mat_off);
                if (!lay.staged) {
                    V* wU = (V*)work;
                    const int DD = 1 << (2 * op.k);
                    for (int e = threadIdx.x; e < DD; e += blockDim.x) wU[e] = sU[e];
                    __syncthreads();
                    sU = wU;
                }
                switch (op.k) {
                case 1: tile_dense<V, 1>(tile, m, op, sU); break;
                case 2: tile_dense<V, 2>(tile, m, op, sU); break;
                case 3: tile_dense<V, 3>(tile, m, op, sU); break;
                case 4: tile_dense<V, 4>(tile, m, op, sU); break;
                default: tile_dense<V, 5>(tile, m, op, sU); break;
                }
            } else {
                tile_diag<V, R>(tile, P, base, (const uint64_t*)(reg + op.diag_off), work, s_ap, &s_c);
            }
            __syncthreads();
        }
        store_tile(tile, psi, base, rowoff, m, L);
        __syncthreads();
        if (lay.nbuf == 2) cur ^= 1;
    }
    if (tc_k) {
        tc::fence_before();
        __syncthreads();
        if (threadIdx.x < 32) tc::tmem_dealloc(tmem_base, tc_cols);
    }
}

// Shared memory a pass may stage (its region) and the CTA budget that keeps
// two CTAs per SM when the tile is double-buffered.
constexpr int kTwoCtaBudget = 112 * 1024;
constexpr int kMaxDynSmem = 225 * 1024;  // 227 KB per block less the kernel's static variables
constexpr int kSmemPerSm = 228 * 1024;   // shared memory of one SM

static int round128(size_t v) { return (int)((v + 127) & ~(size_t)127); }

PassLayout pass_layout(int dtype, const PassDev& P) {
    const size_t csz = dtype == SV_C64 ? 8 : 16;
    const size_t usz = dtype == SV_C64 ? 4 : 8;
    const int m = P.m;
    const int nrows = 1 << (m - P.L);
    PassLayout lay;
    lay.tile_bytes = round128(csz << m);
    lay.tc_res = P.tc_res;
    lay.staged = P.region_bytes <= kStageCap;
    // Drop the staged payloads, then the resident B operands, until the CTA
    // fits the per-block shared-memory limit (static variables included).
    for (int attempt = 0; attempt < 3; ++attempt) {
        lay.stage_bytes = lay.staged ? P.region_bytes : (P.ops_bytes <= kStageCap ? P.ops_bytes : 0);
        // work: the diagonal runs' per-tile table, non-resident tensor-core B
        // operands, and without staging the per-op payload copies
        size_t work = usz * (size_t)diag_table_elems(m);
        if (P.tc_k && !lay.tc_res) work = std::max(work, (size_t)tc_floats(P.tc_k) * 4);
        if (!lay.staged) {
            work = std::max(work, csz * (size_t)(1 << (2 * kMaxK)));
            work = std::max(work, csz * kMaxGateData + sizeof(GateRec) * kMaxGateRecs);
        }
        const int rest = round128(4 * (size_t)nrows) + round128(4 * (size_t)lay.tc_res) + round128(lay.stage_bytes) +
                         round128(work);
        lay.nbuf = 2 * lay.tile_bytes + rest <= kTwoCtaBudget ? 2 : 1;
        lay.rowoff_off = lay.nbuf * lay.tile_bytes;
        lay.bres_off = lay.rowoff_off + round128(4 * (size_t)nrows);
        lay.stage_off = lay.bres_off + round128(4 * (size_t)lay.tc_res);
        lay.work_off = lay.stage_off + round128(lay.stage_bytes);
        lay.total = lay.work_off + round128(work);
        if (lay.total <= kMaxDynSmem) break;
        if (attempt == 0) lay.staged = 0;
        else lay.tc_res = 0;
    }
    // Blocks of 5 qubits take 256 TMEM columns per CTA: at most two CTAs may
    // share an SM (512 columns), so such passes ask for enough shared memory
    // to keep a third one away.
    if (P.tc_k >= 5 && lay.total < 80 * 1024) lay.total = 80 * 1024;
    return lay;
}

// Register pass fed by TMA.  The CTA keeps a ring of S tile slots: warp 0
// issues the tensor copies of a tile's rows into a free slot (completion
// counted in bytes on the slot's mbarrier) S-1 tiles ahead, every thread
// works on the oldest loaded slot in registers, and warp 0 writes the slot
// back with tensor stores, whose shared-memory reads are awaited before the
// slot is loaded again.  The copies use the 128-byte swizzle, which places
// each 16-byte chunk exactly where swz() puts it.  All waits are bounded; on
// expiry the kernel records an error, lets its copies in flight land and
// returns.
constexpr int kMaxSlots = 4;
constexpr uint32_t kTmaWaitLimit = 1u << 22;

struct RingLayout {
    int slots;
    int tile_bytes;
    int box_rows;   // rows per tensor copy
    int rowoff_off;
    int stage_off;
    int stage_bytes;
    int work_off;
    int total;
};

template <typename R, int RB, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_rpass_tma(int n, const PassDev* __restrict__ pdp,
                                                       const unsigned char* __restrict__ blob,
                                                       const __grid_constant__ CUtensorMap tmap, const RingLayout lay,
                                                       int* __restrict__ err) {
    using V = typename CT<R>::V;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // slots start on a 1024-byte boundary (the period of the 128-byte swizzle);
    // the layout reserves the kilobyte this may skip
    unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ PassDev P;
    __shared__ __align__(8) uint64_t full[kMaxSlots];
    __shared__ uint32_t tbase[3][256];
    {
        const int* src = (const int*)pdp;
        int* dst = (int*)&P;
        for (int i = threadIdx.x; i < (int)(sizeof(PassDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int m = P.m, L = P.L, nd = P.ndiag, S = lay.slots;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t* rowoff = (uint32_t*)(smem + lay.rowoff_off);
    unsigned char* stage = smem + lay.stage_off;
    uint64_t* fold = (uint64_t*)(smem + lay.work_off);  // nd x (m + 1)
    int* dofs = (int*)(fold + (size_t)nd * (m + 1));
    const unsigned char* greg = blob + P.region_off;
    for (int e = tid; e < lay.stage_bytes / 16; e += blockDim.x) cp_async16(stage + 16 * e, greg + 16 * e);
    cp_async_commit();
    const int nrows = 1 << (m - L);
    for (int r = tid; r < nrows; r += blockDim.x) {
        uint32_t o = 0;
        for (int b = 0; b < m - L; ++b)
            if ((r >> b) & 1) o |= 1u << (P.tq[L + b] - L);
        rowoff[r] = o;
    }
    build_base_tables(tbase, P);
    if (tid == 0) {
        for (int s = 0; s < S; ++s) tc::mbar_init(&full[s], 1);
        tc::fence_mbar_init();
    }
    cp_async_wait_group<0>();
    __syncthreads();
    const OpDev* ops = (const OpDev*)stage;
    if (tid == 0)
        for (int i = 0; i < P.nops; ++i)
            if (ops[i].kind == OP_DIAG) dofs[ops[i].ord] = ops[i].diag_off;
    const uint64_t ntiles = 1ull << (n - m);
    const int nloc = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);  // this CTA's tiles
    const int BR = lay.box_rows, ngroups = nrows / BR;
    auto tile_of = [&](int j) { return (uint64_t)blockIdx.x + (uint64_t)j * gridDim.x; };
    auto row0_of = [&](uint64_t t) { return (int)(table_base(tbase, t, L) >> L); };
    auto issue_load = [&](int j) {  // warp 0: tile j of this CTA into slot j % S
        const int s = j % S;
        if (lane == 0) tma::mbar_arrive_expect_tx(&full[s], (uint32_t)lay.tile_bytes);
        __syncwarp();
        const int row0 = row0_of(tile_of(j));
        unsigned char* dst = smem + (size_t)s * lay.tile_bytes;
        for (int g = lane; g < ngroups; g += 32)
            tma::load_2d(dst + (size_t)g * BR * 128, &tmap, 0, row0 + (int)rowoff[g * BR], &full[s]);
    };
    if (warp == 0)
        for (int j = 0; j < S - 1 && j < nloc; ++j) issue_load(j);
    __syncthreads();  // the expect_tx arrivals precede any wait
    V v[1 << RB];
    RegLayout<V, RB> Lg;
    int done = 0;  // tiles whose slots were consumed
    bool aborted = false;
    for (int j = 0; j < nloc; ++j) {
        const int s = j % S;
        if (warp == 0 && j + S - 1 < nloc) {
            if (j >= 1) tma::store_wait_read();  // the store of tile j-1 has left slot (j+S-1) % S
            __syncwarp();
            issue_load(j + S - 1);
        }
        const bool ok = tc::mbar_wait_bounded(&full[s], (uint32_t)((j / S) & 1), kTmaWaitLimit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            aborted = true;
            break;
        }
        const uint64_t t = tile_of(j);
        V* tile = (V*)(smem + (size_t)s * lay.tile_bytes);
        if (P.ndiag) fold_diags<R>(P, stage, fold, dofs, t);
        TcCtx T0{0u, nullptr, nullptr, err, 0u, nullptr, nullptr};  // (TMA-fed passes carry no tensor-core blocks)
        InterpOps<false>::tile<V, R, RB>(v, tile, P, stage, fold, Lg, nullptr, T0);
        if (P.scale != 1.0) {
            const R sc = (R)P.scale;
#pragma unroll
            for (int k = 0; k < (1 << RB); ++k) {
                v[k].x *= sc;
                v[k].y *= sc;
            }
        }
        __syncthreads();
        reg_write<V, RB>(v, tile, Lg);
        tc::fence_proxy_async();
        __syncthreads();
        if (warp == 0) {
            const int row0 = row0_of(t);
            for (int g = lane; g < ngroups; g += 32)
                tma::store_2d(&tmap, 0, row0 + (int)rowoff[g * BR], (const unsigned char*)tile + (size_t)g * BR * 128);
            tma::store_commit();
        }
        done = j + 1;
    }
    if (warp == 0) {
        tma::store_wait_all();
        if (aborted)  // let the loads already issued land before the CTA's shared memory goes away
            for (int j = done; j < nloc && j < done + S - 1; ++j)
                tc::mbar_wait_bounded(&full[j % S], (uint32_t)((j / S) & 1), kTmaWaitLimit);
    }
}

PassLayout rpass_layout(int dtype, const PassDev& P, bool single) {
    const size_t csz = dtype == SV_C64 ? 8 : 16;
    const int m = P.m;
    const int nrows = 1 << (m - P.L);
    PassLayout lay;
    memset(&lay, 0, sizeof(lay));
    lay.tile_bytes = round128(csz << m);
    lay.staged = 1;
    lay.stage_bytes = P.region_bytes;
    const size_t work = sizeof(uint64_t) * (size_t)P.ndiag * (m + 1) + sizeof(int) * (size_t)P.ndiag;
    const int rest = round128(4 * (size_t)nrows) + round128(lay.stage_bytes) + round128(work);
    // double-buffered while two CTAs per SM still fit; and also when even one
    // single-buffered CTA leaves no room for a second (a pass staging several
    // tensor-core matrices): the SM's only CTA then loads the next tile while
    // it computes the current one
    const bool two_single = lay.tile_bytes + rest <= kTwoCtaBudget;
    lay.nbuf = !single && (2 * lay.tile_bytes + rest <= kTwoCtaBudget ||
                           (!two_single && 2 * lay.tile_bytes + rest + 4096 <= kMaxDynSmem)) ? 2 : 1;
    lay.rowoff_off = lay.nbuf * lay.tile_bytes;
    lay.bres_off = lay.rowoff_off + round128(4 * (size_t)nrows);
    lay.stage_off = lay.bres_off;
    lay.work_off = lay.stage_off + round128(lay.stage_bytes);
    lay.total = lay.work_off + round128(work);
    if (P.tc_k > 0) {
        // a CTA with tensor-core blocks holds 128 TMEM columns per 128 threads
        // for its whole (persistent) run: ask for enough shared memory that no
        // more CTAs share an SM than its 512 columns serve, so no allocation
        // ever waits for a co-resident CTA to finish
        const int groups = std::max(1, (1 << (m - reg_bits(dtype))) >> 7);
        const int fit = std::max(1, 4 / groups);
        const int need = kSmemPerSm / (fit + 1) + 1024;
        if (lay.total < need) lay.total = need;
    }
    return lay;
}

int resident_ctas(int threads, int regs, int smem) {
    const int warps = (threads + 31) / 32;
    const int regs_warp = ((std::max(regs, 1) * 32 + 255) / 256) * 256;  // allocated per warp in units of 256
    const int by_regs = 65536 / std::max(1, regs_warp * warps);
    const int by_smem = kSmemPerSm / std::max(1, smem + 1024);          // 1 KB per CTA reserved by the driver
    const int by_tmem = 4 / std::max(1, threads >> 7);                    // 512 columns, 128 per 128 threads
    const int by_warps = 64 / std::max(1, warps);
    return std::max(1, std::min(std::min(by_regs, by_smem), std::min(by_tmem, by_warps)));
}

// ---------------------------------------------------------------------------
// Batched circuits whose whole state fits one CTA's shared memory (the
// paper's parallel mode of many small circuits, Sec. 2.4): one persistent
// launch; each CTA takes circuits from a work counter, starts from |0...0>,
// applies the circuit's single tile pass (every qubit in the tile), and
// writes <Z_i> and the shots straight from shared memory.  Shots follow the
// library's rule min{x : C_x > u C_{N-1}} with the CDF built over blocks of
// 32 amplitudes in FP64; circuit c (index gidx[c] in the caller's batch)
// draws its uniforms with seed + gidx[c].
// ---------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ double prob_d(V a) {
    const double x = (double)a.x, y = (double)a.y;
    return fma(x, x, y * y);
}

size_t batch_small_smem_bytes(int dtype, int mmax) {
    const size_t csz = dtype == SV_C64 ? 8 : 16;
    const size_t rsz = dtype == SV_C64 ? 4 : 8;
    size_t work = csz * (1 << (2 * kMaxK));
    const size_t dt = rsz * diag_table_elems(mmax);
    if (dt > work) work = dt;
    return (csz << mmax) + work + 8 * 256;
}

template <typename R>
__global__ void __launch_bounds__(kPassThreads) k_batch_small(const PassDev* __restrict__ pd, int C,
                                                             const unsigned char* __restrict__ blob, int mmax,
                                                             uint64_t shots, uint64_t seed,
                                                             const int* __restrict__ gidx,
                                                             uint64_t* __restrict__ samples,
                                                             double* __restrict__ expz, int nmax,
                                                             int* __restrict__ counter) {
    using V = typename CT<R>::V;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ PassDev P;
    __shared__ uint64_t s_ap[kMaxTileM];
    __shared__ uint64_t s_c;
    __shared__ int s_circ;
    __shared__ double s_red[8][kMaxTileM + 2];
    V* tile = (V*)smem;
    R* work = (R*)(smem + (sizeof(V) << mmax));
    double* cdf = (double*)(smem + (sizeof(V) << mmax) +
                            ((size_t)(sizeof(V) << (2 * kMaxK)) > sizeof(R) * diag_table_elems(mmax)
                                 ? (size_t)(sizeof(V) << (2 * kMaxK))
                                 : sizeof(R) * diag_table_elems(mmax)));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_circ = atomicAdd(counter, 1);
        __syncthreads();
        const int c = s_circ;
        if (c >= C) break;
        {
            const int* src = (const int*)(pd + c);
            int* dst = (int*)&P;
            for (int i = tid; i < (int)(sizeof(PassDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        const int m = P.m;  // = the circuit's qubit count
        const int N = 1 << m;
        for (int i = tid; i < N; i += blockDim.x) {
            V v = czero<V>();
            if (i == 0) v.x = 1;
            tile[swz<V>(i)] = v;
        }
        __syncthreads();
        const unsigned char* greg = blob + P.region_off;
        const OpDev* ops = (const OpDev*)greg;
        for (int oi = 0; oi < P.nops; ++oi) {
            const OpDev op = ops[oi];
            if (op.kind == OP_GATES) {
                V* sd = (V*)work;
                GateRec* sr = (GateRec*)(sd + kMaxGateData);
                const V* gd = (const V*)(greg + op.mat_off);
                const GateRec* gr = (const GateRec*)(greg + op.rec_off);
                for (int e = tid; e < op.ndata; e += blockDim.x) sd[e] = gd[e];
                for (int e = tid; e < op.nrec; e += blockDim.x) sr[e] = gr[e];
                __syncthreads();
                switch (op.k) {  // k <= smem_gates_max_k: 4 (complex64), 3 (complex128)
                case 1: tile_gates<V, 1>(tile, m, op, sr, sd); break;
                case 2: tile_gates<V, 2>(tile, m, op, sr, sd); break;
                case 3: tile_gates<V, 3>(tile, m, op, sr, sd); break;
                default: if constexpr (sizeof(V) == 8) tile_gates<V, 4>(tile, m, op, sr, sd); break;
                }
            } else if (op.kind == OP_DENSE) {
                V* sU = (V*)work;
                const int DD = 1 << (2 * op.k);
                const V* gU = (const V*)(greg + op.mat_off);
                for (int e = tid; e < DD; e += blockDim.x) sU[e] = gU[e];
                __syncthreads();
                switch (op.k) {
                case 1: tile_dense<V, 1>(tile, m, op, sU); break;
                case 2: tile_dense<V, 2>(tile, m, op, sU); break;
                case 3: tile_dense<V, 3>(tile, m, op, sU); break;
                case 4: tile_dense<V, 4>(tile, m, op, sU); break;
                default: tile_dense<V, 5>(tile, m, op, sU); break;
                }
            } else {
                tile_diag<V, R>(tile, P, 0ull, (const uint64_t*)(greg + op.diag_off), work, s_ap, &s_c);
            }
            __syncthreads();
        }
        if (expz) {
            double tot = 0.0, sb[kMaxTileM];
#pragma unroll
            for (int b = 0; b < kMaxTileM; ++b) sb[b] = 0.0;
            for (int i = tid; i < N; i += blockDim.x) {
                const double p = prob_d(tile[swz<V>(i)]);
                tot += p;
#pragma unroll
                for (int b = 0; b < kMaxTileM; ++b)
                    if ((i >> b) & 1) sb[b] += p;
            }
#pragma unroll
            for (int b = 0; b <= kMaxTileM; ++b) {
                double v = b < kMaxTileM ? sb[b] : tot;
#pragma unroll
                for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
                if (lane == 0) s_red[warp][b] = v;
            }
            __syncthreads();
            if (tid < m) {
                double s = 0.0, t = 0.0;
                for (int w = 0; w < 8; ++w) {
                    s += s_red[w][tid];
                    t += s_red[w][kMaxTileM];
                }
                expz[(size_t)c * nmax + tid] = t - 2.0 * s;
            }
            __syncthreads();
        }
        if (samples && shots) {
            const int blen = N < 32 ? N : 32;
            const int nblk = N / blen;
            for (int b = warp; b < nblk; b += 8) {
                double p = lane < blen ? prob_d(tile[swz<V>(b * blen + lane)]) : 0.0;
#pragma unroll
                for (int sh = 16; sh > 0; sh >>= 1) p += __shfl_xor_sync(0xffffffffu, p, sh);
                if (lane == 0) cdf[b] = p;
            }
            __syncthreads();
            if (tid == 0) {
                double a = 0.0;
                for (int b = 0; b < nblk; ++b) {
                    a += cdf[b];
                    cdf[b] = a;
                }
            }
            __syncthreads();
            const double S = cdf[nblk - 1];
            for (uint64_t s = tid; s < shots; s += blockDim.x) {
                const double t = philox_uniform(seed + (uint64_t)gidx[c], s) * S;
                int lo = 0, hi = nblk - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cdf[mid] > t) hi = mid;
                    else lo = mid + 1;
                }
                double acc = lo ? cdf[lo - 1] : 0.0;
                int pick = -1, last_nz = lo * blen;
                for (int l = 0; l < blen; ++l) {
                    const double p = prob_d(tile[swz<V>(lo * blen + l)]);
                    if (p > 0.0) last_nz = lo * blen + l;
                    acc += p;
                    if (acc > t && p > 0.0) {
                        pick = lo * blen + l;
                        break;
                    }
                }
                samples[(size_t)c * shots + s] = (uint64_t)(pick >= 0 ? pick : last_nz);
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_batch_small(int dtype, const void* blob_dev, const PlanBlob& blob, int C, int mmax,
                               uint64_t shots, uint64_t seed, const int* gidx, uint64_t* samples, double* expz,
                               int nmax, int* counter, cudaStream_t st) {
    const size_t smem = batch_small_smem_bytes(dtype, mmax);
    const unsigned char* b = (const unsigned char*)blob_dev;
    int per_sm = 1;
    cudaError_t e;
    if (dtype == SV_C64) {
        e = cudaFuncSetAttribute(k_batch_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_small<float>, kPassThreads, smem);
    } else {
        e = cudaFuncSetAttribute(k_batch_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_small<double>, kPassThreads, smem);
    }
    if (per_sm < 1) per_sm = 1;
    const int sms = device_sms();
    int grid = sms * per_sm;
    if (grid > C) grid = C;
    count_launch();
    if (dtype == SV_C64)
        k_batch_small<float><<<grid, kPassThreads, smem, st>>>(
            (const PassDev*)(b + blob.pass_off), C, b, mmax, shots, seed, gidx,
            samples, expz, nmax, counter);
    else
        k_batch_small<double><<<grid, kPassThreads, smem, st>>>(
            (const PassDev*)(b + blob.pass_off), C, b, mmax, shots, seed, gidx,
            samples, expz, nmax, counter);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
namespace {
int num_sms() { return device_sms(); }
unsigned grid_for(uint64_t items, int per_thread = UNR) {
    const uint64_t want = (items + (uint64_t)256 * per_thread - 1) / ((uint64_t)256 * per_thread);
    const uint64_t cap = (uint64_t)num_sms() * 16;
    uint64_t g = want < cap ? want : cap;
    return (unsigned)(g ? g : 1);
}
}  // namespace
int num_sms_pub() { return num_sms(); }

cudaError_t launch_init_basis(sv_state* h, uint64_t x) {
    const uint64_t N = 1ull << h->n;
    count_launch();
    if (h->dtype == SV_C64)
        k_init_basis<float2><<<grid_for(N, 1), 256, 0, h->stream>>>((float2*)h->amps, N, x);
    else
        k_init_basis<double2><<<grid_for(N, 1), 256, 0, h->stream>>>((double2*)h->amps, N, x);
    return cudaGetLastError();
}

template <typename V>
static cudaError_t plain_op_t(sv_state* h, const PlainOp& op) {
    V* psi = (V*)h->amps;
    const int n = h->n;
    const uint64_t N = 1ull << n;
    cudaStream_t st = h->stream;
    count_launch();
    switch (op.kind) {
    case PK_1Q:
        k_plain_1q<V><<<grid_for(N / 2), 256, 0, st>>>(psi, N / 2, op.q0, to_dev<V>(op.m[0]), to_dev<V>(op.m[1]),
                                                       to_dev<V>(op.m[2]), to_dev<V>(op.m[3]));
        break;
    case PK_CX: {
        const int lo = op.q0 < op.q1 ? op.q0 : op.q1, hi = op.q0 < op.q1 ? op.q1 : op.q0;
        const uint64_t A = 1ull << op.q0, B = A | (1ull << op.q1);
        k_plain_swap<V><<<grid_for(N / 4), 256, 0, st>>>(psi, N / 4, lo, hi, A, B);
        break;
    }
    case PK_SWAP: {
        const int lo = op.q0 < op.q1 ? op.q0 : op.q1, hi = op.q0 < op.q1 ? op.q1 : op.q0;
        k_plain_swap<V><<<grid_for(N / 4), 256, 0, st>>>(psi, N / 4, lo, hi, 1ull << op.q0, 1ull << op.q1);
        break;
    }
    case PK_CPHASE: {
        const int lo = op.q0 < op.q1 ? op.q0 : op.q1, hi = op.q0 < op.q1 ? op.q1 : op.q0;
        k_plain_phase<V><<<grid_for(N / 4), 256, 0, st>>>(psi, N / 4, lo, hi, (1ull << lo) | (1ull << hi),
                                                          to_dev<V>(op.m[0]));
        break;
    }
    case PK_PHASE1:
        k_plain_phase<V><<<grid_for(N / 2), 256, 0, st>>>(psi, N / 2, op.q0, op.q0, 1ull << op.q0,
                                                          to_dev<V>(op.m[0]));
        break;
    case PK_DIAG1:
        k_plain_diag1<V><<<grid_for(N), 256, 0, st>>>(psi, N, op.q0, to_dev<V>(op.m[0]), to_dev<V>(op.m[1]));
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_op(sv_state* h, const PlainOp& op) {
    if (h->dtype == SV_C64) return plain_op_t<float2>(h, op);
    return plain_op_t<double2>(h, op);
}

template <typename R, bool TC>
static cudaError_t pass_t(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass, const HostPass& hp) {
    using V = typename CT<R>::V;
    const int m = (int)hp.tile.size();
    const PassDev* pdh = (const PassDev*)(blob.bytes.data() + blob.pass_off) + pass;
    const PassLayout lay = pass_layout(h->dtype, *pdh);
    static int attr_bytes = 0;  // dynamic shared memory the kernel is currently allowed
    if (lay.total > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_pass<R, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total);
        if (e != cudaSuccess) return e;
        attr_bytes = lay.total;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass<R, TC>, kPassThreads, lay.total);
    if (per_sm < 1) per_sm = 1;
    if (TC && pdh->tc_k >= 5 && per_sm > 2) per_sm = 2;  // 256 TMEM columns per CTA
    const uint64_t ntiles = 1ull << (h->n - m);
    uint64_t grid = (uint64_t)num_sms() * per_sm;
    if (grid > ntiles) grid = ntiles;
    const unsigned char* b = (const unsigned char*)blob_dev;
    count_launch();
    k_pass<R, TC><<<(unsigned)grid, kPassThreads, lay.total, h->stream>>>(
        (V*)h->amps, h->n, (const PassDev*)(b + blob.pass_off) + pass, b, (const float*)(b + blob.tc_off),
        (int*)h->err.ptr, lay);
    return cudaGetLastError();
}

template <typename R, int RB, int MAXT, int MINB, bool TC>
static cudaError_t rpass_t(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass) {
    using V = typename CT<R>::V;
    const PassDev* pdh = (const PassDev*)(blob.bytes.data() + blob.pass_off) + pass;
    const PassLayout lay = rpass_layout(h->dtype, *pdh);
    if (lay.total > kMaxDynSmem) return cudaErrorInvalidValue;
    static int attr_bytes = 0;
    if (lay.total > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_rpass<R, RB, MAXT, MINB, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             lay.total);
        if (e != cudaSuccess) return e;
        attr_bytes = lay.total;
    }
    const int threads = 1 << (pdh->m - RB);
    if (threads > MAXT) return cudaErrorInvalidValue;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rpass<R, RB, MAXT, MINB, TC>, threads, lay.total);
    if (per_sm < 1) per_sm = 1;
    if (TC) {  // (see resident_ctas: the query counts one CTA per SM for kernels with TMEM allocations)
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k_rpass<R, RB, MAXT, MINB, TC>) == cudaSuccess)
            per_sm = std::max(per_sm, resident_ctas(threads, fa.numRegs, (int)fa.sharedSizeBytes + lay.total));
    }
    const uint64_t ntiles = 1ull << (h->n - pdh->m);
    uint64_t grid = (uint64_t)num_sms() * per_sm;
    if (grid > ntiles) grid = ntiles;
    const unsigned char* b = (const unsigned char*)blob_dev;
    count_launch();
    k_rpass<R, RB, MAXT, MINB, TC><<<(unsigned)grid, threads, lay.total, h->stream>>>(
        (V*)h->amps, h->n, (const PassDev*)(b + blob.pass_off) + pass, b, lay, (int*)h->err.ptr);
    return cudaGetLastError();
}

template <typename R, int RB, bool TC>
static cudaError_t rpass_tc(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass, int m) {
    const int tb = m - RB;
    if (tb <= 7) return rpass_t<R, RB, 128, 2, TC>(h, blob_dev, blob, pass);
    if (tb == 8) return rpass_t<R, RB, 256, 2, TC>(h, blob_dev, blob, pass);
    return rpass_t<R, RB, 512, 1, TC>(h, blob_dev, blob, pass);
}
// Passes with tensor-core blocks run the instance that holds the TMEM code.
template <typename R, int RB>
static cudaError_t rpass_any(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass, int m) {
    const PassDev* pdh = (const PassDev*)(blob.bytes.data() + blob.pass_off) + pass;
    if constexpr (sizeof(R) == 4 && RB == 5)
        if (pdh->tc_k > 0) return rpass_tc<R, RB, true>(h, blob_dev, blob, pass, m);
    return rpass_tc<R, RB, false>(h, blob_dev, blob, pass, m);
}

// ---------------------------------------------------------------------------
// Persistent executor of a wave of circuits (the paper's parallel mode of
// many circuits, Sec. 2.4; see WaveItem).  A CTA takes items from a device
// counter in order, waits until the item's circuit has finished its earlier
// passes (the per-circuit counter of finished items reaches `need`; bounded),
// stages the pass's region when the pass changes, runs its tiles (or
// multiplexor columns) and counts the item finished.  An item only ever waits
// for items of smaller index, which CTAs that are running hold, so the queue
// cannot deadlock; a wait that gives up sets *err = 2 and every CTA stops.
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Multiplexor columns of an item.
template <typename T, typename V>
__device__ __forceinline__ void wave_mux(const unsigned char* __restrict__ region, V* __restrict__ psi, uint64_t lo,
                                      uint64_t hi) {
    const MuxDev& D = *(const MuxDev*)region;
    switch (D.K) {
    case 1: mux_columns<T, V, 1>(D, region, psi, lo, hi, threadIdx.x, blockDim.x); break;
    case 2: mux_columns<T, V, 2>(D, region, psi, lo, hi, threadIdx.x, blockDim.x); break;
    case 3: mux_columns<T, V, 3>(D, region, psi, lo, hi, threadIdx.x, blockDim.x); break;
    case 4: mux_columns<T, V, 4>(D, region, psi, lo, hi, threadIdx.x, blockDim.x); break;
    default: mux_columns<T, V, 5>(D, region, psi, lo, hi, threadIdx.x, blockDim.x); break;
    }
}

// MUX: the instance for waves with multiplexor passes.  One CTA per SM: the
// interpreting tile body and the 2^K-amplitude columns keep their registers
// (measured: at two CTAs per SM the spills' local-memory traffic outweighed
// the state's).  The other instance runs two CTAs per SM: its spills stay in
// L1, and at one CTA per SM a sweep of 4096 20-qubit circuits ran 1.24x
// slower.
template <typename R, int RB, bool MUX>
__global__ void __launch_bounds__(256, MUX ? 1 : 2) k_wave(typename CT<R>::V* __restrict__ base, const uint64_t* __restrict__ offs,
                                                 const int* __restrict__ nq, const unsigned char* __restrict__ blob,
                                                 const PassDev* __restrict__ pds, const WaveItem* __restrict__ items,
                                                 int nitems, int* __restrict__ head, int* __restrict__ done,
                                                 int* __restrict__ err, const PassLayout lay, unsigned limit) {
    using V = typename CT<R>::V;
    using T = decltype(V().x);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ PassDev P;
    __shared__ uint32_t tbase[3][256];
    __shared__ double2 ttab[sizeof(R) == 8 ? 256 : 1];
    __shared__ int s_item, s_stop, s_staged;
    V* tile = (V*)smem;
    uint32_t* rowoff = (uint32_t*)(smem + lay.rowoff_off);
    unsigned char* stage = smem + lay.stage_off;
    uint64_t* fold = (uint64_t*)(smem + lay.work_off);
    const int tid = threadIdx.x;
    if (tid == 0) s_staged = -1;
    if constexpr (sizeof(R) == 8) build_turn_table(ttab);
    TcCtx T0{0u, nullptr, nullptr, err, 0u, nullptr, nullptr};
    V v[1 << RB];
    RegLayout<V, RB> Lg;
    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(head, 1);
            s_stop = 0;
            if (s_item < nitems) {
                const WaveItem& I = items[s_item];
                if (I.need > 0) {
                    unsigned k = 0;
                    while (ld_acquire(&done[I.circ]) < I.need && ld_acquire(err) == 0) {
                        if (++k > limit) {
                            atomicExch(err, 2);
                            break;
                        }
                        __nanosleep(128);
                    }
                }
                if (ld_acquire(err) != 0) s_stop = 1;
            }
        }
        __syncthreads();
        const int it = s_item;
        if (it >= nitems || s_stop) break;
        const WaveItem I = items[it];
        V* psi = base + offs[I.circ];
        if (I.kind == 1) {  // multiplexor columns
            if constexpr (MUX) wave_mux<T, V>(blob + pds[I.pass].region_off, psi, I.lo, I.hi);
        } else {
            if (I.pass != s_staged) {  // stage the pass: record, region, row offsets, base tables
                __syncthreads();
                const int* src = (const int*)(pds + I.pass);
                int* dst = (int*)&P;
                for (int i = tid; i < (int)(sizeof(PassDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
                __syncthreads();
                const unsigned char* greg = blob + P.region_off;
                for (int e = tid; e < P.region_bytes / 16; e += blockDim.x) cp_async16(stage + 16 * e, greg + 16 * e);
                cp_async_commit();
                const int nrows = 1 << (P.m - P.L);
                for (int r = tid; r < nrows; r += blockDim.x) {
                    uint32_t o = 0;
                    for (int b = 0; b < P.m - P.L; ++b)
                        if ((r >> b) & 1) o |= 1u << (P.tq[P.L + b] - P.L);
                    rowoff[r] = o;
                }
                build_base_tables(tbase, P);
                cp_async_wait_group<0>();
                __syncthreads();
                if (tid == 0) s_staged = I.pass;
            }
            const OpDev* ops = (const OpDev*)stage;
            int* dofs = (int*)(fold + (size_t)P.ndiag * (P.m + 1));
            if (tid == 0)
                for (int i = 0; i < P.nops; ++i)
                    if (ops[i].kind == OP_DIAG) dofs[ops[i].ord] = ops[i].diag_off;
            __syncthreads();
            for (uint64_t t = I.lo; t < I.hi; ++t) {
                const uint64_t b = table_base(tbase, t, P.L);
                rissue_tile(tile, psi, b, rowoff, P.L);
                cp_async_commit();
                cp_async_wait_group<0>();
                __syncthreads();
                if (P.ndiag) fold_diags<R>(P, stage, fold, dofs, t);
                InterpOps<false>::tile<V, R, RB>(v, tile, P, stage, fold, Lg, sizeof(R) == 8 ? ttab : nullptr, T0);
                InterpOps<false>::finish<V, R, RB>(v, tile, P, Lg, T0);
                __syncthreads();
                rstore_tile(tile, psi, b, rowoff, P.L);
                __syncthreads();
            }
        }
        __syncthreads();
        if (tid == 0) {  // the item's writes before the count (release)
            __threadfence();
            atomicAdd(&done[I.circ], 1);
        }
    }
}
}  // namespace

namespace {
// |0...0> for every circuit of a wave (the buffer zeroed beforehand).
template <typename V> __global__ void k_wave_init(V* __restrict__ base, const uint64_t* __restrict__ offs, int C) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) base[offs[c]].x = 1;
}
}  // namespace

cudaError_t launch_wave_init(int dtype, void* base, const uint64_t* offs, int C, cudaStream_t st) {
    count_launch();
    const unsigned g = (unsigned)((C + 127) / 128);
    if (dtype == SV_C64) k_wave_init<float2><<<g, 128, 0, st>>>((float2*)base, offs, C);
    else k_wave_init<double2><<<g, 128, 0, st>>>((double2*)base, offs, C);
    return cudaGetLastError();
}

PassLayout wave_layout(int dtype, const PlanBlob& blob) {
    PassLayout lay;
    memset(&lay, 0, sizeof(lay));
    const size_t csz = dtype == SV_C64 ? 8 : 16;
    int m = 0, nrows = 1, region = 16, work = 16;
    for (int p = 0; p < blob.npasses; ++p) {
        const PassDev& P = ((const PassDev*)(blob.bytes.data() + blob.pass_off))[p];
        if (P.rmode != 1) continue;
        m = std::max(m, P.m);
        nrows = std::max(nrows, 1 << (P.m - P.L));
        region = std::max(region, P.region_bytes);
        work = std::max(work, (int)(sizeof(uint64_t) * (size_t)P.ndiag * (P.m + 1) + sizeof(int) * (size_t)P.ndiag));
    }
    lay.nbuf = 1;
    lay.tile_bytes = round128(csz << m);
    lay.rowoff_off = lay.tile_bytes;
    lay.bres_off = lay.rowoff_off + round128(4 * (size_t)nrows);
    lay.stage_off = lay.bres_off;
    lay.stage_bytes = region;
    lay.staged = 1;
    lay.work_off = lay.stage_off + round128(region);
    lay.total = lay.work_off + round128(work);
    return lay;
}

template <typename R, int RB, bool MUX>
static cudaError_t wave_t(void* base, const uint64_t* offs, const int* nq, const unsigned char* b, const PassDev* pds,
                          const WaveItem* items, int nitems, int* head, int* done, int* err, const PassLayout& lay,
                          unsigned limit, cudaStream_t st) {
    int per_sm = 1;
    cudaError_t e = cudaFuncSetAttribute(k_wave<R, RB, MUX>, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total);
    if (e == cudaSuccess) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wave<R, RB, MUX>, 256, lay.total);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int grid = std::max(1, std::min(num_sms() * per_sm, nitems));
    count_launch();
    k_wave<R, RB, MUX><<<grid, 256, lay.total, st>>>((typename CT<R>::V*)base, offs, nq, b, pds, items, nitems, head,
                                                    done, err, lay, limit);
    return cudaGetLastError();
}

cudaError_t launch_wave(int dtype, void* base, const uint64_t* offs, const int* nq, const void* blob_dev,
                        const PlanBlob& blob, const WaveItem* items, int nitems, int* head, int* done, int* err,
                        unsigned limit, cudaStream_t st) {
    const PassLayout lay = wave_layout(dtype, blob);
    if (lay.total > kMaxDynSmem) return cudaErrorInvalidValue;
    const unsigned char* b = (const unsigned char*)blob_dev;
    const PassDev* pds = (const PassDev*)(b + blob.pass_off);
    bool mux = false;
    for (int p = 0; p < blob.npasses; ++p)
        mux |= ((const PassDev*)(blob.bytes.data() + blob.pass_off))[p].rmode == kRmodeMux;
    if (dtype == SV_C64) {
        if (mux) return wave_t<float, 5, true>(base, offs, nq, b, pds, items, nitems, head, done, err, lay, limit, st);
        return wave_t<float, 5, false>(base, offs, nq, b, pds, items, nitems, head, done, err, lay, limit, st);
    }
    if (mux) return wave_t<double, 4, true>(base, offs, nq, b, pds, items, nitems, head, done, err, lay, limit, st);
    return wave_t<double, 4, false>(base, offs, nq, b, pds, items, nitems, head, done, err, lay, limit, st);
}

// ---- TMA-fed register passes: tensor map and ring layout -----------------
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    }
    return fn;
}

// Rows of 128 bytes (2^L amplitudes) per tensor copy: the run of tile qubits
// L, L+1, ... makes consecutive tile rows consecutive in global memory.
int box_rows(const PassDev& P) {
    int run = 0;
    while (P.L + run < P.m && P.tq[P.L + run] == P.L + run) ++run;
    return 1 << std::min(run, 8);
}
}  // namespace

// The ring: as many slots (2..4) as keep the most warps per SM busy.
static bool ring_layout(int dtype, const PassDev& P, RingLayout* out, int* ctas_per_sm) {
    const size_t csz = dtype == SV_C64 ? 8 : 16;
    const int m = P.m, nrows = 1 << (m - P.L), threads = 1 << (m - reg_bits(dtype));
    RingLayout lay;
    memset(&lay, 0, sizeof(lay));
    lay.tile_bytes = (int)(csz << m);
    if (lay.tile_bytes % 1024) return false;  // slots must stay 1024-byte aligned for the swizzle
    lay.box_rows = std::min(box_rows(P), nrows);
    lay.stage_bytes = P.region_bytes;
    const size_t work = sizeof(uint64_t) * (size_t)P.ndiag * (m + 1) + sizeof(int) * (size_t)P.ndiag;
    const int rest = round128(4 * (size_t)nrows) + round128(lay.stage_bytes) + round128(work) + 1024;
    int best_score = -1;
    for (int S = kMaxSlots; S >= 2; --S) {
        const int total = S * lay.tile_bytes + rest;
        if (total > kMaxDynSmem) continue;
        const int ctas = std::max(1, std::min(8, (228 * 1024) / (total + 1024)));
        const int warps = std::min(16, ctas * threads / 32);
        const int score = warps * 8 + S;
        if (score > best_score) {
            best_score = score;
            lay.slots = S;
            *ctas_per_sm = ctas;
        }
    }
    if (best_score < 0) return false;
    lay.rowoff_off = lay.slots * lay.tile_bytes;
    lay.stage_off = lay.rowoff_off + round128(4 * (size_t)nrows);
    lay.work_off = lay.stage_off + round128(lay.stage_bytes);
    lay.total = lay.work_off + round128(work) + 1024;  // + alignment of the slots
    *out = lay;
    return true;
}

template <typename R, int RB, int MAXT>
static cudaError_t rpass_tma_t(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass, bool* used) {
    *used = false;
    const PassDev* pdh = (const PassDev*)(blob.bytes.data() + blob.pass_off) + pass;
    RingLayout lay;
    int ctas = 1;
    EncodeTiledFn enc = encode_fn();
    // the tensor map's rows are 128 bytes: passes with other row widths stay
    // on the copy-based kernel
    if (pdh->L != (h->dtype == SV_C64 ? 4 : 3)) return cudaSuccess;
    if (!enc || !ring_layout(h->dtype, *pdh, &lay, &ctas)) return cudaSuccess;
    const int threads = 1 << (pdh->m - RB);
    if (threads > MAXT || ((uintptr_t)h->amps & 15)) return cudaSuccess;
    const size_t csz = h->dtype == SV_C64 ? 8 : 16;
    CUtensorMap tmap;
    const cuuint64_t dims[2] = {16, (cuuint64_t)((csz << h->n) / 128)};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {16, (cuuint32_t)lay.box_rows};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, h->amps, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return cudaSuccess;  // not expressible: the caller falls back to the copy-based kernel
    static int attr_bytes = 0;
    if (lay.total > attr_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_rpass_tma<R, RB, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             lay.total);
        if (e != cudaSuccess) return e;
        attr_bytes = lay.total;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rpass_tma<R, RB, MAXT>, threads, lay.total);
    if (per_sm < 1) per_sm = 1;
    const uint64_t ntiles = 1ull << (h->n - pdh->m);
    uint64_t grid = (uint64_t)num_sms() * per_sm;
    if (grid > ntiles) grid = ntiles;
    const unsigned char* b = (const unsigned char*)blob_dev;
    count_launch();
    k_rpass_tma<R, RB, MAXT><<<(unsigned)grid, threads, lay.total, h->stream>>>(
        h->n, (const PassDev*)(b + blob.pass_off) + pass, b, tmap, lay, (int*)h->err.ptr);
    *used = true;
    return cudaGetLastError();
}

template <typename R, int RB>
static cudaError_t rpass_tma_any(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass, int m, bool* used) {
    const int tb = m - RB;
    if (tb <= 7) return rpass_tma_t<R, RB, 128>(h, blob_dev, blob, pass, used);
    if (tb == 8) return rpass_tma_t<R, RB, 256>(h, blob_dev, blob, pass, used);
    return rpass_tma_t<R, RB, 512>(h, blob_dev, blob, pass, used);
}

cudaError_t launch_pass(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass, const HostPass& hp) {
    const PassDev* pdh = (const PassDev*)(blob.bytes.data() + blob.pass_off) + pass;
    if (pdh->rmode == kRmodeMux) return launch_mux(h, blob_dev, blob, pass);
    if (pdh->rmode) {
        bool used = false;
        cudaError_t e = cudaSuccess;
        if (pdh->rmode == 2) {  // the TMA-fed register kernel was asked for
            e = h->dtype == SV_C64 ? rpass_tma_any<float, 5>(h, blob_dev, blob, pass, pdh->m, &used)
                                   : rpass_tma_any<double, 4>(h, blob_dev, blob, pass, pdh->m, &used);
            if (e != cudaSuccess || used) return e;
        }
        if (h->dtype == SV_C64) return rpass_any<float, 5>(h, blob_dev, blob, pass, pdh->m);
        return rpass_any<double, 4>(h, blob_dev, blob, pass, pdh->m);
    }
    if (h->dtype == SV_C64) {
        if (pdh->tc_k) return pass_t<float, true>(h, blob_dev, blob, pass, hp);
        return pass_t<float, false>(h, blob_dev, blob, pass, hp);
    }
    return pass_t<double, false>(h, blob_dev, blob, pass, hp);
}

}  // namespace sv
