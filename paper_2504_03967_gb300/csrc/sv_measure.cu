// Read-out kernels: FP64 probability block sums, the block CDF scan, the shot
// sampler, <Z_i> and full probabilities.
//
// Sampling (Sec. 3: shots per circuit) draws outcome = min{x : C_x > u S},
// C the inclusive CDF of p_x = |a_x|^2 and S = C_{N-1}: a binary search over
// the FP64 block CDF finds the block, then one warp rescans that block's
// 2^B amplitudes in FP64, 32 consecutive amplitudes per step (a coalesced
// load, a warp scan on top of the running CDF, a ballot for the first lane
// above u S).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "sv_internal.h"
#include "sv_philox.cuh"

namespace sv {

namespace {
constexpr int kBlogMax = 10;  // 1024 amplitudes per probability block

template <typename V> __device__ __forceinline__ double prob(V a) {
    const double x = (double)a.x, y = (double)a.y;
    return fma(x, x, y * y);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// ---- block statistics: totals and within-block bit sums in one pass ------
// One warp per block of 2^blog amplitudes; lane l takes amplitudes l + 32 j,
// so index bits 0..4 are the lane and bits 5..9 the loop counter j.  For
// complex64, |a|^2 is formed exactly as an unevaluated float pair (products
// by fma, the sum by TwoSum) and accumulated in double-float, so the FP64
// block value carries the same information as an FP64 sum, at FP32 speed
// (this GPU's FP64 rate is a small fraction of its FP32 rate).  complex128
// accumulates in FP64.  bits (optional, nblocks x 10) receives, for each
// block, the probability mass with index bit i set, i < min(blog, 10).
struct FF {
    float hi, lo;
};
__device__ __forceinline__ void ff_add(FF& a, float x, float xl) {
    const float s = a.hi + x;
    const float bb = s - a.hi;
    a.lo += ((a.hi - (s - bb)) + (x - bb)) + xl;
    a.hi = s;
}
__device__ __forceinline__ double ff_val(FF a) { return (double)a.hi + (double)a.lo; }
// A double as a float pair (hi + lo carries about 48 of its bits).
__device__ __forceinline__ FF ff_of(double d) {
    const float h = (float)d;
    return FF{h, (float)(d - (double)h)};
}
// |a|^2 of a complex64 amplitude as an unevaluated float pair: the squares
// exactly by fma, their sum by TwoSum.
__device__ __forceinline__ FF ff_prob(float2 v) {
    const float r2 = v.x * v.x, r2e = fmaf(v.x, v.x, -r2);
    const float i2 = v.y * v.y, i2e = fmaf(v.y, v.y, -i2);
    const float sum = r2 + i2, bb = sum - r2;
    return FF{sum, ((r2 - (sum - bb)) + (i2 - bb)) + r2e + i2e};
}
// Sum over the warp in double-float (every lane gets it); no FP64 instruction.
__device__ __forceinline__ FF ff_allreduce(FF a) {
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, a.hi, sh), l = __shfl_xor_sync(0xffffffffu, a.lo, sh);
        ff_add(a, h, l);
    }
    return a;
}

// Full 1024-amplitude blocks of complex64 with bit sums.  Lane l holds
// p_j = |a|^2 of amplitudes l + 32 j as float pairs; a pairwise tree over j
// gives the lane's total and its sums over j with bit b set (57 double-float
// additions for 32 amplitudes), and one reduce-scatter across the warp sums
// the 11 per-lane values (total, total where lane bit b is set, the 5 j-bit
// sums): each of the first four exchange steps halves the values a lane
// keeps, so lane 2e (e < 11) ends with value e summed over all 32 lanes.
__device__ __forceinline__ void block_stats_c64_full(const float2* __restrict__ psi, uint64_t wid, int lane,
                                                     double* __restrict__ tot, double* __restrict__ bits) {
    const uint64_t b0 = wid << 10;
    FF p[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const float2 v = psi[b0 + lane + 32 * j];
        const float r2 = v.x * v.x, r2e = fmaf(v.x, v.x, -r2);
        const float i2 = v.y * v.y, i2e = fmaf(v.y, v.y, -i2);
        const float sum = r2 + i2, bb = sum - r2;
        p[j].hi = sum;
        p[j].lo = ((r2 - (sum - bb)) + (i2 - bb)) + r2e + i2e;
    }
    FF e[16];
#pragma unroll
    for (int lev = 0; lev < 5; ++lev) {
        const int half = 16 >> lev;
        FF odd = p[1];
#pragma unroll
        for (int i = 1; i < half; ++i) ff_add(odd, p[2 * i + 1].hi, p[2 * i + 1].lo);
        e[6 + lev] = odd;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            FF t = p[2 * i];
            ff_add(t, p[2 * i + 1].hi, p[2 * i + 1].lo);
            p[i] = t;
        }
    }
    e[0] = p[0];
#pragma unroll
    for (int b = 0; b < 5; ++b) e[1 + b] = ((lane >> b) & 1) ? p[0] : FF{0.f, 0.f};
#pragma unroll
    for (int k = 11; k < 16; ++k) e[k] = FF{0.f, 0.f};
#pragma unroll
    for (int st = 0; st < 4; ++st) {  // lane bits 4, 3, 2, 1
        const int h = 8 >> st, mask = 16 >> st;
        const bool up = (lane & mask) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const FF send = up ? e[k] : e[k + h];
            FF keep = up ? e[k + h] : e[k];
            const float rh = __shfl_xor_sync(0xffffffffu, send.hi, mask);
            const float rl = __shfl_xor_sync(0xffffffffu, send.lo, mask);
            ff_add(keep, rh, rl);
            e[k] = keep;
        }
    }
    ff_add(e[0], __shfl_xor_sync(0xffffffffu, e[0].hi, 1), __shfl_xor_sync(0xffffffffu, e[0].lo, 1));
    const int idx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    if (!(lane & 1) && idx < 11) {
        const double val = ff_val(e[0]);
        if (idx == 0) tot[wid] = val;
        else bits[wid * 10 + (idx - 1)] = val;  // 1..5: lane bits 0..4; 6..10: j bits = index bits 5..9
    }
}

template <typename V>
__global__ void __launch_bounds__(256) k_block_stats(const V* __restrict__ psi, int blog, uint64_t nblocks,
                                                     double* __restrict__ tot, double* __restrict__ bits) {
    const int lane = threadIdx.x & 31;
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= nblocks) return;
    const uint64_t b0 = wid << blog;
    const int len = 1 << blog;
    const int jn = len >= 32 ? len / 32 : 1;
    if constexpr (sizeof(V) == 8) {
        if (bits && blog == 10) {
            block_stats_c64_full((const float2*)psi, wid, lane, tot, bits);
            return;
        }
        FF acc = {0.f, 0.f}, ab[5];
#pragma unroll
        for (int b = 0; b < 5; ++b) ab[b] = FF{0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j < jn && lane + 32 * j < len) {
                const V v = psi[b0 + lane + 32 * j];
                const float r2 = v.x * v.x, r2e = fmaf(v.x, v.x, -r2);
                const float i2 = v.y * v.y, i2e = fmaf(v.y, v.y, -i2);
                const float s = r2 + i2, bb = s - r2;
                const float sl = ((r2 - (s - bb)) + (i2 - bb)) + r2e + i2e;
                ff_add(acc, s, sl);
#pragma unroll
                for (int b = 0; b < 5; ++b)
                    if ((j >> b) & 1) ff_add(ab[b], s, sl);
            }
        }
        // Warp sums in double-float; lane 0 converts the total and lanes 1..10
        // the bit sums, so each block costs one FP64 conversion instruction.
        FF mine = ff_allreduce(acc);
        if (bits) {
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                const FF lb = ff_allreduce(((lane >> b) & 1) ? acc : FF{0.f, 0.f});
                const FF jb = ff_allreduce(ab[b]);
                if (lane == 1 + b) mine = lb;
                if (lane == 6 + b) mine = jb;
            }
        }
        const double val = ff_val(mine);
        if (lane == 0) tot[wid] = val;
        if (bits && lane >= 1 && lane <= 10) bits[wid * 10 + lane - 1] = lane - 1 < blog ? val : 0.0;
    } else {
        double t = 0.0, bj[5];
#pragma unroll
        for (int b = 0; b < 5; ++b) bj[b] = 0.0;
        for (int j = 0; j < jn; ++j) {
            if (lane + 32 * j < len) {
                const double p = prob(psi[b0 + lane + 32 * j]);
                t += p;
#pragma unroll
                for (int b = 0; b < 5; ++b)
                    if ((j >> b) & 1) bj[b] += p;
            }
        }
        const double total = warp_sum(t);
        if (bits) {
            double out[10];
#pragma unroll
            for (int b = 0; b < 5; ++b) out[b] = warp_sum(((lane >> b) & 1) ? t : 0.0);
#pragma unroll
            for (int b = 0; b < 5; ++b) out[5 + b] = warp_sum(bj[b]);
            if (lane == 0)
                for (int b = 0; b < 10; ++b) bits[wid * 10 + b] = b < blog ? out[b] : 0.0;
        }
        if (lane == 0) tot[wid] = total;
    }
}

// <Z_i> = S - 2 * (mass with bit i set) from the block records.  Stage 1:
// CTA (i, g) reduces chunk g of the block records for qubit i (fixed order);
// stage 2: one thread per qubit adds its chunk partials in order.
constexpr int kExpzChunks = 64;
__global__ void __launch_bounds__(256) k_expz_blocks(const double* __restrict__ tot, const double* __restrict__ bits,
                                                     uint64_t nblocks, int blog, double* __restrict__ part) {
    __shared__ double s1[256], s2[256];
    const int i = blockIdx.x, g = blockIdx.y;
    const uint64_t per = (nblocks + kExpzChunks - 1) / kExpzChunks;
    const uint64_t k0 = (uint64_t)g * per, k1 = k0 + per < nblocks ? k0 + per : nblocks;
    double a = 0.0, b = 0.0;
    for (uint64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const double tk = tot[k];
        a += tk;
        if (i < blog) b += bits[k * 10 + i];
        else if ((k >> (i - blog)) & 1) b += tk;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * (i * kExpzChunks + g)] = s1[0];
        part[2 * (i * kExpzChunks + g) + 1] = s2[0];
    }
}
__global__ void k_expz_final(const double* __restrict__ part, int n, double* __restrict__ out) {
    const int i = threadIdx.x;
    if (i >= n) return;
    double a = 0.0, b = 0.0;
    for (int g = 0; g < kExpzChunks; ++g) {
        a += part[2 * (i * kExpzChunks + g)];
        b += part[2 * (i * kExpzChunks + g) + 1];
    }
    out[i] = a - 2.0 * b;
}

// ---- inclusive scan of doubles -------------------------------------------
// One CTA of 1024 threads scans CH = 8192 consecutive values in place
// (8 per thread sequentially, then a CTA scan of the thread totals), adding
// "offset" (an exclusive prefix from the chunk scan, or 0).
constexpr int kScanT = 1024;
constexpr int kScanPer = 8;
constexpr int kScanCh = kScanT * kScanPer;

__device__ double cta_exclusive_scan(double v, double* total) {
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double x = v;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, s);
        if (lane >= s) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        double t = lane < nw ? ws[lane] : 0.0;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, t, s);
            if (lane >= s) t += y;
        }
        ws[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const double before_warp = w ? ws[w - 1] : 0.0;
    if (total) *total = ws[(blockDim.x >> 5) - 1];
    const double excl = before_warp + x - v;
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kScanT) k_scan_chunks(double* __restrict__ a, uint64_t len,
                                                        const double* __restrict__ offsets) {
    const uint64_t c0 = (uint64_t)blockIdx.x * kScanCh;
    const uint64_t i0 = c0 + (uint64_t)threadIdx.x * kScanPer;
    double loc[kScanPer];
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        loc[j] = (i0 + j < len) ? a[i0 + j] : 0.0;
        s += loc[j];
        loc[j] = s;
    }
    const double ex = cta_exclusive_scan(s, nullptr) + (offsets ? offsets[blockIdx.x] : 0.0);
#pragma unroll
    for (int j = 0; j < kScanPer; ++j)
        if (i0 + j < len) a[i0 + j] = loc[j] + ex;
}

__global__ void __launch_bounds__(kScanT) k_chunk_totals(const double* __restrict__ a, uint64_t len,
                                                         double* __restrict__ tot) {
    const uint64_t c0 = (uint64_t)blockIdx.x * kScanCh;
    const uint64_t i0 = c0 + (uint64_t)threadIdx.x * kScanPer;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j)
        if (i0 + j < len) s += a[i0 + j];
    double t;
    cta_exclusive_scan(s, &t);
    if (threadIdx.x == 0) tot[blockIdx.x] = t;
}

// Exclusive scan of chunk totals (one CTA, sequential per thread).
__global__ void __launch_bounds__(kScanT) k_scan_totals(double* __restrict__ tot, int nch) {
    const int per = (nch + kScanT - 1) / kScanT;
    const int i0 = threadIdx.x * per;
    double s = 0.0;
    for (int j = 0; j < per; ++j)
        if (i0 + j < nch) s += tot[i0 + j];
    const double ex = cta_exclusive_scan(s, nullptr);
    double run = ex;
    for (int j = 0; j < per; ++j)
        if (i0 + j < nch) {
            const double v = tot[i0 + j];
            tot[i0 + j] = run;
            run += v;
        }
}

// ---------------------------------------------------------------------------
// Relabelled qubits: logical qubit q is stored at bit map.phys[q].  The
// logical index x lives at P(x) = sum_q x_q 2^phys[q]; P is evaluated with
// per-byte tables of x in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void build_byte_tables(uint64_t (*T)[256], const QubitMap& map) {
    for (int e = threadIdx.x; e < 5 * 256; e += blockDim.x) {
        const int b = e >> 8, v = e & 255;
        uint64_t o = 0;
        for (int i = 0; i < 8; ++i) {
            const int q = 8 * b + i;
            if (q < map.n && ((v >> i) & 1)) o |= 1ull << map.phys[q];
        }
        T[b][v] = o;
    }
}
__device__ __forceinline__ uint64_t phys_index(const uint64_t (*T)[256], uint64_t x) {
    return T[0][x & 255] | T[1][(x >> 8) & 255] | T[2][(x >> 16) & 255] | T[3][(x >> 24) & 255] |
           T[4][(x >> 32) & 255];
}

// ---- logical-order block totals of a relabelled state ----------------------
// The sampler's rule min{x : C_x > u S} runs over the LOGICAL index x.  Logical
// block j holds x = j 2^B .. (j + 1) 2^B - 1; its amplitudes are the physical
// ones whose bits phys[0..B-1] (the set S) vary while the other physical bits
// spell j.  The state is read once in physical order, in chunks of 2^c
// contiguous amplitudes: a chunk's bits outside S (K_low) select different
// blocks and its bits in S (S_low) are summed; the physical bits above the
// chunk outside S (K_high) number the units the CTAs take, and those in S
// (S_high) are summed by a loop over all chunks of a unit.  Every sum has a
// fixed order, so the totals are bitwise reproducible.
struct LogicalBlocks {
    int c;          // chunk bits (physical bits 0..c-1)
    int nkh;        // physical bits >= c outside S
    int kh[40];     // their positions, ascending
    int khb[40];    // the block-index bit each one spells
    uint64_t shmask;  // physical bits >= c inside S
    int nkl, nsl;   // chunk bits outside / inside S
    int kl[10], klb[10], sl[10];
};

// Probability accumulator of one chunk position: complex64 forms |a|^2
// exactly as a float pair and adds in double-float; complex128 adds in FP64.
template <typename V> struct PAcc;
template <> struct PAcc<float2> {
    FF a{0.f, 0.f};
    __device__ __forceinline__ void add(float2 v) {
        const float r2 = v.x * v.x, r2e = fmaf(v.x, v.x, -r2);
        const float i2 = v.y * v.y, i2e = fmaf(v.y, v.y, -i2);
        const float sum = r2 + i2, bb = sum - r2;
        ff_add(a, sum, ((r2 - (sum - bb)) + (i2 - bb)) + r2e + i2e);
    }
    __device__ __forceinline__ double val() const { return ff_val(a); }
};
template <> struct PAcc<double2> {
    double a = 0.0;
    __device__ __forceinline__ void add(double2 v) { a += prob(v); }
    __device__ __forceinline__ double val() const { return a; }
};

template <typename V>
__global__ void __launch_bounds__(256) k_block_tot_logical(const V* __restrict__ psi, const LogicalBlocks lb,
                                                           uint64_t nunits, double* __restrict__ tot) {
    __shared__ double sacc[1 << kBlogMax];
    const int P = 1 << lb.c, tid = threadIdx.x;
    for (uint64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        uint64_t base = 0, jb = 0;
        for (int k = 0; k < lb.nkh; ++k)
            if ((u >> k) & 1) {
                base |= 1ull << lb.kh[k];
                jb |= 1ull << lb.khb[k];
            }
        PAcc<V> a[4];
        uint64_t sub = 0;  // the S_high bits, every subset of shmask in increasing order
        do {
            const V* src = psi + (base | sub);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int pos = tid + 256 * r;
                if (pos < P) a[r].add(src[pos]);
            }
            sub = (sub - lb.shmask) & lb.shmask;
        } while (sub);
        // chunk position -> (K_low pattern t, S_low pattern v) at t 2^nsl + v,
        // then a halving tree over v inside each segment
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int pos = tid + 256 * r;
            if (pos < P) {
                int t = 0, v = 0;
                for (int k = 0; k < lb.nkl; ++k) t |= ((pos >> lb.kl[k]) & 1) << k;
                for (int k = 0; k < lb.nsl; ++k) v |= ((pos >> lb.sl[k]) & 1) << k;
                sacc[(t << lb.nsl) | v] = a[r].val();
            }
        }
        __syncthreads();
        for (int w = (1 << lb.nsl) >> 1; w >= 1; w >>= 1) {
            for (int q = tid; q < P / 2; q += blockDim.x) {
                const int seg = q / w, o = q - seg * w;
                sacc[seg * 2 * w + o] += sacc[seg * 2 * w + o + w];
            }
            __syncthreads();
        }
        for (int t = tid; t < (1 << lb.nkl); t += blockDim.x) {
            uint64_t j = jb;
            for (int k = 0; k < lb.nkl; ++k)
                if ((t >> k) & 1) j |= 1ull << lb.klb[k];
            tot[j] = sacc[t << lb.nsl];
        }
        __syncthreads();
    }
}

// ---- sampler: one warp per shot ------------------------------------------
// PERM (a relabelled state): cdf is the block CDF in LOGICAL order (from
// k_block_tot_logical) and the chosen block is rescanned in logical order,
// amplitude x read at its physical index; the outcome is the logical x.
template <typename V, bool PERM>
__global__ void __launch_bounds__(256) k_sample(const V* __restrict__ psi, int n, int blog,
                                                const double* __restrict__ cdf, uint64_t nblocks,
                                                uint64_t shots, uint64_t seed, const double* __restrict__ u_in,
                                                uint64_t* __restrict__ out, const QubitMap map) {
    __shared__ uint64_t qt[PERM ? 5 : 1][256];
    if constexpr (PERM) {
        build_byte_tables(qt, map);
        __syncthreads();
    }
    auto amp = [&](uint64_t x) -> V {
        if constexpr (PERM) return psi[phys_index(qt, x)];
        else return psi[x];
    };
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const double S = cdf[nblocks - 1];
    const uint64_t len = 1ull << blog;
    for (uint64_t s = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < shots; s += warps) {
        const double u = u_in ? u_in[s] : philox_uniform(seed, s);
        const double t = u * S;
        // first block j with cdf[j] > t (the last block if rounding leaves
        // none): a 32-way search, each lane testing one of 32 evenly spaced
        // entries of [lo, hi), so 2^18 blocks take four steps; the answer
        // stays in [lo, hi) and lane 31 always tests hi - 1
        uint64_t lo = 0, hi = nblocks;
        while (hi - lo > 1) {
            const uint64_t step = (hi - lo + 31) >> 5;
            const uint64_t at = min(lo + (uint64_t)(lane + 1) * step, hi) - 1;
            const unsigned yes = __ballot_sync(0xffffffffu, at == nblocks - 1 || cdf[at] > t);
            const int f = __ffs(yes) - 1;
            const uint64_t at_f = __shfl_sync(0xffffffffu, at, f);
            const uint64_t at_p = __shfl_sync(0xffffffffu, at, f > 0 ? f - 1 : 0);
            hi = at_f + 1;
            if (f > 0) lo = at_p + 1;
        }
        const uint64_t j = lo;
        const double before = j ? cdf[j - 1] : 0.0;
        const uint64_t b0 = j << blog;
        // rescan the block 32 amplitudes at a time (one coalesced load per
        // step): a warp scan of the step's probabilities on top of the
        // running CDF, and the first lane whose CDF exceeds t (and whose
        // probability is not zero) is the outcome.  complex64: |a|^2 as an
        // exact float pair and the scan in double-float (about 48 bits; no
        // FP64 instruction in the loop) when the state's total lies well
        // inside FP32's range; complex128, or a far from normalised state:
        // FP64.
        uint64_t pick = UINT64_MAX, last_nz = b0;
        if constexpr (sizeof(V) == 8) {
            if (S > 1e-20 && S < 1e20) {
                const FF tf = ff_of(t);
                FF base = ff_of(before);
                for (uint64_t c = 0; c < len; c += 32) {
                    const bool valid = c + lane < len;
                    FF p = {0.f, 0.f};
                    if (valid) p = ff_prob(amp(b0 + c + lane));
                    FF inc = p;
#pragma unroll
                    for (int sh = 1; sh < 32; sh <<= 1) {
                        const float h = __shfl_up_sync(0xffffffffu, inc.hi, sh);
                        const float l = __shfl_up_sync(0xffffffffu, inc.lo, sh);
                        if (lane >= sh) ff_add(inc, h, l);
                    }
                    FF cum = base;
                    ff_add(cum, inc.hi, inc.lo);
                    const float above = (cum.hi - tf.hi) + (cum.lo - tf.lo);  // sign of cum - t
                    const unsigned hit = __ballot_sync(0xffffffffu, valid && p.hi > 0.f && above > 0.f);
                    if (hit) {
                        pick = b0 + c + (uint64_t)(__ffs(hit) - 1);
                        break;
                    }
                    const unsigned nz = __ballot_sync(0xffffffffu, p.hi > 0.f);
                    if (nz) last_nz = b0 + c + (uint64_t)(31 - __clz(nz));
                    ff_add(base, __shfl_sync(0xffffffffu, inc.hi, 31), __shfl_sync(0xffffffffu, inc.lo, 31));
                }
                if (lane == 0) out[s] = pick == UINT64_MAX ? last_nz : pick;
                continue;
            }
        }
        double base = before;
        for (uint64_t c = 0; c < len; c += 32) {
            const bool valid = c + lane < len;
            const double p = valid ? prob(amp(b0 + c + lane)) : 0.0;
            double inc = p;
#pragma unroll
            for (int sh = 1; sh < 32; sh <<= 1) {
                const double y = __shfl_up_sync(0xffffffffu, inc, sh);
                if (lane >= sh) inc += y;
            }
            const unsigned hit = __ballot_sync(0xffffffffu, valid && p > 0.0 && base + inc > t);
            if (hit) {
                pick = b0 + c + (uint64_t)(__ffs(hit) - 1);
                break;
            }
            const unsigned nz = __ballot_sync(0xffffffffu, p > 0.0);
            if (nz) last_nz = b0 + c + (uint64_t)(31 - __clz(nz));  // fallback when rounding leaves no x above t
            base += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) out[s] = pick == UINT64_MAX ? last_nz : pick;
    }
}

template <typename V>
__global__ void __launch_bounds__(256) k_probs(const V* __restrict__ psi, uint64_t N, double* __restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) out[i] = prob(psi[i]);
}

int sms() { return device_sms(); }

// Scratch layout in h->red: [block sums/cdf: nblocks][chunk totals: nch][expz partials]
size_t nblocks_of(int n, int* blog, int cap = kBlogMax) {
    *blog = n < cap ? n : cap;
    return (size_t)1 << (n - *blog);
}

// Block size for sampling: a shot scans one block, so with many shots
// smaller blocks keep the shots' work (shots * 2^blog amplitudes) within
// one read of the state; the block CDF then has more entries to search.
int sample_blog(int n, uint64_t shots) {
    int b = kBlogMax;
    while (b > 5 && ldexp((double)shots, b) > ldexp(1.0, n)) --b;
    return b;
}
}  // namespace

// Inclusive FP64 scan of a[0..len) in place; chunks: (len + kScanCh - 1) / kScanCh doubles of scratch.
static void scan_in_place(double* a, size_t len, double* chunks, cudaStream_t st) {
    const size_t nch = (len + kScanCh - 1) / kScanCh;
    if (nch <= 1) {
        count_launch();
        k_scan_chunks<<<1, kScanT, 0, st>>>(a, len, nullptr);
    } else {
        count_launch(3);
        k_chunk_totals<<<(unsigned)nch, kScanT, 0, st>>>(a, len, chunks);
        k_scan_totals<<<1, kScanT, 0, st>>>(chunks, (int)nch);
        k_scan_chunks<<<(unsigned)nch, kScanT, 0, st>>>(a, len, chunks);
    }
}

// Block CDF in LOGICAL order of a relabelled state (blocks of 2^blog
// consecutive logical indices), in h->lcdf: [cdf: nb][chunk totals: nch].
static int logical_block_cdf(sv_state* h, int blog, double** cdf_out, int64_t* nb_out) {
    const int n = h->n;
    const size_t nb = (size_t)1 << (n - blog);
    const size_t nch = (nb + kScanCh - 1) / kScanCh;
    int rc = ensure_scratch(&h->lcdf, sizeof(double) * (nb + nch), h->stream);
    if (rc) return rc;
    double* cdf = (double*)h->lcdf.ptr;
    const QubitMap map = qubit_map(h);
    int inv[64];  // physical bit -> logical qubit
    for (int q = 0; q < n; ++q) inv[map.phys[q]] = q;
    uint64_t smask = 0;  // physical bits of the in-block logical qubits
    for (int q = 0; q < blog; ++q) smask |= 1ull << map.phys[q];
    auto unit_bits = [&](int c) {
        int k = 0;
        for (int b = c; b < n; ++b) k += !((smask >> b) & 1);
        return k;
    };
    // chunk bits: up to 10; fewer (down to 8) when the units would not fill the GPU
    int c = n < kBlogMax ? n : kBlogMax;
    while (c > 8 && ((uint64_t)1 << unit_bits(c)) < (uint64_t)4 * sms()) --c;
    LogicalBlocks lb{};
    lb.c = c;
    for (int b = 0; b < n; ++b) {
        const bool in_s = (smask >> b) & 1;
        if (b < c) {
            if (in_s) lb.sl[lb.nsl++] = b;
            else {
                lb.kl[lb.nkl] = b;
                lb.klb[lb.nkl++] = inv[b] - blog;
            }
        } else if (in_s) {
            lb.shmask |= 1ull << b;
        } else {
            lb.kh[lb.nkh] = b;
            lb.khb[lb.nkh++] = inv[b] - blog;
        }
    }
    const uint64_t nunits = 1ull << lb.nkh;
    const uint64_t cap = (uint64_t)sms() * 8;
    const unsigned g = (unsigned)(nunits < cap ? nunits : cap);
    count_launch();
    if (h->dtype == SV_C64)
        k_block_tot_logical<float2><<<g, 256, 0, h->stream>>>((const float2*)h->amps, lb, nunits, cdf);
    else
        k_block_tot_logical<double2><<<g, 256, 0, h->stream>>>((const double2*)h->amps, lb, nunits, cdf);
    scan_in_place(cdf, nb, cdf + nb, h->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "logical block statistics");
    *cdf_out = cdf;
    *nb_out = (int64_t)nb;
    return SV_OK;
}

// Block statistics in h->red: [raw block totals: nb][inclusive CDF: nb]
// [chunk totals: nch][bit sums: 10 nb, when asked for].
static int block_stats(sv_state* h, bool want_bits, double** tot_out, double** cdf_out, double** bits_out,
                       int* blog_out, int64_t* nb_out, int blog_cap = kBlogMax) {
    int blog;
    const size_t nb = nblocks_of(h->n, &blog, blog_cap);
    const size_t nch = (nb + kScanCh - 1) / kScanCh;
    const size_t need = sizeof(double) * (2 * nb + nch + 64 + (want_bits ? 10 * nb : 0));
    int rc = ensure_scratch(&h->red, need, h->stream);
    if (rc) return rc;
    double* tot = (double*)h->red.ptr;
    double* cdf = tot + nb;
    double* chunks = cdf + nb;
    double* bits = want_bits ? chunks + nch + 64 : nullptr;
    const unsigned g = (unsigned)((nb * 32 + 255) / 256);
    count_launch();
    if (h->dtype == SV_C64)
        k_block_stats<float2><<<g, 256, 0, h->stream>>>((const float2*)h->amps, blog, nb, tot, bits);
    else
        k_block_stats<double2><<<g, 256, 0, h->stream>>>((const double2*)h->amps, blog, nb, tot, bits);
    cudaError_t e = cudaMemcpyAsync(cdf, tot, sizeof(double) * nb, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "block totals copy");
    scan_in_place(cdf, nb, chunks, h->stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "block statistics");
    if (tot_out) *tot_out = tot;
    *cdf_out = cdf;
    if (bits_out) *bits_out = bits;
    *blog_out = blog;
    *nb_out = (int64_t)nb;
    return SV_OK;
}

namespace {
template <typename V>
__global__ void __launch_bounds__(256) k_probs_logical(const V* __restrict__ psi, uint64_t N, double* __restrict__ out,
                                                       const QubitMap map) {
    __shared__ uint64_t T[5][256];
    build_byte_tables(T, map);
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride) {
        const V a = psi[phys_index(T, x)];
        const double re = (double)a.x, im = (double)a.y;
        out[x] = fma(re, re, im * im);
    }
}

template <typename V>
__global__ void __launch_bounds__(256) k_gather_logical(const V* __restrict__ psi, uint64_t x0, uint64_t cnt,
                                                        V* __restrict__ out, const QubitMap map) {
    __shared__ uint64_t T[5][256];
    build_byte_tables(T, map);
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride)
        out[i] = psi[phys_index(T, x0 + i)];
}

__global__ void k_logical_expz(const double* __restrict__ phys, double* __restrict__ out, const QubitMap map) {
    const int q = threadIdx.x;
    if (q < map.n) out[q] = phys[map.phys[q]];
}

unsigned grid_n(uint64_t n, int cap_per_sm) {
    uint64_t g = (n + 255) / 256;
    const uint64_t cap = (uint64_t)sms() * cap_per_sm;
    if (g > cap) g = cap;
    return (unsigned)(g ? g : 1);
}

}  // namespace

cudaError_t launch_gather_logical(sv_state* h, uint64_t x0, uint64_t cnt, void* dev_out) {
    count_launch();
    if (h->dtype == SV_C64)
        k_gather_logical<float2><<<grid_n(cnt, 16), 256, 0, h->stream>>>((const float2*)h->amps, x0, cnt,
                                                                        (float2*)dev_out, qubit_map(h));
    else
        k_gather_logical<double2><<<grid_n(cnt, 16), 256, 0, h->stream>>>((const double2*)h->amps, x0, cnt,
                                                                          (double2*)dev_out, qubit_map(h));
    return cudaGetLastError();
}

int measure_block_sums(sv_state* h, double** cdf, int* blog_out, int64_t* nb_out, int blog_cap) {
    return block_stats(h, false, nullptr, cdf, nullptr, blog_out, nb_out, blog_cap);
}

cudaError_t launch_probs(sv_state* h, double* dev_out) {
    const uint64_t N = 1ull << h->n;
    unsigned g = (unsigned)((N + 255) / 256);
    if (g > (unsigned)sms() * 16) g = (unsigned)sms() * 16;
    count_launch();
    if (h->permuted) {
        if (h->dtype == SV_C64)
            k_probs_logical<float2><<<g, 256, 0, h->stream>>>((const float2*)h->amps, N, dev_out, qubit_map(h));
        else
            k_probs_logical<double2><<<g, 256, 0, h->stream>>>((const double2*)h->amps, N, dev_out, qubit_map(h));
        return cudaGetLastError();
    }
    if (h->dtype == SV_C64)
        k_probs<float2><<<g, 256, 0, h->stream>>>((const float2*)h->amps, N, dev_out);
    else
        k_probs<double2><<<g, 256, 0, h->stream>>>((const double2*)h->amps, N, dev_out);
    return cudaGetLastError();
}

int measure_norm(sv_state* h, double* host_out) {
    double* cdf;
    int blog;
    int64_t nb;
    int rc = measure_block_sums(h, &cdf, &blog, &nb);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(host_out, cdf + nb - 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "norm readback");
    return SV_OK;
}

// Shots from a block CDF; logical = the CDF is in logical order (relabelled
// state) and the outcomes come out as logical indices.
static cudaError_t launch_sample(sv_state* h, int blog, const double* cdf, int64_t nb, uint64_t shots,
                                 uint64_t seed, const double* dev_u, uint64_t* dev_out, bool logical = false) {
    uint64_t g = (shots * 32 + 255) / 256;
    const uint64_t cap = (uint64_t)sms() * 16;
    if (g > cap) g = cap;
    count_launch();
    const QubitMap map = qubit_map(h);
    const unsigned gg = (unsigned)g;
    if (h->dtype == SV_C64) {
        const float2* a = (const float2*)h->amps;
        if (logical) k_sample<float2, true><<<gg, 256, 0, h->stream>>>(a, h->n, blog, cdf, nb, shots, seed, dev_u, dev_out, map);
        else k_sample<float2, false><<<gg, 256, 0, h->stream>>>(a, h->n, blog, cdf, nb, shots, seed, dev_u, dev_out, map);
    } else {
        const double2* a = (const double2*)h->amps;
        if (logical) k_sample<double2, true><<<gg, 256, 0, h->stream>>>(a, h->n, blog, cdf, nb, shots, seed, dev_u, dev_out, map);
        else k_sample<double2, false><<<gg, 256, 0, h->stream>>>(a, h->n, blog, cdf, nb, shots, seed, dev_u, dev_out, map);
    }
    return cudaGetLastError();
}

// Shots of a relabelled state: logical-order block CDF, logical rescan.
static int sample_logical(sv_state* h, int blog, uint64_t shots, uint64_t seed, const double* dev_u,
                          uint64_t* dev_out) {
    double* cdf;
    int64_t nb;
    int rc = logical_block_cdf(h, blog, &cdf, &nb);
    if (rc) return rc;
    cudaError_t e = launch_sample(h, blog, cdf, nb, shots, seed, dev_u, dev_out, true);
    if (e != cudaSuccess) return cuda_fail(e, "sample (relabelled state)");
    return SV_OK;
}

// Shots and <Z_i> from ONE pass over the state (either output may be NULL).
int measure_readout(sv_state* h, uint64_t shots, uint64_t seed, uint64_t* dev_samples, double* dev_expz) {
    double *tot, *cdf, *bits;
    int blog;
    int64_t nb;
    int rc = block_stats(h, dev_expz != nullptr, &tot, &cdf, &bits, &blog, &nb);
    if (rc) return rc;
    if (dev_expz) {
        // chunk partials, then (relabelled qubits) the physical-bit values
        rc = ensure_scratch(&h->perm_tmp, sizeof(double) * (2 * 64 * kExpzChunks + 64), h->stream);
        if (rc) return rc;
        double* part = (double*)h->perm_tmp.ptr;
        double* ez = h->permuted ? part + 2 * 64 * kExpzChunks : dev_expz;
        count_launch(2);
        k_expz_blocks<<<dim3(h->n, kExpzChunks), 256, 0, h->stream>>>(tot, bits, (uint64_t)nb, blog, part);
        k_expz_final<<<1, 64, 0, h->stream>>>(part, h->n, ez);
        if (h->permuted) {
            count_launch();
            k_logical_expz<<<1, 64, 0, h->stream>>>(ez, dev_expz, qubit_map(h));
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "read-out");
    if (dev_samples && shots) {
        // a relabelled state samples from its logical-order CDF (a second
        // read of the state; <Z> above used the physical block statistics)
        if (h->permuted) return sample_logical(h, blog, shots, seed, nullptr, dev_samples);
        e = launch_sample(h, blog, cdf, nb, shots, seed, nullptr, dev_samples);
        if (e != cudaSuccess) return cuda_fail(e, "read-out");
    }
    return SV_OK;
}

int measure_expect_z(sv_state* h, double* dev_out) { return measure_readout(h, 0, 0, nullptr, dev_out); }

int measure_sample(sv_state* h, uint64_t shots, uint64_t seed, const double* dev_u, uint64_t* dev_out) {
    if (shots == 0) return SV_OK;
    const int sb = sample_blog(h->n, shots);
    if (h->permuted) return sample_logical(h, h->n < sb ? h->n : sb, shots, seed, dev_u, dev_out);
    double* cdf;
    int blog;
    int64_t nb;
    int rc = measure_block_sums(h, &cdf, &blog, &nb, sb);
    if (rc) return rc;
    cudaError_t e = launch_sample(h, blog, cdf, nb, shots, seed, dev_u, dev_out);
    if (e != cudaSuccess) return cuda_fail(e, "sample");
    return SV_OK;
}

}  // namespace sv

// ---------------------------------------------------------------------------
// Sampling without any device allocation.
//
// Some callers cannot allocate device memory while they run: a serving
// process whose device memory is handed out up front by its own allocator
// (so a cudaMalloc here could fail or break its budget), or a caller that
// cannot accept the implicit device-wide synchronisation of cudaFree.  For
// them sv_sample_uniforms_noalloc keeps its only scratch (the probability
// block sums / block CDF and the chunk totals of the scan) in the fixed
// array below, which every GPU that loads this library holds until the
// process exits.  The caller passes the state, the uniforms and the output
// buffer, all in device memory.
// ---------------------------------------------------------------------------
namespace sv {
namespace {
constexpr int kNoAllocMaxQubits = 24;  // 2^(24-10) = 16384 block sums
constexpr size_t kNoAllocDoubles = ((size_t)1 << (kNoAllocMaxQubits - kBlogMax)) + 64;

// 128 KiB + 512 B of device memory per GPU; shared by every call.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up
// once per device, with that device current).  In host code the array's
// name only stands in for the symbol, so the address must come from
// cudaGetSymbolAddress.
int noalloc_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(SV_EUNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[dev] = (double*)p;
    }
    *out = g_noalloc_ptr[dev];
    return SV_OK;
}
}  // namespace

}  // namespace sv

extern "C" int sv_sample_uniforms_noalloc(const void* dev_amps, int n, sv_dtype dt, const double* dev_u,
                                          uint64_t shots, uint64_t* dev_out, void* cuda_stream) {
    using namespace sv;
    if (dt != SV_C64 && dt != SV_C128) return set_error(SV_EINVAL, "unknown dtype");
    if (n < 1 || n > kNoAllocMaxQubits)
        return set_error(SV_EINVAL, "sv_sample_uniforms_noalloc: n = " + std::to_string(n) +
                                        " outside 1..24 (its fixed scratch holds 2^14 block sums)");
    if (!dev_amps) return set_error(SV_EINVAL, "NULL state pointer");
    if (((uintptr_t)dev_amps & 15) != 0) return set_error(SV_EINVAL, "state pointer not 16-byte aligned");
    if (shots == 0) return SV_OK;
    if (!dev_u || !dev_out) return set_error(SV_EINVAL, "NULL uniforms or output pointer");
    double* bs = nullptr;
    int rc = noalloc_scratch(&bs);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int blog;
    const size_t nb = nblocks_of(n, &blog);
    const size_t nch = (nb + kScanCh - 1) / kScanCh;
    double* tot = bs + nb;  // nb + nch <= kNoAllocDoubles
    // Every scratch element is written before it is read within this call,
    // so nothing needs clearing; calls that overlap on the GPU race on it.
    const unsigned g = (unsigned)((nb * 32 + 255) / 256);
    count_launch();
    if (dt == SV_C64)
        k_block_stats<float2><<<g, 256, 0, st>>>((const float2*)dev_amps, blog, nb, bs, nullptr);
    else
        k_block_stats<double2><<<g, 256, 0, st>>>((const double2*)dev_amps, blog, nb, bs, nullptr);
    if (nch <= 1) {
        count_launch();
        k_scan_chunks<<<1, kScanT, 0, st>>>(bs, nb, nullptr);
    } else {
        count_launch(3);
        k_chunk_totals<<<(unsigned)nch, kScanT, 0, st>>>(bs, nb, tot);
        k_scan_totals<<<1, kScanT, 0, st>>>(tot, (int)nch);
        k_scan_chunks<<<(unsigned)nch, kScanT, 0, st>>>(bs, nb, tot);
    }
    uint64_t gs = (shots * 32 + 255) / 256;
    const uint64_t cap = (uint64_t)sms() * 16;
    if (gs > cap) gs = cap;
    count_launch();
    if (dt == SV_C64)
        k_sample<float2, false><<<(unsigned)gs, 256, 0, st>>>((const float2*)dev_amps, n, blog, bs, (uint64_t)nb,
                                                             shots, 0, dev_u, dev_out, QubitMap{});
    else
        k_sample<double2, false><<<(unsigned)gs, 256, 0, st>>>((const double2*)dev_amps, n, blog, bs,
                                                              (uint64_t)nb, shots, 0, dev_u, dev_out, QubitMap{});
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sv_sample_uniforms_noalloc");
    return SV_OK;
}

