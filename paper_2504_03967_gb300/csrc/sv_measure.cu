// Read-out kernels: FP64 probability block sums, the block CDF scan, the shot
// sampler, <Z_i> and full probabilities.
//
// Sampling (Sec. 3: shots per circuit) draws outcome = min{x : C_x > u S},
// C the inclusive CDF of p_x = |a_x|^2 and S = C_{N-1}: a binary search over
// the FP64 block CDF finds the block, then one warp rescans that block's
// 2^B amplitudes in FP64 (lane partial sums, warp scan, sequential finish in
// the chosen lane).
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

// ---- block sums: one warp per block of 2^blog amplitudes -----------------
template <typename V>
__global__ void __launch_bounds__(256) k_block_sums(const V* __restrict__ psi, uint64_t N, int blog,
                                                    uint64_t nblocks, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= nblocks) return;
    const uint64_t b0 = wid << blog;
    const uint64_t len = 1ull << blog;
    double acc = 0.0;
    for (uint64_t i = lane; i < len; i += 32) acc += prob(psi[b0 + i]);
    acc = warp_sum(acc);
    if (lane == 0) out[wid] = acc;
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

// ---- sampler: one warp per shot ------------------------------------------
template <typename V>
__global__ void __launch_bounds__(256) k_sample(const V* __restrict__ psi, int n, int blog,
                                                const double* __restrict__ cdf, uint64_t nblocks,
                                                uint64_t shots, uint64_t seed, const double* __restrict__ u_in,
                                                uint64_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const double S = cdf[nblocks - 1];
    const uint64_t len = 1ull << blog;
    const int per = (int)(len >= 32 ? len / 32 : 1);
    for (uint64_t s = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < shots; s += warps) {
        const double u = u_in ? u_in[s] : philox_uniform(seed, s);
        const double t = u * S;
        // first block j with cdf[j] > t
        uint64_t lo = 0, hi = nblocks - 1;
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        const uint64_t j = lo;
        const double before = j ? cdf[j - 1] : 0.0;
        const uint64_t b0 = j << blog;
        // lane chunk sums over contiguous sub-ranges of the block
        const uint64_t c0 = b0 + (uint64_t)lane * per;
        double ls = 0.0;
        if ((uint64_t)lane * per < len)
            for (int i = 0; i < per; ++i) ls += prob(psi[c0 + i]);
        double inc = ls;
#pragma unroll
        for (int sh = 1; sh < 32; sh <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, inc, sh);
            if (lane >= sh) inc += y;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, before + inc > t && (uint64_t)lane * per < len);
        // last lane holding a non-zero probability (fallback when rounding
        // leaves no lane above t)
        const unsigned nz = __ballot_sync(0xffffffffu, ls > 0.0);
        int L = hit ? __ffs(hit) - 1 : (nz ? 31 - __clz(nz) : 0);
        if (lane == L) {
            double acc = before + (inc - ls);
            const uint64_t cb = b0 + (uint64_t)L * per;
            uint64_t pick = UINT64_MAX, last_nz = cb;
            for (int i = 0; i < per && (uint64_t)L * per + i < len; ++i) {
                const double p = prob(psi[cb + i]);
                if (p > 0.0) last_nz = cb + i;
                acc += p;
                if (acc > t && p > 0.0) {
                    pick = cb + i;
                    break;
                }
            }
            out[s] = pick == UINT64_MAX ? last_nz : pick;
        }
    }
}

// ---- <Z_i>: warp-per-segment partial sums --------------------------------
// Segment = 32 x 32 amplitudes.  Lane bits 0..4 are fixed per lane, so each
// lane keeps its own total; bits >= 5 are constant over each 32-amplitude
// row, whose warp sum is added to bit accumulators held one per lane.
template <typename V>
__global__ void __launch_bounds__(256) k_expz_partial(const V* __restrict__ psi, int n, uint64_t N,
                                                      double* __restrict__ part /* [grid][n+1] */) {
    __shared__ double sh[8][40];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    double lane_tot = 0.0;   // sum over this lane's amplitudes
    double bitacc = 0.0;     // lane b: sum of rows with bit (5 + b) set
    double bitacc2 = 0.0;    // lane b: bit (37 + b) (unused for n <= 37)
    const uint64_t rows = N >= 32 ? N / 32 : 1;
    for (uint64_t r = gw; r < rows; r += nw) {
        const uint64_t x = r * 32 + lane;
        const double p = x < N ? prob(psi[x]) : 0.0;
        lane_tot += p;
        const double rs = warp_sum(p);
        const uint64_t xb = r * 32;
        if (lane + 5 < n && ((xb >> (lane + 5)) & 1)) bitacc += rs;
        (void)bitacc2;
    }
    sh[w][lane] = bitacc;
    // totals of lane bits: bit i (< 5) set lanes
    for (int i = 0; i < 5; ++i) {
        const double v = warp_sum(((lane >> i) & 1) ? lane_tot : 0.0);
        if (lane == 0) sh[w][32 + i] = v;
    }
    const double tot = warp_sum(lane_tot);
    if (lane == 0) sh[w][37] = tot;
    __syncthreads();
    if (threadIdx.x < 40) {
        double v = 0.0;
        for (int k = 0; k < 8; ++k) v += sh[k][threadIdx.x];
        // layout per CTA: [0..n-1] = sum of p with bit i set, [n] = total
        const int t = threadIdx.x;
        double* P = part + (uint64_t)blockIdx.x * (n + 1);
        if (t < 32) {
            if (t + 5 < n) P[t + 5] = v;
        } else if (t < 37) {
            if (t - 32 < n) P[t - 32] = v;
        } else if (t == 37) {
            P[n] = v;
        }
    }
}

__global__ void k_expz_final(const double* __restrict__ part, int nparts, int n, double* __restrict__ out) {
    const int i = threadIdx.x;
    if (i >= n) return;
    double s1 = 0.0, tot = 0.0;
    for (int k = 0; k < nparts; ++k) {
        s1 += part[(uint64_t)k * (n + 1) + i];
        tot += part[(uint64_t)k * (n + 1) + n];
    }
    out[i] = tot - 2.0 * s1;
}

template <typename V>
__global__ void __launch_bounds__(256) k_probs(const V* __restrict__ psi, uint64_t N, double* __restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) out[i] = prob(psi[i]);
}

int sms() {
    static int s = 0;
    if (!s) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        if (s <= 0) s = 148;
    }
    return s;
}

// Scratch layout in h->red: [block sums/cdf: nblocks][chunk totals: nch][expz partials]
size_t nblocks_of(int n, int* blog) {
    *blog = n < kBlogMax ? n : kBlogMax;
    return (size_t)1 << (n - *blog);
}
}  // namespace

// Block sums -> inclusive block CDF, in h->red.
int measure_block_sums(sv_state* h, double** cdf, int* blog_out, int64_t* nb_out) {
    int blog;
    const size_t nb = nblocks_of(h->n, &blog);
    const size_t nch = (nb + kScanCh - 1) / kScanCh;
    const size_t need = sizeof(double) * (nb + nch + 64);
    int rc = ensure_scratch(&h->red, need, h->stream);
    if (rc) return rc;
    double* bs = (double*)h->red.ptr;
    double* tot = bs + nb;
    const uint64_t N = 1ull << h->n;
    const unsigned g = (unsigned)((nb * 32 + 255) / 256);
    count_launch();
    if (h->dtype == SV_C64)
        k_block_sums<float2><<<g, 256, 0, h->stream>>>((const float2*)h->amps, N, blog, nb, bs);
    else
        k_block_sums<double2><<<g, 256, 0, h->stream>>>((const double2*)h->amps, N, blog, nb, bs);
    if (nch <= 1) {
        count_launch();
        k_scan_chunks<<<1, kScanT, 0, h->stream>>>(bs, nb, nullptr);
    } else {
        count_launch(3);
        k_chunk_totals<<<(unsigned)nch, kScanT, 0, h->stream>>>(bs, nb, tot);
        k_scan_totals<<<1, kScanT, 0, h->stream>>>(tot, (int)nch);
        k_scan_chunks<<<(unsigned)nch, kScanT, 0, h->stream>>>(bs, nb, tot);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "block sums");
    *cdf = bs;
    *blog_out = blog;
    *nb_out = (int64_t)nb;
    return SV_OK;
}

cudaError_t launch_probs(sv_state* h, double* dev_out) {
    const uint64_t N = 1ull << h->n;
    unsigned g = (unsigned)((N + 255) / 256);
    if (g > (unsigned)sms() * 16) g = (unsigned)sms() * 16;
    count_launch();
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

int measure_expect_z(sv_state* h, double* dev_out) {
    const uint64_t N = 1ull << h->n;
    const uint64_t rows = N >= 32 ? N / 32 : 1;
    uint64_t g = (rows + 7) / 8;
    const uint64_t cap = (uint64_t)sms() * 8;
    if (g > cap) g = cap;
    const size_t need = sizeof(double) * (size_t)g * (h->n + 1);
    int rc = ensure_scratch(&h->red, need, h->stream);
    if (rc) return rc;
    double* part = (double*)h->red.ptr;
    count_launch(2);
    if (h->dtype == SV_C64)
        k_expz_partial<float2><<<(unsigned)g, 256, 0, h->stream>>>((const float2*)h->amps, h->n, N, part);
    else
        k_expz_partial<double2><<<(unsigned)g, 256, 0, h->stream>>>((const double2*)h->amps, h->n, N, part);
    k_expz_final<<<1, 64, 0, h->stream>>>(part, (int)g, h->n, dev_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "expect_z");
    return SV_OK;
}

int measure_sample(sv_state* h, uint64_t shots, uint64_t seed, const double* dev_u, uint64_t* dev_out) {
    if (shots == 0) return SV_OK;
    double* cdf;
    int blog;
    int64_t nb;
    int rc = measure_block_sums(h, &cdf, &blog, &nb);
    if (rc) return rc;
    uint64_t g = (shots * 32 + 255) / 256;
    const uint64_t cap = (uint64_t)sms() * 16;
    if (g > cap) g = cap;
    count_launch();
    if (h->dtype == SV_C64)
        k_sample<float2><<<(unsigned)g, 256, 0, h->stream>>>((const float2*)h->amps, h->n, blog, cdf, (uint64_t)nb,
                                                            shots, seed, dev_u, dev_out);
    else
        k_sample<double2><<<(unsigned)g, 256, 0, h->stream>>>((const double2*)h->amps, h->n, blog, cdf,
                                                             (uint64_t)nb, shots, seed, dev_u, dev_out);
    cudaError_t e = cudaGetLastError();
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
    const uint64_t N = 1ull << n;
    // Every scratch element is written before it is read within this call,
    // so nothing needs clearing; calls that overlap on the GPU race on it.
    const unsigned g = (unsigned)((nb * 32 + 255) / 256);
    count_launch();
    if (dt == SV_C64)
        k_block_sums<float2><<<g, 256, 0, st>>>((const float2*)dev_amps, N, blog, nb, bs);
    else
        k_block_sums<double2><<<g, 256, 0, st>>>((const double2*)dev_amps, N, blog, nb, bs);
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
        k_sample<float2><<<(unsigned)gs, 256, 0, st>>>((const float2*)dev_amps, n, blog, bs, (uint64_t)nb, shots,
                                                      0, dev_u, dev_out);
    else
        k_sample<double2><<<(unsigned)gs, 256, 0, st>>>((const double2*)dev_amps, n, blog, bs, (uint64_t)nb,
                                                       shots, 0, dev_u, dev_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sv_sample_uniforms_noalloc");
    return SV_OK;
}

