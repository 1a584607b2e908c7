// QCrank read-out on the device (Sec. 3 image encoding, App. D.3, Table 2).
//
// A QCrank state holds a uniform superposition over the a address qubits
// (bits 0..a-1) with data qubit k (bit a + k) rotated by RY(pi * pixel_jk),
// so P(bit a+k = 1 | address j) = sin^2(pi * pixel_jk / 2).  The image
// comes back from shots as pixel_jk = (2/pi) * arcsin(sqrt(ones_jk / count_j))
// with count_j the shots at address j and ones_jk those of them with data
// bit k set.  Table 2 takes 3000 shots per address: up to ~10^8 shots, which
// this path histograms where they were drawn, in HBM.
//
// Histogram: per-CTA counters in shared memory (32-bit) when the 2^a (d + 1)
// of them fit, flushed once per CTA with 64-bit global atomics; global
// 64-bit atomics per shot otherwise.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kHistThreads = 512;
constexpr size_t kHistSmemMax = 200 * 1024;

__global__ void __launch_bounds__(kHistThreads) k_qc_hist_smem(const uint64_t* __restrict__ x, uint64_t shots,
                                                               int a, int d, unsigned long long* __restrict__ counts,
                                                               unsigned long long* __restrict__ ones) {
    extern __shared__ unsigned int hs[];  // [2^a counts][2^a * d ones]
    const uint32_t J = 1u << a;
    const uint32_t tot = J * (uint32_t)(d + 1);
    for (uint32_t i = threadIdx.x; i < tot; i += blockDim.x) hs[i] = 0u;
    __syncthreads();
    const uint32_t dmask = d >= 32 ? 0xffffffffu : (1u << d) - 1u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots; s += stride) {
        const uint64_t v = __ldg(x + s);
        const uint32_t j = (uint32_t)v & (J - 1u);
        atomicAdd(&hs[j], 1u);
        for (uint32_t db = (uint32_t)(v >> a) & dmask; db; db &= db - 1u)
            atomicAdd(&hs[J + j * (uint32_t)d + (uint32_t)(__ffs(db) - 1)], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tot; i += blockDim.x) {
        const unsigned int c = hs[i];
        if (c) atomicAdd(i < J ? counts + i : ones + (i - J), (unsigned long long)c);
    }
}

__global__ void __launch_bounds__(256) k_qc_hist_global(const uint64_t* __restrict__ x, uint64_t shots, int a,
                                                        int d, unsigned long long* __restrict__ counts,
                                                        unsigned long long* __restrict__ ones) {
    const uint64_t J = 1ull << a;
    const uint32_t dmask = d >= 32 ? 0xffffffffu : (1u << d) - 1u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots; s += stride) {
        const uint64_t v = __ldg(x + s);
        const uint64_t j = v & (J - 1);
        atomicAdd(counts + j, 1ull);
        for (uint32_t db = (uint32_t)(v >> a) & dmask; db; db &= db - 1u)
            atomicAdd(ones + j * (uint64_t)d + (uint64_t)(__ffs(db) - 1), 1ull);
    }
}

__global__ void __launch_bounds__(256) k_qc_pixels(const unsigned long long* __restrict__ counts,
                                                   const unsigned long long* __restrict__ ones, int a, int d,
                                                   double* __restrict__ pix) {
    const uint64_t total = (uint64_t)d << a;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = counts[i / (uint64_t)d];
        // (2/pi) asin(sqrt(p)); no estimate without shots
        pix[i] = c ? 0.63661977236758134308 * asin(sqrt((double)ones[i] / (double)c)) : __longlong_as_double(0x7ff8000000000000ull);
    }
}

int qc_sms() { return device_sms(); }

}  // namespace

cudaError_t launch_qcrank_decode(const uint64_t* samples, uint64_t shots, int a, int d, uint64_t* counts,
                                 uint64_t* ones, double* pixels, cudaStream_t st) {
    const size_t J = (size_t)1 << a;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint64_t) * J, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ones, 0, sizeof(uint64_t) * J * d, st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(unsigned int) * J * (size_t)(d + 1);
    if (shots) {
        if (smem <= kHistSmemMax) {
            static size_t attr = 0;
            if (smem > 48 * 1024 && smem > attr) {
                e = cudaFuncSetAttribute(k_qc_hist_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                attr = smem;
            }
            // enough CTAs to cover the shots, at most one per SM: every CTA
            // flushes its whole histogram once
            const uint64_t want = (shots + (uint64_t)kHistThreads * 64 - 1) / ((uint64_t)kHistThreads * 64);
            const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)qc_sms()));
            k_qc_hist_smem<<<grid, kHistThreads, smem, st>>>(samples, shots, a, d, (unsigned long long*)counts,
                                                             (unsigned long long*)ones);
        } else {
            const unsigned grid = (unsigned)std::min<uint64_t>((shots + 255) / 256, (uint64_t)qc_sms() * 16);
            k_qc_hist_global<<<grid, 256, 0, st>>>(samples, shots, a, d, (unsigned long long*)counts,
                                                   (unsigned long long*)ones);
        }
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const uint64_t total = (uint64_t)d << a;
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)qc_sms() * 8);
    k_qc_pixels<<<grid, 256, 0, st>>>((const unsigned long long*)counts, (const unsigned long long*)ones, a, d,
                                      pixels);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sv
