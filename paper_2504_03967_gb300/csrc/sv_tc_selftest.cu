// Self-test of the tcgen05 building blocks used by the tensor-core dense
// apply: one CTA computes D (128 x 64) = A (128 x 64, in TMEM) x B^T (B: 64 x
// 64, K-major in shared memory, no-swizzle canonical layout) with kind::tf32
// MMAs of K = 8.  Host code compares D with its own product of the same
// inputs.  Every wait is bounded and the TMEM is always freed.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "sv_internal.h"
#include "sv_selftest.h"  // from include/
#include "sv_tc.cuh"

namespace sv {

namespace {

constexpr int TM = 128, TN = 64, TK = 64;
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kColA = 0, kColD = 128;

// Byte offset of element (n, k) of a K-major operand in the no-swizzle
// canonical layout with the given leading/stride byte offsets.
__device__ __forceinline__ uint32_t kmajor_off(int n, int k, uint32_t lbo, uint32_t sbo) {
    return (uint32_t)(n >> 3) * sbo + (uint32_t)(k >> 2) * lbo + (uint32_t)(n & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

__global__ void __launch_bounds__(128) k_tc_selftest(const float* __restrict__ A, const float* __restrict__ B,
                                                     float* __restrict__ D, uint32_t kstride, uint32_t nstride,
                                                     int swap_fields, int* __restrict__ status) {
    __shared__ __align__(1024) float sB[TN * TK + 1024];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        tc::tmem_alloc(&s_taddr, kTmemCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&s_mbar, 1);
        tc::fence_mbar_init();
    }
    // B into shared memory in the canonical layout (offsets stay inside sB
    // for the lbo/sbo values the host allows).
    for (int e = tid; e < TN * TK; e += blockDim.x) {
        const int n = e / TK, k = e % TK;
        const uint32_t off = kmajor_off(n, k, kstride, nstride);
        if (off + 4 <= sizeof(sB)) sB[off / 4] = B[e];
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_taddr;
    const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
    // A row (this thread's lane) into TMEM columns kColA..kColA+63
    const int row = tid;
    for (int c = 0; c < TK; c += 16) {
        uint32_t v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = __float_as_uint(A[row * TK + c + j]);
        tc::tmem_st16(lane_base + kColA + c, v);
    }
    tc::tmem_wait_st();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
        const uint32_t idesc = tc::idesc_tf32(TM, TN);
        const uint32_t sb = tc::smem_u32(sB);
        for (int kk = 0; kk < TK / 8; ++kk) {
            const uint32_t lbo = swap_fields ? nstride : kstride, sbo = swap_fields ? kstride : nstride;
            const uint64_t bd = tc::sdesc_noswz(sb + (uint32_t)(kk * 2) * kstride, lbo, sbo);
            tc::mma_tf32_ts(tbase + kColD, tbase + kColA + kk * 8, bd, idesc, kk > 0);
        }
        tc::mma_commit(&s_mbar);
    }
    const bool ok = tc::mbar_wait_bounded(&s_mbar, 0, 1u << 22);
    tc::fence_after();
    if (!ok) {
        if (tid == 0) atomicExch(status, 1);
    } else {
        for (int c = 0; c < TN; c += 16) {
            uint32_t v[16];
            tc::tmem_ld16(lane_base + kColD + c, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) D[row * TN + c + j] = __uint_as_float(v[j]);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

}  // namespace
}  // namespace sv

extern "C" int sv_selftest_tc_tf32(const float* host_a, const float* host_b, float* host_d, int kstride,
                                   int nstride, int swap_fields, int* host_status) {
    using namespace sv;
    if (!host_a || !host_b || !host_d || !host_status) return set_error(SV_EINVAL, "NULL argument");
    // offsets must keep every operand byte inside the 17 KiB staging buffer
    const long big = kstride > nstride ? kstride : nstride;
    const long maxoff = (long)(TN / 8 - 1) * nstride + (long)(TK / 4 - 1) * kstride + 7 * 16 + 12;
    // with either field assignment the tensor core reads at most: start of
    // the last K step + one K core + 7 row groups, each stride <= big
    const long maxread = (long)(TK / 8 - 1) * 2 * kstride + big + 7 * big + 128;
    if (kstride <= 0 || nstride <= 0 || (kstride & 15) || (nstride & 15) ||
        maxoff + 4 > (long)sizeof(float) * (TN * TK + 1024) || maxread > (long)sizeof(float) * (TN * TK + 1024))
        return set_error(SV_EINVAL, "strides out of range for the self-test buffer");
    float *dA = nullptr, *dB = nullptr, *dD = nullptr;
    int* dS = nullptr;
    cudaError_t e = cudaMalloc(&dA, sizeof(float) * TM * TK);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(float) * TN * TK);
    if (e == cudaSuccess) e = cudaMalloc(&dD, sizeof(float) * TM * TN);
    if (e == cudaSuccess) e = cudaMalloc(&dS, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dA, host_a, sizeof(float) * TM * TK, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, host_b, sizeof(float) * TN * TK, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dD, 0, sizeof(float) * TM * TN);
    if (e == cudaSuccess) e = cudaMemset(dS, 0, sizeof(int));
    if (e == cudaSuccess) {
        count_launch();
        k_tc_selftest<<<1, 128>>>(dA, dB, dD, (uint32_t)kstride, (uint32_t)nstride, swap_fields, dS);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host_d, dD, sizeof(float) * TM * TN, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(host_status, dS, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dS);
    if (e != cudaSuccess) return cuda_fail(e, "tcgen05 self-test");
    return SV_OK;
}

// ---------------------------------------------------------------------------
// The kind::f16 form used by the tensor-core dense op of the register passes:
// A (128 x 64 FP16, two values per TMEM column, value 2j in the low half of
// column j unless swap_halves) in TMEM, B (64 x 64 FP16, K-major, no-swizzle
// core matrices of 8 rows x 8 values: 128 bytes between K-adjacent ones,
// 1024 bytes between 8-row groups) in shared memory, four MMAs of K = 16.
// ---------------------------------------------------------------------------
namespace sv {
namespace {
__global__ void __launch_bounds__(128) k_tc_f16_selftest(const uint16_t* __restrict__ A,
                                                         const uint16_t* __restrict__ B, float* __restrict__ D,
                                                         int swap_halves, int* __restrict__ status) {
    __shared__ __align__(1024) uint16_t sB[64 * 64];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        tc::tmem_alloc(&s_taddr, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&s_mbar, 1);
        tc::fence_mbar_init();
    }
    for (int e = tid; e < 64 * 64; e += blockDim.x) {
        const int n = e / 64, k = e % 64;
        sB[((n >> 3) * 1024 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) / 2] = B[e];
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_taddr;
    const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
    const int row = tid;
    {
        uint32_t v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const uint32_t lo = A[row * 64 + 2 * j], hi = A[row * 64 + 2 * j + 1];
            v[j] = swap_halves ? (lo << 16) | hi : (hi << 16) | lo;
        }
        tc::tmem_st32(lane_base, v);
    }
    tc::tmem_wait_st();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
        const uint32_t idesc = tc::idesc_f16(128, 64);
        const uint32_t sb = tc::smem_u32(sB);
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_f16_ts(tbase + 128, tbase + kk * 8, tc::sdesc_noswz(sb + kk * 256, 128, 1024), idesc, kk > 0);
        tc::mma_commit(&s_mbar);
    }
    const bool ok = tc::mbar_wait_bounded(&s_mbar, 0, 1u << 22);
    tc::fence_after();
    if (!ok) {
        if (tid == 0) atomicExch(status, 1);
    } else {
        uint32_t v[32];
        tc::tmem_ld32(lane_base + 128, v);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) D[row * 64 + j] = __uint_as_float(v[j]);
        tc::tmem_ld32(lane_base + 160, v);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) D[row * 64 + 32 + j] = __uint_as_float(v[j]);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 256);
}
}  // namespace
}  // namespace sv

extern "C" int sv_selftest_tc_f16(const uint16_t* host_a, const uint16_t* host_b, float* host_d, int swap_halves,
                                  int* host_status) {
    using namespace sv;
    if (!host_a || !host_b || !host_d || !host_status) return set_error(SV_EINVAL, "NULL argument");
    uint16_t *dA = nullptr, *dB = nullptr;
    float* dD = nullptr;
    int* dS = nullptr;
    cudaError_t e = cudaMalloc(&dA, 2 * 128 * 64);
    if (e == cudaSuccess) e = cudaMalloc(&dB, 2 * 64 * 64);
    if (e == cudaSuccess) e = cudaMalloc(&dD, sizeof(float) * 128 * 64);
    if (e == cudaSuccess) e = cudaMalloc(&dS, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dA, host_a, 2 * 128 * 64, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, host_b, 2 * 64 * 64, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dD, 0, sizeof(float) * 128 * 64);
    if (e == cudaSuccess) e = cudaMemset(dS, 0, sizeof(int));
    if (e == cudaSuccess) {
        count_launch();
        k_tc_f16_selftest<<<1, 128>>>(dA, dB, dD, swap_halves, dS);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host_d, dD, sizeof(float) * 128 * 64, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(host_status, dS, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dS);
    if (e != cudaSuccess) return cuda_fail(e, "tcgen05 f16 self-test");
    return SV_OK;
}

// ---------------------------------------------------------------------------
// Failure detection without a fault: one CTA waits on an mbarrier that no
// thread or copy ever arrives at, through the same bounded wait the
// tensor-core pass uses, and records the expiry in a device status word
// before returning normally.
// ---------------------------------------------------------------------------
namespace {
__global__ void k_wait_selftest(uint32_t limit, int* __restrict__ status) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) {
        sv::tc::mbar_init(&mbar, 1);
        sv::tc::fence_mbar_init();
    }
    __syncthreads();
    const bool ok = sv::tc::mbar_wait_bounded(&mbar, 0u, limit);
    if (!ok && threadIdx.x == 0) atomicExch(status, 1);
}
}  // namespace

extern "C" int sv_selftest_wait_timeout(unsigned limit, int* host_status) {
    using namespace sv;
    if (!host_status) return set_error(SV_EINVAL, "NULL argument");
    if (limit == 0 || limit > (1u << 22)) return set_error(SV_EINVAL, "limit must be in 1..2^22");
    int* dS = nullptr;
    cudaError_t e = cudaMalloc(&dS, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(dS, 0, sizeof(int));
    if (e == cudaSuccess) {
        count_launch();
        k_wait_selftest<<<1, 32>>>((uint32_t)limit, dS);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host_status, dS, sizeof(int), cudaMemcpyDeviceToHost);
    if (dS) cudaFree(dS);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
    return SV_OK;
}
