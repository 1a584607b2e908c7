// Multiplexor pass: up to kMuxMaxTargets uniformly controlled rotations that
// share one read and one write of the state.
//
// Each thread owns one column: the 2^K amplitudes whose indices differ only
// in the K target bits.  The control bits of the column's index select the
// angle of every target (one table entry per target, read through L2); the
// rotation and the X flip of each target act on register pairs.  Columns of
// consecutive threads are consecutive in the non-target bits, so every one of
// the 2^K loads and stores of a warp is coalesced whenever the lowest qubits
// are not targets (QCrank: address qubits low, data qubits high).
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>

#include "sv_internal.h"
#include "sv_mux.cuh"

namespace sv {
namespace {

template <typename T, typename C, int K>
// Two CTAs per SM (at most 128 registers) except for FP64 columns of 16 or 32
// amplitudes, which would spill heavily there.
__global__ void __launch_bounds__(256, (sizeof(T) == 8 && K >= 4) ? 1 : 2) k_mux(const MuxDev D, const unsigned char* __restrict__ region,
                                             C* __restrict__ amps, int n) {
    mux_columns<T, C, K>(D, region, amps, 0, 1ull << (n - K), (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                         (uint64_t)gridDim.x * blockDim.x);
}

int mux_sms() { return device_sms(); }

template <typename T, typename C>
cudaError_t mux_t(sv_state* h, const unsigned char* region, const MuxDev& D) {
    const uint64_t ncols = 1ull << (h->n - D.K);
    const uint64_t cap = (uint64_t)mux_sms() * 8;
    const unsigned grid = (unsigned)std::min<uint64_t>(cap, (ncols + 255) / 256);
    C* a = (C*)h->amps;
    switch (D.K) {
    case 1: k_mux<T, C, 1><<<grid, 256, 0, h->stream>>>(D, region, a, h->n); break;
    case 2: k_mux<T, C, 2><<<grid, 256, 0, h->stream>>>(D, region, a, h->n); break;
    case 3: k_mux<T, C, 3><<<grid, 256, 0, h->stream>>>(D, region, a, h->n); break;
    case 4: k_mux<T, C, 4><<<grid, 256, 0, h->stream>>>(D, region, a, h->n); break;
    default: k_mux<T, C, 5><<<grid, 256, 0, h->stream>>>(D, region, a, h->n); break;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mux(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass) {
    const PassDev* pd = (const PassDev*)(blob.bytes.data() + blob.pass_off) + pass;
    MuxDev D;
    memcpy(&D, blob.bytes.data() + pd->region_off, sizeof(D));
    if (D.K < 1 || D.K > kMuxMaxTargets || D.K >= h->n) return cudaErrorInvalidValue;
    const unsigned char* region = (const unsigned char*)blob_dev + pd->region_off;
    if (h->dtype == SV_C64) return mux_t<float, float2>(h, region, D);
    return mux_t<double, double2>(h, region, D);
}

}  // namespace sv
