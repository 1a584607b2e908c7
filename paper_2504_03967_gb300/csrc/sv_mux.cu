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

namespace sv {
namespace {

__device__ __forceinline__ void sin_cos(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sin_cos(double a, double* s, double* c) { sincos(a, s, c); }

template <typename T, typename C, int K>
__global__ void __launch_bounds__(256) k_mux(const MuxDev D, const unsigned char* __restrict__ region,
                                             C* __restrict__ amps, int n) {
    constexpr int S = 1 << K;
    const uint64_t ncols = 1ull << (n - K);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t tb[K];
#pragma unroll
    for (int k = 0; k < K; ++k) tb[k] = 1ull << D.t[k];
    for (uint64_t col = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; col < ncols; col += stride) {
        // insert a zero bit at every target position (ascending)
        uint64_t x = col;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint64_t lo = x & (tb[k] - 1);
            x = ((x ^ lo) << 1) | lo;
        }
        uint32_t j = 0;
        for (int r = 0; r < D.nruns; ++r) j |= (uint32_t)((x >> D.rs[r]) & ((1ull << D.rw[r]) - 1)) << D.ro[r];
        C v[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            uint64_t a = x;
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (s >> k & 1) a |= tb[k];
            v[s] = amps[a];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool f = ((__popc(j & D.flip[k]) ^ D.flip_c[k]) & 1) != 0;
            const T* tab = (const T*)(region + D.tab_off[k]);
            if (D.family[k] == MUX_Y) {
                T sn, cs;
                sin_cos(__ldg(tab + j) * (T)0.5, &sn, &cs);
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    if (s >> k & 1) continue;
                    const C a = v[s], b = v[s | (1 << k)];
                    C u, w;  // RY(phi): (a, b) -> (c a - s b, s a + c b)
                    u.x = cs * a.x - sn * b.x;
                    u.y = cs * a.y - sn * b.y;
                    w.x = sn * a.x + cs * b.x;
                    w.y = sn * a.y + cs * b.y;
                    v[s] = f ? w : u;
                    v[s | (1 << k)] = f ? u : w;
                }
            } else {
                T s0, c0, s1, c1;
                sin_cos(__ldg(tab + 2 * j), &s0, &c0);
                sin_cos(__ldg(tab + 2 * j + 1), &s1, &c1);
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    if (s >> k & 1) continue;
                    const C a = v[s], b = v[s | (1 << k)];
                    C u, w;  // (a, b) -> (e^{i phi0} a, e^{i phi1} b)
                    u.x = c0 * a.x - s0 * a.y;
                    u.y = c0 * a.y + s0 * a.x;
                    w.x = c1 * b.x - s1 * b.y;
                    w.y = c1 * b.y + s1 * b.x;
                    v[s] = f ? w : u;
                    v[s | (1 << k)] = f ? u : w;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            uint64_t a = x;
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (s >> k & 1) a |= tb[k];
            amps[a] = v[s];
        }
    }
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
