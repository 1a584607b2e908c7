// Multiplexor pass body (device code shared by the multiplexor kernel and the
// batch executor): columns [c0, c1) of the state, column c0 + start, then
// every stride-th.  Each column is the 2^K amplitudes whose indices differ
// only in the K target bits; the control bits of its index select each
// target's angle (one table entry per target), and the rotation and the X
// flip of each target act on register pairs.
#pragma once

#include "sv_internal.h"

namespace sv {

__device__ __forceinline__ void mux_sin_cos(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void mux_sin_cos(double a, double* s, double* c) { sincos(a, s, c); }

template <typename T, typename C, int K>
__device__ __forceinline__ void mux_columns(const MuxDev& D, const unsigned char* __restrict__ region,
                                            C* __restrict__ amps, uint64_t c0, uint64_t c1, uint64_t start,
                                            uint64_t stride) {
    constexpr int S = 1 << K;
    uint64_t tb[K];
#pragma unroll
    for (int k = 0; k < K; ++k) tb[k] = 1ull << D.t[k];
    for (uint64_t col = c0 + start; col < c1; col += stride) {
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
                mux_sin_cos(__ldg(tab + j) * (T)0.5, &sn, &cs);
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
                mux_sin_cos(__ldg(tab + 2 * j), &s0, &c0);
                mux_sin_cos(__ldg(tab + 2 * j + 1), &s1, &c1);
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

}  // namespace sv
