// Autotuner: measure every candidate plan of one circuit on the caller's
// state and keep the fastest, with a JSON-lines cache of earlier results.
//
// The knobs are the fusion width k_max (App. D.2's "gate fusion = 5" as the
// upper bound), the tile width m and, for complex64, whether dense blocks of
// 3..5 qubits run on the tensor cores.  Every candidate is an exact plan, so
// the choice changes only the time.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "sv_internal.h"

namespace sv {
namespace {

std::mutex g_file_mu;

uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
    const unsigned char* p = (const unsigned char*)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

std::string cache_key(const sv_state* h, const sv_gate* gates, size_t count) {
    cudaDeviceProp prop;
    int dev = 0;
    std::string devname = "unknown";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
        devname = std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount);
    cudaGetLastError();
    for (char& c : devname)
        if (c == '"' || c == '\\') c = '_';
    char buf[160];
    snprintf(buf, sizeof(buf), "n%d-dt%d-g%zu-%016llx", h->n, h->dtype, count,
             (unsigned long long)fnv1a(gates, count * sizeof(sv_gate), 1469598103934665603ull));
    return std::string(buf) + "@" + devname;
}

// Returns true and fills the options if the file has a line for key.
bool cache_lookup(const char* path, const std::string& key, sv_options* o, double* ms) {
    std::lock_guard<std::mutex> lk(g_file_mu);
    FILE* f = fopen(path, "r");
    if (!f) return false;
    const std::string tag = "\"key\": \"" + key + "\"";
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        if (!strstr(line, tag.c_str())) continue;
        int k = 0, m = 0, t = 0;
        double v = 0.0;
        const char* pk = strstr(line, "\"k_max\": ");
        const char* pm = strstr(line, "\"tile_m\": ");
        const char* pt = strstr(line, "\"tensor\": ");
        const char* pv = strstr(line, "\"ms\": ");
        const char* pp = strstr(line, "\"pass_kernel\": ");
        int kern = 0;
        if (pp && sscanf(pp + 15, "%d", &kern) != 1) kern = 0;
        if (pk && pm && pt && pv && sscanf(pk + 9, "%d", &k) == 1 && sscanf(pm + 10, "%d", &m) == 1 &&
            sscanf(pt + 10, "%d", &t) == 1 && sscanf(pv + 6, "%lf", &v) == 1 && k >= 1 && k <= kMaxK &&
            m >= 1 && m <= kMaxTileM && (t == 1 || t == -1)) {
            memset(o, 0, sizeof(*o));
            o->k_max = k;
            o->tile_m = m;
            o->tensor = t;
            o->pass_kernel = kern == 1 ? 1 : 0;
            o->planner = SV_PLAN_GREEDY;
            *ms = v;
            found = true;  // the last matching line wins
        }
    }
    fclose(f);
    return found;
}

void cache_append(const char* path, const std::string& key, const sv_options& o, double ms) {
    std::lock_guard<std::mutex> lk(g_file_mu);
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"k_max\": %d, \"tile_m\": %d, \"tensor\": %d, \"pass_kernel\": %d, \"ms\": %.6f}\n",
            key.c_str(), o.k_max, o.tile_m, o.tensor, o.pass_kernel, ms);
    fclose(f);
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" int sv_autotune(sv_handle h, const sv_gate* gates, size_t count, const char* cache_path,
                           sv_options* best, double* best_ms) {
    if (!h) return set_error(SV_EINVAL, "NULL handle");
    if (h->bad) return set_error(SV_ESTATE, "state flagged by an earlier CUDA failure; re-initialise it");
    if (!best || (count && !gates)) return set_error(SV_EINVAL, "bad arguments");
    int rc = SV_OK;
    std::vector<CGate> cg;
    size_t bad = 0;
    if (canonicalise(h->n, gates, count, &cg, &bad) != SV_OK)
        return set_error(SV_EINVAL, "invalid gate record at index " + std::to_string(bad));
    const std::string key = cache_key(h, gates, count);
    double ms = 0.0;
    if (cache_path && cache_lookup(cache_path, key, best, &ms)) {
        if (best_ms) *best_ms = ms;
        return SV_OK;
    }
    std::vector<sv_options> cands;
    const int m0 = h->dtype == SV_C64 ? 11 : 10;
    for (int k = 2; k <= kMaxK; ++k)
        for (int m = m0; m < m0 + 4; ++m)
            for (int t = -1; t <= 1; t += 2)
                for (int pk = 0; pk <= 1; ++pk) {
                    if (t == 1 && (h->dtype != SV_C64 || k < kMinTcK)) continue;
                    sv_options o;
                    memset(&o, 0, sizeof(o));
                    o.k_max = k;
                    o.tile_m = std::min(m, h->n);
                    o.tensor = t;
                    o.pass_kernel = pk;
                    o.planner = SV_PLAN_GREEDY;
                    bool dup = false;
                    for (const sv_options& c : cands)
                        dup |= c.k_max == o.k_max && c.tile_m == o.tile_m && c.tensor == o.tensor &&
                               c.pass_kernel == o.pass_kernel;
                    if (!dup) cands.push_back(o);
                }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    double best_t = -1.0;
    for (const sv_options& o : cands) {
        double t_best = -1.0;
        for (int rep = 0; rep < 2 && rc == SV_OK; ++rep) {
            e = cudaEventRecord(e0, h->stream);
            if (e == cudaSuccess) rc = apply_canonical(h, gates, count, cg, &o);
            if (rc != SV_OK) break;
            if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "autotune timing");
                break;
            }
            if (t_best < 0.0 || t < t_best) t_best = t;
        }
        if (rc != SV_OK) break;
        if (best_t < 0.0 || t_best < best_t) {
            best_t = t_best;
            *best = o;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SV_OK) return rc;
    if (best_ms) *best_ms = best_t;
    if (cache_path) cache_append(cache_path, key, *best, best_t);
    return SV_OK;
}
