// Batched execution of many independent circuits of uneven size (the paper's
// parallel mode, Sec. 2.4, where many small circuits run side by side, and
// its fixed-size circuit tensor of App. B Lemma 2).
//
//  * circuits whose whole state fits one CTA's shared memory are planned on
//    host threads into single-tile plans and run by ONE persistent kernel,
//    launched from a CUDA graph: each CTA takes circuits from a device work
//    counter and writes <Z_i> and the shots straight from shared memory;
//  * larger circuits run through the fused tile-pass path, spread over a few
//    streams that each own a state buffer, with the read-outs kept on the
//    device until a single copy back at the end.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <thread>

#include "sv_internal.h"

namespace sv {
namespace {

int small_limit(int dtype) { return dtype == SV_C64 ? 13 : 12; }

template <typename F>
void parallel_for(int n, F f) {
    const int T = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t)
        th.emplace_back([&]() {
            for (int i; (i = next.fetch_add(1)) < n;) f(i);
        });
    for (auto& x : th) x.join();
}

struct Prepared {
    Plan plan;
    PlanBlob blob;
};

struct Slot {
    cudaStream_t st = nullptr;
    void* buf = nullptr;
    sv_state h{};
};

}  // namespace

// ---------------------------------------------------------------------------
// Waves: up to kWaveCircuits circuits whose every pass runs in the persistent
// wave kernel (register tile passes of 256 threads, multiplexor passes).
// ---------------------------------------------------------------------------
constexpr int kWaveCircuits = 256;
// Items hold as many of a pass's tiles (1..64; a CTA stages the pass's region
// once per item) or multiplexor columns (at least 1024) as make about four
// items per CTA at each pass level.
constexpr unsigned kWaveWaitLimit = 1u << 24;  // polls of about 128 ns: a wait gives up after about 2 s

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// One blob from several (passes in order): the pass records first, then
// every blob's region area, region offsets moved with it.  Tensor-core B
// operands of the shared-memory kernel are not carried (wave passes have none).
void merge_blobs(const std::vector<const PlanBlob*>& bl, PlanBlob* out) {
    int np = 0;
    for (const PlanBlob* b : bl) np += b->npasses;
    out->npasses = np;
    out->pass_off = 0;
    out->tc_off = align16(sizeof(PassDev) * (size_t)np);
    size_t cur = out->tc_off, total = cur;
    std::vector<size_t> r0(bl.size(), 0);
    for (size_t i = 0; i < bl.size(); ++i) {
        const PassDev* pd = (const PassDev*)(bl[i]->bytes.data() + bl[i]->pass_off);
        size_t lo = bl[i]->bytes.size();
        for (int p = 0; p < bl[i]->npasses; ++p) lo = std::min(lo, (size_t)pd[p].region_off);
        r0[i] = lo;
        total += bl[i]->bytes.size() - lo;
    }
    out->bytes.assign(total, 0);
    out->max_region = 0;
    PassDev* dst = (PassDev*)(out->bytes.data() + out->pass_off);
    int k = 0;
    for (size_t i = 0; i < bl.size(); ++i) {
        const PlanBlob& b = *bl[i];
        const PassDev* pd = (const PassDev*)(b.bytes.data() + b.pass_off);
        for (int p = 0; p < b.npasses; ++p, ++k) {
            dst[k] = pd[p];
            dst[k].region_off = (int)(pd[p].region_off - r0[i] + cur);
        }
        if (b.bytes.size() > r0[i]) memcpy(out->bytes.data() + cur, b.bytes.data() + r0[i], b.bytes.size() - r0[i]);
        cur += b.bytes.size() - r0[i];
        out->max_region = std::max(out->max_region, b.max_region);
    }
}

bool build_wave(int dtype, const std::vector<const Plan*>& plans, WaveHost* w,
                const std::vector<const PlanBlob*>* blobs) {
    if (blobs) merge_blobs(*blobs, &w->blob);
    else serialise_plans(plans, &w->blob);
    const int RB = reg_bits(dtype);
    const unsigned char* b = w->blob.bytes.data();
    const PassDev* pds = (const PassDev*)(b + w->blob.pass_off);
    for (int p = 0; p < w->blob.npasses; ++p)
        if (!(pds[p].rmode == kRmodeMux || (pds[p].rmode == 1 && pds[p].m - RB == 8 && pds[p].tc_k == 0)))
            return false;
    const int C = (int)plans.size();
    std::vector<int> first(C + 1, 0);
    for (int c = 0; c < C; ++c) first[c + 1] = first[c] + (int)plans[c]->passes.size();
    w->offs.resize(C);
    w->nq.resize(C);
    w->amps = 0;
    int levels = 0;
    for (int c = 0; c < C; ++c) {
        w->offs[c] = w->amps;
        w->nq[c] = plans[c]->n;
        w->amps += 1ull << plans[c]->n;
        levels = std::max(levels, first[c + 1] - first[c]);
    }
    w->items.clear();
    std::vector<int> cum(C, 0);
    const uint64_t target = (uint64_t)device_sms() * 2 * 4;  // about four items per CTA per pass level
    for (int l = 0; l < levels; ++l) {
        uint64_t tiles = 0, cols = 0;  // the level's work
        for (int c = 0; c < C; ++c) {
            const int p = first[c] + l;
            if (p >= first[c + 1]) continue;
            if (pds[p].rmode == kRmodeMux) {
                MuxDev D;
                memcpy(&D, b + pds[p].region_off, sizeof(D));
                cols += 1ull << (plans[c]->n - D.K);
            } else {
                tiles += 1ull << (plans[c]->n - pds[p].m);
            }
        }
        const uint64_t tper = std::min<uint64_t>(64, std::max<uint64_t>(1, tiles / target));
        const uint64_t cper = std::max<uint64_t>(1024, cols / target);
        for (int c = 0; c < C; ++c) {
            const int p = first[c] + l;
            if (p >= first[c + 1]) continue;
            const int need = cum[c];
            WaveItem I;
            I.circ = c;
            I.pass = p;
            I.need = need;
            if (pds[p].rmode == kRmodeMux) {
                MuxDev D;
                memcpy(&D, b + pds[p].region_off, sizeof(D));
                const uint64_t ncols = 1ull << (plans[c]->n - D.K);
                I.kind = 1;
                const uint64_t per = cper;
                for (uint64_t c0 = 0; c0 < ncols; c0 += per) {
                    I.lo = c0;
                    I.hi = std::min(ncols, c0 + per);
                    w->items.push_back(I);
                    ++cum[c];
                }
            } else {
                const uint64_t ntiles = 1ull << (plans[c]->n - pds[p].m);
                I.kind = 0;
                const uint64_t per = tper;
                for (uint64_t t0 = 0; t0 < ntiles; t0 += per) {
                    I.lo = t0;
                    I.hi = std::min(ntiles, t0 + per);
                    w->items.push_back(I);
                    ++cum[c];
                }
            }
        }
    }
    return true;
}

void WaveKeep::release() {
    for (cudaGraphExec_t x : execs) cudaGraphExecDestroy(x);
    for (cudaGraph_t g : graphs) cudaGraphDestroy(g);
    for (void* p : pinned) cudaFreeHost(p);
    if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    execs.clear();
    graphs.clear();
    pinned.clear();
    ev = nullptr;
    cs = nullptr;
    cudaGetLastError();
}

int enqueue_wave(int dtype, const WaveHost& w, cudaStream_t st, unsigned limit, int* dev_err, WaveKeep* keep,
                 void** dev_base) {
    *dev_base = nullptr;
    const size_t csz = dtype == SV_C64 ? 8 : 16, C = w.offs.size();
    void *base = nullptr, *blob = nullptr, *pin = nullptr;
    uint64_t* offs = nullptr;
    int *nq = nullptr, *cnt = nullptr;
    WaveItem* items = nullptr;
    const size_t ib = sizeof(WaveItem) * w.items.size(), ob = sizeof(uint64_t) * C, nb = sizeof(int) * C;
    const size_t pinb = w.blob.bytes.size() + ib + ob + nb;
    cudaError_t e = cudaMallocAsync(&base, csz * w.amps, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&blob, w.blob.bytes.size(), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&items, ib, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&offs, ob, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&nq, nb, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&cnt, sizeof(int) * (C + 1), st);  // head, done[C]
    if (e == cudaSuccess) e = cudaMallocHost(&pin, pinb);
    if (pin) keep->pinned.push_back(pin);
    auto free_tmp = [&]() {  // stream-ordered: after the wave
        if (blob) cudaFreeAsync(blob, st);
        if (items) cudaFreeAsync(items, st);
        if (offs) cudaFreeAsync(offs, st);
        if (nq) cudaFreeAsync(nq, st);
        if (cnt) cudaFreeAsync(cnt, st);
    };
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_tmp();
        if (base) cudaFreeAsync(base, st);
        cudaGetLastError();
        return set_error(SV_ENOMEM, "sv_batch_run: wave allocation failed");
    }
    unsigned char* pc = (unsigned char*)pin;
    memcpy(pc, w.blob.bytes.data(), w.blob.bytes.size());
    memcpy(pc + w.blob.bytes.size(), w.items.data(), ib);
    memcpy(pc + w.blob.bytes.size() + ib, w.offs.data(), ob);
    memcpy(pc + w.blob.bytes.size() + ib + ob, w.nq.data(), nb);
    e = cudaMemcpyAsync(blob, pc, w.blob.bytes.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(items, pc + w.blob.bytes.size(), ib, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(offs, pc + w.blob.bytes.size() + ib, ob, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nq, pc + w.blob.bytes.size() + ib + ob, nb, cudaMemcpyHostToDevice, st);
    // the counters, the |0...0> states and the persistent launch, from one graph
    // captured on a private stream (the caller's may be the legacy stream)
    if (e == cudaSuccess && !keep->cs) e = cudaStreamCreateWithFlags(&keep->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess && !keep->ev) e = cudaEventCreateWithFlags(&keep->ev, cudaEventDisableTiming);
    cudaStream_t cs = keep->cs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    if (e == cudaSuccess) e = cudaEventRecord(keep->ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, keep->ev, 0);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(cnt, 0, sizeof(int) * (C + 1), cs);
        cudaMemsetAsync(base, 0, csz * w.amps, cs);
        launch_wave_init(dtype, base, offs, (int)C, cs);
        launch_wave(dtype, base, offs, nq, blob, w.blob, items, (int)w.items.size(), cnt, cnt + 1, dev_err, limit,
                    cs);
        e = cudaStreamEndCapture(cs, &graph);
    }
    if (graph) keep->graphs.push_back(graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
    if (gexec) keep->execs.push_back(gexec);
    if (e == cudaSuccess) e = cudaGraphLaunch(gexec, cs);
    if (e == cudaSuccess) e = cudaEventRecord(keep->ev, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, keep->ev, 0);
    free_tmp();
    if (e != cudaSuccess) {
        cudaFreeAsync(base, st);
        cudaGetLastError();
        return cuda_fail(e, "wave");
    }
    *dev_base = base;
    return SV_OK;
}

}  // namespace sv

using namespace sv;

extern "C" int sv_batch_run(int C, const int* n_qubits, const int64_t* gate_offsets, const int64_t* gate_counts,
                            const sv_gate* gates, sv_dtype dt, uint64_t shots, uint64_t seed,
                            const sv_options* opt, uint64_t* host_samples, double* host_expz, int nmax,
                            void* cuda_stream) {
    if (C < 1 || !n_qubits || !gate_offsets || !gate_counts || !gates)
        return set_error(SV_EINVAL, "sv_batch_run: NULL argument or C < 1");
    if (dt != SV_C64 && dt != SV_C128) return set_error(SV_EINVAL, "unknown dtype");
    if (host_samples && shots == 0) host_samples = nullptr;
    int nbig = 0;
    for (int c = 0; c < C; ++c) {
        const int n = n_qubits[c];
        if (n < 1 || n > (dt == SV_C64 ? kMaxQubitsC64 : kMaxQubitsC128))
            return set_error(SV_EINVAL, "circuit " + std::to_string(c) + ": n out of range");
        if (gate_counts[c] < 0 || gate_offsets[c] < 0) return set_error(SV_EINVAL, "negative gate offset/count");
        nbig = std::max(nbig, n);
    }
    if (host_expz && nmax < nbig) return set_error(SV_EINVAL, "nmax below the largest circuit");
    if (!host_expz) nmax = 1;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // 1. validate and canonicalise every circuit on host threads; circuits
    //    for the tile-pass path are planned and serialised there too (their
    //    canonical lists are dropped as soon as the plan exists)
    std::vector<std::vector<CGate>> cg(C);
    std::vector<int> bad(C, 0);
    const PlanOptions probe = resolve_options(1, dt, opt);
    const bool host_plans = probe.planner == SV_PLAN_GREEDY && !probe.relabel;
    // Run-time compiled passes only when asked for (jit = 1): a batch of
    // mostly different circuits would spend its time compiling.
    sv_options bopt;
    memset(&bopt, 0, sizeof(bopt));
    if (opt) bopt = *opt;
    if (bopt.jit != 1) bopt.jit = -1;
    opt = &bopt;
    std::vector<std::unique_ptr<Prepared>> prep(C);
    parallel_for(C, [&](int c) {
        size_t b = 0;
        const int n = n_qubits[c];
        bad[c] = canonicalise(n, gates + gate_offsets[c], (size_t)gate_counts[c], &cg[c], &b) != SV_OK;
        if (bad[c] || n <= small_limit(dt) || !host_plans) return;
        PlanOptions po = resolve_options(n, dt, opt);
        po.tc_auto = 0;  // the wave kernel runs the interpreting pass body, without tensor-core blocks
        if (po.tensor == 0) po.tensor = -1;
        std::vector<CGate>& g = cg[c];
        drop_small_phases(&g, po.drop_phase_below);
        std::vector<CGate> muxed;
        std::vector<Mux> muxes;
        const bool rec = recognise_mux(n, g, &muxed, &muxes, po.mux);
        std::unique_ptr<Prepared> P(new Prepared);
        plan_greedy(n, dt, rec ? muxed : g, po, &P->plan, &muxes);
        serialise_plan(P->plan, &P->blob);
        for (Mux& M : P->plan.muxes) {  // the blob holds the tables now
            std::vector<double>().swap(M.phi0);
            std::vector<double>().swap(M.phi1);
        }
        prep[c] = std::move(P);
        std::vector<CGate>().swap(g);
    });
    for (int c = 0; c < C; ++c)
        if (bad[c]) return set_error(SV_EINVAL, "circuit " + std::to_string(c) + ": invalid gate record");

    std::vector<int> small, large;
    for (int c = 0; c < C; ++c) (n_qubits[c] <= small_limit(dt) ? small : large).push_back(c);
    const int Cs = (int)small.size();
    std::vector<int> slot(C);  // row of circuit c in the device outputs: [small..., large...]
    for (int i = 0; i < Cs; ++i) slot[small[i]] = i;
    for (size_t i = 0; i < large.size(); ++i) slot[large[i]] = Cs + (int)i;

    // device outputs in [small..., large...] order
    uint64_t* d_samples = nullptr;
    double* d_expz = nullptr;
    int* d_counter = nullptr;
    int* d_gidx = nullptr;
    void* d_blob = nullptr;
    cudaError_t e = cudaSuccess;
    if (host_samples) e = cudaMallocAsync((void**)&d_samples, sizeof(uint64_t) * (size_t)C * shots, st);
    if (e == cudaSuccess && host_expz) e = cudaMallocAsync((void**)&d_expz, sizeof(double) * (size_t)C * nmax, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_counter, sizeof(int), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(SV_ENOMEM, "sv_batch_run: output allocation failed");
    }
    int rc = SV_OK;
    std::vector<Slot> slots;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    void* pin = nullptr;

    // 2. small circuits: single-tile plans -> one persistent launch
    if (Cs > 0) {
        std::vector<Plan> plans(Cs);
        int mmax = 1;
        parallel_for(Cs, [&](int i) {
            const int c = small[i];
            PlanOptions po = resolve_options(n_qubits[c], dt, opt);
            if (!opt || opt->k_max == 0) po.k_max = 3;  // CUDA-core blocks: k = 3 is the cheapest fused width
            po.tile_m = n_qubits[c];
            po.tensor = -1;
            plan_greedy(n_qubits[c], dt, cg[c], po, &plans[i]);
        });
        std::vector<const Plan*> pp;
        for (int i = 0; i < Cs; ++i) {
            if (plans[i].passes.size() > 1) return set_error(SV_EINVAL, "internal: small circuit needs one pass");
            if (plans[i].passes.empty()) {  // empty circuit: an identity pass
                HostPass hp;
                for (int q = 0; q < plans[i].n; ++q) hp.tile.push_back(q);
                hp.L = std::min(plans[i].n, dt == SV_C64 ? 4 : 3);
                plans[i].passes.push_back(hp);
            }
            mmax = std::max(mmax, plans[i].n);
            plans[i].no_register_passes = true;  // the batch kernel reads the shared-memory region format
            pp.push_back(&plans[i]);
        }
        PlanBlob blob;
        serialise_plans(pp, &blob);
        const size_t gbytes = sizeof(int) * (size_t)Cs;
        e = cudaMallocAsync(&d_blob, blob.bytes.size(), st);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_gidx, gbytes, st);
        if (e == cudaSuccess) e = cudaMallocHost(&pin, blob.bytes.size() + gbytes);
        if (e == cudaSuccess) {
            memcpy(pin, blob.bytes.data(), blob.bytes.size());
            memcpy((char*)pin + blob.bytes.size(), small.data(), gbytes);
            e = cudaMemcpyAsync(d_blob, pin, blob.bytes.size(), cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_gidx, (char*)pin + blob.bytes.size(), gbytes, cudaMemcpyHostToDevice, st);
        // the persistent launch (and its work-counter reset) from a graph
        cudaStream_t cs = nullptr;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        cudaEvent_t ready = nullptr;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ready, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready, 0);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(d_counter, 0, sizeof(int), cs);
            launch_batch_small(dt, d_blob, blob, Cs, mmax, host_samples ? shots : 0, seed, d_gidx, d_samples, d_expz,
                               nmax, d_counter, cs);
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(gexec, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ready, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ready, 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (ready) cudaEventDestroy(ready);
        if (cs) cudaStreamDestroy(cs);
        if (e != cudaSuccess) rc = cuda_fail(e, "batched small circuits");
    }

    // 3a. large circuits planned on the host: waves of up to kWaveCircuits
    //     circuits (and a bounded state budget), each one persistent launch
    std::vector<int> rest;
    if (rc == SV_OK) {
        size_t freeb = 0, totb = 0;
        cudaMemGetInfo(&freeb, &totb);
        const uint64_t budget = std::max<uint64_t>(freeb / 4, 1ull << 28);
        const size_t csz = dt == SV_C64 ? 8 : 16;
        // views of one circuit's state for its read-outs, on 4 streams
        constexpr int kViews = 4;
        sv_state hv[kViews] = {};
        cudaStream_t vs[kViews] = {};
        cudaEvent_t vev = nullptr;
        cudaEventCreateWithFlags(&vev, cudaEventDisableTiming);
        for (int v = 0; v < kViews; ++v) {
            cudaStreamCreateWithFlags(&vs[v], cudaStreamNonBlocking);
            hv[v].dtype = dt;
            hv[v].stream = vs[v];
            hv[v].pending_basis = -1;
        }
        int* d_err = nullptr;  // a wait of any wave gave up (2)
        if (cudaMallocAsync((void**)&d_err, sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(SV_ENOMEM, "sv_batch_run: wave error word");
        }
        WaveKeep keep;
        size_t i = 0;
        while (rc == SV_OK && i < large.size()) {
            std::vector<int> wc;
            std::vector<const Plan*> plans;
            uint64_t bytes = 0;
            for (; i < large.size() && (int)wc.size() < kWaveCircuits; ++i) {
                const int c = large[i];
                const uint64_t sb = (uint64_t)csz << n_qubits[c];
                if (!prep[c] || prep[c]->plan.passes.empty()) {
                    rest.push_back(c);
                    continue;
                }
                if (!wc.empty() && bytes + sb > budget) break;
                wc.push_back(c);
                plans.push_back(&prep[c]->plan);
                bytes += sb;
            }
            if (wc.empty()) continue;
            WaveHost w;
            std::vector<const PlanBlob*> blobs;
            for (int c : wc) blobs.push_back(&prep[c]->blob);
            if (!build_wave(dt, plans, &w, &blobs)) {
                rest.insert(rest.end(), wc.begin(), wc.end());
                continue;
            }
            void* base = nullptr;
            rc = enqueue_wave(dt, w, st, kWaveWaitLimit, d_err, &keep, &base);
            if (rc == SV_OK) {  // the read-out streams start after the wave
                cudaEventRecord(vev, st);
                for (int v = 0; v < kViews; ++v) cudaStreamWaitEvent(vs[v], vev, 0);
            }
            for (size_t k = 0; rc == SV_OK && k < wc.size(); ++k) {
                const int c = wc[k];
                const int idx = slot[c];
                sv_state& h = hv[k % kViews];
                h.n = n_qubits[c];
                h.amps = (char*)base + csz * w.offs[k];
                reset_perm(&h);
                if (host_samples)
                    rc = measure_sample(&h, shots, seed + (uint64_t)c, nullptr, d_samples + (size_t)idx * shots);
                if (rc == SV_OK && host_expz) rc = measure_expect_z(&h, d_expz + (size_t)idx * nmax);
            }
            for (int v = 0; v < kViews; ++v) {  // the wave's buffer is freed after its read-outs
                cudaEventRecord(vev, vs[v]);
                cudaStreamWaitEvent(st, vev, 0);
            }
            if (base) cudaFreeAsync(base, st);
            for (int c : wc) prep[c].reset();
        }
        int herr = 0;
        if (d_err) {
            if (cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) herr = -1;
            cudaFreeAsync(d_err, st);
        }
        const cudaError_t es = cudaStreamSynchronize(st);
        if (rc == SV_OK && es != cudaSuccess) rc = cuda_fail(es, "waves");
        else if (rc == SV_OK && herr == 2) rc = set_error(SV_ETIMEOUT, "sv_batch_run: a wait of the wave kernel gave up");
        keep.release();
        for (int v = 0; v < kViews; ++v) {
            cudaStreamSynchronize(vs[v]);
            if (hv[v].red.ptr) cudaFree(hv[v].red.ptr);
            if (hv[v].perm_tmp.ptr) cudaFree(hv[v].perm_tmp.ptr);
            if (hv[v].lcdf.ptr) cudaFree(hv[v].lcdf.ptr);
            cudaStreamDestroy(vs[v]);
        }
        cudaEventDestroy(vev);
    }
    // 3b. the other large circuits: fused passes on a few streams
    if (rc == SV_OK && !rest.empty()) {
        int nl = 0;
        for (int c : rest) nl = std::max(nl, n_qubits[c]);
        const size_t bytes = (size_t)(dt == SV_C64 ? 8 : 16) << nl;
        size_t freeb = 0, totb = 0;
        cudaMemGetInfo(&freeb, &totb);
        int ns = (int)std::min<size_t>(std::min<size_t>(4, rest.size()), std::max<size_t>(1, freeb / (2 * bytes)));
        slots.resize(ns);
        for (int s = 0; e == cudaSuccess && s < ns; ++s) {
            e = cudaStreamCreateWithFlags(&slots[s].st, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaMalloc(&slots[s].buf, bytes);
            slots[s].h.dtype = dt;
            slots[s].h.amps = slots[s].buf;
            slots[s].h.stream = slots[s].st;
            slots[s].h.owned = false;
            slots[s].h.bad = false;
            slots[s].h.ev_used = 0;
            slots[s].h.upload_ev = nullptr;
            slots[s].h.upload_pending = false;
            slots[s].h.pending_basis = -1;
            slots[s].h.plans = nullptr;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(SV_ENOMEM, "sv_batch_run: large-circuit state buffers");
        }
        for (size_t i = 0; rc == SV_OK && i < rest.size(); ++i) {
            const int c = rest[i];
            const int idx = slot[c];
            sv_state* h = &slots[i % slots.size()].h;
            h->n = n_qubits[c];
            reset_perm(h);
            if (launch_init_basis(h, 0) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "init");
            if (rc == SV_OK && prep[c]) {
                if (prep[c]->blob.npasses > 0) rc = launch_plan(h, prep[c]->plan, prep[c]->blob, false, nullptr, nullptr);
                prep[c].reset();
            } else if (rc == SV_OK) {
                rc = apply_canonical(h, gates + gate_offsets[c], (size_t)gate_counts[c], cg[c], opt);
            }
            if (rc == SV_OK && host_samples)
                rc = measure_sample(h, shots, seed + (uint64_t)c, nullptr, d_samples + (size_t)idx * shots);
            if (rc == SV_OK && host_expz) rc = measure_expect_z(h, d_expz + (size_t)idx * nmax);
        }
    }

    // 4. one copy back, then scatter to the caller's circuit order
    for (auto& s : slots)
        if (s.st) cudaStreamSynchronize(s.st);
    e = cudaStreamSynchronize(st);
    if (rc == SV_OK && e != cudaSuccess) rc = cuda_fail(e, "batch");
    std::vector<int> order(small);
    order.insert(order.end(), large.begin(), large.end());
    if (rc == SV_OK && host_samples) {  // straight into the caller's rows (no staging copy)
        for (int i = 0; rc == SV_OK && i < C; ++i) {
            e = cudaMemcpy(host_samples + (size_t)order[i] * shots, d_samples + (size_t)i * shots,
                           sizeof(uint64_t) * shots, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) rc = cuda_fail(e, "samples readback");
        }
    }
    if (rc == SV_OK && host_expz) {
        std::vector<double> tmp((size_t)C * nmax);
        e = cudaMemcpy(tmp.data(), d_expz, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "expz readback");
        for (int i = 0; rc == SV_OK && i < C; ++i)
            memcpy(host_expz + (size_t)order[i] * nmax, tmp.data() + (size_t)i * nmax, sizeof(double) * nmax);
    }
    for (auto& s : slots) {
        if (s.h.plan_dev.ptr) cudaFree(s.h.plan_dev.ptr);
        if (s.h.red.ptr) cudaFree(s.h.red.ptr);
        if (s.h.err.ptr) cudaFree(s.h.err.ptr);
        if (s.h.host_pin.ptr) cudaFreeHost(s.h.host_pin.ptr);
        if (s.h.upload_ev) cudaEventDestroy(s.h.upload_ev);
        for (cudaEvent_t ev : s.h.ev_pool) cudaEventDestroy(ev);
        if (s.buf) cudaFree(s.buf);
        if (s.st) cudaStreamDestroy(s.st);
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (pin) cudaFreeHost(pin);
    if (d_blob) cudaFree(d_blob);
    if (d_samples) cudaFree(d_samples);
    if (d_expz) cudaFree(d_expz);
    if (d_counter) cudaFree(d_counter);
    if (d_gidx) cudaFree(d_gidx);
    cudaGetLastError();
    return rc;
}

// ---------------------------------------------------------------------------
// Failure detection of the wave kernel without a GPU fault: one circuit of 14
// qubits (an H on every qubit, one pass of 2 tiles) whose first item is made
// to wait for more finished items of its circuit than there can be:
// the bounded wait gives up after `limit` polls, the kernel records it and
// returns, and the call reports SV_ETIMEOUT.  *host_status = 1 when it did.
// ---------------------------------------------------------------------------
extern "C" int sv_selftest_wave_timeout(unsigned limit, int* host_status) {
    if (!host_status) return set_error(SV_EINVAL, "NULL argument");
    if (limit == 0 || limit > (1u << 22)) return set_error(SV_EINVAL, "limit must be in 1..2^22");
    const int n = 14;
    std::vector<sv_gate> g(n);
    for (int q = 0; q < n; ++q) {
        memset(&g[q], 0, sizeof(sv_gate));
        g[q].type = SV_H;
        g[q].nq = 1;
        g[q].q[0] = (uint32_t)q;
    }
    std::vector<CGate> cg;
    size_t bad = 0;
    if (canonicalise(n, g.data(), g.size(), &cg, &bad) != SV_OK) return set_error(SV_EINVAL, "internal: circuit");
    PlanOptions po = resolve_options(n, SV_C64, nullptr);
    po.tc_auto = 0;
    Plan plan;
    plan_greedy(n, SV_C64, cg, po, &plan);
    WaveHost w;
    if (!build_wave(SV_C64, {&plan}, &w) || w.items.empty()) return set_error(SV_EINVAL, "internal: wave");
    // the unsatisfiable dependency: as many finished items as the wave has,
    // which cannot happen while this one waits
    w.items[0].need = (int)w.items.size();
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "stream");
    void* base = nullptr;
    int* d_err = nullptr;
    int herr = 0;
    WaveKeep keep;
    int rc = SV_OK;
    if (cudaMallocAsync((void**)&d_err, sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "error word");
    if (rc == SV_OK) rc = enqueue_wave(SV_C64, w, st, limit, d_err, &keep, &base);
    if (base) cudaFreeAsync(base, st);
    if (d_err) {
        cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(d_err, st);
    }
    const cudaError_t e2 = cudaStreamSynchronize(st);
    keep.release();
    cudaStreamDestroy(st);
    if (rc == SV_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "wave self-test");
    cudaGetLastError();
    *host_status = herr == 2 ? 1 : 0;
    return rc;
}
