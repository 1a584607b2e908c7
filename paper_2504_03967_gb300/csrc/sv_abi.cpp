// C ABI entry points of libsv (declared in include/sv.h).
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>
#include <new>
#include <string>

#include "sv_internal.h"

namespace sv {

namespace {
thread_local std::string t_err;
std::atomic<uint64_t> g_launches{0};
}  // namespace

int set_error(int code, const std::string& msg) {
    t_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return set_error(SV_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void count_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// SM count of the current device, looked up once per device ordinal.
int device_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    if (dev < 0 || dev >= 64) dev = 0;
    int s = cache[dev].load(std::memory_order_relaxed);
    if (s <= 0) {
        if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0) {
            cudaGetLastError();
            s = 148;
        }
        cache[dev].store(s, std::memory_order_relaxed);
    }
    return s;
}

void reset_perm(sv_state* h) {
    for (int q = 0; q < 64; ++q) h->perm[q] = q;
    h->permuted = false;
}

QubitMap qubit_map(const sv_state* h) {
    QubitMap m;
    m.n = h->n;
    for (int q = 0; q < 40; ++q) m.phys[q] = q < h->n ? h->perm[q] : q;
    return m;
}

int ensure_scratch(Scratch* s, size_t bytes, cudaStream_t st) {
    if (s->cap >= bytes) return SV_OK;
    if (s->ptr) {
        cudaError_t e = cudaFreeAsync(s->ptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync(scratch)");
        s->ptr = nullptr;
        s->cap = 0;
    }
    size_t cap = bytes < 4096 ? 4096 : bytes;
    cudaError_t e = cudaMallocAsync(&s->ptr, cap, st);
    if (e != cudaSuccess) {
        s->ptr = nullptr;
        cudaGetLastError();
        return set_error(SV_ENOMEM, "scratch allocation of " + std::to_string(cap) + " bytes failed");
    }
    s->cap = cap;
    return SV_OK;
}

int ensure_pinned(Scratch* s, size_t bytes) {
    if (s->cap >= bytes) return SV_OK;
    if (s->ptr) cudaFreeHost(s->ptr);
    s->ptr = nullptr;
    s->cap = 0;
    size_t cap = bytes < 65536 ? 65536 : bytes * 2;
    cudaError_t e = cudaMallocHost(&s->ptr, cap);
    if (e != cudaSuccess) {
        s->ptr = nullptr;
        cudaGetLastError();
        return set_error(SV_ENOMEM, "pinned staging allocation failed");
    }
    s->cap = cap;
    return SV_OK;
}

// The fields of each gate record the library reads: type, nq, the first nq
// qubits and the type's parameters (three for U3, one for RX, RY, RZ, P and
// CP, none otherwise); every other entry is zeroed, so records that differ
// only in ignored entries share a plan.
void used_fields(const sv_gate* gates, size_t count, std::vector<sv_gate>* out) {
    out->assign(count, sv_gate{});
    for (size_t i = 0; i < count; ++i) {
        const sv_gate& g = gates[i];
        sv_gate& r = (*out)[i];
        r.type = g.type;
        r.nq = g.nq;
        for (uint32_t a = 0; a < g.nq && a < 3; ++a) r.q[a] = g.q[a];
        const uint32_t t = g.type;
        const int np = t == SV_U3 ? 3 : ((t == SV_RX || t == SV_RY || t == SV_RZ || t == SV_P || t == SV_CP) ? 1 : 0);
        for (int a = 0; a < np; ++a) r.p[a] = g.p[a];
    }
}

// Key of a plan: FNV-1a over the used fields of the gate records, the
// options that shape the plan, the state's size and type, and the qubit map
// it starts from.  A cache hit also compares the records themselves.
uint64_t plan_key(const sv_state* h, const std::vector<sv_gate>& recs, const sv_options* opt) {
    uint64_t k = 1469598103934665603ull;
    auto mix = [&k](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) k = (k ^ b[i]) * 1099511628211ull;
    };
    for (const sv_gate& r : recs) {
        mix(&r.type, sizeof(uint32_t) * 5);  // type, nq, q[3]
        mix(r.p, sizeof(double) * 3);
    }
    const int hdr[3] = {h->n, h->dtype, h->permuted ? 1 : 0};
    mix(hdr, sizeof(hdr));
    if (opt) {
        const int f[9] = {opt->k_max, opt->tile_m, opt->planner, opt->tensor, opt->pass_kernel, opt->relabel, opt->mux,
                          opt->jit, 1};
        mix(f, sizeof(f));
        mix(&opt->drop_phase_below, sizeof(double));
    }
    if (h->permuted) mix(h->perm, sizeof(int) * h->n);
    return k ? k : 1;
}

bool same_records(const std::vector<sv_gate>& a, const std::vector<sv_gate>& b) {
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
        if (memcmp(&a[i].type, &b[i].type, sizeof(uint32_t) * 5) || memcmp(a[i].p, b[i].p, sizeof(double) * 3))
            return false;
    return true;
}

int flush_init(sv_state* h) {
    if (h->pending_basis < 0) return SV_OK;
    const uint64_t x = (uint64_t)h->pending_basis;
    h->pending_basis = -1;
    cudaError_t e = launch_init_basis(h, x);
    if (e != cudaSuccess) {
        h->bad = true;
        return cuda_fail(e, "init_basis");
    }
    return SV_OK;
}

}  // namespace sv

using namespace sv;

namespace {

int check_handle_noflush(sv_handle h) {
    if (!h) return set_error(SV_EINVAL, "NULL handle");
    if (h->bad) return set_error(SV_ESTATE, "state flagged by an earlier CUDA failure; re-initialise it");
    return SV_OK;
}

// Entry points that use the amplitudes first write a deferred basis state.
int check_handle(sv_handle h) {
    int rc = check_handle_noflush(h);
    if (rc == SV_OK) rc = flush_init(h);
    return rc;
}

int max_qubits(int dt) { return dt == SV_C64 ? kMaxQubitsC64 : kMaxQubitsC128; }

size_t amp_bytes(int dt) { return dt == SV_C64 ? 8 : 16; }

int make_handle(int n, sv_dtype dt, void* amps, bool owned, void* stream, sv_handle* out) {
    sv_state* h = new (std::nothrow) sv_state();
    if (!h) return set_error(SV_ENOMEM, "host allocation failed");
    h->n = n;
    h->dtype = dt;
    h->amps = amps;
    h->owned = owned;
    h->stream = (cudaStream_t)stream;
    h->bad = false;
    h->ev_used = 0;
    h->upload_ev = nullptr;
    h->upload_pending = false;
    h->pending_basis = -1;
    h->plans = nullptr;
    reset_perm(h);
    memset(&h->last_opts, 0, sizeof(h->last_opts));
    *out = h;
    return SV_OK;
}

// Next free event of the recorder pool (created on demand).
cudaEvent_t next_event(sv_handle h) {
    if (h->ev_used == (int)h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

int fail_state(sv_handle h, int rc) {
    if (rc == SV_ECUDA || rc == SV_ETIMEOUT) h->bad = true;
    return rc;
}

// Copy a result to the host and wait; also reads the device error word that
// the kernels' bounded waits set when they give up (SV_ETIMEOUT).
int sync_d2h(sv_handle h, void* host, const void* dev, size_t bytes, const char* what) {
    int dev_err = 0;
    cudaError_t e = cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && h->err.ptr)
        e = cudaMemcpyAsync(&dev_err, h->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail_state(h, cuda_fail(e, what));
    if (dev_err) {
        cudaMemsetAsync(h->err.ptr, 0, sizeof(int), h->stream);
        return fail_state(h, set_error(SV_ETIMEOUT, "a bounded device wait gave up (tensor-core pass)"));
    }
    return SV_OK;
}

}  // namespace

extern "C" {

int sv_version(void) { return 100; }

const char* sv_last_error(void) { return t_err.c_str(); }

uint64_t sv_launch_count(void) { return g_launches.load(); }

int sv_alloc(int n, sv_dtype dt, void* cuda_stream, sv_handle* out) {
    if (!out) return set_error(SV_EINVAL, "NULL output handle pointer");
    *out = nullptr;
    if (dt != SV_C64 && dt != SV_C128) return set_error(SV_EINVAL, "unknown dtype");
    if (n < 1 || n > max_qubits(dt))
        return set_error(SV_EINVAL, "n = " + std::to_string(n) + " out of range 1.." + std::to_string(max_qubits(dt)));
    const size_t bytes = amp_bytes(dt) << n;
    size_t freeb = 0, totalb = 0;
    cudaError_t e = cudaMemGetInfo(&freeb, &totalb);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    if (bytes > freeb)
        return set_error(SV_ENOMEM, "state of " + std::to_string(bytes) + " bytes exceeds free device memory " +
                                        std::to_string(freeb));
    void* p = nullptr;
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(SV_ENOMEM, std::string("cudaMalloc(state): ") + cudaGetErrorString(e));
    }
    int rc = make_handle(n, dt, p, true, cuda_stream, out);
    if (rc) cudaFree(p);
    return rc;
}

int sv_attach(int n, sv_dtype dt, void* dev_amps, void* cuda_stream, sv_handle* out) {
    if (!out) return set_error(SV_EINVAL, "NULL output handle pointer");
    *out = nullptr;
    if (!dev_amps) return set_error(SV_EINVAL, "NULL device pointer");
    if (((uintptr_t)dev_amps & 15) != 0) return set_error(SV_EINVAL, "device pointer not 16-byte aligned");
    if (dt != SV_C64 && dt != SV_C128) return set_error(SV_EINVAL, "unknown dtype");
    if (n < 1 || n > max_qubits(dt)) return set_error(SV_EINVAL, "n out of range");
    return make_handle(n, dt, dev_amps, false, cuda_stream, out);
}

int sv_free(sv_handle h) {
    if (!h) return SV_OK;
    cudaStreamSynchronize(h->stream);
    if (h->owned && h->amps) cudaFree(h->amps);
    if (h->plan_dev.ptr) cudaFree(h->plan_dev.ptr);
    if (h->red.ptr) cudaFree(h->red.ptr);
    if (h->out_dev.ptr) cudaFree(h->out_dev.ptr);
    if (h->err.ptr) cudaFree(h->err.ptr);
    if (h->perm_tmp.ptr) cudaFree(h->perm_tmp.ptr);
    if (h->aux.ptr) cudaFree(h->aux.ptr);
    if (h->lcdf.ptr) cudaFree(h->lcdf.ptr);
    delete h->plans;
    if (h->host_pin.ptr) cudaFreeHost(h->host_pin.ptr);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->upload_ev) cudaEventDestroy(h->upload_ev);
    cudaGetLastError();
    delete h;
    return SV_OK;
}

int sv_set_stream(sv_handle h, void* cuda_stream) {
    if (!h) return set_error(SV_EINVAL, "NULL handle");
    if (!h->bad) flush_init(h);
    cudaStreamSynchronize(h->stream);
    h->stream = (cudaStream_t)cuda_stream;
    return SV_OK;
}

int sv_info(sv_handle h, int* n, int* dtype, void** dev_amps) {
    if (!h) return set_error(SV_EINVAL, "NULL handle");
    if (dev_amps && !h->bad) {  // the caller may read the amplitudes through the pointer
        const int rc = flush_init(h);
        if (rc) return rc;
    }
    if (n) *n = h->n;
    if (dtype) *dtype = h->dtype;
    if (dev_amps) *dev_amps = h->amps;
    return SV_OK;
}

int sv_init_basis(sv_handle h, uint64_t x) {
    if (!h) return set_error(SV_EINVAL, "NULL handle");
    if (x >> h->n) return set_error(SV_EINVAL, "basis index out of range");
    // Deferred: the next apply's first compiled pass builds its tiles from x
    // (no write and read of the state); anything else writes it first.
    h->pending_basis = (long long)x;
    h->bad = false;
    reset_perm(h);
    return SV_OK;
}

int sv_load_state(sv_handle h, const void* host_amps) {
    if (!h) return set_error(SV_EINVAL, "NULL handle");
    if (!host_amps) return set_error(SV_EINVAL, "NULL host buffer");
    h->pending_basis = -1;
    cudaError_t e = cudaMemcpyAsync(h->amps, host_amps, amp_bytes(h->dtype) << h->n, cudaMemcpyHostToDevice,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        h->bad = true;
        return cuda_fail(e, "load_state");
    }
    h->bad = false;
    reset_perm(h);
    return SV_OK;
}

int sv_store_state(sv_handle h, void* host_amps) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!host_amps) return set_error(SV_EINVAL, "NULL host buffer");
    if (!h->permuted) return sync_d2h(h, host_amps, h->amps, amp_bytes(h->dtype) << h->n, "store_state");
    // relabelled qubits: gather logical order chunk by chunk through device staging
    const uint64_t N = 1ull << h->n, chunk = std::min<uint64_t>(N, 1ull << 22);
    rc = ensure_scratch(&h->out_dev, amp_bytes(h->dtype) * chunk, h->stream);
    if (rc) return rc;
    for (uint64_t x0 = 0; x0 < N; x0 += chunk) {
        cudaError_t e = launch_gather_logical(h, x0, chunk, h->out_dev.ptr);
        if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "store_state gather"));
        rc = sync_d2h(h, (char*)host_amps + amp_bytes(h->dtype) * x0, h->out_dev.ptr, amp_bytes(h->dtype) * chunk,
                      "store_state");
        if (rc) return rc;
    }
    return SV_OK;
}

int sv_plan_circuit(int n, sv_dtype dt, const sv_gate* gates, size_t count, const sv_options* opt,
                    sv_plan_info* info) {
    if (!info) return set_error(SV_EINVAL, "NULL info");
    if (dt != SV_C64 && dt != SV_C128) return set_error(SV_EINVAL, "unknown dtype");
    if (n < 1 || n > max_qubits(dt)) return set_error(SV_EINVAL, "n out of range");
    if (count && !gates) return set_error(SV_EINVAL, "NULL gate list");
    std::vector<CGate> cg;
    size_t bad = 0;
    if (canonicalise(n, gates, count, &cg, &bad) != SV_OK)
        return set_error(SV_EINVAL, "invalid gate record at index " + std::to_string(bad));
    const PlanOptions po = resolve_options(n, dt, opt);
    const size_t before = cg.size();
    drop_small_phases(&cg, po.drop_phase_below);
    Plan plan;
    if (po.planner == SV_PLAN_PLAIN) {
        plan_plain(n, dt, cg, &plan);
    } else {
        std::vector<CGate> muxed;
        std::vector<Mux> muxes;
        const bool rec = recognise_mux(n, cg, &muxed, &muxes, po.mux);
        plan_greedy(n, dt, rec ? muxed : cg, po, &plan, &muxes);
    }
    plan.gates = (int64_t)(count - (before - cg.size()));
    plan_summary(plan, info);
    if (!plan.plain) {  // which passes the register-resident kernel takes
        PlanBlob blob;
        serialise_plan(plan, &blob);
        const PassDev* pd = (const PassDev*)(blob.bytes.data() + blob.pass_off);
        for (int i = 0; i < blob.npasses; ++i) {
            if (pd[i].rmode != 1 && pd[i].rmode != 2) continue;
            info->reg_passes++;
            const OpDev* od = (const OpDev*)(blob.bytes.data() + pd[i].region_off);
            for (int o = 0; o < pd[i].nops; ++o) {
                info->remaps += od[o].kind == OP_REMAP;
                info->warp_remaps += od[o].kind == OP_REMAP && od[o].nrec == 1;
            }
        }
    }
    return SV_OK;
}

int sv_plan_ops(int n, sv_dtype dt, const sv_gate* gates, size_t count, const sv_options* opt, sv_plan_op* ops,
                size_t ops_cap, size_t* nops, int* recs, size_t recs_cap, size_t* nrecs, double* data,
                size_t data_cap, size_t* ndata) {
    if (!nops || !nrecs || !ndata) return set_error(SV_EINVAL, "NULL count");
    if (dt != SV_C64 && dt != SV_C128) return set_error(SV_EINVAL, "unknown dtype");
    if (n < 1 || n > max_qubits(dt)) return set_error(SV_EINVAL, "n out of range");
    if (count && !gates) return set_error(SV_EINVAL, "NULL gate list");
    std::vector<CGate> cg;
    size_t bad = 0;
    if (canonicalise(n, gates, count, &cg, &bad) != SV_OK)
        return set_error(SV_EINVAL, "invalid gate record at index " + std::to_string(bad));
    const PlanOptions po = resolve_options(n, dt, opt);
    if (po.planner != SV_PLAN_GREEDY) return set_error(SV_EUNSUPPORTED, "sv_plan_ops describes greedy plans");
    drop_small_phases(&cg, po.drop_phase_below);
    std::vector<CGate> muxed;
    std::vector<Mux> muxes;
    const bool rec = recognise_mux(n, cg, &muxed, &muxes, po.mux);
    Plan plan;
    plan_greedy(n, dt, rec ? muxed : cg, po, &plan, &muxes);
    size_t no = 0, nr = 0, nd = 0;
    auto put_d = [&](double v) {
        if (data && nd < data_cap) data[nd] = v;
        ++nd;
    };
    for (size_t pi = 0; pi < plan.passes.size(); ++pi) {
        const HostPass& hp = plan.passes[pi];
        std::vector<sv_plan_op> out;
        for (int mi : hp.mux) {
            const Mux& M = plan.muxes[(size_t)mi];
            sv_plan_op r;
            memset(&r, 0, sizeof(r));
            r.pass = (int)pi;
            r.kind = 3;
            r.k = 1;
            r.q[0] = M.target;
            r.rec_off = (int)nr;
            r.data_off = (int64_t)nd;
            put_d(M.family);
            put_d((double)M.flip);
            put_d(M.flip_c);
            put_d((double)M.controls.size());
            for (int c : M.controls) put_d(c);
            for (double v : M.phi0) put_d(v);
            if (M.family != MUX_Y)
                for (double v : M.phi1) put_d(v);
            out.push_back(r);
        }
        for (const HostOp& o : hp.ops) {
            sv_plan_op r;
            memset(&r, 0, sizeof(r));
            r.pass = (int)pi;
            r.rec_off = (int)nr;
            r.data_off = (int64_t)nd;
            if (o.kind == OP_DIAG) {
                r.kind = 1;
                put_d(o.diag.c);
                for (int q = 0; q < n; ++q) put_d(o.diag.a[(size_t)q]);
                for (size_t i = 0; i < (size_t)n * n; ++i) put_d(o.diag.b[i]);
            } else {
                r.k = (int)o.qubits.size();
                for (int i = 0; i < r.k && i < 5; ++i) r.q[i] = o.qubits[(size_t)i];
                if (o.kind == OP_GATES) {
                    r.kind = 2;
                    r.nrec = (int)o.recs.size();
                    for (const GateRec& g : o.recs) {
                        const int w[4] = {g.kind, g.a, g.b, g.off};
                        for (int j = 0; j < 4; ++j) {
                            if (recs && nr < recs_cap) recs[nr] = w[j];
                            ++nr;
                        }
                    }
                    for (const cd& v : o.gdata) put_d(v.real()), put_d(v.imag());
                } else {
                    r.kind = 0;
                    for (const cd& v : o.mat) put_d(v.real()), put_d(v.imag());
                }
            }
            out.push_back(r);
        }
        for (const sv_plan_op& r : out) {
            if (ops && no < ops_cap) ops[no] = r;
            ++no;
        }
    }
    *nops = no;
    *nrecs = nr;
    *ndata = nd;
    if (no > ops_cap || nr > recs_cap || nd > data_cap)
        return set_error(SV_EINVAL, "buffers too small (the counts are returned)");
    return SV_OK;
}

int sv_apply_circuit(sv_handle h, const sv_gate* gates, size_t count, const sv_options* opt) {
    int rc = check_handle_noflush(h);
    if (rc) return rc;
    if (count && !gates) return set_error(SV_EINVAL, "NULL gate list");
    // the plain planner has no plan; the cost-model planner's plans are kept
    // once its judge has settled on a candidate for the circuit
    const bool cacheable = count && (!opt || opt->planner != SV_PLAN_PLAIN);
    uint64_t key = 0;
    std::vector<sv_gate> recs;
    if (cacheable) {
        used_fields(gates, count, &recs);
        key = plan_key(h, recs, opt);
        if (h->plans) {
            for (auto& kv : h->plans->entries) {
                if (kv.first != key) continue;
                CachedPlan& c = kv.second;
                if (!same_records(c.recs, recs)) continue;  // a hash collision: not this circuit
                c.stamp = ++h->plans->clock;
                memcpy(h->perm, c.perm_after, sizeof(h->perm));
                h->permuted = c.permuted_after;
                h->last_opts = c.last_opts;
                return launch_plan(h, c.plan, c.blob, opt && opt->record, nullptr, nullptr, &c.jit_srcs);
            }
        }
    }
    std::vector<CGate> cg;
    size_t bad = 0;
    if (canonicalise(h->n, gates, count, &cg, &bad) != SV_OK)
        return set_error(SV_EINVAL, "invalid gate record at index " + std::to_string(bad));
    return sv::apply_canonical(h, gates, count, cg, opt, key, &recs);
}

}  // extern "C"

namespace sv {

int apply_canonical(sv_state* h, const sv_gate* gates, size_t count, const std::vector<CGate>& cg,
                    const sv_options* opt, uint64_t cache_key, const std::vector<sv_gate>* recs) {
    int rc = SV_OK;
    if (cg.empty()) return SV_OK;
    PlanOptions po = resolve_options(h->n, h->dtype, opt);
    memset(&h->last_opts, 0, sizeof(h->last_opts));
    // Relabelling: gates act on the physical bits of their logical qubits; with
    // relabel on, a SWAP only exchanges two entries of the map.
    uint64_t salt = 0;
    std::vector<CGate> mapped;
    const std::vector<CGate>* gl = &cg;
    std::vector<CGate> approx;
    if (po.drop_phase_below > 0.0) {
        approx = cg;
        drop_small_phases(&approx, po.drop_phase_below);
        gl = &approx;
        salt ^= 0x51ed270b27f1c0d5ull ^ (uint64_t)(po.drop_phase_below * 1e12);
    }
    if (po.relabel || h->permuted) {
        if (h->permuted) {
            uint64_t ps = 1469598103934665603ull;
            for (int q = 0; q < h->n; ++q) ps = (ps ^ (uint64_t)h->perm[q]) * 1099511628211ull;
            salt ^= ps;
        }
        if (po.relabel) salt ^= 0x9e3779b97f4a7c15ull;
        mapped.reserve(gl->size());
        for (const CGate& g : *gl) {
            if (po.relabel && g.type == SV_SWAP) {
                std::swap(h->perm[g.q[0]], h->perm[g.q[1]]);
                continue;
            }
            CGate x = g;
            for (int i = 0; i < g.nq; ++i) x.q[i] = h->perm[g.q[i]];
            mapped.push_back(x);
        }
        h->permuted = false;
        for (int q = 0; q < h->n; ++q) h->permuted |= h->perm[q] != q;
        gl = &mapped;
        if (mapped.empty()) return SV_OK;
    }
    Plan plan;
    if (po.planner == SV_PLAN_PLAIN) {
        rc = flush_init(h);
        if (rc) return rc;
        const std::vector<CGate>& cgm = *gl;
        plan_plain(h->n, h->dtype, cgm, &plan);
        for (const PlainOp& op : plan.plain_ops) {
            cudaError_t e = launch_plain_op(h, op);
            if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "plain gate kernel"));
        }
        return SV_OK;
    }
    std::vector<CGate> muxed;
    std::vector<Mux> muxes;
    if (recognise_mux(h->n, *gl, &muxed, &muxes, po.mux)) {
        gl = &muxed;
        salt ^= 0x2545f4914f6cdd1dull + (uint64_t)po.mux;
    }
    const std::vector<CGate>& cgm = *gl;
    cudaEvent_t judge0 = nullptr, judge1 = nullptr;
    std::shared_ptr<const Plan> learned;
    if (po.planner == SV_PLAN_MLP)
        po = mlp_plan_options(h, gates, count, cgm, &muxes, po, salt, &judge0, &judge1, &learned);
    if (learned) plan = *learned;
    else plan_greedy(h->n, h->dtype, cgm, po, &plan, &muxes);
    h->last_opts.k_max = po.k_max;
    h->last_opts.tile_m = po.tile_m;
    h->last_opts.planner = opt ? opt->planner : SV_PLAN_GREEDY;
    h->last_opts.tensor = po.tensor == 0 ? 1 : (po.tc_auto ? 0 : -1);
    h->last_opts.pass_kernel = po.pass_kernel;
    h->last_opts.relabel = po.relabel;
    h->last_opts.mux = po.mux;
    h->last_opts.jit = po.jit;
    h->last_opts.drop_phase_below = po.drop_phase_below;
    PlanBlob blob;
    serialise_plan(plan, &blob);
    if (cache_key && recs && !judge0) {  // keep it for the next apply of the same circuit (not while the judge times)
        if (!h->plans) h->plans = new (std::nothrow) PlanCache();
        if (h->plans) {
            auto& es = h->plans->entries;
            if ((int)es.size() >= kPlanCacheEntries) {
                size_t old = 0;
                for (size_t i = 1; i < es.size(); ++i)
                    if (es[i].second.stamp < es[old].second.stamp) old = i;
                es.erase(es.begin() + old);
            }
            es.emplace_back(cache_key, CachedPlan());
            CachedPlan& c = es.back().second;
            c.plan = plan;
            c.blob = blob;
            if (recs) c.recs = *recs;
            memcpy(c.perm_after, h->perm, sizeof(h->perm));
            c.permuted_after = h->permuted;
            c.last_opts = h->last_opts;
            c.stamp = ++h->plans->clock;
        }
    }
    return launch_plan(h, plan, blob, opt && opt->record, judge0, judge1);
}

int launch_plan(sv_state* h, const Plan& plan, const PlanBlob& blob, bool rec, cudaEvent_t judge0,
                cudaEvent_t judge1, std::vector<std::string>* jit_srcs) {
    int rc = SV_OK;
    // Compiled kernels (compiles happen here, before any timing event).  A
    // deferred |x> is built by pass 0's tile loads when that pass has a
    // compiled kernel for it; otherwise it is written now.
    std::vector<void*> jit_fns;
    void* fill0 = nullptr;
    jit_prepare(h, blob, plan.jit, h->pending_basis, &jit_fns, &fill0, jit_srcs);
    // the judge times everything the call puts on the stream from here on
    // (a deferred |x> written by its own kernel included), as a caller does
    if (judge0) cudaEventRecord(judge0, h->stream);
    long long basis = -1;
    if (h->pending_basis >= 0) {
        if (fill0) {
            basis = h->pending_basis;
            jit_fns[0] = fill0;
            h->pending_basis = -1;
        } else {
            rc = flush_init(h);
            if (rc) return rc;
        }
    }
    // Stage through pinned memory; only the previous upload from it has to
    // be finished (the passes of earlier calls may still be running).
    cudaError_t e = cudaSuccess;
    if (h->upload_pending) {
        e = cudaEventSynchronize(h->upload_ev);
        if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "upload event"));
        h->upload_pending = false;
    }
    if (!h->upload_ev) {
        e = cudaEventCreateWithFlags(&h->upload_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
    rc = ensure_pinned(&h->host_pin, blob.bytes.size());
    if (rc) return rc;
    rc = ensure_scratch(&h->plan_dev, blob.bytes.size(), h->stream);
    if (rc) return rc;
    if (!h->err.ptr) {
        rc = ensure_scratch(&h->err, 64, h->stream);
        if (rc) return rc;
        e = cudaMemsetAsync(h->err.ptr, 0, 64, h->stream);
        if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "error word"));
    }
    memcpy(h->host_pin.ptr, blob.bytes.data(), blob.bytes.size());
    if (basis >= 0) ((PassDev*)((char*)h->host_pin.ptr + blob.pass_off))[0].basis = basis;
    e = cudaMemcpyAsync(h->plan_dev.ptr, h->host_pin.ptr, blob.bytes.size(), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "plan upload"));
    e = cudaEventRecord(h->upload_ev, h->stream);
    if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "upload event"));
    h->upload_pending = true;
    for (int p = 0; p < blob.npasses; ++p) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (rec && (e0 = next_event(h)) && (e1 = next_event(h))) cudaEventRecord(e0, h->stream);
        bool jitted = false;
        e = jit_launch(h, jit_fns[p], h->plan_dev.ptr, blob, p, &jitted);
        if (e == cudaSuccess && jitted && p == 0 && basis >= 0) jit_count_fill();
        if (e == cudaSuccess && !jitted) e = launch_pass(h, h->plan_dev.ptr, blob, p, plan.passes[p]);
        if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "tile pass kernel"));
        if (rec && e1) {
            cudaEventRecord(e1, h->stream);
            const PassDev* pd = (const PassDev*)(blob.bytes.data() + blob.pass_off) + p;
            h->rec_feat.push_back(pass_features(h->n, h->dtype, plan.passes[p], plan.tensor == 0, pd->rmode == 1 || pd->rmode == 2));
        }
    }
    if (judge1) cudaEventRecord(judge1, h->stream);
    return SV_OK;
}

}  // namespace sv

extern "C" {

int sv_pass_times(sv_handle h, double* host_ms, float* host_feat, int cap, int* count) {
    if (!h || !count) return set_error(SV_EINVAL, "NULL argument");
    const int np = h->ev_used / 2;
    *count = np;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "stream sync"));
    for (int i = 0; i < np && i < cap; ++i) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        if (host_ms) host_ms[i] = ms;
        if (host_feat)
            for (int f = 0; f < kFeatures; ++f) host_feat[(size_t)i * kFeatures + f] = h->rec_feat[i][f];
    }
    h->ev_used = 0;
    h->rec_feat.clear();
    return SV_OK;
}

int sv_feature_count(void) { return kFeatures; }

int sv_probs_device(sv_handle h, double* dev_out) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!dev_out) return set_error(SV_EINVAL, "NULL output");
    cudaError_t e = launch_probs(h, dev_out);
    if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "probs"));
    return SV_OK;
}

int sv_probs(sv_handle h, double* host_out) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!host_out) return set_error(SV_EINVAL, "NULL output");
    const size_t bytes = sizeof(double) << h->n;
    rc = ensure_scratch(&h->out_dev, bytes, h->stream);
    if (rc) return rc;
    cudaError_t e = launch_probs(h, (double*)h->out_dev.ptr);
    if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "probs"));
    return sync_d2h(h, host_out, h->out_dev.ptr, bytes, "probs readback");
}

int sv_norm(sv_handle h, double* host_out) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!host_out) return set_error(SV_EINVAL, "NULL output");
    return fail_state(h, measure_norm(h, host_out));
}

int sv_expect_z_device(sv_handle h, double* dev_out) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!dev_out) return set_error(SV_EINVAL, "NULL output");
    return fail_state(h, measure_expect_z(h, dev_out));
}

int sv_expect_z(sv_handle h, double* host_out) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!host_out) return set_error(SV_EINVAL, "NULL output");
    rc = ensure_scratch(&h->out_dev, sizeof(double) * 64, h->stream);
    if (rc) return rc;
    rc = measure_expect_z(h, (double*)h->out_dev.ptr);
    if (rc) return fail_state(h, rc);
    return sync_d2h(h, host_out, h->out_dev.ptr, sizeof(double) * h->n, "expect_z readback");
}

int sv_sample_device(sv_handle h, uint64_t shots, uint64_t seed, uint64_t* dev_out) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (shots && !dev_out) return set_error(SV_EINVAL, "NULL output");
    return fail_state(h, measure_sample(h, shots, seed, nullptr, dev_out));
}

int sv_sample(sv_handle h, uint64_t shots, uint64_t seed, uint64_t* host_out) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (shots == 0) return SV_OK;
    if (!host_out) return set_error(SV_EINVAL, "NULL output");
    rc = ensure_scratch(&h->out_dev, sizeof(uint64_t) * shots, h->stream);
    if (rc) return rc;
    rc = measure_sample(h, shots, seed, nullptr, (uint64_t*)h->out_dev.ptr);
    if (rc) return fail_state(h, rc);
    return sync_d2h(h, host_out, h->out_dev.ptr, sizeof(uint64_t) * shots, "sample readback");
}

int sv_qcrank_decode_device(const uint64_t* samples, uint64_t shots, int a, int d, uint64_t* counts, uint64_t* ones,
                            double* pixels, void* stream) {
    if (a < 1 || d < 1 || d > 32 || a > kQcrankMaxAddr || a + d > 63) return set_error(SV_EINVAL, "a or d out of range");
    if ((shots && !samples) || !counts || !ones || !pixels) return set_error(SV_EINVAL, "NULL buffer");
    cudaError_t e = launch_qcrank_decode(samples, shots, a, d, counts, ones, pixels, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "qcrank decode");
    return SV_OK;
}

int sv_qcrank_reconstruct(sv_handle h, int a, int d, uint64_t shots, uint64_t seed, double* host_pixels,
                          uint64_t* host_counts) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (a < 1 || d < 1 || d > 32 || a > kQcrankMaxAddr || a + d > h->n) return set_error(SV_EINVAL, "a or d out of range");
    if (!host_pixels) return set_error(SV_EINVAL, "NULL output");
    const size_t J = (size_t)1 << a;
    const size_t bytes = sizeof(uint64_t) * (shots + J + J * d) + sizeof(double) * J * d;
    rc = ensure_scratch(&h->aux, bytes, h->stream);
    if (rc) return rc;
    uint64_t* samples = (uint64_t*)h->aux.ptr;
    uint64_t* counts = samples + shots;
    uint64_t* ones = counts + J;
    double* pixels = (double*)(ones + J * d);
    rc = measure_sample(h, shots, seed, nullptr, samples);
    if (rc) return fail_state(h, rc);
    cudaError_t e = launch_qcrank_decode(samples, shots, a, d, counts, ones, pixels, h->stream);
    if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "qcrank decode"));
    if (host_counts) {
        rc = sync_d2h(h, host_counts, counts, sizeof(uint64_t) * J, "qcrank counts");
        if (rc) return rc;
    }
    return sync_d2h(h, host_pixels, pixels, sizeof(double) * J * d, "qcrank pixels");
}

int sv_sample_uniforms(sv_handle h, const double* host_u, uint64_t shots, uint64_t* host_out) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (shots == 0) return SV_OK;
    if (!host_u || !host_out) return set_error(SV_EINVAL, "NULL buffer");
    for (uint64_t s = 0; s < shots; ++s)
        if (!(host_u[s] >= 0.0 && host_u[s] < 1.0)) return set_error(SV_EINVAL, "uniform outside [0,1)");
    rc = ensure_scratch(&h->out_dev, 16 * shots, h->stream);
    if (rc) return rc;
    double* du = (double*)h->out_dev.ptr;
    uint64_t* dout = (uint64_t*)(du + shots);
    cudaError_t e = cudaMemcpyAsync(du, host_u, sizeof(double) * shots, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "uniforms upload"));
    rc = measure_sample(h, shots, 0, du, dout);
    if (rc) return fail_state(h, rc);
    return sync_d2h(h, host_out, dout, sizeof(uint64_t) * shots, "sample readback");
}


int sv_qubit_map(sv_handle h, int* map) {
    if (!h) return set_error(SV_EINVAL, "NULL handle");
    if (!map) return set_error(SV_EINVAL, "NULL output");
    for (int q = 0; q < h->n; ++q) map[q] = h->perm[q];
    return SV_OK;
}

int sv_materialize(sv_handle h) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->permuted) return SV_OK;
    // physical SWAPs that bring every logical qubit to its own bit
    int perm[64];
    for (int q = 0; q < h->n; ++q) perm[q] = h->perm[q];
    std::vector<sv_gate> sw;
    for (int q = 0; q < h->n; ++q) {
        if (perm[q] == q) continue;
        int q2 = 0;
        while (perm[q2] != q) ++q2;  // the logical qubit stored at bit q
        sv_gate g;
        memset(&g, 0, sizeof(g));
        g.type = SV_SWAP;
        g.nq = 2;
        g.q[0] = (uint32_t)perm[q];
        g.q[1] = (uint32_t)q;
        sw.push_back(g);
        perm[q2] = perm[q];
        perm[q] = q;
    }
    std::vector<CGate> cg;
    size_t bad = 0;
    if (canonicalise(h->n, sw.data(), sw.size(), &cg, &bad) != SV_OK) return set_error(SV_EINVAL, "internal: swap list");
    reset_perm(h);  // the swaps below act on physical bits
    sv_options o;
    memset(&o, 0, sizeof(o));
    return apply_canonical(h, sw.data(), sw.size(), cg, &o);
}

int sv_last_plan(sv_handle h, sv_options* out) {
    if (!h) return set_error(SV_EINVAL, "NULL handle");
    if (!out) return set_error(SV_EINVAL, "NULL output");
    *out = h->last_opts;
    return SV_OK;
}

}  // extern "C"

extern "C" int sv_measure_device(sv_handle h, uint64_t shots, uint64_t seed, uint64_t* dev_samples,
                                 double* dev_expz) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (shots && !dev_samples) return set_error(SV_EINVAL, "NULL samples output");
    return fail_state(h, measure_readout(h, dev_samples ? shots : 0, seed, dev_samples, dev_expz));
}

// Host outputs of sv_measure_device: one read of the state for both.
extern "C" int sv_measure(sv_handle h, uint64_t shots, uint64_t seed, uint64_t* host_samples, double* host_expz) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (shots && !host_samples) return set_error(SV_EINVAL, "NULL samples output");
    if (!host_samples) shots = 0;
    const size_t sb = sizeof(uint64_t) * shots, eb = host_expz ? sizeof(double) * h->n : 0;
    if (!sb && !eb) return SV_OK;
    rc = ensure_scratch(&h->out_dev, sb + eb, h->stream);
    if (rc) return rc;
    uint64_t* ds = sb ? (uint64_t*)h->out_dev.ptr : nullptr;
    double* de = eb ? (double*)((char*)h->out_dev.ptr + sb) : nullptr;
    rc = measure_readout(h, shots, seed, ds, de);
    if (rc) return fail_state(h, rc);
    if (eb && sb) {
        cudaError_t e = cudaMemcpyAsync(host_samples, ds, sb, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return fail_state(h, cuda_fail(e, "samples readback"));
        return sync_d2h(h, host_expz, de, eb, "expz readback");
    }
    return sb ? sync_d2h(h, host_samples, ds, sb, "samples readback") : sync_d2h(h, host_expz, de, eb, "expz readback");
}
