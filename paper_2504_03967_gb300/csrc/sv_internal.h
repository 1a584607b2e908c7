// Internal declarations shared by the libsv translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <memory>
#include <string>
#include <vector>

#include "sv.h"
#include "sv_dev.h"

namespace sv {

using cd = std::complex<double>;

constexpr int kMaxQubitsC64 = 34;
constexpr int kMaxQubitsC128 = 33;
constexpr int kQcrankMaxAddr = 26;  // address qubits of the QCrank read-out

// ---------------------------------------------------------------------------
// Canonical gates (host, FP64).  A gate is either dense (a 2^k x 2^k matrix,
// local bit i <-> qubit q[i]) or diagonal (phase e^{i ph[j]} on local index
// j, same bit convention).  MEASURE records are dropped.
// ---------------------------------------------------------------------------
// GK_MUX: a recognised multiplexor standing for a run of gates (q[0] = its
// target, mux = index into the recognised set).
enum GateKind { GK_DENSE = 0, GK_DIAG = 1, GK_MUX = 2 };

struct CGate {
    int kind;
    int nq;
    int q[2];
    cd m[16];       // dense: row-major 2^nq x 2^nq
    double ph[4];   // diag: phases (radians) per local index
    uint32_t type;  // original sv_gate_type
    double p[3];
    int mux;        // GK_MUX: index of the multiplexor
};

// Validate and canonicalise; returns SV_OK or SV_EINVAL with *bad = index.
int canonicalise(int n, const sv_gate* g, size_t count, std::vector<CGate>* out, size_t* bad);

// ---------------------------------------------------------------------------
// Plans.  A pass loads every tile of 2^m amplitudes whose index varies only in
// the tile qubits T (sorted, always holding bits 0..L-1 so that each row of
// 2^L amplitudes is contiguous), applies its ops in shared memory and writes
// the tile back: one HBM read and one write of the state per pass.
// ---------------------------------------------------------------------------
// Widest gate-sequence block: its 2^k amplitudes per thread stay in
// registers (64 registers of data at the bound, for both dtypes).  The
// shared-memory pass kernel, which holds more state per thread, takes one
// qubit less and runs wider blocks from their dense matrix.
inline int max_gates_k(int dtype) { return dtype == SV_C64 ? 5 : 4; }
inline int smem_gates_max_k(int dtype) { return dtype == SV_C64 ? 4 : 3; }
// Tile rows: qubits 0..L-1 are always tile qubits, so a tile is made of rows
// of 2^L contiguous amplitudes, 128 bytes (the TMA-fed kernel's tensor-map
// row).  256-byte rows copy faster when the other tile qubits are far apart
// (in-place tile copies at n=30: 0.94 of a plain copy against 0.73), but a
// 60-layer random circuit at n=30 then needed 11% more 13-qubit passes for 9%
// faster passes, and the QFT's passes slowed: 128 bytes it is.
inline int row_bits(int dtype, int pass_kernel) {
    (void)pass_kernel;
    return dtype == SV_C64 ? 4 : 3;
}

struct DiagForm {
    // phase(x) = c + sum_q a[q] x_q + sum_{p<q} b[p*n+q] x_p x_q  (radians)
    double c = 0.0;
    std::vector<double> a, b;
    std::vector<char> support;
    void init(int n) {
        c = 0.0;
        a.assign(n, 0.0);
        b.assign((size_t)n * n, 0.0);
        support.assign(n, 0);
    }
    bool empty() const {
        for (char s : support)
            if (s) return false;
        return c == 0.0;
    }
};

struct HostOp {
    int kind;
    std::vector<int> qubits;  // dense / gates: sorted ascending, block bit i <-> qubits[i]
    std::vector<cd> mat;      // dense: the block's 2^k x 2^k matrix, row-major (gates: formed on demand
                              // from seq, see op_matrix)
    std::vector<CGate> seq;   // gates: the block's gates in order
    std::vector<cd> gdata;    // gates: the records' complex data
    DiagForm diag;            // diag
    std::vector<GateRec> recs;  // gates
    int ngates = 0;           // logical gates folded into the op
    bool tc = false;          // dense: run on the tensor cores (register passes: OP_DENSE_TC for 4-5 qubits)
};

// ---------------------------------------------------------------------------
// Multiplexors (uniformly controlled rotations, the building block of the
// QCrank encoder, App. D.3, and of the Mottonen et al. decompositions the
// paper cites).  A run of gates on one target t whose other qubits are only
// CX controls collapses to: for each value j of the control bits,
//     U_j = X^(popcount(j & flip) ^ flip_c)  R_j
// with R_j = RY(phi[j]) (family Y: RY and X gates) or
// R_j = diag(e^{i phi0[j]}, e^{i phi1[j]}) (family D: RZ, P, Z and X gates).
// The angles are one Walsh-Hadamard transform of the run's angles indexed
// by the CX-parity mask in force at each rotation.
// ---------------------------------------------------------------------------
enum MuxFamily { MUX_Y = 0, MUX_D = 1 };
constexpr int kMuxMaxControls = 16;   // table of 2^16 entries per target at most
constexpr int kMuxMaxTargets = 5;     // targets per multiplexor pass (2^5 amplitudes per thread)
constexpr int kMuxMinGates = 64;      // shorter runs stay in the fused tile passes (mux = 0)

struct Mux {
    int target = -1;
    std::vector<int> controls;  // ascending; bit b of j <-> controls[b]
    int family = MUX_Y;
    uint32_t flip = 0;          // X-parity mask over the j bits at the end of the run
    int flip_c = 0;             // X gates on the target itself, mod 2
    std::vector<double> phi0, phi1;  // Y: phi0 = RY angle; D: the two phases
    int ngates = 0;
    int type_count[14] = {0};
};

// Rewrite g into *rewritten, replacing each qualifying run with one GK_MUX
// gate (placed where the run's last gate was; every gate in between commutes
// with the run).  mode: 0 runs of at least kMuxMinGates gates, 1 runs of at
// least 4 gates, -1 none.  Returns false (and leaves *rewritten alone) when
// no run qualifies.
bool recognise_mux(int n, const std::vector<CGate>& g, std::vector<CGate>* rewritten, std::vector<Mux>* muxes,
                   int mode);

struct HostPass {
    std::vector<int> mux;   // multiplexor pass: indices into Plan::muxes (no tile ops)
    std::vector<int> tile;  // sorted ascending
    int L = 0;              // bits 0..L-1 are in the tile
    std::vector<HostOp> ops;
    int ngates = 0;
    int type_count[14] = {0};  // logical gates of each sv_gate_type in the pass
};

// Plain (unfused) per-gate kernels over the whole state.
enum PlainKind { PK_1Q = 0, PK_CX, PK_SWAP, PK_CPHASE, PK_DIAG1, PK_PHASE1 };

struct PlainOp {
    int kind;
    int q0, q1;
    cd m[4];  // PK_1Q: 2x2; PK_DIAG1: m[0], m[1] = d0, d1; PK_PHASE1/PK_CPHASE: m[0]
};

struct Plan {
    int n = 0;
    int dtype = 0;
    bool plain = false;
    std::vector<HostPass> passes;
    std::vector<PlainOp> plain_ops;
    int64_t gates = 0;
    int tensor = -1;  // 0: dense blocks of k >= kMinTcK go to the tensor cores
    bool no_register_passes = false;
    bool use_tma = false;  // register passes move tiles with TMA tensor copies
    int jit = 0;           // PlanOptions::jit
    std::vector<Mux> muxes;
};

// Default of the tensor-core choice (sv_options.tensor = 0): 1 = 4- and
// 5-qubit blocks go to the tensor cores where their estimated cost is below
// the gate sequence's, 0 = CUDA cores only.  CUDA cores: with warp-local
// remaps and direct tile copies the CUDA-core passes ran a 30-qubit random
// U3+CX circuit 4% faster than the estimate's tensor-core mix (the cost-model
// planner still weighs both).
constexpr int kTcAutoDefault = 0;

struct PlanOptions {
    int k_max = 5;
    int tile_m = 13;
    int planner = SV_PLAN_GREEDY;
    int tensor = -1;  // 0: tensor cores for c64 blocks of k >= 3; -1: CUDA cores only
    int pass_kernel = 0;  // 1: shared-memory pass kernel only; 2: register passes fed by TMA
    int relabel = 0;      // SWAP gates relabel qubits
    double drop_phase_below = 0.0;  // approximation: smaller P/RZ/CP angles are dropped
    int mux = 0;          // multiplexor recognition: 0 long runs, 1 any run of 4+ gates, -1 off
    int jit = 0;          // run-time compiled register passes: 0 on repeat, 1 always, -1 never
    int tc_auto = 0;      // tensor-core dense blocks where their estimated cost is below the gate sequence's
};
// The approximation for negligible rotations: the gates kept.
void drop_small_phases(std::vector<CGate>* g, double eps);

PlanOptions resolve_options(int n, int dtype, const sv_options* opt);
// GK_MUX gates index muxes (may be null when there are none); the plan keeps
// a copy of the multiplexors its passes use.
void plan_greedy(int n, int dtype, const std::vector<CGate>& gates, const PlanOptions& po, Plan* out,
                 const std::vector<Mux>* muxes = nullptr);
void plan_plain(int n, int dtype, const std::vector<CGate>& gates, Plan* out);
// One greedy pass from the front of `remaining` (see plan_greedy); the gates
// it leaves for later in *deferred_out.  form_matrices = false keeps dense
// blocks as their gate list (HostOp::seq) until form_dense_matrices.
void greedy_pass(int n, int dtype, const std::vector<CGate>& gates, const std::vector<Mux>& muxes,
                 const PlanOptions& po, const std::vector<int>& remaining, HostPass* pass_out,
                 std::vector<int>* deferred_out, bool form_matrices);
void form_dense_matrices(HostPass* hp);
// The cost model's own plan (SV_PLAN_MLP): passes chosen one at a time by
// predicted time (see sv_costplan.cpp).  False without a model.
bool plan_learned(int n, int dtype, const std::vector<CGate>& gates, const std::vector<Mux>* muxes,
                  const PlanOptions& base, Plan* out, double* predicted_ms);
void plan_summary(const Plan& p, sv_plan_info* info);

// Cost-model features of one pass (fixed length kFeatures): qubit count,
// dtype, tile width, dense blocks per width, diagonal runs, logical gates per
// type (the paper's one-hot gate-type encoding, App. D.1 Eq. "onehot",
// summed over the pass), arithmetic and byte volume, and a bias input.
constexpr int kFeatures = 32;
std::vector<float> pass_features(int n, int dtype, const HostPass& p, bool tensor_cores, bool register_pass);
// Whether the register-resident kernel can take the pass (the serialiser's
// structural conditions; a region too large to stage is checked there).
bool register_pass_eligible(const Plan& p, const HostPass& hp);

// Options for an apply under SV_PLAN_MLP; ev0/ev1 receive events to record
// around the passes when the judge times this call (else nullptr).
// *learned (may stay null): the model's per-pass plan to run instead of
// plan_greedy with the returned options.
PlanOptions mlp_plan_options(sv_state* h, const sv_gate* g, size_t count, const std::vector<CGate>& cg,
                             const std::vector<Mux>* muxes, const PlanOptions& base, uint64_t salt, cudaEvent_t* ev0,
                             cudaEvent_t* ev1, std::shared_ptr<const Plan>* learned);

// Multiplexor pass (PassDev::rmode == kRmodeMux): the region is MuxDev
// followed by one angle table per target: 2^nc entries of the state's real
// type (float for complex64, double for complex128), phi for family Y and
// (phi0, phi1) pairs for family D, at byte offset tab_off[k] from the region.
constexpr int kRmodeMux = 3;
struct MuxDev {
    int K;                          // targets
    int nc;                         // control bits
    int nruns;                      // runs of consecutive control qubits
    int pad0;
    int t[kMuxMaxTargets];          // target qubits, ascending
    int family[kMuxMaxTargets];
    int flip_c[kMuxMaxTargets];
    uint32_t flip[kMuxMaxTargets];
    int tab_off[kMuxMaxTargets];
    int rs[kMuxMaxControls];        // run r: j bits [ro, ro + rw) = index bits [rs, rs + rw)
    int rw[kMuxMaxControls];
    int ro[kMuxMaxControls];
    int pad1[3];
};
static_assert(sizeof(MuxDev) % 16 == 0, "tables after MuxDev stay 16-byte aligned");

__host__ __device__ inline size_t diag_doubles(int m, int no) { return (size_t)DiagLayout(m, no).total; }

struct PlanBlob {
    std::vector<unsigned char> bytes;
    size_t pass_off = 0, tc_off = 0;
    int npasses = 0;
    int max_region = 0;  // largest pass region (bytes)
};

void serialise_plan(const Plan& p, PlanBlob* blob);
// Region of a multiplexor pass (MuxDev and its tables); sets P->rmode.
void mux_region(const Plan& p, const HostPass& hp, PassDev* P, std::vector<unsigned char>* out);
// Several plans (same dtype) in one blob, passes in order.
void serialise_plans(const std::vector<const Plan*>& plans, PlanBlob* blob);

// ---------------------------------------------------------------------------
// Handle.
// ---------------------------------------------------------------------------
struct Scratch {
    void* ptr = nullptr;
    size_t cap = 0;
};
struct PlanCache;

}  // namespace sv

struct sv_state {
    int n;
    int dtype;
    void* amps;
    bool owned;
    cudaStream_t stream;
    bool bad;
    sv::Scratch plan_dev;    // device plan blob
    sv::Scratch red;         // reduction scratch (block sums, CDF, partials)
    sv::Scratch out_dev;     // device staging for host outputs
    sv::Scratch host_pin;    // pinned staging for plan uploads
    sv::Scratch err;         // device error word of bounded waits (int)
    cudaEvent_t upload_ev;   // recorded after the last plan upload from host_pin
    bool upload_pending;
    // recorder: CUDA events around each pass of applies made with record=1
    std::vector<cudaEvent_t> ev_pool;
    int ev_used;             // events in use (pairs: begin, end)
    std::vector<std::vector<float>> rec_feat;  // per recorded pass features
    int perm[64];            // logical qubit -> physical bit of the stored amplitudes
    bool permuted;           // perm is not the identity
    sv::Scratch perm_tmp;    // device scratch of the permuted read-outs
    sv::Scratch aux;         // device scratch of the QCrank read-out (shots, counters, pixels)
    sv::Scratch lcdf;        // device scratch of the logical-order block CDF of a relabelled state
    long long pending_basis; // >= 0: sv_init_basis(x) not written yet (the next apply's first pass or any other
                             // use of the state writes it)
    sv::PlanCache* plans;    // recent plans of this handle (sv_apply_circuit)
    sv_options last_opts;    // options of the last planned apply
};

namespace sv {

// Logical -> physical qubit map handed to the read-out kernels by value.
struct QubitMap {
    int n;
    int phys[40];
};
void reset_perm(sv_state* h);
QubitMap qubit_map(const sv_state* h);

// Error handling (thread-local message).
int set_error(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
void count_launch(uint64_t k = 1);
// SM count of the current device (cached per device ordinal).
int device_sms();

// Write a deferred sv_init_basis to the state (no-op when none is pending).
int flush_init(sv_state* h);
void used_fields(const sv_gate* gates, size_t count, std::vector<sv_gate>* out);
uint64_t plan_key(const sv_state* h, const std::vector<sv_gate>& recs, const sv_options* opt);
bool same_records(const std::vector<sv_gate>& a, const std::vector<sv_gate>& b);

// The body of sv_apply_circuit after validation: plan and launch on h's stream.
// cache_key != 0: keep the plan under that key (see PlanCache).
// recs: the used fields of the records (see used_fields), kept with a cached plan.
int apply_canonical(sv_state* h, const sv_gate* gates, size_t count, const std::vector<CGate>& cg,
                    const sv_options* opt, uint64_t cache_key = 0, const std::vector<sv_gate>* recs = nullptr);

// Recent plans of a handle: the same gate records, options and qubit map
// give the same plan, so a repeated apply skips validation, planning and
// serialisation (and the compiled-kernel lookup reuses its sources).
struct CachedPlan {
    Plan plan;
    PlanBlob blob;
    int perm_after[64];
    bool permuted_after;
    sv_options last_opts;
    uint64_t stamp;
    std::vector<std::string> jit_srcs;  // compiled-kernel sources of its passes (filled on first launch)
    std::vector<sv_gate> recs;          // the used fields of the circuit's gate records (compared on a hit)
};
struct PlanCache {
    std::vector<std::pair<uint64_t, CachedPlan>> entries;  // small: linear search, least recently used evicted
    uint64_t clock = 0;
};
constexpr int kPlanCacheEntries = 8;

// Upload a serialised plan through h's pinned staging and launch its passes
// on h's stream (rec: events around each pass; judge0/1: around all of them).
int launch_plan(sv_state* h, const Plan& plan, const PlanBlob& blob, bool rec, cudaEvent_t judge0,
                cudaEvent_t judge1, std::vector<std::string>* jit_srcs = nullptr);

int ensure_scratch(Scratch* s, size_t bytes, cudaStream_t st);
int ensure_pinned(Scratch* s, size_t bytes);

// Kernel launchers (sv_kernels.cu).  All return cudaError_t of the launch.
cudaError_t launch_init_basis(sv_state* h, uint64_t x);
cudaError_t launch_plain_op(sv_state* h, const PlainOp& op);
cudaError_t launch_pass(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass,
                        const HostPass& hp);
cudaError_t launch_mux(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass);
PassLayout rpass_layout(int dtype, const PassDev& P, bool single = false);  // single: one tile buffer
// CTAs of `threads` threads an SM holds by registers (regs per thread),
// shared memory (smem bytes per CTA, static + dynamic) and TMEM columns (128
// per 128 threads, for passes with tensor-core blocks).
int resident_ctas(int threads, int regs, int smem);
int num_sms_pub();
// Run-time compiled register passes (sv_jit.cpp).  jit_prepare: per pass of
// the blob, the compiled kernel ready for it (else nullptr); policy 1
// compiles missing ones now, 0 once a structure is seen a second time on a
// state of 22 or more qubits (compiles finish inside the call), -1 never.
// jit_launch: run the pass on it (*used = false: the caller runs the
// interpreting kernel).
// basis >= 0: *fill0 = a kernel for pass 0 that builds its tiles from |basis>
// instead of reading them (nullptr when not ready).
// srcs (optional): the pass sources of this blob, written on first use and
// reused after (a cached plan keeps them).
void jit_prepare(sv_state* h, const PlanBlob& blob, int policy, long long basis, std::vector<void*>* fns,
                 void** fill0, std::vector<std::string>* srcs = nullptr);
cudaError_t jit_launch(sv_state* h, void* entry, const void* blob_dev, const PlanBlob& blob, int pass, bool* used);
void jit_count_fill();
// One persistent launch for circuits of at most mmax qubits (single-tile
// plans, one pass each, in blob order); outputs per circuit c at
// samples + c*shots and expz + c*nmax (either may be NULL).
cudaError_t launch_batch_small(int dtype, const void* blob_dev, const PlanBlob& blob, int C, int mmax,
                               uint64_t shots, uint64_t seed, const int* gidx, uint64_t* samples, double* expz,
                               int nmax, int* counter, cudaStream_t st);
size_t batch_small_smem_bytes(int dtype, int mmax);

// Persistent executor of a wave of circuits (sv_batch_run): one launch runs
// every pass of every circuit of the wave.  Items are (circuit, pass, range)
// in pass-level order; an item may start once `need` items of its circuit
// have finished (its earlier passes).  kind 0: register tile pass over tiles
// [lo, hi) (all tile passes of a wave have the same tile width, 2^(m - RB) =
// 256 threads); kind 1: multiplexor pass over columns [lo, hi).
struct WaveItem {
    int circ;
    int pass;
    int need;
    int kind;
    uint64_t lo, hi;
};
// States of the wave's circuits at base + offs[c] (amplitudes), n qubits
// nq[c]; counters: head (1 int, zero) and done (one int per circuit, zero);
// err set to 2 when a wait gives up after `limit` polls (every CTA then
// stops taking items).  Launch on st; the caller captures it in a graph.
cudaError_t launch_wave(int dtype, void* base, const uint64_t* offs, const int* nq, const void* blob_dev,
                        const PlanBlob& blob, const WaveItem* items, int nitems, int* head, int* done, int* err,
                        unsigned limit, cudaStream_t st);
// Dynamic shared memory of the wave kernel for a blob's register passes.
PassLayout wave_layout(int dtype, const PlanBlob& blob);
// Amplitude 0 of every circuit of a wave set to 1 (the buffer zeroed first).
cudaError_t launch_wave_init(int dtype, void* base, const uint64_t* offs, int C, cudaStream_t st);
// A wave's plans and item list (host).  Returns false when some pass cannot
// run in the wave kernel (a pass not register-resident with 2^(m - RB) = 256
// threads, nor a multiplexor pass).
struct WaveHost {
    PlanBlob blob;
    std::vector<WaveItem> items;
    std::vector<uint64_t> offs;  // amplitudes, per circuit
    std::vector<int> nq;
    uint64_t amps = 0;           // total
};
// blobs (optional): the plans' serialised blobs, merged instead of
// serialising the plans again (the batch frees a plan's multiplexor tables
// once its blob holds them).
bool build_wave(int dtype, const std::vector<const Plan*>& plans, WaveHost* w,
                const std::vector<const PlanBlob*>* blobs = nullptr);
// Host objects of enqueued waves (pinned staging, graphs, the capture stream),
// released once the caller's stream has been synchronised.
struct WaveKeep {
    std::vector<void*> pinned;
    std::vector<cudaGraphExec_t> execs;
    std::vector<cudaGraph_t> graphs;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    void release();
};
// Enqueue a built wave on st (one captured graph; nothing waits on the host).
// The states land in *dev_base (allocated on st, Σ 2^n amplitudes; the caller
// frees it, stream-ordered).  A wait that gives up after `limit` polls sets
// *dev_err = 2 (device memory, zeroed by the caller); every CTA of every later
// wave then stops at once.
int enqueue_wave(int dtype, const WaveHost& w, cudaStream_t st, unsigned limit, int* dev_err, WaveKeep* keep,
                 void** dev_base);

// Read-out (sv_measure.cu).  Device outputs; scratch comes from h->red.
int measure_block_sums(sv_state* h, double** block_sums, int* blog, int64_t* nblocks, int blog_cap = 10);
cudaError_t launch_probs(sv_state* h, double* dev_out);
// Amplitudes of logical indices x0 .. x0+cnt-1 into dev_out (the handle's dtype).
cudaError_t launch_gather_logical(sv_state* h, uint64_t x0, uint64_t cnt, void* dev_out);
int measure_norm(sv_state* h, double* host_out);
int measure_expect_z(sv_state* h, double* dev_out);
// Shots and <Z_i> from one pass over the state (either output may be NULL).
int measure_readout(sv_state* h, uint64_t shots, uint64_t seed, uint64_t* dev_samples, double* dev_expz);

// QCrank read-out (sv_qcrank.cu): counts[2^a], ones[2^a * d] and pixels
// [2^a * d] from shots, all device memory, enqueued on st.
cudaError_t launch_qcrank_decode(const uint64_t* samples, uint64_t shots, int a, int d, uint64_t* counts,
                                 uint64_t* ones, double* pixels, cudaStream_t st);
int measure_sample(sv_state* h, uint64_t shots, uint64_t seed, const double* dev_u, uint64_t* dev_out);

}  // namespace sv
