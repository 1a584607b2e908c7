// Internal declarations shared by the libsv translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "sv.h"

namespace sv {

using cd = std::complex<double>;

constexpr int kMaxQubitsC64 = 34;
constexpr int kMaxQubitsC128 = 33;
constexpr int kQcrankMaxAddr = 26;  // address qubits of the QCrank read-out
constexpr int kMaxK = 5;         // widest fused dense block
constexpr int kMaxTileM = 14;    // qubits per shared-memory tile
constexpr int kPassThreads = 256;

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
enum OpKind { OP_DENSE = 0, OP_DIAG = 1, OP_GATES = 2, OP_REMAP = 3 };

// Register-resident passes: each thread holds 2^kRegBits amplitudes of the
// tile in registers; the other m - kRegBits tile bits index the thread.
__host__ __device__ inline int reg_bits(int dtype) { return dtype == SV_C64 ? 5 : 4; }
constexpr int kRegDenseMaxK = 3;  // dense blocks in registers (wider ones run as gate sequences)
constexpr int kStageCap = 48 * 1024;  // bytes of a pass region staged in shared memory

// Gate-sequence block records (positions are block-local bits, data offsets
// index the op's own complex values).
enum GateRecKind { GR_U = 0, GR_UR = 1, GR_DT = 2, GR_CX = 3, GR_SWAP = 4, GR_H = 5, GR_HD = 6 };
// GR_HD (register passes only): GR_H on position a followed by the phase table
// at off with entry mask b (one dispatch for the pair).
// GR_H (register passes only): the Hadamard without its 1/sqrt(2), a + b and
// a - b; the pass multiplies its amplitudes by the product of the dropped
// factors once, when it writes them back (PassDev::scale).
struct GateRec {
    int kind, a, b, off;
};
constexpr int kMaxGateRecs = 64;     // records per gate-sequence op
constexpr int kMaxGateData = 768;    // complex values per gate-sequence op
// Widest gate-sequence block: its 2^k amplitudes per thread stay in
// registers (64 registers of data at the bound, for both dtypes).  The
// shared-memory pass kernel, which holds more state per thread, takes one
// qubit less and runs wider blocks from their dense matrix.
inline int max_gates_k(int dtype) { return dtype == SV_C64 ? 5 : 4; }
inline int smem_gates_max_k(int dtype) { return dtype == SV_C64 ? 4 : 3; }

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
    std::vector<cd> mat;      // dense and gates: the block's 2^k x 2^k matrix, row-major
    std::vector<cd> gdata;    // gates: the records' complex data
    DiagForm diag;            // diag
    std::vector<GateRec> recs;  // gates
    int ngates = 0;           // logical gates folded into the op
};

// ---------------------------------------------------------------------------
// Multiplexors (uniformly controlled rotations, the building block of the
// QCrank encoder, Sec. 2.3, and of the Mottonen et al. decompositions the
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
    std::vector<Mux> muxes;
};

struct PlanOptions {
    int k_max = 5;
    int tile_m = 13;
    int planner = SV_PLAN_GREEDY;
    int tensor = -1;  // 0: tensor cores for c64 blocks of k >= 3; -1: CUDA cores only
    int pass_kernel = 0;  // 1: shared-memory pass kernel only; 2: register passes fed by TMA
    int relabel = 0;      // SWAP gates relabel qubits
    double drop_phase_below = 0.0;  // approximation: smaller P/RZ/CP angles are dropped
    int mux = 0;          // multiplexor recognition: 0 long runs, 1 any run of 4+ gates, -1 off
};
// The approximation for negligible rotations: the gates kept.
void drop_small_phases(std::vector<CGate>* g, double eps);

PlanOptions resolve_options(int n, int dtype, const sv_options* opt);
// GK_MUX gates index muxes (may be null when there are none); the plan keeps
// a copy of the multiplexors its passes use.
void plan_greedy(int n, int dtype, const std::vector<CGate>& gates, const PlanOptions& po, Plan* out,
                 const std::vector<Mux>* muxes = nullptr);
void plan_plain(int n, int dtype, const std::vector<CGate>& gates, Plan* out);
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
PlanOptions mlp_plan_options(sv_state* h, const sv_gate* g, size_t count, const std::vector<CGate>& cg,
                             const std::vector<Mux>* muxes, const PlanOptions& base, uint64_t salt, cudaEvent_t* ev0,
                             cudaEvent_t* ev1);

// ---------------------------------------------------------------------------
// Device-side plan blob: [PassDev x P][tensor-core B operands][pass regions].
// Each pass owns one contiguous region [OpDev x nops | payloads], every piece
// 16-byte aligned, so a CTA can copy the whole region into shared memory once
// and run all its tiles from there.  Payload offsets are bytes from the start
// of the region.
// ---------------------------------------------------------------------------
struct OpDev {
    int kind;
    int k;
    int mat_off;   // dense / gates: byte offset of the matrix / the records' complex data
    int diag_off;  // diag: byte offset of the run's words (DiagLayout)
    int lq[kMaxK]; // dense / gates: local tile positions, ascending
    int ngates;
    int tc;        // dense on the tensor cores (c64, k >= 3)
    int tc_off;    // float offset of its B operands [hi | lo] in the tc section
    int nrec;      // gates: number of records
    int rec_off;   // gates: byte offset of the records
    int ndata;     // gates: complex values at mat_off
    int ord;       // register passes, diag: ordinal of the run within the pass
};
static_assert(sizeof(OpDev) % 16 == 0, "OpDev array must keep 16-byte alignment");

// Tensor-core dense block of k qubits (D = 2^k): B operand = [Ur; Ui], N = 2D
// rows x K = D columns, FP32 values laid out as the tcgen05 no-swizzle
// K-major canonical layout (8-row x 4-element core matrices of 128 bytes;
// 128 bytes between K-adjacent core matrices, (K/4)*128 between 8-row
// groups), stored twice: hi = value with the low 13 mantissa bits cleared
// (what the tensor core reads from an FP32 input) and lo = value - hi.
constexpr int kMinTcK = 3;
constexpr int kTcResidentFloats = 8192;  // 32 KiB of B operands kept per CTA
__host__ __device__ inline int tc_floats(int k) { return 2 * (2 << k) * (1 << k); }  // hi + lo
__host__ __device__ inline int tc_kmajor_index(int n, int kk, int K) {
    return ((n >> 3) * (K >> 2) + (kk >> 2)) * 32 + (n & 7) * 4 + (kk & 3);
}

struct PassDev {
    double scale;        // register passes: factor applied at write-back (1 unless GR_H records)
    int n;               // qubits of the state the pass runs on
    int m;
    int L;
    int rmode;           // register-resident pass (region in the register format): 1 fed by
                         // cp.async copies, 2 by TMA tensor copies; 0: shared-memory kernel;
                         // kRmodeMux: multiplexor pass
    int ndiag;           // register passes: diagonal runs (each folded once per tile)
    int nops;            // ops in the pass's region
    int region_off;      // byte offset of the region in the blob
    int region_bytes;    // its size (multiple of 16)
    int ops_bytes;       // size of its OpDev array (multiple of 16)
    int tc_k;            // widest tensor-core block in the pass (0: none)
    int tc_base;         // float offset of the pass's first tensor-core B operands
    int tc_res;          // floats of B operands kept resident in shared memory (0: loaded per op)
    int tq[kMaxTileM];   // tile qubits ascending
    int nother;
    int oq[40];          // non-tile qubits ascending
};

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

// Layout (in 8-byte words of fixed-point turns, 2^-64 turn units) of one
// diagonal run inside a pass
// with m tile qubits and no = n - m other qubits:
//   c | a_t[m] | a_o[no] | Bo[m][no] | Boo[no][no] | Qlo[2^h] | Qhi[2^(m-h)]
//   | Rt[(m-h)][2^h]
// with h = min(m, 7): the tile index splits into lo = bits 0..h-1 and hi.
struct DiagLayout {
    int h, mh, c, at, ao, bo, boo, qlo, qhi, rt, total;
    __host__ __device__ DiagLayout(int m, int no) {
        h = m < 7 ? m : 7;
        mh = m - h;
        c = 0;
        at = 1;
        ao = at + m;
        bo = ao + no;
        boo = bo + m * no;
        qlo = boo + no * no;
        qhi = qlo + (1 << h);
        rt = qhi + (1 << mh);
        total = rt + (mh << h);
    }
};
__host__ __device__ inline size_t diag_doubles(int m, int no) { return (size_t)DiagLayout(m, no).total; }

// Diagonal run of a register pass (8-byte words of fixed-point turns), for
// the register layout in force: rpos[b] = tile position of register bit b,
// tpos[t] = tile position of thread bit t (t < m - r; lo = thread bits 0..3,
// hi = the rest, at most 5):
//   c | a_t[m] | a_o[no] | Bo[m][no] | Boo[no][no]        (per-tile fold)
//   | TQlo[16] | TQhi[32] | TR[5][16]                       (thread-thread couplings)
//   | TAlo[5][16] | TAhi[5][32]                             (register-thread couplings)
//   | beta[5][5]                                            (register-register couplings)
struct RDiagLayout {
    int c, at, ao, bo, boo, tqlo, tqhi, tr, talo, tahi, beta, total;
    __host__ __device__ RDiagLayout(int m, int no) {
        c = 0;
        at = 1;
        ao = at + m;
        bo = ao + no;
        boo = bo + m * no;
        tqlo = boo + no * no;
        tqhi = tqlo + 16;
        tr = tqhi + 32;
        talo = tr + 5 * 16;
        tahi = talo + 5 * 16;
        beta = tahi + 5 * 32;
        total = beta + 25;
    }
};

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

// The body of sv_apply_circuit after validation: plan and launch on h's stream.
int apply_canonical(sv_state* h, const sv_gate* gates, size_t count, const std::vector<CGate>& cg,
                    const sv_options* opt);

// Upload a serialised plan through h's pinned staging and launch its passes
// on h's stream (rec: events around each pass; judge0/1: around all of them).
int launch_plan(sv_state* h, const Plan& plan, const PlanBlob& blob, bool rec, cudaEvent_t judge0,
                cudaEvent_t judge1);

int ensure_scratch(Scratch* s, size_t bytes, cudaStream_t st);
int ensure_pinned(Scratch* s, size_t bytes);

// Kernel launchers (sv_kernels.cu).  All return cudaError_t of the launch.
cudaError_t launch_init_basis(sv_state* h, uint64_t x);
cudaError_t launch_plain_op(sv_state* h, const PlainOp& op);
cudaError_t launch_pass(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass,
                        const HostPass& hp);
cudaError_t launch_mux(sv_state* h, const void* blob_dev, const PlanBlob& blob, int pass);
// One persistent launch for circuits of at most mmax qubits (single-tile
// plans, one pass each, in blob order); outputs per circuit c at
// samples + c*shots and expz + c*nmax (either may be NULL).
cudaError_t launch_batch_small(int dtype, const void* blob_dev, const PlanBlob& blob, int C, int mmax,
                               uint64_t shots, uint64_t seed, const int* gidx, uint64_t* samples, double* expz,
                               int nmax, int* counter, cudaStream_t st);
size_t batch_small_smem_bytes(int dtype, int mmax);

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
