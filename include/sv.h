/*
 * libsv: GB300-native (sm_103a) state-vector simulator, C ABI.
 *
 * The computation is the one the paper (Q-GEAR, arXiv 2504.03967) accelerates
 * by turning a circuit's gate list into GPU kernels: apply a gate list to a
 * 2^n-amplitude complex state (App. A, Eq. "hilbert": |psi> = sum_i a_i |i>,
 * sum |a_i|^2 = 1) and then read probabilities, <Z_i> or measurement shots
 * (Sec. 3, shots per circuit).  One process drives one GPU; every call is
 * asynchronous on the handle's CUDA stream unless it writes host memory, in
 * which case it returns after the result has been copied.
 *
 * Conventions
 *   - Qubit q is bit q of the amplitude index (LSB = qubit 0).  An outcome x
 *     returned by the samplers is that index, so bit q of x is qubit q.
 *   - Amplitudes are interleaved (re, im): SV_C64 = 2 x float (8 bytes),
 *     SV_C128 = 2 x double (16 bytes), 2^n of them, index order.
 *   - Every call returns SV_OK (0) or a negative sv_status.  sv_last_error()
 *     gives a message for the calling thread's last failure.  Validation
 *     failures (SV_EINVAL, SV_EUNSUPPORTED, SV_ENOMEM before any launch) leave
 *     the state unchanged.  After SV_ECUDA or SV_ETIMEOUT the state content is
 *     undefined and the handle is flagged: later calls other than sv_free and
 *     sv_init_* return SV_ESTATE until the state is re-initialised.
 *   - Pointers named dev_* are device pointers, host_* are host pointers.
 *     Nothing returned is owned by the caller unless stated; the caller owns
 *     every buffer it passes in and must keep it alive for the call.
 */
#ifndef SV_H_
#define SV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sv_state *sv_handle;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

typedef enum {
    SV_OK = 0,
    SV_EINVAL = -1,       /* bad argument: n out of range, qubit >= n,
                             duplicate qubits, unknown gate type, wrong arity,
                             NULL pointer */
    SV_ENOMEM = -2,       /* device or pinned allocation failed */
    SV_EUNSUPPORTED = -3, /* valid request this build does not provide */
    SV_ECUDA = -4,        /* a CUDA runtime call or kernel launch failed */
    SV_ETIMEOUT = -5,     /* a bounded device-side wait gave up */
    SV_ESTATE = -6        /* handle flagged by an earlier SV_ECUDA/SV_ETIMEOUT */
} sv_status;

/* Gate alphabet.  The paper's one-hot gate set h, ry, rz, cx, measure
 * (App. D.1, Eq. "onehot"), cr1 = SV_CP (App. D.2, Eq. "cr1"), and the
 * single-qubit rotations Rx (App. A) and U3 used by the random circuits.
 * Matrices (c = cos(t/2), s = sin(t/2)):
 *   H = [[1,1],[1,-1]]/sqrt2, X, Y = [[0,-i],[i,0]], Z = diag(1,-1),
 *   RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]],
 *   RZ(f) = diag(e^{-if/2}, e^{if/2}), P(l) = diag(1, e^{il}),
 *   U3(t,f,l) = [[c, -e^{il}s], [e^{if}s, e^{i(f+l)}c]],
 *   CX(control q[0], target q[1]) flips the target where the control is 1
 *   (App. A, Eq. "cx" and its 3-qubit example), CZ = diag(1,1,1,-1),
 *   CP(l) = CR1(l) = diag(1,1,1,e^{il}), SWAP exchanges the two qubits.
 * SV_MEASURE is terminal: accepted, validated and ignored by the apply calls
 * (sampling always measures every qubit). */
typedef enum {
    SV_H = 0, SV_X = 1, SV_Y = 2, SV_Z = 3, SV_RX = 4, SV_RY = 5, SV_RZ = 6,
    SV_P = 7, SV_U3 = 8, SV_CX = 9, SV_CZ = 10, SV_CP = 11, SV_SWAP = 12,
    SV_MEASURE = 13
} sv_gate_type;

/* One gate: the (type, control, target, params) record of the paper's circuit
 * tensor (Sec. 2.1 "Circuit encoding"; App. D.1 gate_type / gate_param).
 * nq must equal the type's arity (1 or 2); q[0] is the control of CX/CP.
 * Unused q[] and p[] entries are ignored.  48 bytes. */
typedef struct {
    uint32_t type;
    uint32_t nq;
    uint32_t q[3];
    double p[3];
} sv_gate;

/* Planner choice for sv_apply_circuit. */
typedef enum {
    SV_PLAN_GREEDY = 0, /* greedy tile passes with fixed fusion width k_max */
    SV_PLAN_MLP = 1,    /* cost-model-guided plan; greedy when no model */
    SV_PLAN_PLAIN = 2   /* one kernel per gate over the whole state */
} sv_planner;

/* Options for sv_apply_circuit; pass NULL for defaults.  A zero field means
 * "default".  k_max: widest fused dense block, 1..5 (App. D.2: gate fusion =
 * 5); tile_m: qubits per shared-memory tile pass (c64 9..14, c128 9..13);
 * planner: sv_planner; record: store per-pass CUDA-event times for the cost
 * model (sv_pass_times); tensor: 1 = complex64 dense blocks run on the
 * tensor cores (register passes: 4..5 qubits, FP16 hi/lo splits, three
 * products; shared-memory passes: 3..5 qubits, 3xTF32; FP32 accumulation),
 * -1 = CUDA cores only, 0 = the library's default (CUDA cores; the
 * cost-model planner may choose either).
 * pass_kernel: 0 = default (passes run register-resident where they can:
 * every thread keeps 2^5 (c64) / 2^4 (c128) amplitudes of the tile in
 * registers; tiles move by 16-byte cp.async copies, or, in compiled passes
 * whose first / last register layout has coalesced warp accesses, straight
 * between the state and registers), 1 = always the
 * shared-memory pass kernel, 2 = register-resident passes whose tiles move by
 * TMA tensor copies through a ring of tile slots (one CTA per SM).  Results
 * agree within rounding whichever kernel runs.  relabel: 1 = SWAP gates
 * become a relabelling of the state's qubits instead of data movement (see
 * sv_qubit_map); 0 = SWAPs move amplitudes.  drop_phase_below: the
 * approximation for negligible rotations (App. D.2): P, RZ and CP gates whose
 * angle, reduced modulo the gate's period (2 pi; 4 pi for RZ, as RZ(2 pi) =
 * -I), is smaller in magnitude than this many radians are left out; the result then differs from the exact circuit by at most
 * the sum of the dropped angles over 2 in norm (0, a negative value or NaN =
 * exact).  mux: multiplexor recognition (QCrank's uniformly
 * controlled rotations, App. D.3): a run of RY (or RZ / P / Z) and X gates on one
 * target interleaved with CX gates into it, whose controls nothing else
 * changes meanwhile, becomes one block-diagonal operator with per-control-value
 * angles from a Walsh-Hadamard transform, and up to five such targets share
 * one pass over the state; exact up to rounding.  0 = runs of at least 64
 * gates, 1 = runs of at least 4 gates, -1 = off.  At most 16 controls.
 * jit: register-resident passes as kernels compiled at run time (NVRTC) for
 * their structure -- op sequence, gate positions, table masks and register
 * layouts fixed in the code, the data still read from the plan -- and cached
 * for the process: 0 = compile a structure the second time it runs on a
 * state of 22 or more qubits (the first run, one-off circuits and small
 * states stay on the library's interpreting kernel), 1 = compile on first
 * use, -1 = never.  A compile (about a second, the passes of one plan in
 * parallel) happens inside the apply that needs it.  Results agree with the interpreting
 * kernel to rounding; where NVRTC is missing the interpreting kernel runs. */
typedef struct {
    int k_max;
    int tile_m;
    int planner;
    int record;
    int tensor;
    int pass_kernel;
    int relabel;
    int mux;
    double drop_phase_below;
    int jit;
} sv_options;

/* Plan summary returned by sv_plan_circuit (host only, no device work). */
typedef struct {
    int64_t gates;        /* gate records given (MEASURE included), less those drop_phase_below removes */
    int64_t passes;       /* HBM passes the plan makes over the state */
    int64_t dense_ops;    /* fused dense blocks over all passes */
    int64_t diag_ops;     /* diagonal-phase runs over all passes */
    int64_t max_k;        /* widest dense block */
    int64_t bytes_moved;  /* algorithmic HBM bytes: sum over passes of the
                             amplitudes each pass reads and writes */
    int64_t gate_ops;     /* of dense_ops, the blocks applied as their gate
                             sequence in registers instead of a 2^k matrix */
    int64_t reg_passes;   /* passes run by the register-resident kernel */
    int64_t remaps;       /* register-layout exchanges over all such passes
                             (per tile) */
    int64_t mux_ops;      /* recognised multiplexors (each one target) */
    int64_t mux_passes;   /* passes that apply multiplexors */
    int64_t tc_ops;       /* of dense_ops, the blocks applied on the tensor cores */
    int64_t warp_remaps;  /* of remaps, those that keep every warp's amplitudes
                             within the warp (ordered by a warp barrier) */
} sv_plan_info;

/* ---- state lifetime (App. A, Eq. "hilbert") ---------------------------- */

/* Allocate a library-owned 2^n state of dtype dt on the current device.
 * n: 1..34 (c64) or 1..33 (c128).  cuda_stream: a cudaStream_t to run on
 * (NULL = the legacy default stream).  The state content is undefined until
 * an sv_init_* or sv_load_state call.  SV_ENOMEM if the device cannot hold
 * it (checked before any allocation touches the device). */
int sv_alloc(int n, sv_dtype dt, void *cuda_stream, sv_handle *out);

/* Wrap caller-owned device memory (e.g. a torch tensor) of 2^n amplitudes of
 * dtype dt, 16-byte aligned.  The library never frees dev_amps; the caller
 * keeps it alive until sv_free. */
int sv_attach(int n, sv_dtype dt, void *dev_amps, void *cuda_stream, sv_handle *out);

/* Release the handle and any memory the library allocated for it. */
int sv_free(sv_handle h);

/* Change the stream later calls on h run on. */
int sv_set_stream(sv_handle h, void *cuda_stream);

/* Number of qubits / dtype / device pointer of the state (for interop). */
int sv_info(sv_handle h, int *n, int *dtype, void **dev_amps);

/* Qubit relabelling.  After an apply with opt->relabel = 1 the amplitude of
 * logical basis state x may sit at a permuted index in device memory: logical
 * qubit q is stored at bit map[q].  Every read-out (probabilities, norm, <Z>,
 * shots, sv_store_state) and every later sv_apply_circuit honours the map, so
 * results are those of the logical circuit; only code that reads the device
 * buffer directly (sv_info, sv_attach memory, sv_sample_uniforms_noalloc)
 * sees the physical order.  sv_init_basis and sv_load_state reset the map to
 * the identity.  Shots under a non-identity map follow the sampling rule
 * over the LOGICAL index, exactly as for the materialised state: the block
 * CDF is formed in logical order from one more read of the state and the
 * chosen block is rescanned in logical order through the map.
 * sv_qubit_map writes map[0..n-1]; sv_materialize moves the amplitudes into
 * logical order (fused SWAP passes) and resets the map. */
int sv_qubit_map(sv_handle h, int *map);
int sv_materialize(sv_handle h);

/* Options the last sv_apply_circuit on h planned with (for SV_PLAN_MLP, the
 * candidate the cost model and its judge picked for that call). */
int sv_last_plan(sv_handle h, sv_options *out);

/* |x>: all amplitudes 0 except a_x = 1.  SV_EINVAL if x >= 2^n.  The write
 * is deferred: the next sv_apply_circuit whose first pass runs on a compiled
 * register kernel (see sv_options.jit) builds that pass's tiles from x
 * instead of reading the state, and every other call that uses the state
 * (read-outs, sv_store_state, other applies, sv_info asking for the device
 * pointer, sv_set_stream) writes |x> first.  Code that reads attached memory
 * directly must therefore take the pointer from sv_info after the init, or
 * call a read-out, before reading it. */
int sv_init_basis(sv_handle h, uint64_t x);

/* Copy 2^n amplitudes (interleaved, the handle's dtype) from host memory to
 * the state / from the state to host memory. */
int sv_load_state(sv_handle h, const void *host_amps);
int sv_store_state(sv_handle h, void *host_amps);

/* ---- gate application (App. A Eqs. "tp", "cx"; App. D.2 Eq. "cr1") ---- */

/* Apply count gate records in list order to the state.  The result equals
 * applying each gate's matrix to every group of amplitudes that differ only
 * in the gate's qubit bits, one gate after the other; the planner may fuse
 * consecutive gates into dense blocks of <= k_max qubits (App. D.2, "gate
 * fusion = 5") and diagonal-phase runs, which is exact up to rounding.  All
 * records are validated before any device work. */
int sv_apply_circuit(sv_handle h, const sv_gate *gates, size_t count, const sv_options *opt);

/* Run-time compiled passes: kernels compiled, compiles that failed, passes
 * launched on them and host milliseconds spent compiling (process totals);
 * sv_jit_fills: passes that built their tiles from a deferred basis state
 * instead of reading the state.  sv_jit_wait returns at once (compiles finish
 * inside the apply that starts them). */
int sv_jit_stats(uint64_t *compiled, uint64_t *failed, uint64_t *launched, double *compile_ms);
int sv_jit_fills(uint64_t *filled);
/* Of the passes launched on compiled kernels (process totals): those whose
 * kernel loads the pass's first register layout straight from the state, and
 * those that store its last layout straight back (no shared-memory copy),
 * which it does when the layout's warp accesses cover runs of 32 bytes or
 * more. */
int sv_jit_direct(uint64_t *loads, uint64_t *stores);
int sv_jit_wait(void);
/* Host-only check of the pass compiler (no GPU needed): plan the circuit,
 * write the run-time kernel source of every register-resident pass (and of
 * pass 0 building its tiles from a basis state) and compile it with NVRTC for
 * sm_<arch>a.  *compiled = kernels compiled; log (cap bytes) receives the
 * compiler's output (with the source when a compile fails).  SV_EUNSUPPORTED
 * without NVRTC.  sv_jit_last_log: the last run-time compile's log. */
int sv_jit_check(int n, sv_dtype dt, const sv_gate *gates, size_t count, const sv_options *opt, int arch,
                 int *compiled, char *log, size_t cap);
int sv_jit_last_log(char *buf, size_t cap);

/* Plan without running: fills *info for a circuit on n qubits of dtype dt.
 * Host only; usable without a GPU. */
int sv_plan_circuit(int n, sv_dtype dt, const sv_gate *gates, size_t count,
                    const sv_options *opt, sv_plan_info *info);

/* One op of a fused plan as the planner built it, in FP64, before the device
 * encoding (register layouts, deferred factors, single precision), so that a
 * plan can be checked against the circuit without a GPU.  The ops of each
 * pass apply in order, passes in order; their product is the circuit's
 * operator (App. D.2 "gate fusion"; Eq. "cr1" for the phase runs).
 *   kind 0, dense block: the 2^k x 2^k matrix on qubits q[0..k-1] (block bit
 *     i <-> q[i]), row-major, 2 * 4^k doubles (re, im) at data_off.
 *   kind 1, phase run: phase(x) = c + sum_q a_q x_q + sum_{p<q} b_pq x_p x_q
 *     radians on every amplitude x; 1 + n + n*n doubles at data_off: c, a[n],
 *     b[n*n] (row p, column q; only p < q is used).  k = 0.
 *   kind 2, gate sequence on the block positions of q[0..k-1]: nrec records
 *     of 4 ints (rkind, a, b, off) from recs[rec_off]; complex values (re, im)
 *     at data + data_off + 2 * off.  rkind 0: 2x2 complex matrix on position
 *     a (4 values, row-major); 1: the same with real entries; 2: a 2^k-entry
 *     diagonal table over the block index (a = mask of the positions it
 *     depends on); 3: CX, control a, target b; 4: SWAP a, b.
 *   kind 3, multiplexor (a uniformly controlled rotation, recognised from a
 *     run of the circuit): q[0] = its target t, k = 1; at data_off: family
 *     (0: RY, 1: diagonal), flip, flip_c, nc, the nc control qubits
 *     (ascending), then phi0[2^nc] and, for the diagonal family, phi1[2^nc].
 *     With j the value of the control bits (bit b <-> control b) it applies
 *     U_j = X^(popcount(j & flip) ^ flip_c) R_j on t, R_j = RY(phi0[j]) or
 *     diag(e^{i phi0[j]}, e^{i phi1[j]}).
 * pass: the pass the op runs in.  Planner SV_PLAN_GREEDY only
 * (SV_EUNSUPPORTED otherwise).  The counts are always written; ops, recs and
 * data are filled where they fit, and SV_EINVAL reports buffers too small
 * (call with zero capacities to size them).  Host only. */
typedef struct {
    int pass;
    int kind;
    int k;
    int q[5];
    int nrec;
    int rec_off;
    int64_t data_off;
} sv_plan_op;

int sv_plan_ops(int n, sv_dtype dt, const sv_gate *gates, size_t count, const sv_options *opt,
                sv_plan_op *ops, size_t ops_cap, size_t *nops, int *recs, size_t recs_cap, size_t *nrecs,
                double *data, size_t data_cap, size_t *ndata);

/* ---- read-out (Sec. 3 shots; App. A Eq. "hilbert") --------------------- */

/* p_x = |a_x|^2 in FP64 for all 2^n x, to host or device memory. */
int sv_probs(sv_handle h, double *host_out);
int sv_probs_device(sv_handle h, double *dev_out);

/* sum_x |a_x|^2 in FP64. */
int sv_norm(sv_handle h, double *host_out);

/* <Z_i> = sum_x p_x (1 - 2 x_i) for i = 0..n-1, FP64, to host or device. */
int sv_expect_z(sv_handle h, double *host_out);
int sv_expect_z_device(sv_handle h, double *dev_out);

/* Draw shots outcomes x with probability p_x / sum p: outcome = min{x :
 * C_x > u * C_{N-1}} with C the inclusive FP64 CDF.  sv_sample draws u from
 * Philox4x64-10 (Salmon et al. SC'11): shot s uses word s mod 4 of block
 * Philox(counter = (s div 4, 0, 0, 0), key = (seed, 0)), u = (w >> 11) 2^-53.
 * sv_sample_uniforms takes the uniforms u[0..shots) from the caller (host).
 * Outcomes are uint64 indices, to host or device memory. */
int sv_sample(sv_handle h, uint64_t shots, uint64_t seed, uint64_t *host_out);
int sv_sample_device(sv_handle h, uint64_t shots, uint64_t seed, uint64_t *dev_out);
int sv_sample_uniforms(sv_handle h, const double *host_u, uint64_t shots, uint64_t *host_out);

/* QCrank read-out (Sec. 3 image encoding, App. D.3, Table 2).  A QCrank state holds a uniform
 * superposition over a address qubits (bits 0..a-1 of an outcome) with data
 * qubit k (bit a+k) rotated by RY(pi * pixel[j][k]), so that
 * P(bit a+k = 1 | address j) = sin^2(pi * pixel[j][k] / 2).  From shots:
 *   counts[j]   = shots whose address bits equal j,
 *   ones[j*d+k] = of those, the shots with bit a+k set,
 *   pixels[j*d+k] = (2/pi) * asin(sqrt(ones[j*d+k] / counts[j])),
 * NaN where counts[j] = 0.  Bits above a+d-1 are ignored.
 * sv_qcrank_decode_device: every pointer is device memory (samples: shots
 * uint64 outcomes; counts: 2^a uint64; ones: 2^a*d uint64; pixels: 2^a*d
 * doubles, row-major [address][data qubit]), owned by the caller; the work
 * is enqueued on `stream` (a cudaStream_t, NULL = legacy default stream)
 * without synchronising and without allocating.
 * sv_qcrank_reconstruct: draws `shots` outcomes of the state as sv_sample
 * does (same seed, same shots), decodes them on the device (the shots never
 * leave it) and copies pixels (2^a*d doubles) and, if host_counts is not
 * NULL, counts (2^a) to the host.  Table 2 uses 3000 * 2^a shots.
 * Errors: SV_EINVAL for NULL buffers, a < 1, d < 1, d > 32, a > 26, a + d > 63
 * (sv_qcrank_reconstruct: a + d > n). */
int sv_qcrank_decode_device(const uint64_t *samples, uint64_t shots, int a, int d, uint64_t *counts,
                            uint64_t *ones, double *pixels, void *stream);
int sv_qcrank_reconstruct(sv_handle h, int a, int d, uint64_t shots, uint64_t seed, double *host_pixels,
                          uint64_t *host_counts);

/* Shots (as sv_sample_device) and <Z_i> (as sv_expect_z_device) from ONE
 * pass over the state: the probability block statistics are computed once
 * and serve both.  Either output may be NULL (shots then ignored). */
int sv_measure_device(sv_handle h, uint64_t shots, uint64_t seed, uint64_t *dev_samples, double *dev_expz);
/* The same with host outputs (shots uint64 values, n doubles); returns when
 * both are in host memory. */
int sv_measure(sv_handle h, uint64_t shots, uint64_t seed, uint64_t *host_samples, double *host_expz);

/* Sampling that allocates nothing.  The paper has no counterpart; this entry
 * point exists for callers of this library that cannot allocate device
 * memory while they run, e.g. a serving process whose device memory is
 * handed out up front by its own allocator (a cudaMalloc here could fail or
 * overrun its budget) or a caller that cannot accept the device-wide
 * synchronisation that cudaFree implies.
 *
 * The same rule as sv_sample_uniforms, outcome = min{x : C_x > u C_{N-1}}
 * over the stored index order, with its own block size (1024 amplitudes),
 * so a draw within rounding of a CDF boundary may differ from that call's.
 * The state (dev_amps: 2^n amplitudes of dtype dt, 16-byte aligned), the
 * uniforms (dev_u: shots doubles in [0,1)) and the outcomes (dev_out: shots
 * uint64) all live in caller-owned device memory, and the call runs
 * asynchronously on cuda_stream (NULL = legacy default stream).  The call
 * reads dev_amps on cuda_stream only: when the state belongs to a handle,
 * order cuda_stream after that handle's stream (or synchronise it) first,
 * including after an sv_info call that wrote a deferred sv_init_basis.
 *
 * Its only scratch (the FP64 block CDF) is a fixed array of 128.5 KiB
 * inside this library, which every GPU that loads the library holds until
 * the process exits; it bounds n to 1..24, and larger n returns SV_EINVAL
 * before any device work.  The first call on a device looks up that array's
 * device address (once per device, with the device current); make that first
 * call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents; every element a call reads it has written
 * first, but calls that overlap on the GPU (e.g. on two streams at once)
 * race on it and must be serialised by the caller. */
int sv_sample_uniforms_noalloc(const void *dev_amps, int n, sv_dtype dt, const double *dev_u,
                               uint64_t shots, uint64_t *dev_out, void *cuda_stream);

/* ---- batches of independent circuits ------------------------------------ */

/* Run C independent circuits of uneven size (the paper's parallel mode of
 * many small circuits, Sec. 2.4), each from |0...0>, and return their shots
 * and <Z_i>.  Circuit c has n_qubits[c] qubits and the gate records
 * gates[gate_offsets[c] .. gate_offsets[c] + gate_counts[c]); the fixed-size
 * circuit tensor of App. B Lemma 2 (C circuits padded to d records) is the
 * case gate_offsets[c] = c * d.  Circuit c draws its shots with seed + c
 * (sv_sample's Philox convention).  host_samples (C x shots uint64, row c =
 * circuit c) and host_expz (C x nmax doubles, row c holds n_qubits[c]
 * values, nmax >= every n_qubits[c]) may each be NULL.
 * Circuits of at most 13 (complex64) / 12 (complex128) qubits run entirely in
 * shared memory inside one persistent kernel launched from a CUDA graph;
 * larger ones run through the fused tile passes.  opt as for
 * sv_apply_circuit (k_max defaults to 3 here).  Synchronous. */
int sv_batch_run(int C, const int *n_qubits, const int64_t *gate_offsets, const int64_t *gate_counts,
                 const sv_gate *gates, sv_dtype dt, uint64_t shots, uint64_t seed, const sv_options *opt,
                 uint64_t *host_samples, double *host_expz, int nmax, void *cuda_stream);

/* ---- recorder (per-pass timings; the cost model's training data) ------- */

/* Timings of the tile passes run by sv_apply_circuit calls made with
 * opt->record = 1 since the last sv_pass_times call on h.  Waits for the
 * stream, then writes min(count, cap) CUDA-event durations in milliseconds
 * (host_ms, may be NULL) and their feature vectors (host_feat, cap x
 * sv_feature_count() floats, may be NULL) in launch order, sets *count to
 * the number recorded and clears the record. */
int sv_pass_times(sv_handle h, double *host_ms, float *host_feat, int cap, int *count);

/* Length of one pass feature vector. */
int sv_feature_count(void);

/* ---- autotuner ---------------------------------------------------------- */

/* Time every candidate plan of this circuit on h's state and return the
 * fastest: fusion width k_max 2..5 (App. D.2's "gate fusion = 5" as the
 * bound) x tile width (11..14 qubits for complex64, 10..13 for complex128,
 * at most n) x, for complex64, tensor cores on or off (blocks of 3..5
 * qubits) x pass kernel (register-resident where it can run, or the
 * shared-memory kernel).  Each candidate runs twice on h's stream and keeps its faster
 * CUDA-event time.  h's amplitudes serve as scratch: their content is
 * undefined afterwards.  cache_path (may be NULL) names a JSON-lines file of
 * earlier results, one object per line {"key", "k_max", "tile_m", "tensor",
 * "pass_kernel", "ms"}; the key holds n, dtype, the gate count, a 64-bit FNV-1a hash of the
 * records and the device name and SM count.  When the file has a line for
 * this key its result is returned without any device work; otherwise the
 * new result is appended (the file is created if missing; a write failure
 * is ignored).  *best receives planner = SV_PLAN_GREEDY and the winning
 * k_max, tile_m, tensor (1 or -1) and pass_kernel, ready for sv_apply_circuit; *best_ms
 * (may be NULL) its time in milliseconds.  Synchronous. */
int sv_autotune(sv_handle h, const sv_gate *gates, size_t count, const char *cache_path, sv_options *best,
                double *best_ms);

/* ---- learned cost model (one per process) -------------------------------
 * A small MLP (32 -> 64 -> 64 -> 1, ReLU) predicts the log time of a tile
 * pass from its feature vector (the recorder's features: qubit count, dtype,
 * tile width, fused blocks per width, diagonal runs, and the paper's one-hot
 * gate-type encoding of App. D.1 Eq. "onehot" summed over the pass's gates).
 * With planner = SV_PLAN_MLP, sv_apply_circuit plans each new circuit with
 * every candidate fusion width k (2..5), tile width m and tensor-core choice,
 * predicts the total time and keeps the fastest; the greedy fixed-width plan
 * is the fallback when no model is loaded and the judge of the prediction:
 * the first 2T calls for a circuit (T trials: the model's per-pass plan and
 * best whole-circuit candidates, and the greedy plan) time every trial twice
 * with CUDA events, rounds interleaved, and later calls use the trial with
 * the fastest time, the greedy plan unless another beats it by more than 1%.
 * Plans are exact either way. */

/* Train on count recorded passes (features count x sv_feature_count()
 * floats, times in ms) on the GPU with the library's own forward, backward and
 * Adam kernels, full batch, for epochs steps of learning rate lr, weights
 * initialised from seed.  The trained model becomes the process's model and
 * is written to weights_path unless it is NULL.  *final_loss (may be NULL)
 * receives the mean squared error on standardised log times. */
int sv_cost_model_train(const float *host_feat, const double *host_ms, int count, int epochs, double lr,
                        uint64_t seed, const char *weights_path, double *final_loss);
int sv_cost_model_save(const char *path);
int sv_cost_model_load(const char *path);
int sv_cost_model_unload(void);
/* 1 if a model is loaded, else 0. */
int sv_cost_model_loaded(void);
/* Predicted times (ms) for count feature rows, computed on the GPU. */
int sv_cost_model_predict(const float *host_feat, int count, double *host_ms);
/* The options SV_PLAN_MLP picks for a circuit and its predicted time, without
 * running it (plans on the host, predicts on the GPU). */
int sv_cost_model_choose(int n, sv_dtype dt, const sv_gate *gates, size_t count, sv_options *chosen,
                         double *predicted_ms);
/* Counters: circuits planned by the model, and judged mispredictions (the
 * judge did not keep the model's first choice). */
int sv_cost_model_stats(int64_t *planned, int64_t *mispredicted);
/* The options the judge settled on for a circuit already applied with
 * SV_PLAN_MLP (the model's first choice until all judged calls are done) and
 * that plan's measured time in ms (-1 if not timed yet). */
int sv_cost_model_judged(int n, sv_dtype dt, const sv_gate *gates, size_t count, sv_options *out,
                         double *measured_ms);

/* The trials the judge timed for the circuit the cost-model planner saw
 * last: trial 0 is the model's own plan (passes chosen one at a time by
 * predicted time) when it found one (*learned = 1), then the model's best
 * whole-circuit option sets, last the greedy plan.  predicted[i] and
 * measured[i] in ms (the faster of its timed calls, -1 where not known) for
 * i < min(cap, *ntrials);
 * *chosen = the trial kept (-1 until every trial was timed). */
int sv_cost_model_last_trials(double *predicted, double *measured, int cap, int *ntrials, int *chosen,
                              int *learned);

/* ---- misc -------------------------------------------------------------- */

/* Message for the calling thread's last failing call ("" if none). */
const char *sv_last_error(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
int sv_version(void);

/* Number of kernel launches this library made on the calling process since
 * load (all handles).  For launch accounting in benchmarks. */
uint64_t sv_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SV_H_ */
