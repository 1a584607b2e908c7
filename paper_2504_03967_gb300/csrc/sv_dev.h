// Plan records the device reads (plan blob: passes, ops, gate records, phase
// word layouts) and the shared-memory layout of a tile-pass CTA.  Plain PODs
// and constants only, so the same definitions serve the library and the pass
// kernels compiled at run time.
#pragma once

namespace sv {

constexpr int kMaxK = 5;         // widest fused dense block
constexpr int kMaxTileM = 14;    // qubits per shared-memory tile
constexpr int kPassThreads = 256;

// OP_DENSE_TC (register passes, complex64): a dense block of 4 or 5 qubits
// on the tensor cores (FP16 hi/lo split, three products, FP32 accumulation).
enum OpKind { OP_DENSE = 0, OP_DIAG = 1, OP_GATES = 2, OP_REMAP = 3, OP_DENSE_TC = 4 };

// Launch bounds of a register pass with tb thread bits: 128 threads at least
// 2 CTAs per SM, 256 threads 2 (128 registers), 512 threads 1.  (A cap of 128
// registers on 128-thread passes measured no faster: it trades spills for
// residency.)
__host__ __device__ inline int pass_max_threads(int tb) { return tb <= 7 ? 128 : (tb == 8 ? 256 : 512); }
__host__ __device__ inline int pass_min_blocks(int tb) { return tb <= 8 ? 2 : 1; }

// Register-resident passes: each thread holds 2^kRegBits amplitudes of the
// tile in registers; the other m - kRegBits tile bits index the thread.
__host__ __device__ inline int reg_bits(int dtype) { return dtype == 0 ? 5 : 4; }  // 0: complex64
constexpr int kRegDenseMaxK = 3;  // dense blocks in registers (wider ones run as gate sequences)
constexpr int kStageCap = 48 * 1024;  // bytes of a pass region staged in shared memory
constexpr int kStageCapTc = 100 * 1024;  // the same for a pass with tensor-core blocks

// Gate-sequence block records (positions are block-local bits, data offsets
// index the op's own complex values).
enum GateRecKind { GR_U = 0, GR_UR = 1, GR_DT = 2, GR_CX = 3, GR_SWAP = 4, GR_H = 5, GR_HD = 6, GR_URS = 7 };
// GR_DT: a = mask of the positions its entries depend on (entry j equals
// entry j & a), b = mask of the entries that differ from 1 (register passes).
// GR_HD (register passes only): GR_H on position a followed by the phase table
// at off with entry mask b (one dispatch for the pair).
// GR_URS (register passes only): a rotation [[c, -s], [s, c]] on position a
// without its larger factor: [[1, -t], [t, 1]] with t = s / c (b = 0) or
// [[t, -1], [1, t]] with t = c / s (b = 1), t at off; the factor joins
// PassDev::scale like GR_H's.
// GR_H (register passes only): the Hadamard without its 1/sqrt(2), a + b and
// a - b; the pass multiplies its amplitudes by the product of the dropped
// factors once, when it writes them back (PassDev::scale).
struct GateRec {
    int kind, a, b, off;
};
constexpr int kMaxGateRecs = 64;     // records per gate-sequence op
constexpr int kMaxGateData = 768;    // complex values per gate-sequence op

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
    int nrec;      // gates: number of records; remap: 1 when every warp's amplitudes stay within the warp
    int rec_off;   // gates: byte offset of the records
    int ndata;     // gates: complex values at mat_off
    int ord;       // register passes, diag: ordinal of the run within the pass
    float tc_scale;  // OP_DENSE_TC: factor applied to the registers before the FP16 split
    int pad[3];
};
static_assert(sizeof(OpDev) % 16 == 0, "OpDev array must keep 16-byte alignment");

// OP_DENSE_TC operand scales: the registers enter the FP16 split as the true
// amplitudes times kTcInScale (room for |a| <= 16 below the FP16 maximum) and
// the matrix is staged times kTcMatScale (its small entries stay normal
// FP16 numbers); the product leaves the registers at kTcInScale * kTcMatScale.
constexpr float kTcInScale = 4096.0f;
constexpr float kTcMatScale = 16.0f;
// Bytes of one OP_DENSE_TC matrix operand (hi or lo) of a k-qubit block: the
// real form, 2^(k+1) x 2^(k+1) FP16 values.
__host__ __device__ inline int tc16_bytes(int k) { return 8 << (2 * k); }

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
    long long basis;     // >= 0: the state is |basis> and this pass's compiled kernel builds its tiles from it
                         // instead of reading them (the deferred sv_init_basis); -1 otherwise
};


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


// Shared-memory layout of one pass CTA, computed on the host:
//   [tile buffer 0 | tile buffer 1 (nbuf = 2) | row offsets | resident
//    tensor-core B operands | staged pass region | work]
// With the whole region staged, every op reads its matrix, records or phase
// words from shared memory for all of the CTA's tiles; otherwise only the
// OpDev array is staged and each op copies its payload into the work area.
// With two tile buffers the next tile's copies are in flight while the
// current one is processed.
struct PassLayout {
    int nbuf;
    int tile_bytes;
    int rowoff_off;
    int bres_off;
    int stage_off;
    int tc_res;       // floats of tensor-core B operands kept resident (0: copied per op)
    int stage_bytes;  // bytes of the region copied (region or its OpDev array)
    int staged;       // 1: the whole region is in shared memory
    int work_off;
    int total;
};

}  // namespace sv
