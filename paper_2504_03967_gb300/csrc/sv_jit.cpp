// Pass kernels compiled at run time (the paper's own route: Q-GEAR turns
// circuits into GPU kernels, Sec. 2.2; here one kernel per pass structure).
//
// The library's register-pass kernel walks a pass's op list at run time: a
// switch per op and per gate record, positions and masks read from shared
// memory, register layouts computed per thread.  For a pass structure that
// recurs (the same circuit again, or circuits of one shape with other
// angles), this file writes the pass as straight-line code -- every op, gate
// position, phase-table mask, data offset and register layout a compile-time
// constant, the data (matrices, tables, phase words) still read from the
// staged region -- compiles it with NVRTC for this GPU's architecture, and
// launches it in place of the interpreting kernel.  The kernel body is the
// same source (sv_rpass.cuh), so both produce the same arithmetic.
//
// NVRTC is loaded with dlopen; where it is missing or a compile fails, the
// pass keeps running on the interpreting kernel (still on the GPU).
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <thread>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "sv_internal.h"

namespace sv {
namespace {

// ---- NVRTC and driver entry points --------------------------------------
struct Nvrtc {
    bool ok = false;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

struct Driver {
    bool ok = false;
    CUresult (*module_load)(CUmodule*, const void*) = nullptr;
    CUresult (*get_function)(CUfunction*, CUmodule, const char*) = nullptr;
    CUresult (*set_attr)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*occupancy)(int*, CUfunction, int, size_t) = nullptr;
    CUresult (*get_attr)(int*, CUfunction_attribute, CUfunction) = nullptr;
    CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                       void**, void**) = nullptr;
};

template <typename F> bool sym(void* lib, const char* name, F* out) {
    *out = (F)dlsym(lib, name);
    return *out != nullptr;
}

const Nvrtc& nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, []() {
        void* lib = nullptr;
        for (const char* nm : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"})
            if ((lib = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!lib) return;
        n.ok = sym(lib, "nvrtcCreateProgram", &n.create) && sym(lib, "nvrtcCompileProgram", &n.compile) &&
               sym(lib, "nvrtcGetProgramLogSize", &n.log_size) && sym(lib, "nvrtcGetProgramLog", &n.log) &&
               sym(lib, "nvrtcGetCUBINSize", &n.cubin_size) && sym(lib, "nvrtcGetCUBIN", &n.cubin) &&
               sym(lib, "nvrtcDestroyProgram", &n.destroy);
    });
    return n;
}

template <typename F> bool entry(const char* name, F* out) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return false;
    }
    *out = (F)p;
    return true;
}

const Driver& driver() {
    static Driver d;
    static std::once_flag once;
    std::call_once(once, []() {
        d.ok = entry("cuModuleLoadData", &d.module_load) && entry("cuModuleGetFunction", &d.get_function) &&
               entry("cuFuncSetAttribute", &d.set_attr) &&
               entry("cuOccupancyMaxActiveBlocksPerMultiprocessor", &d.occupancy) &&
               entry("cuFuncGetAttribute", &d.get_attr) && entry("cuLaunchKernel", &d.launch);
    });
    return d;
}

// Directory of the library's sources (csrc/ next to libsv.so): the include
// path of the run-time compiler.
std::string source_dir() {
    Dl_info info;
    if (!dladdr((void*)&source_dir, &info) || !info.dli_fname) return "";
    std::string p(info.dli_fname);
    const size_t s = p.rfind('/');
    return (s == std::string::npos ? std::string(".") : p.substr(0, s)) + "/csrc";
}

int arch_of_device() {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaGetLastError();
    return 10 * major + minor;
}

// ---- source of one pass ---------------------------------------------------
int swz_host(int dtype, int i) {  // the tile swizzle (sv_rpass.cuh swz)
    return dtype == SV_C64 ? i ^ (((i >> 4) & 7) << 1) : i ^ ((i >> 3) & 7);
}

void emit_ints(std::ostringstream& o, const char* name, const int* a, int cnt) {
    o << "constexpr int " << name << "[" << (cnt ? cnt : 1) << "] = {";
    for (int i = 0; i < cnt; ++i) o << (i ? ", " : "") << a[i];
    if (!cnt) o << "0";
    o << "};\n";
}

// Register layout rp/tp: the swizzled offsets C[k] of register combination
// k, and whether no thread's base can share a bit with any C[k].
struct CtLayout {
    int rp[8], tp[16], C[64];
    bool add;
};
CtLayout ct_layout(int dtype, int RB, int tb, const int* rp, const int* tp) {
    CtLayout L;
    int sbit[8], tmask = 0, cmask = 0;
    for (int b = 0; b < RB; ++b) L.rp[b] = rp[b], sbit[b] = swz_host(dtype, 1 << rp[b]);
    for (int t = 0; t < tb; ++t) L.tp[t] = tp[t], tmask |= swz_host(dtype, 1 << tp[t]);
    for (int k = 0; k < (1 << RB); ++k) {
        int c = 0;
        for (int b = 0; b < RB; ++b)
            if ((k >> b) & 1) c ^= sbit[b];
        L.C[k] = c;
        cmask |= c;
    }
    L.add = (tmask & cmask) == 0;
    return L;
}

// A register layout whose warp accesses to global memory cover runs of at
// least 32 bytes: the lanes (thread bits 0..4) hold tile positions 0 and 1
// (complex64 with position 0 at register bit 0, moved as 16-byte pairs:
// position 1; complex128: position 0).  Tile positions 0..L-1 are qubits
// 0..L-1, contiguous in the state.
bool direct_ok(int dtype, int RB, int tb, const int* rp, const int* tp) {
    const int nl = std::min(5, tb);
    auto lane = [&](int q) { return std::find(tp, tp + nl, q) != tp + nl; };
    (void)RB;
    if (dtype != SV_C64) return lane(0);
    return rp[0] == 0 ? lane(1) : lane(0) && lane(1);
}

// load (name "ld") / store_regs ("st"): the registers of layout rp/tp moved
// straight between the state and registers.  Register k of thread t is
// amplitude base + G(t) + KR[k], G(t) = the thread bits at their qubits; the
// deferred-basis variant (fill) builds |x> in the registers instead.
void emit_direct(std::ostringstream& o, const char* name, const PassDev& P, int dtype, int RB, int tb, const int* rp,
                 const int* tp, bool load, bool fill) {
    const bool pair = dtype == SV_C64 && rp[0] == 0;  // registers 2j, 2j + 1 adjacent in the state
    o << "static constexpr unsigned long long " << name << "_KR[" << (1 << RB) << "] = {";
    for (int k = 0; k < (1 << RB); ++k) {
        unsigned long long off = 0;
        for (int b = 0; b < RB; ++b)
            if ((k >> b) & 1) off |= 1ull << P.tq[rp[b]];
        o << (k ? ", " : "") << off << "ull";
    }
    o << "};\n";
    o << "static constexpr int " << name << "_TQ[" << tb << "] = {";
    for (int t = 0; t < tb; ++t) o << (t ? ", " : "") << P.tq[tp[t]];
    o << "};\n";
    o << "static __device__ __forceinline__ uint64_t " << name << "_goff() {\nuint64_t g = 0;\n#pragma unroll\n"
      << "for (int t = 0; t < " << tb << "; ++t) g |= (uint64_t)((threadIdx.x >> t) & 1) << " << name
      << "_TQ[t];\nreturn g;\n}\n";
    if (load) {
        o << "template <typename V>\nstatic __device__ __forceinline__ void load(V* v, const V* __restrict__ psi, "
             "uint64_t base, const PassDev& P) {\n"
          << "const uint64_t g = base + " << name << "_goff();\n";
        if (fill) {
            o << "const unsigned long long x = (unsigned long long)P.basis;\n#pragma unroll\n"
              << "for (int k = 0; k < " << (1 << RB) << "; ++k) {\nv[k].x = g + " << name
              << "_KR[k] == x ? 1 : 0;\nv[k].y = 0;\n}\n";
        } else if (pair) {
            o << "#pragma unroll\nfor (int k = 0; k < " << (1 << RB) << "; k += 2) {\n"
              << "const float4 q = *reinterpret_cast<const float4*>(psi + g + " << name << "_KR[k]);\n"
              << "v[k].x = q.x;\nv[k].y = q.y;\nv[k + 1].x = q.z;\nv[k + 1].y = q.w;\n}\n";
        } else {
            o << "#pragma unroll\nfor (int k = 0; k < " << (1 << RB) << "; ++k) v[k] = psi[g + " << name
              << "_KR[k]];\n";
        }
        o << "}\n";
    } else {
        o << "template <typename V>\nstatic __device__ __forceinline__ void store_regs(const V* v, V* __restrict__ psi, "
             "uint64_t base) {\n"
          << "const uint64_t g = base + " << name << "_goff();\n";
        if (pair) {
            o << "#pragma unroll\nfor (int k = 0; k < " << (1 << RB) << "; k += 2)\n"
              << "*reinterpret_cast<float4*>(psi + g + " << name
              << "_KR[k]) = make_float4(v[k].x, v[k].y, v[k + 1].x, v[k + 1].y);\n";
        } else {
            o << "#pragma unroll\nfor (int k = 0; k < " << (1 << RB) << "; ++k) psi[g + " << name << "_KR[k]] = v[k];\n";
        }
        o << "}\n";
    }
}

// The pass as straight-line code (mirrors InterpOps op by op).  Returns
// false for a structure it does not take.
bool pass_source(const PassDev& P, const unsigned char* region, int dtype, int maxt, int minb, std::string* out,
                 bool fill = false) {
    const int RB = reg_bits(dtype), tb = P.m - RB, L = P.L, m = P.m, no = P.nother;
    if (tb < 5 || tb > 9 || L < 1) return false;
    const OpDev* ops = (const OpDev*)region;
    const int PER = dtype == SV_C64 ? 2 : 1;  // amplitudes per 16-byte chunk
    const int T = 1 << tb, NCH = (1 << RB) / PER;
    const int istep = PER * T;
    if (istep % (1 << L)) return false;
    std::ostringstream o;
    o << "#include \"sv_rpass.cuh\"\nnamespace sv {\nstruct GenOps {\n";
    // tile copies: thread part of the row index from i0 = PER * tid, chunk
    // part from k * istep (disjoint bits, so the row offsets add)
    {
        uint64_t KO[64];
        int SW[64];
        int swmask = 0, s0mask = 0;
        for (int k = 0; k < NCH; ++k) {
            const int i = k * istep, r = i >> L;
            uint64_t off = 0;
            for (int b = 0; b < m - L; ++b)
                if ((r >> b) & 1) off |= 1ull << P.tq[L + b];
            KO[k] = off;
            SW[k] = swz_host(dtype, i);
            swmask |= SW[k];
        }
        for (int b = 0; (1 << b) < istep; ++b)
            if ((1 << b) >= PER) s0mask |= swz_host(dtype, 1 << b);
        const bool add = (swmask & s0mask) == 0;
        o << "static constexpr unsigned long long KO[" << NCH << "] = {";
        for (int k = 0; k < NCH; ++k) o << (k ? ", " : "") << KO[k] << "ull";
        o << "};\n";
        o << "static constexpr int SW[" << NCH << "] = {";
        for (int k = 0; k < NCH; ++k) o << (k ? ", " : "") << SW[k];
        o << "};\n";
        // per-thread global offset: in-row part and the row bits of i0
        o << "static __device__ __forceinline__ uint64_t thread_goff() {\n"
          << "const int i0 = " << PER << " * (int)threadIdx.x;\n"
          << "uint64_t g = (uint64_t)(i0 & " << ((1 << L) - 1) << ");\n";
        for (int b = 0; (1 << (L + b)) < istep && L + b < m; ++b)
            o << "g |= (uint64_t)((i0 >> " << L + b << ") & 1) << " << P.tq[L + b] << ";\n";
        o << "return g;\n}\n";
        o << "template <typename V>\nstatic __device__ __forceinline__ void issue(V* tile, const V* __restrict__ psi, "
             "uint64_t base, const uint32_t*, int, const PassDev& P) {\n";
        if (fill) {
            // |basis>: is it in this tile, and at which tile position?
            uint64_t tmask = 0;
            for (int p = 0; p < m; ++p) tmask |= 1ull << P.tq[p];
            o << "const unsigned long long x = (unsigned long long)P.basis;\nint ix = -1;\n"
              << "if ((x & ~" << tmask << "ull) == base) {\nix = 0;\n";
            for (int p = 0; p < m; ++p) o << "ix |= (int)((x >> " << P.tq[p] << ") & 1) << " << p << ";\n";
            o << "}\nfill_basis_ct<V, " << NCH << ", " << (add ? "true" : "false") << ">(tile, ix, " << PER
              << " * (int)threadIdx.x, " << istep << ", swz<V>(" << PER << " * (int)threadIdx.x), SW);\n}\n";
        } else {
            o << "issue_ct<V, " << NCH << ", " << (add ? "true" : "false")
              << ">(tile, psi, base + thread_goff(), swz<V>(" << PER << " * (int)threadIdx.x), KO, SW);\n}\n";
        }
        o << "template <typename V>\nstatic __device__ __forceinline__ void store(const V* tile, V* __restrict__ psi, "
             "uint64_t base, const uint32_t*, int) {\n"
          << "store_ct<V, " << NCH << ", " << (add ? "true" : "false")
          << ">(tile, psi, base + thread_goff(), swz<V>(" << PER << " * (int)threadIdx.x), KO, SW);\n}\n";
    }
    o << "template <typename V, typename R, int RB>\n"
         "static __device__ __forceinline__ void tile(V* v, V* tile, const PassDev& P, const unsigned char* stage,\n"
         "                                            const uint64_t* fold, RegLayout<V, RB>& Lg, const double2* ttab,\n"
         "                                            TcCtx& T) {\n";
    int rpos[8] = {0}, tpos[16] = {0}, nrpos[8] = {0}, ntpos[16] = {0}, frpos[8] = {0}, ftpos[16] = {0};
    bool in_regs = false, direct_load = false;
    CtLayout cur;
    int nl = 0;
    auto emit_rw = [&](const char* fn, const CtLayout& Lc, int id) {
        o << "{\n";
        emit_ints(o, "tp", Lc.tp, tb);
        emit_ints(o, "C", Lc.C, 1 << RB);
        // complex64 with tile position 0 at register bit 0: 16-byte accesses
        o << fn << (dtype == SV_C64 && Lc.rp[0] == 0 ? "2" : "") << "<V, RB, " << (Lc.add ? "true" : "false") << ">(v, tile, thread_sbase<V, " << tb
          << ">(tp), C);\n}\n";
        (void)id;
    };
    bool scaled = false;  // the pass holds rotations whose factor joins the scale
    for (int oi = 0; oi < P.nops; ++oi) {
        const OpDev& op = ops[oi];
        switch (op.kind) {
        case OP_REMAP: {
            // no barrier before the write (a warp writes exactly the positions
            // it read last); a warp barrier after it when every warp's
            // amplitudes stay within the warp (nrec = 1), else a block barrier
            for (int b = 0; b < RB; ++b) nrpos[b] = op.lq[b];
            const int* tp = (const int*)(region + op.mat_off);
            for (int t = 0; t < tb; ++t) ntpos[t] = tp[t];
            if (in_regs) {
                emit_rw("reg_write_ct", cur, nl);
                o << (op.nrec == 1 ? "__syncwarp();\n" : "__syncthreads();\n");
            } else {
                // the first layout: loaded straight into registers when its
                // warp accesses cover runs of 32 bytes or more
                direct_load = direct_ok(dtype, RB, tb, nrpos, ntpos);
                std::copy(nrpos, nrpos + RB, frpos);
                std::copy(ntpos, ntpos + tb, ftpos);
                if (!direct_load) o << "__syncthreads();\n";
            }
            std::copy(nrpos, nrpos + RB, rpos);
            std::copy(ntpos, ntpos + tb, tpos);
            cur = ct_layout(dtype, RB, tb, rpos, tpos);
            ++nl;
            if (in_regs || !direct_load) emit_rw("reg_read_ct", cur, nl);
            // passes with tensor-core blocks restore each tile's norm as loaded
            if (!in_regs && P.tc_k) o << "warp_norm_to<RB>((const float2*)v, T.nin);\n";
            in_regs = true;
            break;
        }
        case OP_GATES: {
            if (!in_regs) return false;
            o << "{\nconst V* sd = (const V*)(stage + " << op.mat_off << ");\n";
            const GateRec* recs = (const GateRec*)(region + op.rec_off);
            for (int r = 0; r < op.nrec; ++r) {
                const GateRec& g = recs[r];
                const int f = g.off;
                switch (g.kind) {
                case GR_U:
                    o << "reg_u<V, RB, " << g.a << ">(v, sd[" << f << "], sd[" << f + 1 << "], sd[" << f + 2
                      << "], sd[" << f + 3 << "]);\n";
                    break;
                case GR_UR:
                    o << "reg_ur<V, RB, " << g.a << ", R>(v, sd[" << f << "].x, sd[" << f + 1 << "].x, sd["
                      << f + 2 << "].x, sd[" << f + 3 << "].x);\n";
                    break;
                case GR_DT:
                    // a table on at most three register bits: its (at most 8)
                    // distinct entries are read once
                    if (__builtin_popcount((unsigned)g.a) <= 3)
                        o << "reg_dt_dep<V, RB, 0x" << std::hex << (unsigned)g.b << "u, 0x" << (unsigned)g.a
                          << std::dec << "u>(v, sd + " << f << ");\n";
                    else
                        o << "reg_dt<V, RB, 0x" << std::hex << (unsigned)g.b << std::dec << "u>(v, sd + " << f << ");\n";
                    break;
                case GR_CX: o << "reg_cx<V, RB, " << g.a << ", " << g.b << ">(v);\n"; break;
                case GR_H: o << "reg_h<V, RB, " << g.a << ">(v);\n"; break;
                case GR_URS:
                    o << "reg_urs<V, RB, " << g.a << ", " << g.b << ", R>(v, sd[" << f << "].x);\n";
                    scaled = true;
                    break;
                case GR_HD:
                    o << "reg_h<V, RB, " << g.a << ">(v);\nreg_dt<V, RB, 0x" << std::hex << (unsigned)g.b << std::dec
                      << "u>(v, sd + " << f << ");\n";
                    break;
                case GR_SWAP: o << "reg_swap<V, RB, " << g.a << ", " << g.b << ">(v);\n"; break;
                default: return false;
                }
            }
            o << "}\n";
            break;
        }
        case OP_DENSE:
            if (!in_regs || op.k < 1 || op.k > kRegDenseMaxK) return false;
            o << "reg_dense<V, RB, " << op.k << ">(v, (const V*)(stage + " << op.mat_off << "));\n";
            break;
        case OP_DENSE_TC:
            // the input scale depends on the pass's deferred factors (angles): read from the op record
            if (!in_regs || dtype != SV_C64 || (op.k != 4 && op.k != 5)) return false;
            o << "reg_dense_tc<RB, " << op.k << ">((float2*)v, stage + " << op.mat_off << ", ((const OpDev*)stage)["
              << oi << "].tc_scale, T);\n";
            break;
        case OP_DIAG:
            if (!in_regs) return false;
            o << "{\n";
            emit_ints(o, "rp", rpos, RB);
            emit_ints(o, "tp", tpos, tb);
            o << "reg_diag<V, R, RB>(v, (const uint64_t*)(stage + " << op.diag_off << "), fold + " << op.ord * (m + 1)
              << ", " << m << ", " << no << ", rp, tp, " << tb << ", ttab);\n}\n";
            break;
        default:
            return false;
        }
    }
    if (!in_regs) return false;
    o << "}\n";
    // write-back: the pass's scale, then the last layout.  A scale made of
    // Hadamard factors alone is a constant of the structure; one with rotation
    // factors depends on the angles and is read from the pass record.
    o << "template <typename V, typename R, int RB>\n"
         "static __device__ __forceinline__ void finish(V* v, V* tile, const PassDev& P, const RegLayout<V, RB>&,\n"
         "                                              TcCtx& T) {\n";
    // the last layout goes straight to global memory when its warp accesses
    // cover runs of 32 bytes or more
    const bool direct_store = direct_ok(dtype, RB, tb, rpos, tpos);
    if (P.tc_k) {
        // the tile's norm as loaded (every op is unitary on the tile): the
        // scale is sqrt(in / out) with the sign of the deferred factors, which
        // it also undoes
        o << "warp_norm_to<RB>((const float2*)v, T.nout);\n__syncthreads();\n"
          << "scale_regs<V, RB>(v, copysignf(tile_norm_fix(T.nin, T.nout), (float)P.scale));\n";
    } else if (scaled) {
        o << "scale_regs<V, RB>(v, (R)P.scale);\n";
    } else if (P.scale != 1.0) {
        char buf[64];
        snprintf(buf, sizeof(buf), "%.17g", P.scale);
        o << "scale_regs<V, RB>(v, (R)" << buf << ");\n";
    }
    // else each warp writes back the positions it read last (no barrier needed)
    if (!direct_store) emit_rw("reg_write_ct", cur, nl);
    o << "}\n";
    o << "static constexpr bool kDirectLoad = " << (direct_load ? "true" : "false")
      << ", kDirectStore = " << (direct_store ? "true" : "false") << ";\n";
    if (direct_load) emit_direct(o, "ld", P, dtype, RB, tb, frpos, ftpos, true, fill);
    if (direct_store) emit_direct(o, "st", P, dtype, RB, tb, rpos, tpos, false, false);
    o << "};\n}  // namespace sv\n";
    const char* R = dtype == SV_C64 ? "float" : "double";
    o << "extern \"C\" __global__ void __launch_bounds__(" << maxt << ", " << minb << ") sv_jit_pass(\n"
      << "    sv::CT<" << R << ">::V* __restrict__ psi, int n, const sv::PassDev* __restrict__ pdp,\n"
      << "    const unsigned char* __restrict__ blob, const sv::PassLayout lay, int* __restrict__ err) {\n"
      << "    sv::rpass_body<" << R << ", " << RB << ", sv::GenOps, " << (P.tc_k ? "true" : "false")
      << ">(psi, n, pdp, blob, lay, err);\n}\n";
    *out = o.str();
    return true;
}

// ---- cache ------------------------------------------------------------------
// One entry per pass source.  A structure compiles once per process, inside
// the apply that needs it (the passes of one plan in parallel): on its first
// use with jit = 1, on its second with jit = 0 (the first run of a structure,
// one-off circuits and small states stay on the interpreting kernel).
enum { JIT_NEW = 0, JIT_COMPILING, JIT_READY, JIT_FAILED };
// jit = 0 compiles only for states of at least this many qubits: below it a
// pass takes tens of microseconds, and the compile (about a second) would not
// pay back.
constexpr int kJitAutoMinQubits = 22;
struct Entry {
    int seen = 0;
    int state = JIT_NEW;
    CUfunction fn = nullptr;
    int attr_bytes = 0;
    bool direct_load = false;   // the kernel loads its first layout straight into registers (one tile buffer)
    bool direct_store = false;  // and stores its last layout straight from registers
};

std::mutex g_mu;
std::unordered_map<std::string, Entry> g_cache;
uint64_t g_compiled = 0, g_failed = 0, g_launched = 0, g_filled = 0, g_direct_ld = 0, g_direct_st = 0;
double g_compile_ms = 0.0;
std::string g_last_log;

// NVRTC only (no CUDA call, so any thread may run it): the cubin of src for
// sm_<arch>a, empty on a failure.
std::vector<char> nvrtc_cubin(const std::string& src, int arch, std::string* log) {
    const Nvrtc& nv = nvrtc();
    std::vector<char> cubin;
    const std::string inc = "--include-path=" + source_dir();
    char archo[64];
    snprintf(archo, sizeof(archo), "--gpu-architecture=sm_%da", arch);
    const char* opts[] = {archo, "-std=c++17", inc.c_str(), "-DSV_JIT=1", "-lineinfo"};
    nvrtcProgram prog;
    if (nv.create(&prog, src.c_str(), "sv_jit_pass.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) return cubin;
    const nvrtcResult rc = nv.compile(prog, 5, opts);
    size_t ls = 0;
    nv.log_size(prog, &ls);
    log->assign(ls, '\0');
    if (ls) nv.log(prog, &(*log)[0]);
    if (rc == NVRTC_SUCCESS) {
        size_t cs = 0;
        nv.cubin_size(prog, &cs);
        cubin.resize(cs);
        if (!cs || nv.cubin(prog, cubin.data()) != NVRTC_SUCCESS) cubin.clear();
    }
    nv.destroy(&prog);
    return cubin;
}

// Compile the sources (NVRTC on helper threads that are joined here, one per
// source), load the modules on the calling thread (its current context) and
// publish the results.  No thread outlives the call.
void compile_all(const std::vector<std::string>& srcs) {
    const Driver& dr = driver();
    const int arch = arch_of_device();
    std::vector<std::vector<char>> bins(srcs.size());
    std::vector<std::string> logs(srcs.size());
    const auto c0 = std::chrono::steady_clock::now();
    auto one = [&](size_t i) { bins[i] = nvrtc_cubin(srcs[i], arch, &logs[i]); };
    if (srcs.size() == 1) {
        one(0);
    } else {
        std::vector<std::thread> th;
        for (size_t i = 0; i < srcs.size(); ++i) th.emplace_back(one, i);
        for (auto& t : th) t.join();
    }
    std::vector<CUfunction> fns(srcs.size(), nullptr);
    for (size_t i = 0; i < srcs.size(); ++i) {
        if (bins[i].empty()) continue;
        CUmodule mod = nullptr;  // kept for the life of the process
        if (dr.module_load(&mod, bins[i].data()) != CUDA_SUCCESS ||
            dr.get_function(&fns[i], mod, "sv_jit_pass") != CUDA_SUCCESS)
            fns[i] = nullptr;
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c0).count();
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < srcs.size(); ++i) {
        Entry& e = g_cache[srcs[i]];
        e.fn = fns[i];
        e.direct_load = srcs[i].find("kDirectLoad = true") != std::string::npos;
        e.direct_store = srcs[i].find("kDirectStore = true") != std::string::npos;
        e.state = fns[i] ? JIT_READY : JIT_FAILED;
        (fns[i] ? g_compiled : g_failed)++;
        if (!logs[i].empty()) g_last_log = logs[i];
    }
    g_compile_ms += ms;
}

}  // namespace

void jit_prepare(sv_state* h, const PlanBlob& blob, int policy, long long basis, std::vector<void*>* fns,
                 void** fill0, std::vector<std::string>* memo) {
    fns->assign(blob.npasses, nullptr);
    *fill0 = nullptr;
    // jit = 0 on a small state: nothing to compile or look up (writing the
    // pass sources would cost more than the passes)
    if (policy < 0 || (policy == 0 && h->n < kJitAutoMinQubits) || !nvrtc().ok || !driver().ok) return;
    // sources: one per register pass, plus pass 0 building |basis> (a
    // cached plan keeps them: writing them is most of this function's time)
    std::vector<std::string> local;
    std::vector<std::string>& srcs = memo ? *memo : local;
    const bool fresh = (int)srcs.size() != blob.npasses + 1;
    if (fresh) {
        srcs.assign(blob.npasses + 1, std::string());
        for (int p = 0; p <= blob.npasses; ++p) {
            const bool fill = p == blob.npasses;
            const PassDev* pd = (const PassDev*)(blob.bytes.data() + blob.pass_off) + (fill ? 0 : p);
            if ((fill && blob.npasses == 0) || pd->rmode != 1) continue;
            const int tb = pd->m - reg_bits(h->dtype);
            if (!pass_source(*pd, blob.bytes.data() + pd->region_off, h->dtype, pass_max_threads(tb),
                             pass_min_blocks(tb), &srcs[p], fill))
                srcs[p].clear();
        }
    }
    std::vector<std::string> now;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (int p = 0; p <= blob.npasses; ++p) {
            if (srcs[p].empty() || (p == blob.npasses && basis < 0)) continue;
            Entry& e = g_cache[srcs[p]];
            e.seen++;
            if (e.state == JIT_NEW && (policy == 1 || e.seen >= 2)) {
                e.state = JIT_COMPILING;
                now.push_back(srcs[p]);
            }
        }
    }
    if (!now.empty()) compile_all(now);
    std::lock_guard<std::mutex> lk(g_mu);
    for (int p = 0; p <= blob.npasses; ++p) {
        if (srcs[p].empty() || (p == blob.npasses && basis < 0)) continue;
        auto it = g_cache.find(srcs[p]);
        if (it == g_cache.end() || it->second.state != JIT_READY) continue;
        if (p == blob.npasses) *fill0 = &it->second;
        else (*fns)[p] = &it->second;
    }
}

cudaError_t jit_launch(sv_state* h, void* entry, const void* blob_dev, const PlanBlob& blob, int pass, bool* used) {
    *used = false;
    if (!entry) return cudaSuccess;
    Entry& e = *(Entry*)entry;  // entries are never erased, so the pointer stays valid
    const Driver& dr = driver();
    const PassDev* pd = (const PassDev*)(blob.bytes.data() + blob.pass_off) + pass;
    const int tb = pd->m - reg_bits(h->dtype);
    const PassLayout lay = rpass_layout(h->dtype, *pd, e.direct_load);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (lay.total > e.attr_bytes) {
            if (dr.set_attr(e.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, lay.total) != CUDA_SUCCESS)
                return cudaSuccess;  // stays on the interpreting kernel
            e.attr_bytes = lay.total;
        }
    }
    const int threads = 1 << tb;
    int per_sm = 1;
    if (dr.occupancy(&per_sm, e.fn, threads, (size_t)lay.total) != CUDA_SUCCESS || per_sm < 1) per_sm = 1;
    if (pd->tc_k > 0) {
        // the occupancy query counts one CTA per SM for a kernel with TMEM
        // allocations; the CTAs an SM holds by registers, shared memory and
        // TMEM columns (rpass_layout pads the shared memory so that these
        // never ask for more than the SM's 512 columns)
        int regs = 0, sstat = 0;
        if (dr.get_attr(&regs, CU_FUNC_ATTRIBUTE_NUM_REGS, e.fn) == CUDA_SUCCESS &&
            dr.get_attr(&sstat, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, e.fn) == CUDA_SUCCESS)
            per_sm = std::max(per_sm, resident_ctas(threads, regs, sstat + lay.total));
    }
    const uint64_t ntiles = 1ull << (h->n - pd->m);
    uint64_t grid = (uint64_t)num_sms_pub() * per_sm;
    if (grid > ntiles) grid = ntiles;
    const unsigned char* b = (const unsigned char*)blob_dev;
    void* psi = h->amps;
    int n = h->n;
    const PassDev* pdp = (const PassDev*)(b + blob.pass_off) + pass;
    PassLayout lay_arg = lay;
    int* err = (int*)h->err.ptr;
    void* args[] = {&psi, &n, &pdp, &b, &lay_arg, &err};
    count_launch();
    if (dr.launch(e.fn, (unsigned)grid, 1, 1, (unsigned)threads, 1, 1, (unsigned)lay.total, (CUstream)h->stream, args,
                  nullptr) != CUDA_SUCCESS)
        return cudaErrorLaunchFailure;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        ++g_launched;
        g_direct_ld += e.direct_load;
        g_direct_st += e.direct_store;
    }
    *used = true;
    return cudaSuccess;
}

}  // namespace sv

using namespace sv;

namespace sv {
void jit_count_fill() {
    std::lock_guard<std::mutex> lk(g_mu);
    ++g_filled;
}
}  // namespace sv

// Passes that built their tiles from a deferred basis state (no state read).
extern "C" int sv_jit_fills(uint64_t* filled) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (filled) *filled = g_filled;
    return SV_OK;
}

extern "C" int sv_jit_stats(uint64_t* compiled, uint64_t* failed, uint64_t* launched, double* compile_ms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (compiled) *compiled = g_compiled;
    if (failed) *failed = g_failed;
    if (launched) *launched = g_launched;
    if (compile_ms) *compile_ms = g_compile_ms;
    return SV_OK;
}

extern "C" int sv_jit_direct(uint64_t* loads, uint64_t* stores) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (loads) *loads = g_direct_ld;
    if (stores) *stores = g_direct_st;
    return SV_OK;
}

// Compiles finish inside the apply that starts them; kept for callers that
// wait before timing.
extern "C" int sv_jit_wait(void) { return SV_OK; }

extern "C" int sv_jit_last_log(char* buf, size_t cap) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (buf && cap) {
        const size_t k = std::min(cap - 1, g_last_log.size());
        memcpy(buf, g_last_log.data(), k);
        buf[k] = '\0';
    }
    return SV_OK;
}

// Host-only check of the pass compiler: plan the circuit, write the source
// of every register-resident pass and compile it with NVRTC for sm_<arch>a
// (no module is loaded, so no GPU is needed).  *compiled = passes compiled;
// the last compiler log goes to log.
extern "C" int sv_jit_check(int n, sv_dtype dt, const sv_gate* gates, size_t count, const sv_options* opt, int arch,
                            int* compiled, char* log, size_t cap) {
    if (!compiled || (count && !gates)) return set_error(SV_EINVAL, "bad arguments");
    if (dt != SV_C64 && dt != SV_C128) return set_error(SV_EINVAL, "unknown dtype");
    if (n < 1 || n > (dt == SV_C64 ? kMaxQubitsC64 : kMaxQubitsC128)) return set_error(SV_EINVAL, "n out of range");
    const Nvrtc& nv = nvrtc();
    if (!nv.ok) return set_error(SV_EUNSUPPORTED, "NVRTC not found");
    std::vector<CGate> cg;
    size_t bad = 0;
    if (canonicalise(n, gates, count, &cg, &bad) != SV_OK)
        return set_error(SV_EINVAL, "invalid gate record at index " + std::to_string(bad));
    const PlanOptions po = resolve_options(n, dt, opt);
    Plan plan;
    plan_greedy(n, dt, cg, po, &plan);
    PlanBlob blob;
    serialise_plan(plan, &blob);
    *compiled = 0;
    const std::string inc = "--include-path=" + source_dir();
    char archo[64];
    snprintf(archo, sizeof(archo), "--gpu-architecture=sm_%da", arch);
    // the check also asks ptxas for its register and spill report
    const char* opts[] = {archo, "-std=c++17", inc.c_str(), "-DSV_JIT=1", "-lineinfo", "--ptxas-options=-v"};
    std::string lastlog, alllogs;
    for (int p = 0; p <= blob.npasses; ++p) {  // the last round: pass 0 building its tiles from |x>
        const bool fill = p == blob.npasses;
        if (fill && blob.npasses == 0) break;
        const PassDev* pd = (const PassDev*)(blob.bytes.data() + blob.pass_off) + (fill ? 0 : p);
        if (pd->rmode != 1) continue;
        const int tb = pd->m - reg_bits(dt);
        std::string src;
        if (!pass_source(*pd, blob.bytes.data() + pd->region_off, dt, pass_max_threads(tb), pass_min_blocks(tb),
                         &src, fill))
            continue;
        nvrtcProgram prog;
        if (nv.create(&prog, src.c_str(), "sv_jit_pass.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
            return set_error(SV_EUNSUPPORTED, "nvrtcCreateProgram failed");
        const nvrtcResult rc = nv.compile(prog, 6, opts);
        size_t ls = 0;
        nv.log_size(prog, &ls);
        lastlog.assign(ls, '\0');
        if (ls) nv.log(prog, &lastlog[0]);
        alllogs += lastlog;
        size_t cs = 0;
        if (rc == NVRTC_SUCCESS) nv.cubin_size(prog, &cs);
        nv.destroy(&prog);
        if (rc != NVRTC_SUCCESS || cs == 0) {
            if (log && cap) snprintf(log, cap, "%s\n--- source ---\n%s", lastlog.c_str(), src.c_str());
            return set_error(SV_EINVAL, "pass compile failed");
        }
        ++*compiled;
    }
    if (log && cap) snprintf(log, cap, "%s", alllogs.c_str());
    return SV_OK;
}
