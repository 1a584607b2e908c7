"""GB300-native (sm_103a) state-vector simulator: Python binding of libsv.

Argument marshalling only: every step runs in the CUDA library ``libsv.so``
(built in-tree by ``paper_2504_03967_gb300.build``).  There is no CPU fallback:
importing a function whose library is missing raises.  PyTorch is used by
callers for device memory and streams; pass ``tensor.data_ptr()`` and
``torch.cuda.current_stream().cuda_stream`` where a device pointer or stream is
expected.

The functions carry the names of the C ABI (include/sv.h); each returns the
C status converted to an exception (``SVError``) on failure.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsv.so")

C64, C128 = 0, 1
PLAN_GREEDY, PLAN_MLP, PLAN_PLAIN = 0, 1, 2

STATUS = {0: "SV_OK", -1: "SV_EINVAL", -2: "SV_ENOMEM", -3: "SV_EUNSUPPORTED", -4: "SV_ECUDA",
          -5: "SV_ETIMEOUT", -6: "SV_ESTATE"}

GATE_DTYPE = np.dtype([("type", "<u4"), ("nq", "<u4"), ("q", "<u4", (3,)),
                       ("pad", "<u4"), ("p", "<f8", (3,))])


class SVError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class sv_options(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int), ("tile_m", ctypes.c_int), ("planner", ctypes.c_int),
                ("record", ctypes.c_int), ("tensor", ctypes.c_int), ("pass_kernel", ctypes.c_int),
                ("relabel", ctypes.c_int), ("mux", ctypes.c_int), ("drop_phase_below", ctypes.c_double),
                ("jit", ctypes.c_int)]


class sv_plan_info(ctypes.Structure):
    _fields_ = [("gates", ctypes.c_int64), ("passes", ctypes.c_int64), ("dense_ops", ctypes.c_int64),
                ("diag_ops", ctypes.c_int64), ("max_k", ctypes.c_int64), ("bytes_moved", ctypes.c_int64),
                ("gate_ops", ctypes.c_int64), ("reg_passes", ctypes.c_int64), ("remaps", ctypes.c_int64),
                ("mux_ops", ctypes.c_int64), ("mux_passes", ctypes.c_int64),
                ("tc_ops", ctypes.c_int64), ("warp_remaps", ctypes.c_int64)]


class sv_plan_op(ctypes.Structure):
    _fields_ = [("pass_", ctypes.c_int), ("kind", ctypes.c_int), ("k", ctypes.c_int), ("q", ctypes.c_int * 5),
                ("nrec", ctypes.c_int), ("rec_off", ctypes.c_int), ("data_off", ctypes.c_int64)]


_lib = None


def lib():
    """Load libsv.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsv.so not built: run paper_2504_03967_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t
        P = ctypes.POINTER
        sig = {
            "sv_alloc": [i, i, vp, P(vp)],
            "sv_attach": [i, i, vp, vp, P(vp)],
            "sv_free": [vp],
            "sv_set_stream": [vp, vp],
            "sv_info": [vp, P(i), P(i), P(vp)],
            "sv_qubit_map": [vp, vp],
            "sv_materialize": [vp],
            "sv_last_plan": [vp, vp],
            "sv_init_basis": [vp, u64],
            "sv_load_state": [vp, vp],
            "sv_store_state": [vp, vp],
            "sv_apply_circuit": [vp, vp, sz, P(sv_options)],
            "sv_plan_circuit": [i, i, vp, sz, P(sv_options), P(sv_plan_info)],
            "sv_plan_ops": [i, i, vp, sz, P(sv_options), vp, sz, P(sz), vp, sz, P(sz), vp, sz, P(sz)],
            "sv_probs": [vp, vp],
            "sv_probs_device": [vp, vp],
            "sv_norm": [vp, P(ctypes.c_double)],
            "sv_expect_z": [vp, vp],
            "sv_expect_z_device": [vp, vp],
            "sv_sample": [vp, u64, u64, vp],
            "sv_sample_device": [vp, u64, u64, vp],
            "sv_sample_uniforms": [vp, vp, u64, vp],
            "sv_pass_times": [vp, vp, vp, i, P(i)],
            "sv_sample_uniforms_noalloc": [vp, i, i, vp, u64, vp, vp],
            "sv_qcrank_decode_device": [vp, u64, i, i, vp, vp, vp, vp],
            "sv_qcrank_reconstruct": [vp, i, i, u64, u64, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.sv_last_error.restype = ctypes.c_char_p
        L.sv_version.restype = ctypes.c_int
        L.sv_launch_count.restype = ctypes.c_uint64
        L.sv_feature_count.restype = ctypes.c_int
        _lib = L
    return _lib


def exported_symbols():
    """Names declared in include/sv.h that the loaded library exports."""
    L = lib()
    return [n for n in declared_symbols() if hasattr(L, n)]


def declared_symbols():
    """Entry points declared in every header under include/."""
    import glob
    import re
    names = set()
    for hdr in glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h")):
        with open(hdr) as f:
            txt = f.read()
        names |= set(re.findall(r"^\s*(?:int|const char \*|uint64_t)\s*\*?\s*(sv_\w+)\s*\(", txt, re.M))
    return sorted(names)


def _check(rc):
    if rc != 0:
        raise SVError(rc, lib().sv_last_error().decode())
    return rc


def _opts(k_max=0, tile_m=0, planner=PLAN_GREEDY, record=0, tensor=0, pass_kernel=0, relabel=0, drop_phase_below=0.0,
          mux=0, jit=0):
    o = sv_options()
    o.k_max, o.tile_m, o.planner, o.record, o.tensor = k_max, tile_m, planner, record, tensor
    o.pass_kernel, o.relabel, o.drop_phase_below, o.mux, o.jit = pass_kernel, relabel, drop_phase_below, mux, jit
    return o


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def as_gates(g):
    g = np.ascontiguousarray(g)
    if g.dtype.itemsize != GATE_DTYPE.itemsize:
        raise ValueError("gate records must be 48-byte sv_gate structs")
    return g


# ---- C ABI names ----------------------------------------------------------
def sv_version():
    return lib().sv_version()


def sv_launch_count():
    return lib().sv_launch_count()


def sv_last_error():
    return lib().sv_last_error().decode()


def sv_alloc(n, dtype=C64, stream=None):
    h = ctypes.c_void_p()
    _check(lib().sv_alloc(n, dtype, stream, ctypes.byref(h)))
    return h


def sv_attach(n, dtype, dev_ptr, stream=None):
    h = ctypes.c_void_p()
    _check(lib().sv_attach(n, dtype, ctypes.c_void_p(dev_ptr), stream, ctypes.byref(h)))
    return h


def sv_free(h):
    _check(lib().sv_free(h))


def sv_set_stream(h, stream):
    _check(lib().sv_set_stream(h, stream))


def sv_info(h):
    """(n, dtype, device pointer).  Handing out the pointer writes a deferred
    sv_init_basis first, so the memory holds the state."""
    n, dt, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_void_p()
    _check(lib().sv_info(h, ctypes.byref(n), ctypes.byref(dt), ctypes.byref(p)))
    return n.value, dt.value, p.value


def _n_dtype(h):
    n, dt = ctypes.c_int(), ctypes.c_int()
    _check(lib().sv_info(h, ctypes.byref(n), ctypes.byref(dt), None))
    return n.value, dt.value


def sv_init_basis(h, x=0):
    _check(lib().sv_init_basis(h, int(x)))


def sv_load_state(h, amps):
    n, dt = _n_dtype(h)
    a = np.ascontiguousarray(amps, dtype=np.complex64 if dt == C64 else np.complex128)
    assert a.shape == (1 << n,)
    _check(lib().sv_load_state(h, _ptr(a)))


def sv_store_state(h):
    n, dt = _n_dtype(h)
    a = np.empty(1 << n, dtype=np.complex64 if dt == C64 else np.complex128)
    _check(lib().sv_store_state(h, _ptr(a)))
    return a


def sv_apply_circuit(h, gates, k_max=0, tile_m=0, planner=PLAN_GREEDY, record=0, tensor=0, pass_kernel=0, relabel=0,
                     drop_phase_below=0.0, mux=0, jit=0):
    g = as_gates(gates)
    o = _opts(k_max, tile_m, planner, record, tensor, pass_kernel, relabel, drop_phase_below, mux, jit)
    _check(lib().sv_apply_circuit(h, _ptr(g), len(g), ctypes.byref(o)))


def sv_plan_circuit(n, dtype, gates, k_max=0, tile_m=0, planner=PLAN_GREEDY, tensor=0, pass_kernel=0,
                    drop_phase_below=0.0, mux=0):
    g = as_gates(gates)
    o = _opts(k_max, tile_m, planner, 0, tensor, pass_kernel, 0, drop_phase_below, mux)
    info = sv_plan_info()
    _check(lib().sv_plan_circuit(n, dtype, _ptr(g), len(g), ctypes.byref(o), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in sv_plan_info._fields_}


def sv_plan_ops(n, dtype, gates, k_max=0, tile_m=0, mux=-1, drop_phase_below=0.0, pass_kernel=0, tensor=0):
    """Host only: the greedy plan's ops in FP64 (see sv_plan_op in sv.h), as a
    list of dicts: pass, kind ("dense", "diag", "gates", "mux"), qubits, and
    per kind: mat (2^k x 2^k complex), c / a / b (phase run), recs (rkind, a,
    b, off rows) with vals (complex values), target / family / flip / flip_c /
    controls / phi0 / phi1 (multiplexor)."""
    g = as_gates(gates)
    o = _opts(k_max, tile_m, PLAN_GREEDY, 0, tensor, pass_kernel, 0, drop_phase_below, mux)
    L = lib()
    cnt = [ctypes.c_size_t(0) for _ in range(3)]
    rc = L.sv_plan_ops(n, dtype, _ptr(g), len(g), ctypes.byref(o), None, 0, ctypes.byref(cnt[0]), None, 0,
                       ctypes.byref(cnt[1]), None, 0, ctypes.byref(cnt[2]))
    if rc not in (0, -1) or (rc == -1 and cnt[0].value == 0 and len(g)):
        _check(rc)
    ops = (sv_plan_op * max(1, cnt[0].value))()
    recs = np.zeros(max(1, cnt[1].value), dtype=np.int32)
    data = np.zeros(max(1, cnt[2].value), dtype=np.float64)
    _check(L.sv_plan_ops(n, dtype, _ptr(g), len(g), ctypes.byref(o), ctypes.cast(ops, ctypes.c_void_p), len(ops),
                         ctypes.byref(cnt[0]), _ptr(recs), len(recs), ctypes.byref(cnt[1]), _ptr(data), len(data),
                         ctypes.byref(cnt[2])))
    out = []
    for r in ops[: cnt[0].value]:
        k = r.k
        d = {"pass": r.pass_, "kind": ("dense", "diag", "gates", "mux")[r.kind], "qubits": list(r.q[:k])}
        off = r.data_off
        if r.kind == 0:
            v = data[off: off + 2 * 4 ** k]
            d["mat"] = (v[0::2] + 1j * v[1::2]).reshape(1 << k, 1 << k)
        elif r.kind == 1:
            d["c"] = float(data[off])
            d["a"] = data[off + 1: off + 1 + n].copy()
            d["b"] = data[off + 1 + n: off + 1 + n + n * n].reshape(n, n).copy()
        elif r.kind == 2:
            rr = recs[r.rec_off: r.rec_off + 4 * r.nrec].reshape(-1, 4).copy()
            d["recs"] = rr
            nv = 0
            for rk, _, _, ro in rr:
                nv = max(nv, ro + (4 if rk in (0, 1) else (1 << k) if rk == 2 else 0))
            v = data[off: off + 2 * nv]
            d["vals"] = v[0::2] + 1j * v[1::2]
        else:
            d["target"] = r.q[0]
            fam, flip, flip_c, nc = (int(v) for v in data[off: off + 4])
            J = 1 << nc
            d["family"] = ("ry", "diag")[fam]
            d["flip"], d["flip_c"] = flip, flip_c
            d["controls"] = [int(v) for v in data[off + 4: off + 4 + nc]]
            d["phi0"] = data[off + 4 + nc: off + 4 + nc + J].copy()
            if fam:
                d["phi1"] = data[off + 4 + nc + J: off + 4 + nc + 2 * J].copy()
        out.append(d)
    return out


def sv_qubit_map(h):
    """Physical bit of each logical qubit (identity unless relabelled)."""
    n, _ = _n_dtype(h)
    m = (ctypes.c_int * max(1, n))()
    _check(lib().sv_qubit_map(h, m))
    return [m[i] for i in range(n)]


def sv_materialize(h):
    _check(lib().sv_materialize(h))


def sv_last_plan(h):
    o = sv_options()
    _check(lib().sv_last_plan(h, ctypes.byref(o)))
    return {"k_max": o.k_max, "tile_m": o.tile_m, "planner": o.planner, "tensor": o.tensor,
            "pass_kernel": o.pass_kernel, "relabel": o.relabel}


def sv_probs(h):
    n, _ = _n_dtype(h)
    out = np.empty(1 << n, dtype=np.float64)
    _check(lib().sv_probs(h, _ptr(out)))
    return out


def sv_probs_device(h, dev_out_ptr):
    _check(lib().sv_probs_device(h, ctypes.c_void_p(dev_out_ptr)))


def sv_norm(h):
    v = ctypes.c_double()
    _check(lib().sv_norm(h, ctypes.byref(v)))
    return v.value


def sv_expect_z(h):
    n, _ = _n_dtype(h)
    out = np.empty(n, dtype=np.float64)
    _check(lib().sv_expect_z(h, _ptr(out)))
    return out


def sv_expect_z_device(h, dev_out_ptr):
    _check(lib().sv_expect_z_device(h, ctypes.c_void_p(dev_out_ptr)))


def sv_sample(h, shots, seed):
    out = np.empty(int(shots), dtype=np.uint64)
    _check(lib().sv_sample(h, int(shots), int(seed), _ptr(out)))
    return out


def sv_jit_check(n, dtype, gates, arch=103, **opts):
    """Host-only: write and compile (NVRTC, no GPU) the run-time kernel of
    every register-resident pass of the circuit's plan.  Returns the number
    of passes compiled; raises SVError with the compiler log on a failure."""
    g = as_gates(gates)
    o = _opts(**opts)
    L = lib()
    f = L.sv_jit_check
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(sv_options), ctypes.c_int,
                  ctypes.POINTER(ctypes.c_int), ctypes.c_char_p, ctypes.c_size_t]
    f.restype = ctypes.c_int
    cnt = ctypes.c_int(0)
    buf = ctypes.create_string_buffer(1 << 16)
    rc = f(n, dtype, _ptr(g), len(g), ctypes.byref(o), arch, ctypes.byref(cnt), buf, len(buf))
    if rc != 0:
        raise SVError(rc, L.sv_last_error().decode() + "\n" + buf.value.decode(errors="replace"))
    sv_jit_check.last_log = buf.value.decode(errors="replace")  # ptxas register / spill report
    return cnt.value


def sv_jit_stats():
    """Kernels compiled, compiles failed, passes launched on them, compile ms,
    passes built from a deferred basis state, passes with direct loads/stores."""
    L = lib()
    f = L.sv_jit_stats
    f.argtypes = [ctypes.c_void_p] * 4
    f.restype = ctypes.c_int
    c, fl, ln = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(f(ctypes.byref(c), ctypes.byref(fl), ctypes.byref(ln), ctypes.byref(ms)))
    fi = ctypes.c_uint64()
    g = L.sv_jit_fills
    g.argtypes = [ctypes.c_void_p]
    g.restype = ctypes.c_int
    _check(g(ctypes.byref(fi)))
    dl, ds = ctypes.c_uint64(), ctypes.c_uint64()
    d = L.sv_jit_direct
    d.argtypes = [ctypes.c_void_p] * 2
    d.restype = ctypes.c_int
    _check(d(ctypes.byref(dl), ctypes.byref(ds)))
    return {"compiled": c.value, "failed": fl.value, "launched": ln.value, "compile_ms": ms.value,
            "filled": fi.value, "direct_load": dl.value, "direct_store": ds.value}


def sv_jit_wait():
    """Returns at once: pass compiles finish inside the apply that starts them."""
    _check(lib().sv_jit_wait())


def sv_qcrank_reconstruct(h, a, d, shots, seed):
    """QCrank read-out of the state (shots drawn as sv_sample draws them,
    decoded on the device).  Returns (pixels [2^a, d], counts [2^a])."""
    pix = np.empty((1 << a, d), dtype=np.float64)
    counts = np.empty(1 << a, dtype=np.uint64)
    _check(lib().sv_qcrank_reconstruct(h, int(a), int(d), int(shots), int(seed), _ptr(pix), _ptr(counts)))
    return pix, counts


def sv_qcrank_decode_device(samples_ptr, shots, a, d, counts_ptr, ones_ptr, pixels_ptr, stream=None):
    """Device buffers (integer addresses): shots uint64 outcomes -> counts
    [2^a] uint64, ones [2^a * d] uint64, pixels [2^a * d] float64."""
    vp = ctypes.c_void_p
    _check(lib().sv_qcrank_decode_device(vp(samples_ptr), int(shots), int(a), int(d), vp(counts_ptr), vp(ones_ptr),
                                         vp(pixels_ptr), vp(stream) if stream else None))


def sv_sample_device(h, shots, seed, dev_out_ptr):
    _check(lib().sv_sample_device(h, int(shots), int(seed), ctypes.c_void_p(dev_out_ptr)))


def sv_measure(h, shots, seed, expz=True):
    """Shots and <Z_i> from one read of the state, to host arrays."""
    n, _ = _n_dtype(h)
    L = lib()
    f = L.sv_measure
    f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    samp = np.empty(int(shots), dtype=np.uint64)
    ez = np.empty(n, dtype=np.float64) if expz else None
    _check(f(h, int(shots), int(seed), _ptr(samp) if shots else None, _ptr(ez) if expz else None))
    return samp, ez


def sv_measure_device(h, shots, seed, dev_samples_ptr, dev_expz_ptr):
    L = lib()
    f = L.sv_measure_device
    f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(h, int(shots), int(seed), ctypes.c_void_p(dev_samples_ptr) if dev_samples_ptr else None,
             ctypes.c_void_p(dev_expz_ptr) if dev_expz_ptr else None))


def sv_feature_count():
    return lib().sv_feature_count()


def sv_pass_times(h, cap=1 << 16, features=False):
    """Recorded pass times (ms) [and features] since the last call."""
    ms = np.empty(cap, dtype=np.float64)
    F = sv_feature_count()
    feat = np.empty((cap, F), dtype=np.float32) if features else None
    cnt = ctypes.c_int()
    _check(lib().sv_pass_times(h, _ptr(ms), _ptr(feat) if features else None, cap, ctypes.byref(cnt)))
    k = min(cnt.value, cap)
    return (ms[:k].copy(), feat[:k].copy()) if features else ms[:k].copy()


def sv_autotune(h, gates, cache_path=None):
    """Fastest plan options for this circuit on h's state (h's amplitudes are
    scratch afterwards); returns (options dict, ms)."""
    L = lib()
    f = L.sv_autotune
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_char_p, ctypes.POINTER(sv_options),
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    g = as_gates(gates)
    o = sv_options()
    ms = ctypes.c_double()
    path = cache_path.encode() if cache_path else None
    _check(f(h, _ptr(g), len(g), path, ctypes.byref(o), ctypes.byref(ms)))
    return {"k_max": o.k_max, "tile_m": o.tile_m, "tensor": o.tensor, "pass_kernel": o.pass_kernel}, ms.value


def sv_sample_uniforms_noalloc(dev_amps, n, dtype, dev_u, shots, dev_out, stream=None):
    """Sampling with caller-owned device buffers and no device allocation
    (see include/sv.h): all pointers are device addresses (ints)."""
    _check(lib().sv_sample_uniforms_noalloc(ctypes.c_void_p(dev_amps), int(n), int(dtype),
                                            ctypes.c_void_p(dev_u), int(shots), ctypes.c_void_p(dev_out),
                                            stream))


def sv_sample_uniforms(h, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(len(u), dtype=np.uint64)
    _check(lib().sv_sample_uniforms(h, _ptr(u), len(u), _ptr(out)))
    return out


# ---- learned cost model ---------------------------------------------------
def _cm_lib():
    L = lib()
    if not getattr(L, "_cm_ready", False):
        vp, i, u64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        P = ctypes.POINTER
        for name, args in {
            "sv_cost_model_train": [vp, vp, i, i, d, u64, ctypes.c_char_p, P(d)],
            "sv_cost_model_save": [ctypes.c_char_p],
            "sv_cost_model_load": [ctypes.c_char_p],
            "sv_cost_model_unload": [],
            "sv_cost_model_loaded": [],
            "sv_cost_model_predict": [vp, i, vp],
            "sv_cost_model_choose": [i, i, vp, ctypes.c_size_t, P(sv_options), P(d)],
            "sv_cost_model_stats": [P(ctypes.c_int64), P(ctypes.c_int64)],
            "sv_mlp_gradient": [vp, vp, vp, i, P(d), vp],
            "sv_mlp_adam": [vp, vp, i, d],
            "sv_mlp_param_count": [],
            "sv_selftest_tc_tf32": [vp, vp, vp, i, i, i, P(i)],
        }.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L._cm_ready = True
    return L


def sv_cost_model_train(feat, ms, epochs=2000, lr=3e-3, seed=0, weights_path=None):
    """Train the cost model on recorded passes; returns the final loss."""
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    ms = np.ascontiguousarray(ms, dtype=np.float64)
    assert feat.shape == (len(ms), sv_feature_count())
    loss = ctypes.c_double()
    path = weights_path.encode() if weights_path else None
    _check(_cm_lib().sv_cost_model_train(_ptr(feat), _ptr(ms), len(ms), int(epochs), float(lr), int(seed),
                                         path, ctypes.byref(loss)))
    return loss.value


def sv_cost_model_save(path):
    _check(_cm_lib().sv_cost_model_save(path.encode()))


def sv_cost_model_load(path):
    _check(_cm_lib().sv_cost_model_load(path.encode()))


def sv_cost_model_unload():
    _check(_cm_lib().sv_cost_model_unload())


def sv_cost_model_loaded():
    return bool(_cm_lib().sv_cost_model_loaded())


def sv_cost_model_predict(feat):
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    out = np.empty(len(feat), dtype=np.float64)
    _check(_cm_lib().sv_cost_model_predict(_ptr(feat), len(feat), _ptr(out)))
    return out


def sv_cost_model_choose(n, dtype, gates):
    """(options dict, predicted ms) the cost-model planner picks for a circuit."""
    g = as_gates(gates)
    o = sv_options()
    ms = ctypes.c_double()
    _check(_cm_lib().sv_cost_model_choose(n, dtype, _ptr(g), len(g), ctypes.byref(o), ctypes.byref(ms)))
    return {"k_max": o.k_max, "tile_m": o.tile_m, "tensor": o.tensor, "pass_kernel": o.pass_kernel}, ms.value


def sv_cost_model_judged(n, dtype, gates):
    L = _cm_lib()
    f = L.sv_cost_model_judged
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(sv_options),
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    g = as_gates(gates)
    o = sv_options()
    ms = ctypes.c_double()
    _check(f(n, dtype, _ptr(g), len(g), ctypes.byref(o), ctypes.byref(ms)))
    return {"k_max": o.k_max, "tile_m": o.tile_m, "tensor": o.tensor, "pass_kernel": o.pass_kernel}, ms.value


def sv_cost_model_stats():
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(_cm_lib().sv_cost_model_stats(ctypes.byref(a), ctypes.byref(b)))
    return {"planned": a.value, "mispredicted": b.value}


def sv_mlp_param_count():
    return _cm_lib().sv_mlp_param_count()


def sv_mlp_gradient(params, x, t):
    params = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    g = np.empty(sv_mlp_param_count(), dtype=np.float32)
    loss = ctypes.c_double()
    _check(_cm_lib().sv_mlp_gradient(_ptr(params), _ptr(x), _ptr(t), len(t), ctypes.byref(loss), _ptr(g)))
    return loss.value, g


def sv_mlp_adam(params, grads, steps, lr):
    p = np.array(params, dtype=np.float32, copy=True)
    g = np.ascontiguousarray(grads, dtype=np.float32)
    _check(_cm_lib().sv_mlp_adam(_ptr(p), _ptr(g), int(steps), float(lr)))
    return p


# ---- batches ----------------------------------------------------------------
def sv_batch_run(circuits, dtype=C64, shots=0, seed=0, expz=True, k_max=0, tile_m=0, stream=None, mux=0):
    """circuits: list of (n, gates).  Returns (samples C x shots uint64 or
    None, expz C x nmax float64 or None)."""
    L = lib()
    if not getattr(L, "_batch_ready", False):
        vp = ctypes.c_void_p
        L.sv_batch_run.argtypes = [ctypes.c_int, vp, vp, vp, vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.POINTER(sv_options), vp, vp, ctypes.c_int, vp]
        L.sv_batch_run.restype = ctypes.c_int
        L._batch_ready = True
    C = len(circuits)
    ns = np.array([n for n, _ in circuits], dtype=np.int32)
    counts = np.array([len(g) for _, g in circuits], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    allg = np.ascontiguousarray(np.concatenate([as_gates(g) for _, g in circuits]) if C else
                                np.zeros(0, GATE_DTYPE))
    if len(allg) == 0:
        allg = np.zeros(1, GATE_DTYPE)
    nmax = int(ns.max())
    samp = np.empty((C, shots), dtype=np.uint64) if shots else None
    ez = np.empty((C, nmax), dtype=np.float64) if expz else None
    o = _opts(k_max, tile_m, mux=mux)
    _check(L.sv_batch_run(C, _ptr(ns), _ptr(offs), _ptr(counts), _ptr(allg), dtype, int(shots), int(seed),
                          ctypes.byref(o), _ptr(samp) if samp is not None else None,
                          _ptr(ez) if ez is not None else None, nmax, stream))
    return samp, ez


def sv_cost_model_last_trials(cap=8):
    """Trials the judge timed for the circuit the cost-model planner saw last:
    dict(predicted_ms, measured_ms, chosen, learned)."""
    L = lib()
    f = L.sv_cost_model_last_trials
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
    f.restype = ctypes.c_int
    pred = np.zeros(cap, np.float64)
    meas = np.zeros(cap, np.float64)
    nt, ch, le = ctypes.c_int(0), ctypes.c_int(-1), ctypes.c_int(0)
    _check(f(_ptr(pred), _ptr(meas), cap, ctypes.byref(nt), ctypes.byref(ch), ctypes.byref(le)))
    k = min(cap, nt.value)
    return {"predicted_ms": pred[:k].tolist(), "measured_ms": meas[:k].tolist(), "chosen": ch.value,
            "learned": bool(le.value)}
