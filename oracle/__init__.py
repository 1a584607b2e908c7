"""FP64 CPU oracle for the state-vector simulator (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference arm may import this package.  The product (the CUDA library and its
binding) never does; the two share no code.  The simulator itself is plain C
(``sv_oracle.c``) compiled with gcc; this module compiles it on demand and wraps
it with ctypes.  ``mlp_ref`` holds the FP64 reference of the cost-model MLP.

Conventions are listed in the header of ``sv_oracle.c``; the paper passages
each function follows are cited there (App. A Eqs. "hilbert", "tp", "cx";
App. D.2 Eq. "cr1"; Sec. 3 shot sampling).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_LIB = os.path.join(_HERE, "libsv_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load(path):
    L = ctypes.CDLL(path)
    vp, i64, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64
    L.or_apply_circuit.argtypes = [ctypes.c_int, vp, vp, i64]
    L.or_apply_circuit.restype = i64
    L.or_init_basis.argtypes = [ctypes.c_int, vp, u64]
    L.or_probs.argtypes = [ctypes.c_int, vp, vp]
    L.or_cdf.argtypes = [ctypes.c_int, vp, vp]
    L.or_sample_cdf.argtypes = [ctypes.c_int, vp, vp, i64, vp]
    L.or_expect_z.argtypes = [ctypes.c_int, vp, vp]
    L.or_philox4x64_10.argtypes = [vp, vp, vp]
    L.or_uniforms.argtypes = [u64, i64, vp]
    L.or_gate_matrix.argtypes = [ctypes.c_uint32, vp, vp]
    L.or_gate_matrix.restype = ctypes.c_int
    L.or_set_threads.argtypes = [ctypes.c_int]
    L.or_get_threads.restype = ctypes.c_int
    L.or_gate_struct_size.restype = ctypes.c_int
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """The oracle's functions bound to one compiled copy of ``sv_oracle.c``."""

    def __init__(self, path):
        self.L = _load(path)

    def set_threads(self, t):
        self.L.or_set_threads(int(t))

    def get_threads(self):
        return self.L.or_get_threads()

    def gate_matrix(self, gtype, params=(0.0, 0.0, 0.0)):
        p = np.zeros(3, dtype=np.float64)
        p[: len(params)] = params
        out = np.zeros(32, dtype=np.float64)
        k = self.L.or_gate_matrix(int(gtype), _ptr(p), _ptr(out))
        if k < 0:
            raise ValueError("unknown gate type %d" % gtype)
        if k == 0:
            return None
        d = 1 << k
        return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()

    def basis_state(self, n, x=0):
        psi = np.empty(1 << n, dtype=np.complex128)
        self.L.or_init_basis(n, _ptr(psi), int(x))
        return psi

    def apply_circuit(self, n, gates, psi=None):
        """Apply the gate list one gate at a time; returns a new complex128 state."""
        if psi is None:
            psi = self.basis_state(n, 0)
        else:
            psi = np.array(psi, dtype=np.complex128, copy=True)
            assert psi.shape == (1 << n,)
        g = np.ascontiguousarray(gates)
        assert g.dtype.itemsize == self.L.or_gate_struct_size()
        rc = self.L.or_apply_circuit(n, _ptr(psi), _ptr(g), len(g))
        if rc != 0:
            raise ValueError("invalid gate record at index %d" % (-rc - 1))
        return psi

    def apply_inplace(self, n, gates, psi):
        """The same as apply_circuit, in place on psi (complex128, C-contiguous,
        length 2^n): no copy of the state, for states of tens of GiB."""
        assert psi.dtype == np.complex128 and psi.flags["C_CONTIGUOUS"] and psi.shape == (1 << n,)
        g = np.ascontiguousarray(gates)
        assert g.dtype.itemsize == self.L.or_gate_struct_size()
        rc = self.L.or_apply_circuit(n, _ptr(psi), _ptr(g), len(g))
        if rc != 0:
            raise ValueError("invalid gate record at index %d" % (-rc - 1))
        return psi

    def probs(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        n = int(np.log2(len(psi)))
        p = np.empty(len(psi), dtype=np.float64)
        self.L.or_probs(n, _ptr(psi), _ptr(p))
        return p

    def cdf(self, p):
        p = np.ascontiguousarray(p, dtype=np.float64)
        n = int(np.log2(len(p)))
        c = np.empty_like(p)
        self.L.or_cdf(n, _ptr(p), _ptr(c))
        return c

    def sample_cdf(self, c, u):
        c = np.ascontiguousarray(c, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        n = int(np.log2(len(c)))
        out = np.empty(len(u), dtype=np.uint64)
        self.L.or_sample_cdf(n, _ptr(c), _ptr(u), len(u), _ptr(out))
        return out

    def sample(self, psi, u):
        return self.sample_cdf(self.cdf(self.probs(psi)), u)

    def expect_z(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        n = int(np.log2(len(psi)))
        out = np.empty(n, dtype=np.float64)
        self.L.or_expect_z(n, _ptr(psi), _ptr(out))
        return out

    def philox4x64_10(self, ctr, key):
        c = np.ascontiguousarray(ctr, dtype=np.uint64)
        k = np.ascontiguousarray(key, dtype=np.uint64)
        out = np.empty(4, dtype=np.uint64)
        self.L.or_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
        return out

    def uniforms(self, seed, shots):
        u = np.empty(int(shots), dtype=np.float64)
        self.L.or_uniforms(int(seed), int(shots), _ptr(u))
        return u


def default():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = Oracle(_LIB)
    return _lib


def compile_variant(src_text, out_path):
    """Compile a modified copy of the oracle source (used by the tests that
    plant mistakes in the oracle to show that the pins catch them)."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-o", out_path, c_path, "-lm"])
    return Oracle(out_path)


def source_text():
    with open(_SRC) as f:
        return f.read()


def set_threads(t): default().set_threads(t)
def get_threads(): return default().get_threads()
def gate_matrix(gtype, params=(0.0, 0.0, 0.0)): return default().gate_matrix(gtype, params)
def basis_state(n, x=0): return default().basis_state(n, x)
def apply_circuit(n, gates, psi=None): return default().apply_circuit(n, gates, psi)
def apply_inplace(n, gates, psi): return default().apply_inplace(n, gates, psi)
def probs(psi): return default().probs(psi)
def cdf(p): return default().cdf(p)
def sample_cdf(c, u): return default().sample_cdf(c, u)
def sample(psi, u): return default().sample(psi, u)
def expect_z(psi): return default().expect_z(psi)
def philox4x64_10(ctr, key): return default().philox4x64_10(ctr, key)
def uniforms(seed, shots): return default().uniforms(seed, shots)


def fidelity(a, b):
    """|<a|b>|^2 / (<a|a><b|b>) in FP64."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ov = np.vdot(a, b)
    return float(abs(ov) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def max_abs_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.complex128) - np.asarray(b, np.complex128))))
