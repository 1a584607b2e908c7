"""Seeded synthetic workloads for the state-vector simulator.

This module builds INPUTS only: gate lists in the boundary's record format and
seeded initial states.  It holds none of the simulation arithmetic, so both the
FP64 oracle (``oracle/``) and the CUDA library consume exactly the same inputs
without sharing any code with each other.

Gate record (48 bytes, little endian), the boundary's input format:
    uint32 type; uint32 nq; uint32 q[3]; (4 pad bytes); double p[3]
For two-qubit gates q[0] is the control (CX, CP) and q[1] the target.  This is
the per-gate (type, control, target, params) tuple of the paper's circuit
tensor (Sec. 2.1 "Circuit encoding", App. D.1 ``gate_type``/``gate_param``).

Workload shapes follow the paper's benchmark families: random CX-block
circuits (Sec. 3, App. D.1 Alg. 1), QFT (App. D.2) and QCrank image encoding
(Sec. 3, App. D.3, Table 2), plus a hardware-efficient variational ansatz.
"""
from __future__ import annotations

import numpy as np

# Gate type codes of the boundary's input format.  The alphabet is the paper's
# one-hot gate set h, ry, rz, cx, measure (App. D.1, Eq. "onehot") plus cr1
# (App. D.2, Eq. "cr1" = CP here) and the rotations the configs use (U3, RX).
H, X, Y, Z, RX, RY, RZ, P, U3, CX, CZ, CP, SWAP, MEASURE = range(14)
GATE_NAMES = ["h", "x", "y", "z", "rx", "ry", "rz", "p", "u3", "cx", "cz", "cp",
              "swap", "measure"]
ARITY = {H: 1, X: 1, Y: 1, Z: 1, RX: 1, RY: 1, RZ: 1, P: 1, U3: 1,
         CX: 2, CZ: 2, CP: 2, SWAP: 2, MEASURE: 1}
NPARAMS = {RX: 1, RY: 1, RZ: 1, P: 1, U3: 3, CP: 1}

GATE_DTYPE = np.dtype([("type", "<u4"), ("nq", "<u4"), ("q", "<u4", (3,)),
                       ("pad", "<u4"), ("p", "<f8", (3,))])
assert GATE_DTYPE.itemsize == 48

TWO_PI = 2.0 * np.pi


def gates_from_list(items):
    """[(type, (q...), (p...)), ...] -> structured gate array."""
    g = np.zeros(len(items), dtype=GATE_DTYPE)
    for i, (t, qs, ps) in enumerate(items):
        g[i]["type"] = t
        g[i]["nq"] = len(qs)
        g[i]["q"][: len(qs)] = qs
        g[i]["p"][: len(ps)] = ps
    return g


class _Builder:
    """Append-only gate list with numpy-backed growth."""

    def __init__(self, cap=1024):
        self.g = np.zeros(cap, dtype=GATE_DTYPE)
        self.n = 0

    def add(self, t, qs, ps=()):
        if self.n == len(self.g):
            self.g = np.concatenate([self.g, np.zeros(len(self.g), GATE_DTYPE)])
        r = self.g[self.n]
        r["type"] = t
        r["nq"] = len(qs)
        r["q"][: len(qs)] = qs
        r["p"][: len(ps)] = ps
        self.n += 1

    def done(self):
        return self.g[: self.n].copy()


# --------------------------------------------------------------------------
# Random CX-block circuits (Sec. 3 "random non-Clifford unitaries", App. D.1).
# The configurations use a U3 on every qubit followed by CX on a random
# disjoint pairing; the pairing is a seeded permutation split into
# consecutive (control, target) pairs, one qubit left out when n is odd.
# --------------------------------------------------------------------------
def random_u3_cx(n, layers, seed):
    rng = np.random.default_rng(seed)
    b = _Builder(layers * (n + n // 2))
    for _ in range(layers):
        ang = rng.uniform(0.0, TWO_PI, size=(n, 3))
        for q in range(n):
            b.add(U3, (q,), tuple(ang[q]))
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            b.add(CX, (int(perm[i]), int(perm[i + 1])))
    return b.done()


def random_cx_blocks(n, blocks, seed):
    """The paper's Alg. 1 shape: per block a random ordered pair (q_c, q_t),
    q_t != q_c, sampled with replacement; Ry/Rz rotations with
    theta ~ U[0, 2pi] on both qubits, then CX(q_c, q_t)."""
    rng = np.random.default_rng(seed)
    b = _Builder(blocks * 5)
    for _ in range(blocks):
        qc = int(rng.integers(n))
        qt = int(rng.integers(n - 1))
        qt = qt + 1 if qt >= qc else qt
        th = rng.uniform(0.0, TWO_PI, size=4)
        b.add(RY, (qc,), (th[0],))
        b.add(RZ, (qc,), (th[1],))
        b.add(RY, (qt,), (th[2],))
        b.add(RZ, (qt,), (th[3],))
        b.add(CX, (qc, qt))
    return b.done()


# --------------------------------------------------------------------------
# QFT (App. D.2): Hadamard on each qubit followed by cr1 rotations to the
# remaining qubits with angle 2*pi/2^(d+1) = pi/2^d at qubit distance d, then
# the final swaps that put the output in natural bit order.  With qubit q =
# bit q of the amplitude index the first H goes on the most significant qubit.
# --------------------------------------------------------------------------
def qft(n, swaps=True):
    b = _Builder(n * (n + 1) // 2 + n // 2)
    for j in range(n - 1, -1, -1):
        b.add(H, (j,))
        for k in range(j - 1, -1, -1):
            b.add(CP, (k, j), (np.pi / float(2 ** (j - k)),))
    if swaps:
        for i in range(n // 2):
            b.add(SWAP, (i, n - 1 - i))
    return b.done()


# --------------------------------------------------------------------------
# QCrank image encoding (Sec. 3, App. D.3, Table 2).  Address qubits
# q0..q_{a-1} get H; data qubit k (= q_{a+k}) gets a uniformly controlled
# RY(theta_{j,k}), theta = pi * pixel, decomposed into 2^a alternating RY / CX
# steps (Mottonen et al. 2004): step i applies RY(theta'_i) then CX from the
# address bit that flips between Gray codes g(i) and g(i+1) (cyclically).
# For address j the applied angle is sum_i (-1)^popcount(j & g(i)) theta'_i,
# so theta' = 2^-a M^T theta with M[j, i] = (-1)^popcount(j & g(i)).
# --------------------------------------------------------------------------
def _gray(i):
    return i ^ (i >> 1)


def qcrank_angles(a, theta):
    """Decomposition angles theta' (shape (2^a, d)) for address angles theta.

    theta'_i = 2^-a sum_j (-1)^popcount(j & g(i)) theta_j = 2^-a W[g(i)], with
    W the Walsh-Hadamard transform of theta along the address axis."""
    L = 1 << a
    w = np.array(theta, dtype=np.float64, copy=True).reshape(L, -1)
    h = 1
    while h < L:  # in-place fast Walsh-Hadamard transform
        w = w.reshape(L // (2 * h), 2, h, -1)
        s = w[:, 0] + w[:, 1]
        d = w[:, 0] - w[:, 1]
        w = np.stack([s, d], axis=1).reshape(L, -1)
        h *= 2
    g = np.array([_gray(i) for i in range(L)], dtype=np.int64)
    return w[g] / float(L)


def qcrank(a, d, pixels):
    """Gate list for a QCrank circuit with pixels of shape (2^a, d) in [0,1]."""
    L = 1 << a
    assert pixels.shape == (L, d)
    theta = np.pi * np.asarray(pixels, dtype=np.float64)
    tp = qcrank_angles(a, theta)
    ctrl = np.array([(_gray(i) ^ _gray((i + 1) % L)).bit_length() - 1 for i in range(L)], dtype=np.uint32)
    # H on every address qubit, then for each data qubit t = a + k the ladder
    # RY(theta'_i) on t, CX(ctrl_i, t) for i = 0 .. L-1 (filled column-wise)
    g = np.zeros(a + 2 * d * L, dtype=GATE_DTYPE)
    g["type"][:a] = H
    g["nq"][:a] = 1
    g["q"][:a, 0] = np.arange(a, dtype=np.uint32)
    lad = g[a:].reshape(d, L, 2)
    t = (a + np.arange(d, dtype=np.uint32))[:, None]
    lad["type"][:, :, 0] = RY
    lad["nq"][:, :, 0] = 1
    lad["q"][:, :, 0, 0] = t
    lad["p"][:, :, 0, 0] = tp.T
    lad["type"][:, :, 1] = CX
    lad["nq"][:, :, 1] = 2
    lad["q"][:, :, 1, 0] = ctrl[None, :]
    lad["q"][:, :, 1, 1] = t
    return g


def qcrank_batch(circuits, seed, a_range=(8, 14), d_range=(4, 10)):
    """Uneven QCrank batch: a ~ U{a_range}, d ~ U{d_range}, pixels ~ U[0,1]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(circuits):
        a = int(rng.integers(a_range[0], a_range[1] + 1))
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        pix = rng.uniform(0.0, 1.0, size=(1 << a, d))
        out.append((a, d, pix))
    return out


# --------------------------------------------------------------------------
# Hardware-efficient ansatz: per layer RY(theta_q) then RZ(phi_q) on each
# qubit q = 0..n-1, then the CX ring CX(q, q+1 mod n).
# --------------------------------------------------------------------------
def hea(n, layers, angles):
    """angles: (layers, n, 2) array of (theta, phi)."""
    b = _Builder(layers * 3 * n)
    for l in range(layers):
        for q in range(n):
            b.add(RY, (q,), (float(angles[l, q, 0]),))
            b.add(RZ, (q,), (float(angles[l, q, 1]),))
        for q in range(n):
            b.add(CX, (q, (q + 1) % n))
    return b.done()


def hea_params(sets, n, layers, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, TWO_PI, size=(sets, layers, n, 2))


# --------------------------------------------------------------------------
# Inverse circuit: inverse gates in reverse order (used by reversal tests).
# U3(t, f, l)^dagger = U3(-t, -l, -f).
# --------------------------------------------------------------------------
def inverse(gates):
    inv = gates[::-1].copy()
    for r in inv:
        t = int(r["type"])
        if t in (RX, RY, RZ, P, CP):
            r["p"][0] = -r["p"][0]
        elif t == U3:
            th, ph, la = r["p"]
            r["p"][0], r["p"][1], r["p"][2] = -th, -la, -ph
        elif t == Y or t in (H, X, Z, CX, CZ, SWAP, MEASURE):
            pass
        else:
            raise ValueError(t)
    return inv


# --------------------------------------------------------------------------
# Seeded initial states and uniforms.
# --------------------------------------------------------------------------
def random_basis_index(n, seed):
    return int(np.random.default_rng(seed).integers(0, 1 << n))


def random_state(n, seed):
    """Complex Gaussian amplitudes normalised in FP64 (complex128, length 2^n)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    v /= np.sqrt(np.vdot(v, v).real)
    return v


def uniforms(shots, seed):
    """Oracle-supplied uniforms in [0,1) with 53-bit resolution."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 1 << 53, size=shots, dtype=np.uint64).astype(np.float64)
            * (2.0 ** -53))


# Seeds per configuration: 1000 + configuration number.
SEED = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005}


def config1():
    """n=12, 20 layers of U3 on every qubit + CX on a disjoint pairing."""
    return 12, random_u3_cx(12, 20, SEED[1])


def config2(n=28):
    """QFT with final swaps (n=28: 28 H + 378 CP + 14 SWAP = 420 gates)."""
    return n, qft(n)


def config4(n=32, layers=60):
    return n, random_u3_cx(n, layers, SEED[4])


def config5(n=20, layers=8, sets=4096):
    return n, hea_params(sets, n, layers, SEED[5])
