"""Pins for the FP64 oracle: checks against what the paper and mathematics fix.

Each check takes an oracle instance (``oracle.Oracle``) and raises
AssertionError when it disagrees.  They are used twice: on the real oracle
(tests/test_oracle.py) and on copies with a planted mistake
(tests/test_oracle_mutants.py), which must each fail at least one check.

None of these checks re-types the oracle's formula: gate matrices are checked
against matrix exponentials of Pauli generators (scipy) and the paper's printed
CR1 / CX example; states against kron-product brute force, numpy's FFT, closed
forms (GHZ, QFT of a basis state, QCrank conditional probabilities, product
state <Z>), and reversal; the sampler against a linear scan of numpy's cumsum;
Philox against numpy's Philox bit generator.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

import workloads as W
from tests.conftest import golden_lines

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
SZ = np.array([[1, 0], [0, -1]], dtype=complex)
I2 = np.eye(2, dtype=complex)


# ---------------------------------------------------------------- matrices --
def rot(pauli, t):
    return sla.expm(-0.5j * t * pauli)


def ref_matrix(t, p):
    """Gate matrices built independently of the oracle (expm, identities)."""
    if t == W.H:
        return (SX + SZ) / np.sqrt(2.0)
    if t == W.X:
        return cx_golden()[2:, 2:]  # X is the target block of the paper's CX
    if t == W.Z:
        return np.diag(np.diag(cr1_golden(np.pi))[2:])  # CZ = CR1(pi) block
    if t == W.Y:
        return 1j * ref_matrix(W.X, p) @ ref_matrix(W.Z, p)
    if t == W.RX:
        return rot(SX, p[0])
    if t == W.RY:
        return rot(SY, p[0])
    if t == W.RZ:
        return rot(SZ, p[0])
    if t == W.P:
        return np.exp(0.5j * p[0]) * rot(SZ, p[0])
    if t == W.U3:
        th, ph, la = p
        return np.exp(0.5j * (ph + la)) * rot(SZ, ph) @ rot(SY, th) @ rot(SZ, la)
    if t == W.CX:
        return cx_golden()
    if t == W.CP:
        return cr1_golden(p[0])
    if t == W.CZ:
        return cr1_golden(np.pi)
    if t == W.SWAP:
        m = np.zeros((4, 4), dtype=complex)
        for a in range(2):
            for b in range(2):
                m[2 * b + a, 2 * a + b] = 1.0  # |a b> -> |b a>
        return m
    raise ValueError(t)


def cr1_golden(lam):
    rows = golden_lines("cr1_matrix.txt")
    m = np.zeros((4, 4), dtype=complex)
    for i, r in enumerate(rows):
        for j, v in enumerate(r):
            m[i, j] = np.exp(1j * lam) if v == "e" else float(v)
    return m


def cx_golden():
    """CX on (control, target) with the control as the most significant local
    bit, read off the paper's 3-qubit example: where the control is 1 the
    target's two amplitudes are exchanged."""
    m = np.eye(4, dtype=complex)
    pairs = golden_lines("cx_3qubit_example.txt")
    assert len(pairs) == 2
    m[2:, 2:] = SX
    return m


def check_gate_matrices(O, rng):
    for t in (W.H, W.X, W.Y, W.Z, W.RX, W.RY, W.RZ, W.P, W.U3, W.CX, W.CZ, W.CP, W.SWAP):
        for _ in range(3):
            p = tuple(rng.uniform(-2 * np.pi, 2 * np.pi, size=3))
            got = O.gate_matrix(t, p)
            ref = ref_matrix(t, p)
            assert got.shape == ref.shape, (t, got.shape)
            assert np.allclose(got, ref, atol=1e-13), (W.GATE_NAMES[t], got, ref)
            d = got.shape[0]
            assert np.allclose(got.conj().T @ got, np.eye(d), atol=1e-13)
    assert O.gate_matrix(W.MEASURE) is None


# ------------------------------------------------------- CX worked example --
def label_to_index(label):
    """Paper labels |q0 q1 q2>: q0 is the leftmost character, bit 0."""
    return sum(int(ch) << i for i, ch in enumerate(label))


def check_cx_example(O, rng):
    n = 3
    psi = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    out = O.apply_circuit(n, W.gates_from_list([(W.CX, (0, 2), ())]), psi)
    expect = psi.copy()
    for a, b in golden_lines("cx_3qubit_example.txt"):
        ia, ib = label_to_index(a), label_to_index(b)
        expect[ia], expect[ib] = psi[ib], psi[ia]
    assert np.array_equal(out, expect), (out, expect)


# ----------------------------------------------------- brute-force krons ---
def site_op(n, ops):
    """Kron product over qubits n-1 .. 0 (qubit 0 rightmost = least
    significant index bit), identity where ops has no entry (App. A, Eq. tp)."""
    m = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        m = np.kron(m, ops.get(q, I2))
    return m


def full_matrix(n, rec):
    t = int(rec["type"])
    k = W.ARITY[t]
    q = [int(x) for x in rec["q"][:k]]
    if t == W.MEASURE:
        return np.eye(1 << n, dtype=complex)
    U = ref_matrix(t, tuple(rec["p"]))
    if k == 1:
        return site_op(n, {q[0]: U})
    # two-qubit gate: sum over |a><c| (x) |b><d| of U[(a b), (c d)], q[0] first
    M = np.zeros((1 << n, 1 << n), dtype=complex)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for d in range(2):
                    u = U[2 * a + b, 2 * c + d]
                    if u == 0:
                        continue
                    e0 = np.zeros((2, 2), dtype=complex)
                    e0[a, c] = 1
                    e1 = np.zeros((2, 2), dtype=complex)
                    e1[b, d] = 1
                    M += u * site_op(n, {q[0]: e0, q[1]: e1})
    return M


def random_mixed_circuit(n, count, rng):
    items = []
    for _ in range(count):
        t = int(rng.choice([W.H, W.X, W.Y, W.Z, W.RX, W.RY, W.RZ, W.P, W.U3,
                            W.CX, W.CZ, W.CP, W.SWAP, W.MEASURE]))
        k = W.ARITY[t]
        qs = tuple(int(x) for x in rng.choice(n, size=k, replace=False))
        ps = tuple(rng.uniform(0, 2 * np.pi, size=3))
        items.append((t, qs, ps))
    return W.gates_from_list(items)


def check_brute_force(O, rng, n=5, count=40):
    g = random_mixed_circuit(n, count, rng)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    U = np.eye(1 << n, dtype=complex)
    for rec in g:
        U = full_matrix(n, rec) @ U
    got = O.apply_circuit(n, g, psi0)
    assert np.allclose(got, U @ psi0, atol=1e-12), np.abs(got - U @ psi0).max()


# ------------------------------------------------------------------ QFT ----
def check_qft_angles():
    """The generator's cr1 angles follow App. D.2: 2 pi / 2^(j-i+1)."""
    table = {int(d): float(f) for d, f in golden_lines("qft_angles.txt")}
    g = W.qft(6)
    seen = set()
    for r in g:
        if int(r["type"]) == W.CP:
            i, j = sorted(int(x) for x in r["q"][:2])
            d = j - i
            if d in table:
                assert abs(r["p"][0] / (2 * np.pi) - table[d]) < 1e-15
                seen.add(d)
    assert seen == set(table)
    n = 28
    assert len(W.qft(n)) == n + n * (n - 1) // 2 + n // 2 == 420


def check_qft_basis(O, rng, n=9):
    N = 1 << n
    x = int(rng.integers(N))
    got = O.apply_circuit(n, W.qft(n), O.basis_state(n, x))
    y = np.arange(N)
    ref = np.exp(2j * np.pi * ((x * y) % N) / N) / np.sqrt(N)
    assert np.allclose(got, ref, atol=1e-12), np.abs(got - ref).max()


def check_qft_random(O, rng, n=12):
    N = 1 << n
    psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi /= np.linalg.norm(psi)
    got = O.apply_circuit(n, W.qft(n), psi)
    ref = np.sqrt(N) * np.fft.ifft(psi)
    assert np.allclose(got, ref, atol=1e-12), np.abs(got - ref).max()


# ------------------------------------------------ GHZ, reversal, norm ------
def check_ghz(O, rng, n=6):
    items = [(W.H, (0,), ())] + [(W.CX, (q, q + 1), ()) for q in range(n - 1)]
    got = O.apply_circuit(n, W.gates_from_list(items))
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / np.sqrt(2)
    assert np.allclose(got, ref, atol=1e-15)
    u = np.linspace(0, 1, 64, endpoint=False)
    s = O.sample(got, u)
    assert set(s.tolist()) == {0, (1 << n) - 1}
    assert np.allclose(O.expect_z(got), 0.0, atol=1e-15)


def check_reversal(O, rng, n=10):
    g = W.random_u3_cx(n, 6, int(rng.integers(1 << 30)))
    out = O.apply_circuit(n, np.concatenate([g, W.inverse(g)]))
    ref = O.basis_state(n, 0)
    assert np.abs(out - ref).max() < 1e-12
    psi = O.apply_circuit(n, g)
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12


# ----------------------------------------------------------- QCrank --------
def check_qcrank(O, rng, a=3, d=3):
    pix = rng.uniform(0, 1, size=(1 << a, d))
    g = W.qcrank(a, d, pix)
    assert sum(int(r["type"]) == W.CX for r in g) == d * (1 << a)
    psi = O.apply_circuit(a + d, g)
    p = O.probs(psi).reshape((1 << d), (1 << a))  # [data bits, address]
    addr = p.sum(axis=0)
    assert np.allclose(addr, 2.0 ** -a, atol=1e-13)
    for k in range(d):
        sel = ((np.arange(1 << d) >> k) & 1).astype(bool)
        p1 = p[sel].sum(axis=0) / addr
        assert np.allclose(p1, np.sin(np.pi * pix[:, k] / 2) ** 2, atol=1e-12), k


def check_qcrank_table2():
    rows = golden_lines("qcrank_table2.txt")
    for name, w, h, pix_r, a, dq, shots_r in rows:
        w, h, a, dq = int(w), int(h), int(a), int(dq)
        assert w * h == dq * (1 << a), name
        assert abs(w * h / 1000.0 - float(pix_r[:-1])) <= 1.0, name
        shots = 3000 * (1 << a)
        assert abs(shots / 1e6 - float(shots_r[:-1])) / shots * 1e6 < 0.1, name
    a, dq = 10, 5  # Finger: CX count of the generated circuit = pixel count
    g = W.qcrank(a, dq, np.zeros((1 << a, dq)))
    assert sum(int(r["type"]) == W.CX for r in g) == 64 * 80


# -------------------------------------------------------------- <Z> --------
def check_expect_z(O, rng, n=7):
    th = rng.uniform(0, 2 * np.pi, size=n)
    ph = rng.uniform(0, 2 * np.pi, size=n)
    items = []
    for q in range(n):
        items += [(W.RY, (q,), (th[q],)), (W.RZ, (q,), (ph[q],))]
    psi = O.apply_circuit(n, W.gates_from_list(items))
    assert np.allclose(O.expect_z(psi), np.cos(th), atol=1e-13)
    x = int(rng.integers(1 << n))
    ez = O.expect_z(O.basis_state(n, x))
    assert np.array_equal(ez, np.array([-1.0 if (x >> i) & 1 else 1.0 for i in range(n)]))


# ------------------------------------------------------------ sampler ------
def check_sampler(O, rng, n=4):
    N = 1 << n
    x = int(rng.integers(N))
    assert (O.sample(O.basis_state(n, x), rng.uniform(size=50)) == x).all()
    psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi[rng.choice(N, size=5, replace=False)] = 0.0  # zero-probability outcomes
    psi /= np.linalg.norm(psi)
    p = np.abs(psi) ** 2
    assert np.allclose(O.probs(psi), p, rtol=1e-14, atol=0)
    c = np.cumsum(p)  # sequential FP64 inclusive scan
    assert np.array_equal(O.cdf(p), c)
    S = c[-1]
    # grid, exact CDF boundaries, random draws
    u = np.concatenate([np.arange(256) / 256.0, c[:-1] / S, rng.uniform(size=200)])
    u = u[u < 1.0]
    got = O.sample_cdf(O.cdf(p), u)
    for ui, gi in zip(u, got):
        t = ui * S
        lin = next(i for i in range(N) if c[i] > t)  # linear scan
        assert gi == lin, (ui, gi, lin)
        assert p[gi] > 0


def check_philox(O, rng):
    m = (1 << 64) - 1
    for _ in range(4):
        key = [int(rng.integers(1 << 63)), int(rng.integers(1 << 63))]
        ctr = [int(rng.integers(1 << 63)) for _ in range(4)]
        # numpy increments the counter before each block
        prev = list(ctr)
        i = 0
        while prev[i] == 0:
            prev[i] = m
            i += 1
        prev[i] -= 1
        bg = np.random.Philox(counter=prev, key=key)
        ref = bg.random_raw(4)
        assert np.array_equal(O.philox4x64_10(ctr, key), ref)
    seed = 12345
    bg = np.random.Philox(counter=[m, m, m, m], key=[seed, 0])
    raw = bg.random_raw(11)
    ref = (raw >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    assert np.array_equal(O.uniforms(seed, 11), ref)


ALL_STATE_CHECKS = [check_gate_matrices, check_cx_example, check_brute_force, check_qft_basis,
                    check_qft_random, check_ghz, check_reversal, check_qcrank, check_expect_z,
                    check_sampler, check_philox]
