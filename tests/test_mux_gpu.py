"""Multiplexor recognition (uniformly controlled rotations, QCrank, Sec. 3 image encoding and App. D.3)
through the C ABI against the FP64 oracle, which plays every gate.

Pins: the oracle state element by element; for QCrank also the closed-form
state 2^(-a/2) sum_j |j> prod_k (cos(theta_jk/2)|0> + sin(theta_jk/2)|1>)
(P(data_k = 1 | address j) = sin^2(theta_jk / 2)), computed here with numpy.
"""
import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

DT = [S.C64, S.C128]
DTN = {S.C64: "c64", S.C128: "c128"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    oracle.set_threads(8)
    yield


def qcrank_closed_form(a, d, pix):
    th = np.pi * np.asarray(pix, dtype=np.float64)  # (2^a, d)
    amp = np.full((1 << d, 1 << a), 2.0 ** (-a / 2))
    for k in range(d):
        y = (np.arange(1 << d) >> k) & 1
        amp *= np.where(y[:, None] == 1, np.sin(th[:, k] / 2)[None, :], np.cos(th[:, k] / 2)[None, :])
    return amp.reshape(-1).astype(np.complex128)  # index = j + 2^a * y


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("a,d", [(5, 3), (6, 6), (7, 11)])
def test_qcrank_mux_vs_oracle(dtype, a, d):
    pix = np.random.default_rng(100 + a).uniform(0, 1, size=(1 << a, d))
    g = W.qcrank(a, d, pix)
    n = a + d
    info = S.sv_plan_circuit(n, dtype, g, mux=1)
    assert info["mux_ops"] == d
    assert info["mux_passes"] == -(-d // 5)
    got = U.run_gpu(n, g, dtype, mux=1)
    ref = U.run_oracle(n, g)
    U.assert_close(got, ref, dtype, "qcrank a=%d d=%d" % (a, d))
    U.assert_close(got, qcrank_closed_form(a, d, pix), dtype, "closed form")


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("a,d", [(10, 7), (14, 10)])
def test_qcrank_mux_closed_form_large(dtype, a, d):
    """Config-3 sizes (up to a = 14, d = 10, n = 24) with the default
    recognition threshold: a handful of passes instead of 2 d 2^a gate passes."""
    pix = np.random.default_rng(7 + a).uniform(0, 1, size=(1 << a, d))
    g = W.qcrank(a, d, pix)
    n = a + d
    info = S.sv_plan_circuit(n, dtype, g)
    assert info["mux_ops"] == d and info["passes"] <= 2 + -(-d // 5)
    got = U.run_gpu(n, g, dtype)
    U.assert_close(got, qcrank_closed_form(a, d, pix), dtype, "closed form")


def _ladder_mix(seed):
    """Runs of every recognised shape on n = 10 qubits, started from a random
    state: a Y run (RY, X, CX from non-adjacent controls 0, 2, 3, 5, odd CX
    parity at the end) on qubit 7, a D run (RZ, P, Z, X, CX from 1 and 4) on
    qubit 8, gates in between that commute with both (P and RZ on controls, CX
    from a control into qubit 9, H on 6), an H on control 2 that splits the Y
    run, and a CX into a control that ends the D run."""
    rng = np.random.default_rng(seed)
    items = []
    ty, cy = 7, [0, 2, 3, 5]
    td, cd = 8, [1, 4]
    ang = lambda: float(rng.uniform(-np.pi, np.pi))  # noqa: E731

    def y_step():
        r = rng.integers(0, 4)
        if r == 0:
            items.append((W.X, (ty,), ()))
        elif r == 1:
            items.append((W.CX, (int(rng.choice(cy)), ty), ()))
        else:
            items.append((W.RY, (ty,), (ang(),)))

    def d_step():
        r = rng.integers(0, 6)
        if r == 0:
            items.append((W.X, (td,), ()))
        elif r == 1:
            items.append((W.Z, (td,), ()))
        elif r == 2:
            items.append((W.CX, (int(rng.choice(cd)), td), ()))
        elif r == 3:
            items.append((W.P, (td,), (ang(),)))
        else:
            items.append((W.RZ, (td,), (ang(),)))

    def between():
        r = rng.integers(0, 5)
        if r == 0:
            items.append((W.P, (int(rng.choice(cy + cd)),), (ang(),)))
        elif r == 1:
            items.append((W.RZ, (int(rng.choice(cy + cd)),), (ang(),)))
        elif r == 2:
            items.append((W.CX, (int(rng.choice(cy + cd)), 9), ()))
        elif r == 3:
            items.append((W.H, (6,), ()))
        else:
            items.append((W.CZ, (int(rng.choice(cy)), int(rng.choice(cd))), ()))

    for i in range(60):
        y_step()
        d_step()
        if i % 3 == 0:
            between()
        if i == 30:
            items.append((W.H, (2,), ()))  # non-diagonal on a Y control: the Y run ends here
    items.append((W.CX, (td, 4), ()))      # into a D control: the D run ends here
    for i in range(20):
        y_step()
        d_step()
    items.append((W.CX, (5, ty), ()))      # leave an odd CX parity on control 5
    items += [(W.H, (q,), ()) for q in range(10)] + [(W.CX, (q, (q + 1) % 10), ()) for q in range(10)]
    return W.gates_from_list(items)


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_recognised_runs_vs_oracle(dtype, seed):
    n = 10
    g = _ladder_mix(seed)
    on = S.sv_plan_circuit(n, dtype, g, mux=1)
    assert on["mux_ops"] >= 3, on
    assert S.sv_plan_circuit(n, dtype, g, mux=-1)["mux_ops"] == 0
    assert S.sv_plan_circuit(n, dtype, g)["mux_ops"] == 0  # runs below the default threshold
    psi0 = W.random_state(n, 40 + seed)
    ref = U.run_oracle(n, g, psi0)
    U.assert_close(U.run_gpu(n, g, dtype, psi0=psi0, mux=1), ref, dtype, "mux on")
    U.assert_close(U.run_gpu(n, g, dtype, psi0=psi0, mux=-1), ref, dtype, "mux off")


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
def test_mux_with_relabel_and_other_gates(dtype):
    """A QCrank encoder whose address register was permuted by SWAPs (with
    relabelling the multiplexors see physical controls), followed by a QFT on
    the address qubits (tile passes after the multiplexor passes)."""
    a, d = 6, 5
    pix = np.random.default_rng(9).uniform(0, 1, size=(1 << a, d))
    g = np.concatenate([W.gates_from_list([(W.SWAP, (0, 3), ()), (W.SWAP, (1, 7), ())]), W.qcrank(a, d, pix),
                        W.qft(a, swaps=False)])
    n = a + d
    ref = U.run_oracle(n, g)
    for relabel in (0, 1):
        h = S.sv_alloc(n, dtype)
        try:
            S.sv_init_basis(h, 0)
            S.sv_apply_circuit(h, g, relabel=relabel)
            got = S.sv_store_state(h).astype(np.complex128)
        finally:
            S.sv_free(h)
        U.assert_close(got, ref, dtype, "relabel=%d" % relabel)


def test_qcrank_batch_mux_closed_form():
    """Batched QCrank (config-3 shape, a up to 12): <Z> of the data qubits
    equals mean_j cos(pi pixel_jk) and of the address qubits 0, with and
    without recognition."""
    batch = W.qcrank_batch(24, 77, a_range=(6, 12), d_range=(4, 10))
    circuits = [(a + d, W.qcrank(a, d, pix)) for a, d, pix in batch]
    for mux in (0, -1):
        _, ez = S.sv_batch_run(circuits, dtype=S.C64, shots=0, mux=mux)
        for c, (a, d, pix) in enumerate(batch):
            want = np.cos(np.pi * pix).mean(axis=0)
            assert np.abs(ez[c, a:a + d] - want).max() < 1e-5, (mux, c)
            assert np.abs(ez[c, :a]).max() < 1e-5, (mux, c)
