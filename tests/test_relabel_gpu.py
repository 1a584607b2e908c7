"""SWAP gates as qubit relabelling: every read-out of a relabelled state
(amplitudes, probabilities, <Z>, shots) equals the oracle's for the logical
circuit, later circuits see the logical qubits, and materialising restores
the physical order."""
import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U
from tests.oracle_pins import random_mixed_circuit

pytestmark = pytest.mark.gpu

DT = [S.C64, S.C128]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    oracle.set_threads(8)
    yield


def swap_heavy(n, seed):
    rng = np.random.default_rng(seed)
    L = []
    for layer in range(6):
        for q in range(n):
            L.append((W.U3, (q,), tuple(rng.uniform(0, 6, 3))))
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            L.append((W.SWAP, (int(perm[i]), int(perm[i + 1])), ()))
        L.append((W.CX, (int(perm[0]), int(perm[-1])), ()))
        L.append((W.CP, (int(perm[1]), int(perm[2])), (0.7,)))
    return W.gates_from_list(L)


@pytest.mark.parametrize("dtype", DT, ids=["c64", "c128"])
@pytest.mark.parametrize("planner", [S.PLAN_GREEDY, S.PLAN_PLAIN])
@pytest.mark.parametrize("kind", ["swap_heavy", "qft", "mixed"])
def test_relabelled_readouts(dtype, planner, kind):
    n = 14
    g = {"swap_heavy": lambda: swap_heavy(n, 3), "qft": lambda: W.qft(n),
         "mixed": lambda: random_mixed_circuit(n, 150, np.random.default_rng(9))}[kind]()
    psi0 = W.random_state(n, 11)
    ref = U.run_oracle(n, g, psi0)
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_load_state(h, psi0)
        S.sv_apply_circuit(h, g, planner=planner, relabel=1)
        if kind != "mixed":
            assert S.sv_qubit_map(h) != list(range(n))
        got = S.sv_store_state(h).astype(np.complex128)
        U.assert_close(got, ref, dtype, "%s relabelled" % kind)
        p = S.sv_probs(h)
        assert np.abs(p - np.abs(ref) ** 2).max() < (1e-6 if dtype == S.C64 else 1e-12)
        ez = S.sv_expect_z(h)
        ez_ref = oracle.expect_z(ref)
        assert np.abs(ez - ez_ref).max() < (1e-5 if dtype == S.C64 else 1e-11)
        # shots follow the oracle's rule over the LOGICAL index: outcome =
        # min{x : C_x > u C_{N-1}}.  complex128 end to end against the
        # oracle's own probabilities; complex64 against the oracle's CDF of
        # the GPU's probabilities (its amplitudes differ in the 7th digit)
        c_ref = oracle.cdf(np.abs(ref) ** 2 if dtype == S.C128 else p)
        u = np.random.default_rng(5).random(2000)
        shots = S.sv_sample_uniforms(h, u).astype(np.int64)
        U.compare_samples(shots, u, c_ref, U.BAND)
        # Philox shots (sv_sample and the one-read sv_measure) follow the same rule
        us = oracle.uniforms(77, 3000)
        U.compare_samples(S.sv_sample(h, 3000, 77).astype(np.int64), us, c_ref, U.BAND)
        sm, ezm = S.sv_measure(h, 3000, 77)
        U.compare_samples(sm.astype(np.int64), us, c_ref, U.BAND)
        assert np.abs(ezm - ez_ref).max() < (1e-5 if dtype == S.C64 else 1e-11)
        # a second circuit acts on the logical qubits
        g2 = W.random_u3_cx(n, 2, 44)
        S.sv_apply_circuit(h, g2, planner=planner, relabel=1)
        ref2 = U.run_oracle(n, g2, ref)
        U.assert_close(S.sv_store_state(h).astype(np.complex128), ref2, dtype, "second circuit")
        # materialise: physical order becomes logical order
        S.sv_materialize(h)
        assert S.sv_qubit_map(h) == list(range(n))
        U.assert_close(S.sv_store_state(h).astype(np.complex128), ref2, dtype, "materialised")
    finally:
        S.sv_free(h)


def test_relabel_off_moves_data():
    n = 10
    g = W.gates_from_list([(W.H, (0,), ()), (W.SWAP, (0, 7), ())])
    h = S.sv_alloc(n, S.C64)
    try:
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, g)
        assert S.sv_qubit_map(h) == list(range(n))
        S.sv_apply_circuit(h, g, relabel=1)
        m = S.sv_qubit_map(h)
        assert m[0] == 7 and m[7] == 0
        S.sv_init_basis(h, 0)
        assert S.sv_qubit_map(h) == list(range(n))
    finally:
        S.sv_free(h)
