"""Repeated applies of one circuit reuse the handle's cached plan: the state
after k applies equals the oracle's circuit played k times, with qubit
relabelling (the map a cached plan leaves behind), with another circuit in
between, and after the cache has evicted the entry."""
import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    yield


def _logical(h):
    S.sv_materialize(h)
    return S.sv_store_state(h).astype(np.complex128)


@pytest.mark.parametrize("relabel", [0, 1])
def test_repeated_applies(relabel):
    n = 14
    g = W.qft(n)  # with swaps: relabelling changes the map every time
    g2 = W.random_u3_cx(n, 2, 8)
    psi0 = W.random_state(n, 9)
    ref = psi0
    h = S.sv_alloc(n, S.C64)
    try:
        S.sv_load_state(h, psi0)
        for k in range(3):
            S.sv_apply_circuit(h, g, relabel=relabel, jit=1)
            ref = oracle.apply_circuit(n, g, ref)
        S.sv_apply_circuit(h, g2, relabel=relabel)
        ref = oracle.apply_circuit(n, g2, ref)
        S.sv_apply_circuit(h, g, relabel=relabel, jit=1)
        ref = oracle.apply_circuit(n, g, ref)
        # evict: more distinct circuits than the cache holds, then g again
        for s in range(10):
            gs = W.random_u3_cx(n, 1, 100 + s)
            S.sv_apply_circuit(h, gs, relabel=relabel)
            ref = oracle.apply_circuit(n, gs, ref)
        S.sv_apply_circuit(h, g, relabel=relabel, jit=1)
        ref = oracle.apply_circuit(n, g, ref)
        U.assert_close(_logical(h), ref, S.C64, "relabel=%d" % relabel)
    finally:
        S.sv_free(h)


def test_options_are_part_of_the_key():
    n = 12
    g = W.random_u3_cx(n, 3, 4)
    ref = U.run_oracle(n, g)
    h = S.sv_alloc(n, S.C64)
    try:
        for opts in ({}, {"k_max": 2}, {"tile_m": 9}, {"pass_kernel": 1}, {"k_max": 2}, {}):
            S.sv_init_basis(h, 0)
            S.sv_apply_circuit(h, g, **opts)
            U.assert_close(S.sv_store_state(h).astype(np.complex128), ref, S.C64, str(opts))
        # a phase-dropping threshold changes the circuit
        gq = W.qft(n)
        x = 0b101101110101
        exact = U.run_oracle(n, gq, basis=x)
        S.sv_init_basis(h, x)
        S.sv_apply_circuit(h, gq, drop_phase_below=0.5)
        approx = S.sv_store_state(h).astype(np.complex128)
        S.sv_init_basis(h, x)
        S.sv_apply_circuit(h, gq)
        U.assert_close(S.sv_store_state(h).astype(np.complex128), exact, S.C64, "exact after approximate")
        assert oracle.fidelity(approx, exact) < 1 - 1e-4
    finally:
        S.sv_free(h)


def test_cache_ignores_unused_fields_and_compares_records():
    """Records that differ only in entries the library ignores (unused qubits
    and parameters) share a cached plan; records that differ in a used
    parameter do not, even right after the first circuit's plan was cached."""
    n = 12
    g = W.random_u3_cx(n, 3, 21)
    noisy = g.copy()
    rng = np.random.default_rng(4)
    one_q = noisy["nq"] == 1
    noisy["q"][one_q, 1] = rng.integers(0, 1 << 30, size=int(one_q.sum()))
    noisy["q"][:, 2] = rng.integers(0, 1 << 30, size=len(noisy))
    cx = noisy["type"] == W.CX
    noisy["p"][cx] = rng.standard_normal((int(cx.sum()), 3))
    other = g.copy()
    u3 = np.nonzero(g["type"] == W.U3)[0]
    other["p"][u3[5], 1] += 0.25  # one used parameter changed
    psi0 = W.random_state(n, 3)
    h = S.sv_alloc(n, S.C64)
    try:
        for circ in (g, noisy, other, g):
            S.sv_load_state(h, psi0)
            S.sv_apply_circuit(h, circ)
            U.assert_close(S.sv_store_state(h).astype(np.complex128), U.run_oracle(n, circ, psi0), S.C64)
    finally:
        S.sv_free(h)
