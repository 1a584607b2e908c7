"""The FP64 oracle against its pins (CPU only)."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import oracle_pins as P


@pytest.fixture(scope="module")
def O():
    return oracle.default()


@pytest.mark.parametrize("check", P.ALL_STATE_CHECKS, ids=lambda f: f.__name__)
def test_pin(O, check):
    check(O, np.random.default_rng(hash(check.__name__) % (1 << 32)))


def test_qft_angles_golden():
    P.check_qft_angles()


def test_qcrank_table2_golden():
    P.check_qcrank_table2()


def test_qft_reversal_random_state(O):
    n = 10
    psi = W.random_state(n, 7)
    g = W.qft(n)
    out = O.apply_circuit(n, np.concatenate([g, W.inverse(g)]), psi)
    assert np.abs(out - psi).max() < 1e-13


def test_brute_force_n8(O):
    P.check_brute_force(O, np.random.default_rng(8), n=8, count=12)


def test_invalid_records_rejected(O):
    n = 4
    psi = W.random_state(n, 1)
    bad = [
        [(W.H, (4,), ())],                # qubit >= n
        [(W.CX, (1, 1), ())],             # duplicate qubit
        [(W.H, (0,), ()), (W.CX, (0,), ())],  # arity mismatch
    ]
    for items in bad:
        with pytest.raises(ValueError):
            O.apply_circuit(n, W.gates_from_list(items), psi)
    g = W.gates_from_list([(W.H, (0,), ())])
    g[0]["type"] = 99
    with pytest.raises(ValueError):
        O.apply_circuit(n, g, psi)


def test_threads_do_not_change_results(O):
    n = 14
    g = W.random_u3_cx(n, 4, 3)
    O.set_threads(1)
    a = O.apply_circuit(n, g)
    O.set_threads(4)
    b = O.apply_circuit(n, g)
    O.set_threads(1)
    assert np.array_equal(a, b)
