"""The approximation for negligible rotations (App. D.2): P, RZ and CP gates
below an angle threshold are left out.  The fidelity loss against the exact
oracle grows with the threshold and stays inside the bound from the dropped
angles: || U psi - U' psi || <= sum |lambda| / 2, so 1 - F <= (sum |lambda| / 2)^2."""
import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [S.C64, S.C128], ids=["c64", "c128"])
def test_approximate_qft_fidelity(dtype):
    B.build()
    n = 16
    g = W.qft(n)
    psi0 = W.random_state(n, 12)
    exact = U.run_oracle(n, g, psi0)
    lam = np.array([abs(np.remainder(r["p"][0] + np.pi, 2 * np.pi) - np.pi) for r in g if r["type"] == W.CP])
    losses = []
    for eps in (0.0, 1e-4, 1e-3, 1e-2, 3e-2):
        got = U.run_gpu(n, g, dtype, psi0=psi0, drop_phase_below=eps)
        F = oracle.fidelity(got, exact)
        dropped = lam[lam < eps] if eps > 0 else lam[:0]
        bound = (dropped.sum() / 2) ** 2
        floor = 1e-6 if dtype == S.C64 else 1e-12
        assert 1.0 - F <= bound + floor, (eps, 1.0 - F, bound)
        info = S.sv_plan_circuit(n, dtype, g, drop_phase_below=eps)
        assert info["gates"] == len(g) - len(dropped)
        losses.append(1.0 - F)
    assert losses[-1] > losses[0]  # the approximation is visible at the largest threshold
    assert all(l2 >= l1 - 1e-9 for l1, l2 in zip(losses, losses[1:]))  # monotone in the threshold
