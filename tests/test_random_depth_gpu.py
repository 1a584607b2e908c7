"""Large random circuits at their full depth: 60 layers of U3 on every qubit
and CX on a random disjoint pairing (the random non-Clifford family of Sec. 3,
App. D.1), at n = 20 where the FP64 oracle finishes in seconds, against that
oracle element by element.  Covers the planner's gate reordering within a pass
(blocks grouped by qubit set), U3 blocks written as P RY P with merged phase
tables, compiled and interpreted passes, both dtypes.  Bounds: complex64
1-F <= 1e-6 and max |d psi| <= 1e-5; complex128 1e-12 and 1e-12."""
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

N, LAYERS, SEED = 20, 60, 1004


@pytest.fixture(scope="module")
def ref():
    B.build()
    oracle.set_threads(16)
    g = W.random_u3_cx(N, LAYERS, SEED)
    return g, U.run_oracle(N, g)


@pytest.mark.parametrize("dtype,opts", [
    (S.C64, {}),                              # interpreting kernel (small state)
    (S.C64, {"jit": 1}),                      # compiled passes
    (S.C64, {"jit": 1, "tile_m": 14}),
    (S.C64, {"k_max": 4, "tile_m": 12}),
    (S.C64, {"pass_kernel": 1}),              # shared-memory kernel
    (S.C128, {}),
    (S.C128, {"jit": 1}),
], ids=["c64", "c64-jit", "c64-jit-m14", "c64-k4-m12", "c64-smem", "c128", "c128-jit"])
def test_full_depth_vs_oracle(ref, dtype, opts):
    g, want = ref
    got = U.run_gpu(N, g, dtype, **opts)
    U.assert_close(got, want, dtype, "random n=%d, %d layers %s" % (N, LAYERS, opts))



@pytest.mark.parametrize("dtype,opts", [(S.C64, {}), (S.C64, {"jit": 1}), (S.C128, {})], ids=["c64", "c64-jit", "c128"])
def test_many_rotations_in_one_pass(dtype, opts):
    """250 RY rotations and 50 Hadamards kept apart by CX gates on five
    qubits of a 12-qubit state: one pass whose rotations and Hadamards defer
    more factors than the write-back scale takes (each at least 1/sqrt(2), at
    most 2^40 of growth), so the later ones run with their factor in the
    matrix.  Against the oracle."""
    import numpy as np

    rng = np.random.default_rng(77)
    items = [(W.H, (q,), ()) for q in range(12)]
    for r in range(50):
        for q in range(5):
            items.append((W.RY, (q,), (rng.uniform(np.pi / 4, 3 * np.pi / 4),)))
        items.append((W.H, (r % 5,), ()))
        for q in range(4):
            items.append((W.CX, (q, q + 1), ()))
    g = W.gates_from_list(items)
    got = U.run_gpu(12, g, dtype, **opts)
    U.assert_close(got, U.run_oracle(12, g), dtype, "250 rotations in one pass %s" % opts)
