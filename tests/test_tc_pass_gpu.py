"""Dense 4- and 5-qubit blocks on the tensor cores inside the register
passes (kind::f16 with FP16 hi/lo splits of the amplitudes and the matrix,
three products, FP32 accumulation; App. D.2 "gate fusion = 5"), against the
FP64 oracle within the complex64 bounds: one, two and four 128-thread groups
per CTA (tiles of 12, 13 and 14 qubits), the run-time compiled passes and the
interpreting kernel, blocks after deferred Hadamard factors (QFT), the first
pass built from a deferred basis state, relabelled SWAPs and a long circuit
followed by its inverse."""
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
    oracle.set_threads(8)
    yield


@pytest.mark.parametrize("jit", [1, -1], ids=["compiled", "interpreting"])
@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("tile_m", [12, 13, 14])
def test_tc_blocks_random(jit, k, tile_m):
    n = 18
    g = W.random_u3_cx(n, 8, 40 + k + tile_m)
    info = S.sv_plan_circuit(n, S.C64, g, k_max=k, tile_m=tile_m, tensor=1)
    assert info["tc_ops"] > 0
    psi0 = W.random_state(n, 3)
    got = U.run_gpu(n, g, S.C64, psi0=psi0, k_max=k, tile_m=tile_m, tensor=1, jit=jit)
    U.assert_close(got, U.run_oracle(n, g, psi0), S.C64, "tc random k=%d m=%d jit=%d" % (k, tile_m, jit))


@pytest.mark.parametrize("jit", [1, -1], ids=["compiled", "interpreting"])
def test_tc_blocks_qft_and_cx_blocks(jit):
    n = 17
    q = W.qft(n)
    psi0 = W.random_state(n, 5)
    got = U.run_gpu(n, q, S.C64, psi0=psi0, tensor=1, jit=jit)
    U.assert_close(got, U.run_oracle(n, q, psi0), S.C64, "tc qft")
    c = W.random_cx_blocks(n, 300, 6)
    got = U.run_gpu(n, c, S.C64, tensor=1, jit=jit)
    U.assert_close(got, U.run_oracle(n, c), S.C64, "tc cx blocks")


def test_tc_blocks_from_deferred_basis_with_relabel():
    n = 20
    g = W.qft(n)
    x = W.random_basis_index(n, 12)
    h = S.sv_alloc(n, S.C64)
    try:
        f0 = S.sv_jit_stats()["filled"]
        S.sv_init_basis(h, x)
        S.sv_apply_circuit(h, g, tensor=1, relabel=1, jit=1)
        assert S.sv_jit_stats()["filled"] - f0 == 1
        got = S.sv_store_state(h).astype(np.complex128)  # logical order through the map
    finally:
        S.sv_free(h)
    U.assert_close(got, U.run_oracle(n, g, basis=x), S.C64, "tc qft from |x>")


def test_tc_blocks_reversal():
    n = 20
    g = W.random_u3_cx(n, 30, 9)
    gg = np.concatenate([g, W.inverse(g)])
    got = U.run_gpu(n, gg, S.C64, tensor=1, jit=1)
    U.assert_close(got, oracle.basis_state(n, 0), S.C64, "tc reversal")


def test_tc_readouts_after_tc_pass():
    """Probabilities, <Z> and shots of a state produced by tensor-core passes
    follow the oracle (the sampler on the state's own probabilities)."""
    n = 16
    g = W.random_u3_cx(n, 10, 11)
    ref = U.run_oracle(n, g)
    h = S.sv_alloc(n, S.C64)
    try:
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, g, tensor=1, tile_m=12)
        U.assert_close(S.sv_store_state(h).astype(np.complex128), ref, S.C64, "state")
        assert np.abs(S.sv_expect_z(h) - oracle.expect_z(ref)).max() < 1e-5
        p = S.sv_probs(h)
        u = W.uniforms(3000, 4)
        U.compare_samples(S.sv_sample_uniforms(h, u).astype(np.int64), u, oracle.cdf(p), U.BAND)
    finally:
        S.sv_free(h)
