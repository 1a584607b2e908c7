"""sv_init_basis is deferred: the next apply's first compiled pass builds its
tiles from |x> instead of reading the state, and every other use of the
state writes |x> first.  Each path against the FP64 oracle."""
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
    yield


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("where", ["zero", "low", "high", "last"])
def test_first_pass_builds_the_basis_state(dtype, where):
    n = 18
    x = {"zero": 0, "low": 37, "high": (1 << 17) | 1234, "last": (1 << n) - 1}[where]
    g = W.random_u3_cx(n, 3, 71) if dtype == S.C64 else W.qft(n)
    ref = U.run_oracle(n, g, basis=x)
    before = S.sv_jit_stats()
    for relabel in (0, 1):
        h = S.sv_alloc(n, dtype)
        try:
            S.sv_init_basis(h, x)
            S.sv_apply_circuit(h, g, jit=1, relabel=relabel)
            U.assert_close(S.sv_store_state(h).astype(np.complex128), ref, dtype, where)
        finally:
            S.sv_free(h)
    if S.sv_plan_circuit(n, dtype, g)["reg_passes"]:  # the compiled kernels (and the tile fill) ran
        assert S.sv_jit_stats()["launched"] > before["launched"]


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
def test_other_uses_write_the_basis_first(dtype):
    n, x = 12, 1234
    e = np.zeros(1 << n, np.complex128)
    e[x] = 1
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_init_basis(h, x)
        assert np.array_equal(S.sv_store_state(h).astype(np.complex128), e)
        S.sv_init_basis(h, x)
        p = S.sv_probs(h)
        assert p[x] == 1.0 and p.sum() == 1.0
        S.sv_init_basis(h, x)
        assert (S.sv_sample(h, 50, 3) == x).all()
        S.sv_init_basis(h, x)
        ez = S.sv_expect_z(h)
        assert np.array_equal(ez, [-1.0 if (x >> i) & 1 else 1.0 for i in range(n)])
        # an empty circuit leaves the state |x>
        S.sv_init_basis(h, x)
        S.sv_apply_circuit(h, W.gates_from_list([]))
        assert np.array_equal(S.sv_store_state(h).astype(np.complex128), e)
        # a load replaces a pending |x>
        psi = W.random_state(n, 5)
        S.sv_init_basis(h, x)
        S.sv_load_state(h, psi)
        U.assert_close(S.sv_store_state(h).astype(np.complex128), psi, dtype, "load after init")
        # the one-kernel-per-gate planner and the interpreting kernel write |x> first
        g = W.qft(n)
        ref = U.run_oracle(n, g, basis=x)
        for opts in ({"planner": S.PLAN_PLAIN}, {"jit": -1}, {"pass_kernel": 1}):
            S.sv_init_basis(h, x)
            S.sv_apply_circuit(h, g, **opts)
            U.assert_close(S.sv_store_state(h).astype(np.complex128), ref, dtype, str(opts))
    finally:
        S.sv_free(h)


def test_attached_memory_is_written_before_the_pointer_is_handed_out():
    torch = pytest.importorskip("torch")
    n, x = 10, 77
    t = torch.full((2 << n,), 7.0, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    h = S.sv_attach(n, S.C64, t.data_ptr(), st.cuda_stream)
    try:
        S.sv_init_basis(h, x)
        S.sv_info(h)  # hands out the device pointer: the amplitudes are written
        torch.cuda.synchronize()
        a = t.view(torch.complex64).cpu().numpy()
        e = np.zeros(1 << n, np.complex64)
        e[x] = 1
        assert np.array_equal(a, e)
    finally:
        S.sv_free(h)
