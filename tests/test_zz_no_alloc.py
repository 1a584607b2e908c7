"""The no-allocation sampling entry point against sv_sample_uniforms.

sv_sample_uniforms_noalloc serves callers that cannot allocate device memory
while they run (a serving process whose device memory its own allocator hands
out up front, or a caller that cannot accept cudaFree's device-wide
synchronisation).  It keeps its scratch in a fixed array inside the library,
so it must give the same outcomes as the allocating entry point, call after
call.  The outcomes are integers decided by the same FP64 kernels on the
same data, so they must be equal exactly.  This file is collected last.
"""
import numpy as np
import pytest

import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    B.build()
    return pytest.importorskip("torch")


@pytest.mark.parametrize("dtype", [S.C64, S.C128], ids=["c64", "c128"])
@pytest.mark.parametrize("n", [11, 24])
def test_noalloc_matches_allocating_sampler_twice(torch, dtype, n):
    g = W.random_u3_cx(n, 2, 40 + n)
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, g)
        _, _, dev_amps = S.sv_info(h)
        shots = 3000
        for call in range(2):  # two calls in a row share the fixed scratch
            u = W.uniforms(shots, 100 * n + call)
            ref = S.sv_sample_uniforms(h, u)
            du = torch.from_numpy(u).cuda()
            dout = torch.full((shots,), -1, dtype=torch.int64, device="cuda")
            torch.cuda.synchronize()
            S.sv_sample_uniforms_noalloc(dev_amps, n, dtype, du.data_ptr(), shots, dout.data_ptr(), None)
            torch.cuda.synchronize()
            got = dout.cpu().numpy().view(np.uint64)
            assert np.array_equal(got, ref), "call %d: %d mismatches" % (call, int((got != ref).sum()))
    finally:
        S.sv_free(h)


def test_noalloc_rejects_n_above_limit(torch):
    h = S.sv_alloc(10, S.C64)
    try:
        _, _, dev_amps = S.sv_info(h)
        du = torch.zeros(4, dtype=torch.float64, device="cuda")
        dout = torch.zeros(4, dtype=torch.int64, device="cuda")
        with pytest.raises(S.SVError) as ei:
            S.sv_sample_uniforms_noalloc(dev_amps, 25, S.C64, du.data_ptr(), 4, dout.data_ptr(), None)
        assert ei.value.code == -1
        assert "1..24" in str(ei.value)
    finally:
        S.sv_free(h)
