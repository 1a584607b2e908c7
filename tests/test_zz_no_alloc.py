"""The no-allocation sampling entry point against the oracle's shot rule.

sv_sample_uniforms_noalloc serves callers that cannot allocate device memory
while they run (a serving process whose device memory its own allocator hands
out up front, or a caller that cannot accept cudaFree's device-wide
synchronisation).  It keeps its scratch in a fixed array inside the library.
Its outcomes must follow the rule every sampler here follows, outcome =
min{x : C_x > u C_{N-1}} with C the FP64 CDF, except for draws within 1e-9
of a CDF boundary, call after call while the fixed array is reused: checked
against the oracle's CDF (complex128: of the oracle's own state; complex64:
of the GPU state's probabilities, whose amplitudes differ from the oracle's
in the 7th digit) and, within the same band, against the allocating entry
point, whose block size may differ.  This file is collected last.
"""
import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    B.build()
    return pytest.importorskip("torch")


@pytest.mark.parametrize("dtype", [S.C64, S.C128], ids=["c64", "c128"])
@pytest.mark.parametrize("n", [11, 24])
def test_noalloc_follows_oracle_rule_twice(torch, dtype, n):
    g = W.random_u3_cx(n, 2, 40 + n)
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, g)
        p = S.sv_probs(h)
        if dtype == S.C128:
            oracle.set_threads(8)
            p = np.abs(U.run_oracle(n, g)) ** 2
        c_ref = oracle.cdf(p)
        _, _, dev_amps = S.sv_info(h)
        torch.cuda.synchronize()  # sv_info may flush a deferred init on the handle's stream
        shots = 3000
        for call in range(2):  # two calls in a row share the fixed scratch
            u = W.uniforms(shots, 100 * n + call)
            du = torch.from_numpy(u).cuda()
            dout = torch.full((shots,), -1, dtype=torch.int64, device="cuda")
            torch.cuda.synchronize()
            S.sv_sample_uniforms_noalloc(dev_amps, n, dtype, du.data_ptr(), shots, dout.data_ptr(), None)
            torch.cuda.synchronize()
            got = dout.cpu().numpy().astype(np.int64)
            compared, _ = U.compare_samples(got, u, c_ref, U.BAND)
            assert compared > shots // 2, "call %d" % call
            ref = S.sv_sample_uniforms(h, u).astype(np.int64)
            U.compare_samples(ref, u, c_ref, U.BAND)
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
