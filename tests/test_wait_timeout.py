"""Failure detection without a GPU fault: a bounded wait on an mbarrier that
nothing arrives at gives up, reports it through a status word and returns,
and the context stays usable (a circuit applied afterwards is still exact)."""
import ctypes

import numpy as np
import pytest

import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U


@pytest.mark.gpu
@pytest.mark.parametrize("limit", [1, 64, 4096])
def test_bounded_wait_gives_up_and_context_survives(limit):
    B.build()
    f = S.lib().sv_selftest_wait_timeout
    f.argtypes = [ctypes.c_uint, ctypes.POINTER(ctypes.c_int)]
    f.restype = ctypes.c_int
    st = ctypes.c_int(-1)
    assert f(limit, ctypes.byref(st)) == 0, S.sv_last_error()
    assert st.value == 1
    # the same context still simulates correctly
    n, g = W.config1()
    got = U.run_gpu(n, g, S.C64)
    U.assert_close(got, U.run_oracle(n, g), S.C64, "after timeout self-test")


@pytest.mark.gpu
def test_bounded_wait_rejects_bad_limit():
    B.build()
    f = S.lib().sv_selftest_wait_timeout
    f.argtypes = [ctypes.c_uint, ctypes.POINTER(ctypes.c_int)]
    f.restype = ctypes.c_int
    st = ctypes.c_int(-1)
    assert f(0, ctypes.byref(st)) == -1  # SV_EINVAL
    assert f(1 << 23, ctypes.byref(st)) == -1


@pytest.mark.gpu
@pytest.mark.parametrize("limit", [1, 1000])
def test_wave_wait_gives_up_and_context_survives(limit):
    """The batch executor's persistent kernel: a work item whose dependency
    never finishes gives up after its bounded wait, the wave reports the
    timeout and the context still runs a batch correctly."""
    B.build()
    f = S.lib().sv_selftest_wave_timeout
    f.argtypes = [ctypes.c_uint, ctypes.POINTER(ctypes.c_int)]
    f.restype = ctypes.c_int
    st = ctypes.c_int(-1)
    assert f(limit, ctypes.byref(st)) == 0, S.sv_last_error()
    assert st.value == 1
    circuits = [(14, W.random_u3_cx(14, 3, 70 + i)) for i in range(3)]
    _, ez = S.sv_batch_run(circuits, dtype=S.C64, shots=0)
    for c, (n, g) in enumerate(circuits):
        ref = U.run_oracle(n, g)
        import oracle
        assert np.abs(ez[c, :n] - oracle.expect_z(ref)).max() < 1e-5
