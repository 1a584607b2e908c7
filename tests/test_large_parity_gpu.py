"""Full-state parity at n = 32 (complex64, 32 GiB on the device) against the
FP64 oracle (64 GiB of host memory): the first two layers of the n = 32
random U3 + CX workload (App. D.1 random circuits, Sec. 3), fused on the CUDA
cores and with tensor-core blocks, compared amplitude by amplitude in chunks
(fidelity and max amplitude error within the complex64 bounds).  Skipped
where the host lacks the memory."""
import os

import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _mem_available_gib():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / (1 << 20)
    except OSError:
        pass
    return 0.0


def test_full_state_parity_n32():
    if _mem_available_gib() < 112:
        pytest.skip("needs about 100 GiB of host memory (64 GiB oracle state + 32 GiB device copy)")
    torch = pytest.importorskip("torch")
    B.build()
    n = 32
    g = W.random_u3_cx(n, 60, W.SEED[4])[:2 * (n + n // 2)]  # the first two layers: 96 gates
    oracle.set_threads(len(os.sched_getaffinity(0)))
    ref = oracle.basis_state(n, 0)
    oracle.apply_inplace(n, g, ref)
    state = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    h = S.sv_attach(n, S.C64, state.data_ptr(), torch.cuda.current_stream().cuda_stream)
    try:
        for tensor in (0, 1):
            S.sv_init_basis(h, 0)
            S.sv_apply_circuit(h, g, tensor=tensor, jit=1)
            torch.cuda.synchronize()
            ov, ng, nr, err = 0j, 0.0, 0.0, 0.0
            C = 1 << 27
            st = state.view(torch.complex64)
            for off in range(0, 1 << n, C):
                got = st[off:off + C].cpu().numpy().astype(np.complex128)
                r = ref[off:off + C]
                ov += np.vdot(got, r)
                ng += np.vdot(got, got).real
                nr += np.vdot(r, r).real
                err = max(err, float(np.abs(got - r).max()))
            one_minus_F = 1.0 - abs(ov) ** 2 / (ng * nr)
            fd, ma = U.TOL[S.C64]
            assert one_minus_F <= fd, "tensor=%d: 1-F = %.3e" % (tensor, one_minus_F)
            assert err <= ma, "tensor=%d: max |d psi| = %.3e" % (tensor, err)
    finally:
        S.sv_free(h)
