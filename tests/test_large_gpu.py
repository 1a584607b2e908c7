"""Config-4 sizes (the memory ceiling): random U3 + CX circuits on 32 (complex64,
32 GiB), 34 (complex64, 128 GiB) and 33 (complex128, 128 GiB) qubits, each
followed by its inverse.  The oracle cannot hold these states, so the pin is
the reversal: the result must be |0...0>, checked without reading the state
back: every <Z_i> = 1 (so the mass off |0...0> is at most sum_i (1 - <Z_i>)/2),
the norm is 1, and every shot is 0."""
import numpy as np
import pytest

import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B

pytestmark = pytest.mark.gpu


def free_bytes():
    import torch

    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("n,dtype,layers", [(32, S.C64, 20), (34, S.C64, 2), (33, S.C128, 1)],
                         ids=["n32-c64", "n34-c64", "n33-c128"])
def test_large_state_reversal(n, dtype, layers):
    B.build()
    need = (8 if dtype == S.C64 else 16) << n
    if free_bytes() < need + (4 << 30):
        pytest.skip("device too small for this state")
    g = W.random_u3_cx(n, layers, W.SEED[4])
    circ = np.concatenate([g, W.inverse(g)])
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, circ)
        tol = 1e-5 if dtype == S.C64 else 1e-11
        ez = S.sv_expect_z(h)
        assert np.abs(ez - 1.0).max() < tol, np.abs(ez - 1.0).max()
        assert abs(S.sv_norm(h) - 1.0) < tol
        assert (S.sv_sample(h, 1000, 9) == 0).all()
    finally:
        S.sv_free(h)
