"""Run-time compiled register passes (jit) against the FP64 oracle, and
against the interpreting kernel on the same plan: same bounds as every other
plan (complex64 1-F <= 1e-6, max |d psi| <= 1e-5; complex128 1e-12)."""
import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U
from tests.oracle_pins import random_mixed_circuit

pytestmark = pytest.mark.gpu

DT = [S.C64, S.C128]
DTN = {S.C64: "c64", S.C128: "c128"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    oracle.set_threads(8)
    yield


def _circuits():
    return [
        ("qft16", 16, W.qft(16), {}),
        ("qft18-relabel", 18, W.qft(18), {"relabel": 1}),
        ("random-u3cx", 16, W.random_u3_cx(16, 6, 11), {}),
        ("cx-blocks-k3", 15, W.random_cx_blocks(15, 60, 12), {"k_max": 3}),
        ("hea", 14, W.hea(14, 3, W.hea_params(1, 14, 3, 13)[0]), {}),
        ("mixed", 15, random_mixed_circuit(15, 200, np.random.default_rng(14)), {}),
    ]


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("case", range(6), ids=[c[0] for c in _circuits()])
def test_jit_pass_vs_oracle(dtype, case):
    name, n, g, opts = _circuits()[case]
    psi0 = W.random_state(n, 300 + case)
    ref = U.run_oracle(n, g, psi0)
    before = S.sv_jit_stats()
    got = U.run_gpu(n, g, dtype, psi0=psi0, jit=1, **opts)
    after = S.sv_jit_stats()
    assert after["failed"] == before["failed"]
    info = S.sv_plan_circuit(n, dtype, g[g["type"] != W.SWAP] if opts.get("relabel") else g,
                             k_max=opts.get("k_max", 0))
    if info["reg_passes"]:
        assert after["launched"] > before["launched"], name  # the compiled kernels ran
    if opts.get("relabel"):
        h = S.sv_alloc(n, dtype)
        try:
            S.sv_load_state(h, psi0)
            S.sv_apply_circuit(h, g, jit=1, **opts)
            S.sv_materialize(h)
            got = S.sv_store_state(h).astype(np.complex128)
        finally:
            S.sv_free(h)
    U.assert_close(got, ref, dtype, name)
    interp = U.run_gpu(n, g, dtype, psi0=psi0, jit=-1, **opts) if not opts.get("relabel") else None
    if interp is not None:
        U.assert_close(got, interp, dtype, name + " vs interpreting kernel")


def test_jit_auto_compiles_on_repeat():
    """jit = 0: the first apply of a structure runs the interpreting kernel,
    the second compiles it (states of 22+ qubits), and later applies, also
    with other angles, reuse the kernels."""
    n = 22
    g = W.random_u3_cx(n, 2, 21)  # a structure no other test uses
    psi0 = W.random_state(n, 22)
    ref = U.run_oracle(n, g, psi0)
    s0 = S.sv_jit_stats()
    U.assert_close(U.run_gpu(n, g, S.C64, psi0=psi0), ref, S.C64, "first")
    s1 = S.sv_jit_stats()
    assert s1["launched"] == s0["launched"] and s1["compiled"] == s0["compiled"]
    U.assert_close(U.run_gpu(n, g, S.C64, psi0=psi0), ref, S.C64, "second")
    s2 = S.sv_jit_stats()
    assert s2["compiled"] > s1["compiled"]
    U.assert_close(U.run_gpu(n, g, S.C64, psi0=psi0), ref, S.C64, "third")
    s3 = S.sv_jit_stats()
    assert s3["launched"] > s2["launched"] and s3["compiled"] == s2["compiled"]
    # small states stay on the interpreting kernel under jit = 0
    gs = W.random_u3_cx(14, 2, 23)
    for _ in range(3):
        U.run_gpu(14, gs, S.C64)
    assert S.sv_jit_stats()["compiled"] == s3["compiled"]
    # the same structure with other angles reuses the kernels
    g2 = W.random_u3_cx(n, 2, 21)
    g2["p"] = np.random.default_rng(5).uniform(0, 2 * np.pi, size=g2["p"].shape) * (g2["type"] == W.U3)[:, None]
    U.assert_close(U.run_gpu(n, g2, S.C64, psi0=psi0), U.run_oracle(n, g2, psi0), S.C64, "other angles")
    s4 = S.sv_jit_stats()
    assert s4["compiled"] == s3["compiled"] and s4["launched"] > s3["launched"]


@pytest.mark.parametrize("tile_m", [12, 13])
def test_direct_copies_and_warp_remaps_vs_oracle(tile_m):
    """Compiled passes that load their first register layout straight from
    the state and store their last straight back (no shared-memory copy), and
    plans whose remaps stay within warps (ordered by warp barriers only), give
    the oracle's state: a random U3+CX circuit whose plan has both, from a
    random state and from the deferred |0...0> (its first pass builds the tile
    in registers)."""
    n = 20
    g = W.random_u3_cx(n, 10, 17 + tile_m)
    info = S.sv_plan_circuit(n, S.C64, g, k_max=5, tile_m=tile_m, tensor=-1)
    assert info["warp_remaps"] > 0 and info["warp_remaps"] < info["remaps"]
    psi0 = W.random_state(n, 44)
    before = S.sv_jit_stats()
    got = U.run_gpu(n, g, S.C64, psi0=psi0, jit=1, k_max=5, tile_m=tile_m, tensor=-1)
    after = S.sv_jit_stats()
    assert after["failed"] == before["failed"]
    assert after["direct_load"] > before["direct_load"] and after["direct_store"] > before["direct_store"]
    U.assert_close(got, U.run_oracle(n, g, psi0), S.C64, "direct copies m=%d" % tile_m)
    h = S.sv_alloc(n, S.C64)
    try:
        S.sv_init_basis(h, 0)
        f0 = S.sv_jit_stats()["filled"]
        S.sv_apply_circuit(h, g, jit=1, k_max=5, tile_m=tile_m, tensor=-1)
        got0 = S.sv_store_state(h).astype(np.complex128)
        assert S.sv_jit_stats()["filled"] > f0
    finally:
        S.sv_free(h)
    U.assert_close(got0, U.run_oracle(n, g), S.C64, "direct copies from |0> m=%d" % tile_m)
