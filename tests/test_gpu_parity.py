"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Sizes span several tiles and ragged cases (n below the tile width, n below
the row width, tiles of every allowed width), every planner and fusion width,
both dtypes.  Bounds: complex64 1-F <= 1e-6 and max |d psi| <= 1e-5;
complex128 1e-12 and 1e-12.
"""
import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U
from tests.oracle_pins import random_mixed_circuit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    oracle.set_threads(8)
    yield


DT = [S.C64, S.C128]
DTN = {S.C64: "c64", S.C128: "c128"}


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("planner,k", [(S.PLAN_PLAIN, 0), (S.PLAN_GREEDY, 2), (S.PLAN_GREEDY, 3),
                                       (S.PLAN_GREEDY, 4), (S.PLAN_GREEDY, 5)])
def test_config1_tiny(dtype, planner, k):
    n, g = W.config1()
    got = U.run_gpu(n, g, dtype, planner=planner, k_max=k)
    ref = U.run_oracle(n, g)
    U.assert_close(got, ref, dtype, "config1")


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("tile_m", [9, 10, 12, 13, 14])
@pytest.mark.parametrize("k", [2, 5])
def test_random_multi_tile(dtype, tile_m, k):
    if dtype == S.C128 and tile_m > 13:
        pytest.skip("c128 tiles hold at most 13 qubits")
    n = 17
    g = W.random_u3_cx(n, 5, 77 + tile_m)
    got = U.run_gpu(n, g, dtype, tile_m=tile_m, k_max=k)
    U.assert_close(got, U.run_oracle(n, g), dtype, "random n=17 m=%d k=%d" % (tile_m, k))


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("planner", [S.PLAN_PLAIN, S.PLAN_GREEDY])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 13, 16])
def test_mixed_all_gate_types(dtype, planner, n):
    rng = np.random.default_rng(100 + n)
    g = random_mixed_circuit(n, 60 if n > 1 else 20, rng) if n > 1 else W.gates_from_list(
        [(t, (0,), tuple(rng.uniform(0, 6, 3))) for t in (W.H, W.RX, W.RY, W.RZ, W.P, W.U3, W.X, W.Y, W.Z)])
    psi0 = W.random_state(n, 5 + n)
    got = U.run_gpu(n, g, dtype, psi0=psi0, planner=planner)
    U.assert_close(got, U.run_oracle(n, g, psi0), dtype, "mixed n=%d" % n)


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("k", [2, 3, 4, 5])
@pytest.mark.parametrize("kind", ["mixed", "qft", "cx_blocks"])
def test_gate_sequence_blocks(dtype, k, kind):
    """Blocks applied as their gate sequence in registers (2x2 complex and
    real matrices, phase tables, CX and SWAP moves) next to dense blocks."""
    n = 15
    rng = np.random.default_rng(300 + k)
    g = {"mixed": lambda: random_mixed_circuit(n, 120, rng), "qft": lambda: W.qft(n),
         "cx_blocks": lambda: W.random_cx_blocks(n, 40, 9 + k)}[kind]()
    info = S.sv_plan_circuit(n, dtype, g, k_max=k, tile_m=12)
    assert info["gate_ops"] > 0 or k == 5
    psi0 = W.random_state(n, 17 + k)
    got = U.run_gpu(n, g, dtype, psi0=psi0, k_max=k, tile_m=12)
    U.assert_close(got, U.run_oracle(n, g, psi0), dtype, "%s k=%d" % (kind, k))


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("tb", [5, 6, 8, 9])
@pytest.mark.parametrize("kind", ["mixed", "qft", "random", "cx_blocks"])
def test_register_passes(dtype, tb, kind):
    """Register-resident passes (2^5 / 2^4 amplitudes per thread, remaps
    through shared memory, diagonal runs from the register layout) at every
    thread count, fed by TMA tensor copies and by cp.async copies, and the
    shared-memory kernel, all against the oracle."""
    rb = 5 if dtype == S.C64 else 4
    m = rb + tb
    n = max(m + 3, 15)
    rng = np.random.default_rng(500 + tb)
    g = {"mixed": lambda: random_mixed_circuit(n, 150, rng), "qft": lambda: W.qft(n),
         "random": lambda: W.random_u3_cx(n, 4, 40 + tb), "cx_blocks": lambda: W.random_cx_blocks(n, 60, 7 + tb)}[kind]()
    psi0 = W.random_state(n, 70 + tb)
    ref = U.run_oracle(n, g, psi0)
    for k in (3, 4):
        info = S.sv_plan_circuit(n, dtype, g, k_max=k, tile_m=m)
        assert info["reg_passes"] > 0 and (k > 3 or info["reg_passes"] == info["passes"])
        for pk, what in ((0, "register"), (2, "register+TMA"), (1, "shared-memory")):
            got = U.run_gpu(n, g, dtype, psi0=psi0, k_max=k, tile_m=m, pass_kernel=pk)
            U.assert_close(got, ref, dtype, "%s %s k=%d m=%d" % (kind, what, k, m))


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("planner", [S.PLAN_PLAIN, S.PLAN_GREEDY])
def test_qft_basis_and_random(dtype, planner):
    n = 18
    g = W.qft(n)
    x = W.random_basis_index(n, 3)
    got = U.run_gpu(n, g, dtype, basis=x, planner=planner)
    U.assert_close(got, U.run_oracle(n, g, basis=x), dtype, "qft basis")
    psi0 = W.random_state(n, 4)
    got = U.run_gpu(n, g, dtype, psi0=psi0, planner=planner)
    U.assert_close(got, U.run_oracle(n, g, psi0), dtype, "qft random")


@pytest.mark.parametrize("tensor", [1, -1], ids=["tcgen05", "cuda_cores"])
@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("tile_m", [9, 11, 13, 14])
def test_tensor_core_blocks(tensor, k, tile_m):
    """complex64 dense blocks of 3..5 qubits on the tensor cores (3xTF32)
    and on the CUDA cores, multi-tile, random circuit and QFT."""
    n = 17
    g = W.random_u3_cx(n, 6, 300 + k + tile_m)
    got = U.run_gpu(n, g, S.C64, k_max=k, tile_m=tile_m, tensor=tensor)
    U.assert_close(got, U.run_oracle(n, g), S.C64, "random k=%d m=%d tensor=%d" % (k, tile_m, tensor))
    q = W.qft(n)
    psi0 = W.random_state(n, 9)
    got = U.run_gpu(n, q, S.C64, psi0=psi0, k_max=k, tile_m=tile_m, tensor=tensor)
    U.assert_close(got, U.run_oracle(n, q, psi0), S.C64, "qft k=%d m=%d tensor=%d" % (k, tile_m, tensor))


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
def test_qubit_position_sweep(dtype):
    """Every 1-qubit gate position and every ordered 2-qubit pair, n = 15
    (low, high and mixed positions relative to the tile rows)."""
    n = 15
    rng = np.random.default_rng(9)
    items = []
    for q in range(n):
        items.append((W.U3, (q,), tuple(rng.uniform(0, 6, 3))))
    for a in range(n):
        for b in range(n):
            if a != b:
                t = [W.CX, W.CP, W.SWAP, W.CZ][(a * n + b) % 4]
                items.append((t, (a, b), (float(rng.uniform(0, 6)),)))
                items.append((W.RY, (b,), (float(rng.uniform(0, 6)),)))
    g = W.gates_from_list(items)
    psi0 = W.random_state(n, 11)
    ref = U.run_oracle(n, g, psi0)
    for planner, k, m in [(S.PLAN_PLAIN, 0, 0), (S.PLAN_GREEDY, 2, 10), (S.PLAN_GREEDY, 5, 12)]:
        got = U.run_gpu(n, g, dtype, psi0=psi0, planner=planner, k_max=k, tile_m=m)
        U.assert_close(got, ref, dtype, "sweep planner=%d k=%d" % (planner, k))


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
def test_reversal_returns_zero_state(dtype):
    n = 16
    g = W.random_u3_cx(n, 8, 5)
    gg = np.concatenate([g, W.inverse(g)])
    got = U.run_gpu(n, gg, dtype)
    ref = oracle.basis_state(n, 0)
    U.assert_close(got, ref, dtype, "reversal")


def test_reversal_tensor_cores():
    """The circuit and its reversal (8 + 8 layers at n = 16) through 3xTF32
    blocks of 5 qubits returns |0...0> within the complex64 bounds."""
    n = 16
    g = W.random_u3_cx(n, 4, 6)
    gg = np.concatenate([g, W.inverse(g)])
    got = U.run_gpu(n, gg, S.C64, k_max=5, tensor=1)
    U.assert_close(got, oracle.basis_state(n, 0), S.C64, "reversal tcgen05")


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
def test_readout_probs_norm_expz(dtype):
    n = 14
    g = W.random_u3_cx(n, 4, 21)
    ref = U.run_oracle(n, g)
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, g)
        p = S.sv_probs(h)
        pref = oracle.probs(ref)
        tol = 1e-6 if dtype == S.C64 else 1e-13
        assert np.abs(p - pref).max() <= tol * max(1.0, pref.max())
        assert abs(S.sv_norm(h) - 1.0) <= (1e-5 if dtype == S.C64 else 1e-12)
        ez = S.sv_expect_z(h)
        assert np.abs(ez - oracle.expect_z(ref)).max() <= (1e-5 if dtype == S.C64 else 1e-12)
    finally:
        S.sv_free(h)


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("n", [3, 12, 17])
def test_sampler_oracle_uniforms(dtype, n):
    """With oracle-supplied uniforms the outcomes match exactly except for
    draws within 1e-9 of a CDF boundary: (a) the sampler given the same
    probabilities (the GPU's own probabilities fed to the oracle sampler);
    (b) end to end against the oracle state (c128 band 1e-9; c64 band widened
    by the measured CDF difference)."""
    g = W.random_u3_cx(n, 3, 31 + n)
    ref = U.run_oracle(n, g)
    u = W.uniforms(4096, 17 + n)
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, g)
        got = S.sv_sample_uniforms(h, u)
        pg = S.sv_probs(h)
    finally:
        S.sv_free(h)
    cmp_a, _ = U.compare_samples(got, u, oracle.cdf(pg), U.BAND)
    assert cmp_a > 4000
    cref = oracle.cdf(oracle.probs(ref))
    band = U.BAND if dtype == S.C128 else max(U.BAND, 4 * np.abs(np.cumsum(pg) - cref).max())
    U.compare_samples(got, u, cref, band)


@pytest.mark.parametrize("scale", [1e-12, 1e3], ids=["tiny", "large"])
def test_sampler_unnormalised_state(scale):
    """The rule min{x : C_x > u C_{N-1}} holds for a state far from unit norm
    (complex64: total 1e-24 takes the FP64 rescan, 1e6 the double-float
    one): outcomes equal the oracle sampler's on the stored probabilities
    except within 1e-9 (relative) of a CDF boundary."""
    n = 14
    psi = W.random_state(n, 71) * scale
    u = W.uniforms(4096, 72)
    h = S.sv_alloc(n, S.C64)
    try:
        S.sv_load_state(h, psi)
        got = S.sv_sample_uniforms(h, u)
        pg = S.sv_probs(h)
    finally:
        S.sv_free(h)
    c = oracle.cdf(pg)
    assert abs(c[-1] / scale ** 2 - 1.0) < 1e-5
    cmp, _ = U.compare_samples(got, u, c, U.BAND * c[-1])
    assert cmp > 4000


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
@pytest.mark.parametrize("n", [4, 10, 15])
def test_measure_device_one_pass(dtype, n):
    """Shots and <Z> from one pass equal the separate entry points."""
    torch = pytest.importorskip("torch")
    g = W.random_u3_cx(n, 3, 90 + n)
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, g)
        ds = torch.zeros(3000, dtype=torch.int64, device="cuda")
        dz = torch.zeros(n, dtype=torch.float64, device="cuda")
        S.sv_measure_device(h, 3000, 42, ds.data_ptr(), dz.data_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(ds.cpu().numpy().view(np.uint64), S.sv_sample(h, 3000, 42))
        ez = S.sv_expect_z(h)
        assert np.array_equal(dz.cpu().numpy(), ez)
        hs, hz = S.sv_measure(h, 3000, 42)  # host outputs, one read
        assert np.array_equal(hs, ds.cpu().numpy().view(np.uint64)) and np.array_equal(hz, ez)
        ref = U.run_oracle(n, g)
        assert np.abs(ez - oracle.expect_z(ref)).max() <= (1e-5 if dtype == S.C64 else 1e-12)
    finally:
        S.sv_free(h)


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
def test_sampler_philox_matches_oracle_uniforms(dtype):
    n = 10
    g = W.random_u3_cx(n, 3, 8)
    seed = 123456789
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, g)
        a = S.sv_sample(h, 5000, seed)
        b = S.sv_sample_uniforms(h, oracle.uniforms(seed, 5000))
        pg = S.sv_probs(h)
    finally:
        S.sv_free(h)
    assert np.array_equal(a, b)
    # zero-probability outcomes are never drawn
    assert (pg[a.astype(np.int64)] > 0).all()


@pytest.mark.parametrize("dtype", DT, ids=DTN.get)
def test_sampler_basis_and_ghz(dtype):
    n = 20
    x = 0xABCDE
    h = S.sv_alloc(n, dtype)
    try:
        S.sv_init_basis(h, x)
        assert (S.sv_sample(h, 1000, 5) == x).all()
        items = [(W.H, (0,), ())] + [(W.CX, (q, q + 1), ()) for q in range(n - 1)]
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, W.gates_from_list(items))
        s = S.sv_sample(h, 4000, 6)
        assert set(s.tolist()) == {0, (1 << n) - 1}
        assert 1700 < (s == 0).sum() < 2300
    finally:
        S.sv_free(h)


def test_invalid_records_leave_state_untouched():
    n = 6
    psi0 = W.random_state(n, 2)
    h = S.sv_alloc(n, S.C128)
    try:
        S.sv_load_state(h, psi0)
        bad = [[(W.H, (6,), ())], [(W.CX, (2, 2), ())]]
        for items in bad:
            with pytest.raises(S.SVError) as ei:
                S.sv_apply_circuit(h, W.gates_from_list(items))
            assert ei.value.code == -1
        g = W.gates_from_list([(W.H, (0,), ())])
        g[0]["type"] = 77
        with pytest.raises(S.SVError):
            S.sv_apply_circuit(h, g)
        assert np.array_equal(S.sv_store_state(h), psi0)
        # measure-only and empty circuits are no-ops
        S.sv_apply_circuit(h, W.gates_from_list([(W.MEASURE, (3,), ())]))
        S.sv_apply_circuit(h, np.zeros(0, dtype=W.GATE_DTYPE))
        assert np.array_equal(S.sv_store_state(h), psi0)
        with pytest.raises(S.SVError):
            S.sv_init_basis(h, 1 << n)
    finally:
        S.sv_free(h)


def test_alloc_limits():
    with pytest.raises(S.SVError) as ei:
        S.sv_alloc(40, S.C64)
    assert ei.value.code == -1
    with pytest.raises(S.SVError) as ei:
        S.sv_alloc(0, S.C64)
    assert ei.value.code == -1


def test_torch_memory_and_stream():
    torch = pytest.importorskip("torch")
    n = 16
    t = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    h = S.sv_attach(n, S.C64, t.data_ptr(), st.cuda_stream)
    try:
        g = W.random_u3_cx(n, 4, 3)
        S.sv_init_basis(h, 0)
        S.sv_apply_circuit(h, g)
        st.synchronize()
        got = t.cpu().numpy().view(np.complex64).astype(np.complex128)
        U.assert_close(got, U.run_oracle(n, g), S.C64, "torch memory")
    finally:
        S.sv_free(h)
