"""Host-side checks that need no GPU: the C ABI library loads and exports
every symbol include/sv.h declares; the planner's host logic."""
import numpy as np
import pytest

import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()


def test_exports_every_declared_symbol():
    decl = S.declared_symbols()
    assert len(decl) >= 20
    missing = sorted(set(decl) - set(S.exported_symbols()))
    assert not missing, missing


def test_version_and_feature_count():
    assert S.sv_version() >= 100
    assert S.sv_feature_count() == 32


def test_plan_qft_counts():
    info = S.sv_plan_circuit(28, S.C64, W.qft(28))
    assert info["gates"] == 420
    assert 1 <= info["passes"] <= 8
    assert info["max_k"] <= 5
    assert info["bytes_moved"] == info["passes"] * 16 * (1 << 28)
    plain = S.sv_plan_circuit(28, S.C64, W.qft(28), planner=S.PLAN_PLAIN)
    assert plain["passes"] == 420


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_plan_respects_k(k):
    info = S.sv_plan_circuit(20, S.C64, W.random_u3_cx(20, 10, 3), k_max=k)
    assert info["max_k"] <= k



def test_plan_groups_gates_by_qubit_set():
    """Grouping each pass's gates by qubit set (each qubit's gates kept in
    order) needs far fewer blocks, and so register remaps, than fusing them
    in list order: about one block per four gates of a random U3+CX circuit,
    where list order gives one per two."""
    n = 24
    g = W.random_u3_cx(n, 20, 5)
    info = S.sv_plan_circuit(n, S.C64, g, k_max=5, tile_m=13)
    assert info["dense_ops"] * 3 < len(g), info
    assert info["reg_passes"] == info["passes"]

def test_plan_validation_errors():
    with pytest.raises(S.SVError) as ei:
        S.sv_plan_circuit(4, S.C64, W.gates_from_list([(W.H, (4,), ())]))
    assert ei.value.code == -1
    with pytest.raises(S.SVError):
        S.sv_plan_circuit(0, S.C64, W.qft(3))
    with pytest.raises(S.SVError):
        S.sv_plan_circuit(34, S.C128, W.qft(3))
    g = W.gates_from_list([(W.RX, (0,), (float("nan"),))])
    with pytest.raises(S.SVError):
        S.sv_plan_circuit(2, S.C64, g)


def test_plan_drops_small_phases():
    # QFT n=16 has CP angles pi/2^j, j = 1..15; eps = 1e-3 drops j >= 12
    # (pi/2^12 = 7.7e-4), i.e. 4 + 3 + 2 + 1 = 10 gates; eps = 0 drops none.
    g = W.qft(16)
    assert S.sv_plan_circuit(16, S.C64, g)["gates"] == len(g)
    assert S.sv_plan_circuit(16, S.C64, g, drop_phase_below=1e-3)["gates"] == len(g) - 10
    # 2*pi wraps to zero and is dropped, -pi/2^14 has magnitude below 1e-3
    h = W.gates_from_list([(W.P, (0,), (2 * np.pi,)), (W.RZ, (1,), (-np.pi / 2**14,)),
                           (W.CP, (0, 1), (0.5,)), (W.H, (0,), ())])
    assert S.sv_plan_circuit(2, S.C64, h, drop_phase_below=1e-3)["gates"] == 2
    for off in (0.0, -1.0, float("nan")):  # no approximation
        assert S.sv_plan_circuit(2, S.C64, h, drop_phase_below=off)["gates"] == 4


def test_plan_recognises_qcrank_multiplexors():
    # a = 8, d = 7: every data qubit's ladder (2^9 gates) becomes one
    # multiplexor; five share a pass.
    a, d = 8, 7
    g = W.qcrank(a, d, np.random.default_rng(0).uniform(0, 1, size=(1 << a, d)))
    info = S.sv_plan_circuit(a + d, S.C64, g)
    assert info["mux_ops"] == d and info["mux_passes"] == 2
    assert info["gates"] == len(g)
    assert info["passes"] == 1 + 2  # the Hadamards, then two multiplexor passes
    off = S.sv_plan_circuit(a + d, S.C64, g, mux=-1)
    # without it the ladders fill two tile passes with over a hundred fused blocks
    assert off["mux_ops"] == 0 and off["dense_ops"] > 100 and info["dense_ops"] <= 2
    # runs shorter than the default threshold stay gates; QFT and random
    # U3 + CX circuits have no runs at all
    small = W.qcrank(2, 2, np.full((4, 2), 0.5))
    assert S.sv_plan_circuit(4, S.C64, small)["mux_ops"] == 0
    assert S.sv_plan_circuit(4, S.C64, small, mux=1)["mux_ops"] == 2
    assert S.sv_plan_circuit(20, S.C64, W.qft(20), mux=1)["mux_ops"] == 0
    assert S.sv_plan_circuit(16, S.C64, W.random_u3_cx(16, 10, 3), mux=1)["mux_ops"] == 0


def test_jit_sources_compile_without_gpu():
    # the run-time compiler writes and compiles (NVRTC, no GPU needed) the
    # kernel of every register-resident pass: Hadamard/phase-table records and
    # diagonal runs (QFT), complex 2x2 records (U3), dense blocks, both dtypes
    try:
        assert S.sv_jit_check(14, S.C64, W.qft(14)) >= 1
    except S.SVError as e:
        if "NVRTC not found" in str(e):
            pytest.skip("NVRTC not installed")
        raise
    assert S.sv_jit_check(18, S.C128, W.qft(18)) >= 1
    assert S.sv_jit_check(12, S.C64, W.random_u3_cx(12, 2, 4)) >= 1
    assert S.sv_jit_check(12, S.C64, W.random_cx_blocks(12, 20, 5), k_max=3) >= 1
