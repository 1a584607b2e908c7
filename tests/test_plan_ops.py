"""The fused plan itself, checked on the CPU: the ops the greedy planner
builds (dense blocks, gate sequences with their phase tables, phase runs;
sv_plan_ops, FP64, before the device encoding) are applied here in numpy,
op by op, and the result must equal the oracle's gate-by-gate state to FP64
rounding.  This pins the planner's exact rewrites without a GPU: grouping a
pass's gates by qubit set, phase tables kept pending past gates they commute
with and moved through CX / SWAP, U3 = P(phi) RY(theta) P(lambda), diagonal
gates folded into blocks or runs (App. D.2 "gate fusion", Eq. "cr1"), and
runs recognised as multiplexors (QCrank, App. D.3)."""
import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests.oracle_pins import random_mixed_circuit


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    yield


def _block(psi, n, qubits, mat):
    """Apply a 2^k x 2^k matrix (block bit i <-> qubits[i]) to psi."""
    k = len(qubits)
    offs = np.zeros(1 << k, dtype=np.int64)
    for j in range(1 << k):
        for i, q in enumerate(qubits):
            if (j >> i) & 1:
                offs[j] |= 1 << q
    idx = np.arange(1 << n)
    mask = 0
    for q in qubits:
        mask |= 1 << q
    bases = idx[(idx & mask) == 0]
    sel = bases[:, None] + offs[None, :]
    psi[sel] = psi[sel] @ np.asarray(mat).T
    return psi


def _apply_ops(n, ops, psi):
    psi = psi.astype(np.complex128).copy()
    idx = np.arange(1 << n)
    bits = (idx[:, None] >> np.arange(n)[None, :]) & 1
    for op in ops:
        qs = op["qubits"]
        if op["kind"] == "dense":
            psi = _block(psi, n, qs, op["mat"])
        elif op["kind"] == "diag":
            ph = op["c"] + bits @ op["a"] + np.einsum("ip,pq,iq->i", bits, np.triu(op["b"], 1), bits)
            psi *= np.exp(1j * ph)
        elif op["kind"] == "gates":
            vals = op["vals"]
            jblk = np.zeros(1 << n, dtype=np.int64)
            for i, q in enumerate(qs):
                jblk |= ((idx >> q) & 1) << i
            for rk, a, b, off in op["recs"]:
                if rk in (0, 1):
                    psi = _block(psi, n, [qs[a]], vals[off:off + 4].reshape(2, 2))
                elif rk == 2:
                    psi *= vals[off + jblk]
                elif rk == 3:
                    c, t = qs[a], qs[b]
                    src = np.where((idx >> c) & 1, idx ^ (1 << t), idx)
                    psi = psi[src]
                elif rk == 4:
                    p, q = qs[a], qs[b]
                    diff = ((idx >> p) ^ (idx >> q)) & 1
                    psi = psi[np.where(diff == 1, idx ^ (1 << p) ^ (1 << q), idx)]
                else:
                    raise AssertionError("unknown record kind %d" % rk)
        else:  # multiplexor: U_j = X^(popcount(j & flip) ^ flip_c) R_j on the target
            t = op["target"]
            i0 = idx[((idx >> t) & 1) == 0]
            i1 = i0 | (1 << t)
            j = np.zeros(len(i0), dtype=np.int64)
            for b, c in enumerate(op["controls"]):
                j |= ((i0 >> c) & 1) << b
            a0, a1 = psi[i0].copy(), psi[i1].copy()
            if op["family"] == "ry":
                cs, sn = np.cos(op["phi0"][j] / 2), np.sin(op["phi0"][j] / 2)
                y0, y1 = cs * a0 - sn * a1, sn * a0 + cs * a1
            else:
                y0, y1 = np.exp(1j * op["phi0"][j]) * a0, np.exp(1j * op["phi1"][j]) * a1
            par = np.array([bin(v).count("1") & 1 for v in (j & op["flip"])]) ^ op["flip_c"]
            psi[i0] = np.where(par == 1, y1, y0)
            psi[i1] = np.where(par == 1, y0, y1)
    return psi


CASES = {
    "random-u3cx": lambda: (11, W.random_u3_cx(11, 12, 3)),
    "qft": lambda: (10, W.qft(10)),
    "cx-blocks": lambda: (10, W.random_cx_blocks(10, 120, 5)),
    "ansatz": lambda: (10, W.hea(10, 4, W.hea_params(1, 10, 4, 9)[0])),
    "mixed": lambda: (9, random_mixed_circuit(9, 160, np.random.default_rng(4))),
}


@pytest.mark.parametrize("k,tile_m", [(5, 7), (3, 7), (5, 9), (2, 6)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_plan_ops_reproduce_the_circuit(case, k, tile_m):
    n, g = CASES[case]()
    ops = S.sv_plan_ops(n, S.C64, g, k_max=k, tile_m=tile_m)
    assert ops and (tile_m >= n or max(op["pass"] for op in ops) >= 1)  # several passes
    rng = np.random.default_rng(n + k)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    got = _apply_ops(n, ops, psi0)
    want = oracle.apply_circuit(n, g, psi0)
    assert np.abs(got - want).max() < 1e-12, (case, np.abs(got - want).max())


@pytest.mark.parametrize("case", ["random-u3cx", "mixed", "qft"])
@pytest.mark.parametrize("dtype,pass_kernel", [(S.C128, 0), (S.C64, 1)], ids=["c128", "c64-smem-kernel"])
def test_plan_ops_other_dtype_and_kernel(case, dtype, pass_kernel):
    """complex128 plans (4-qubit blocks by default) and plans for the
    shared-memory kernel (wide blocks may stay dense) reproduce the circuit."""
    n, g = CASES[case]()
    ops = S.sv_plan_ops(n, dtype, g, tile_m=7, pass_kernel=pass_kernel)
    if dtype == S.C128:
        assert max(len(op["qubits"]) for op in ops) <= 4
    rng = np.random.default_rng(3)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    got = _apply_ops(n, ops, psi0)
    assert np.abs(got - oracle.apply_circuit(n, g, psi0)).max() < 1e-12


def test_phase_tables_depend_only_on_their_mask():
    """Compiled passes read entry j of a phase table as entry j & a: every
    table must satisfy that exactly."""
    n, g = CASES["random-u3cx"]()
    seen = 0
    for op in S.sv_plan_ops(n, S.C64, g, k_max=5, tile_m=9):
        if op["kind"] != "gates":
            continue
        for rk, a, _, off in op["recs"]:
            if rk != 2:
                continue
            t = op["vals"][off: off + (1 << len(op["qubits"]))]
            j = np.arange(len(t))
            assert np.array_equal(t, t[j & a])
            seen += 1
    assert seen > 0


def test_u3_blocks_take_the_p_ry_p_form():
    """Random U3+CX blocks come out as real rotations and phase tables, with
    fewer tables than rotations (phases wait past gates they commute with)."""
    n, g = CASES["random-u3cx"]()
    kinds = np.concatenate([op["recs"][:, 0] for op in S.sv_plan_ops(n, S.C64, g, k_max=5, tile_m=9)
                            if op["kind"] == "gates"])
    ur, dt, u = (kinds == 1).sum(), (kinds == 2).sum(), (kinds == 0).sum()
    assert ur >= 0.9 * (g["type"] == W.U3).sum() and u == 0
    assert 0 < dt < ur


def test_dropped_rotations_are_the_near_identity_ones():
    """drop_phase_below leaves out P, RZ and CP gates within eps of the
    identity: angles near 0 or 2 pi for P and CP, near 0 or 4 pi for RZ
    (RZ(2 pi) = -I stays).  The plan equals the oracle run of the kept gates."""
    eps = 1e-6
    items = [(W.H, (q,), ()) for q in range(4)]
    items += [(W.P, (0,), (5e-7,)), (W.P, (1,), (2 * np.pi - 5e-7,)), (W.CP, (0, 1), (-3e-7,)),
              (W.RZ, (2,), (4 * np.pi - 2e-7,)), (W.RZ, (3,), (2 * np.pi - 2e-7,)), (W.RZ, (1,), (0.3,)),
              (W.CP, (2, 3), (2e-6,))]
    g = W.gates_from_list(items)
    kept = W.gates_from_list([items[i] for i in (0, 1, 2, 3, 8, 9, 10)])
    ops = S.sv_plan_ops(4, S.C64, g, drop_phase_below=eps)
    psi0 = oracle.basis_state(4, 0)
    got = _apply_ops(4, ops, psi0)
    assert np.abs(got - oracle.apply_circuit(4, kept, psi0)).max() < 1e-12
    assert np.abs(got - oracle.apply_circuit(4, g, psi0)).max() < 1e-6  # within the dropped angles


def test_plan_ops_arguments():
    with pytest.raises(S.SVError):
        S.sv_plan_ops(0, S.C64, W.qft(3))
    with pytest.raises(S.SVError):
        S.sv_plan_ops(4, S.C64, W.gates_from_list([(W.H, (4,), ())]))
    assert S.sv_plan_ops(4, S.C64, W.gates_from_list([])) == []


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_multiplexors_reproduce_the_circuit(seed):
    """Runs of both recognised families (RY with X and CX from scattered
    controls; RZ, P, Z, X and CX), interleaved with gates that commute with
    them, become multiplexors whose angles (one Walsh-Hadamard transform of
    the run's angles, QCrank's uniformly controlled rotations, App. D.3) reproduce the
    oracle's gate-by-gate state."""
    from tests.test_mux_gpu import _ladder_mix

    g = _ladder_mix(seed)
    ops = S.sv_plan_ops(10, S.C64, g, mux=1)
    fams = sorted(op["family"] for op in ops if op["kind"] == "mux")
    assert "ry" in fams and "diag" in fams
    rng = np.random.default_rng(seed)
    psi0 = rng.normal(size=1 << 10) + 1j * rng.normal(size=1 << 10)
    psi0 /= np.linalg.norm(psi0)
    got = _apply_ops(10, ops, psi0)
    assert np.abs(got - oracle.apply_circuit(10, g, psi0)).max() < 1e-12


def test_plan_ops_name_the_multiplexor_targets():
    """A QCrank circuit (a address qubits in superposition, d data qubits
    under uniformly controlled RY) plans as Hadamard blocks plus one
    multiplexor per data qubit."""
    a, d = 8, 6
    pix = np.random.default_rng(1).uniform(0, 1, size=(1 << a, d))
    ops = S.sv_plan_ops(a + d, S.C64, W.qcrank(a, d, pix), mux=1)
    assert sorted(op["target"] for op in ops if op["kind"] == "mux") == list(range(a, a + d))
    assert all(op["kind"] in ("mux", "gates", "dense") for op in ops)
    psi0 = np.zeros(1 << (a + d), dtype=complex)
    psi0[0] = 1.0
    got = _apply_ops(a + d, ops, psi0)
    assert np.abs(got - oracle.apply_circuit(a + d, W.qcrank(a, d, pix), psi0)).max() < 1e-12


@pytest.mark.parametrize("case", ["random", "qft", "cx-blocks"])
@pytest.mark.parametrize("tile_m", [12, 13])
def test_tensor_core_plans_reproduce_the_circuit(case, tile_m):
    """Plans with tensor-core blocks (tensor = 1: every 4- and 5-qubit block
    dense, with no cap on its gate count) reproduce the circuit in FP64."""
    n = 14
    g = {"random": lambda: W.random_u3_cx(n, 10, 7), "qft": lambda: W.qft(n),
         "cx-blocks": lambda: W.random_cx_blocks(n, 200, 8)}[case]()
    info = S.sv_plan_circuit(n, S.C64, g, k_max=5, tile_m=tile_m, tensor=1)
    assert info["tc_ops"] > 0
    ops = S.sv_plan_ops(n, S.C64, g, k_max=5, tile_m=tile_m, tensor=1)
    rng = np.random.default_rng(tile_m)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    got = _apply_ops(n, ops, psi0)
    assert np.abs(got - oracle.apply_circuit(n, g, psi0)).max() < 1e-12


def test_register_layouts_keep_some_remaps_within_warps():
    """Host plan summary of the register passes' layouts (no GPU): on random
    U3+CX circuits some remaps keep every warp's amplitudes within the warp
    (ordered by warp barriers), never all of them (a pass's first layout and
    blocks whose qubits sit at warp bits need the block), and the CUDA-core
    default plans every pass register-resident."""
    for n, m in ((20, 12), (22, 13), (24, 13)):
        g = W.random_u3_cx(n, 12, 60 + n)
        info = S.sv_plan_circuit(n, S.C64, g, k_max=5, tile_m=m)
        assert info["reg_passes"] == info["passes"]
        assert info["tc_ops"] == 0  # CUDA cores by default
        assert info["remaps"] >= info["passes"]  # every register pass starts with one
        assert 0 < info["warp_remaps"] <= info["remaps"] - info["passes"]
