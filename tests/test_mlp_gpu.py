"""The learned cost model on the GPU.

- gradient and Adam kernels against the FP64 reference (oracle/mlp_ref.py);
- training on recorded pass timings lowers the loss;
- the cost-model planner (SV_PLAN_MLP) picks plans that run no slower than
  the greedy fixed-width plan on held-out circuits (timing noise aside), its
  results stay within the oracle bounds, and the judge records its decisions.
"""
import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from oracle import mlp_ref as M
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    yield


def test_gradient_matches_fp64_reference():
    assert S.sv_mlp_param_count() == M.NPARAMS
    rng = np.random.default_rng(3)
    p = (rng.standard_normal(M.NPARAMS) * 0.2).astype(np.float32)
    X = rng.uniform(0, 1, size=(96, M.F)).astype(np.float32)
    t = rng.standard_normal(96).astype(np.float32)
    loss_gpu, g_gpu = S.sv_mlp_gradient(p, X, t)
    loss_ref, g_ref = M.grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss_gpu - loss_ref) <= 1e-5 * max(1.0, loss_ref)
    scale = np.abs(g_ref).max()
    assert np.abs(g_gpu - g_ref).max() <= 1e-4 * scale, np.abs(g_gpu - g_ref).max() / scale


def test_adam_matches_fp64_reference():
    rng = np.random.default_rng(4)
    p = rng.standard_normal(M.NPARAMS).astype(np.float32)
    g = rng.standard_normal(M.NPARAMS).astype(np.float32)
    got = S.sv_mlp_adam(p, g, 5, 1e-3)
    ref, m, v = p.astype(np.float64), np.zeros(M.NPARAMS), np.zeros(M.NPARAMS)
    for step in range(1, 6):
        ref, m, v = M.adam(ref, g.astype(np.float64), m, v, step, 1e-3)
    assert np.abs(got - ref).max() <= 1e-6


def test_training_fits_a_smooth_target(tmp_path):
    rng = np.random.default_rng(5)
    X = rng.uniform(0, 1, size=(512, M.F)).astype(np.float32)
    ms = np.exp(1.5 * X[:, 0] - 0.7 * X[:, 3] + 0.4 * X[:, 5] * X[:, 6])
    loss = S.sv_cost_model_train(X, ms, epochs=1500, lr=3e-3, seed=1, weights_path=str(tmp_path / "m.bin"))
    assert loss < 0.05, loss
    pred = S.sv_cost_model_predict(X[:64])
    assert np.abs(np.log(pred) - np.log(ms[:64])).max() < 0.6
    S.sv_cost_model_unload()
    assert not S.sv_cost_model_loaded()
    S.sv_cost_model_load(str(tmp_path / "m.bin"))
    assert np.allclose(S.sv_cost_model_predict(X[:64]), pred, rtol=1e-6)
    S.sv_cost_model_unload()


CANDS = [(k, m, t) for k in (4, 5) for m in (12, 13, 14) for t in (-1, 1)]


def record_timings(h, n, g):
    """Pass timings of the run-time compiled passes (the kernels the library
    runs) for every candidate; each candidate's first apply compiles."""
    feats, times = [], []
    for k, m, t in CANDS:
        for rec in (0, 1):
            S.sv_init_basis(h, 1)
            S.sv_apply_circuit(h, g, k_max=k, tile_m=m, tensor=t, record=rec, jit=1)
        ms, f = S.sv_pass_times(h, features=True)
        feats.append(f)
        times.append(ms)
    return np.concatenate(feats), np.concatenate(times)


def timed(h, g, **kw):
    """Best of five applies on the compiled passes (compiles done first)."""
    import torch
    kw.setdefault("jit", 1)
    S.sv_init_basis(h, 1)
    S.sv_apply_circuit(h, g, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 1e30
    for _ in range(5):
        S.sv_init_basis(h, 1)
        torch.cuda.synchronize()
        e0.record()
        S.sv_apply_circuit(h, g, **kw)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def test_cost_model_planner_beats_greedy(tmp_path):
    """Trained on compiled-pass timings of other circuits, the cost-model
    planner (its per-pass plan, the model's best whole-circuit candidates and
    the greedy plan, judged by measured time on the first calls) runs held-out
    circuits no slower than the greedy fixed-width plan (within timing noise),
    within the oracle's bounds."""
    pytest.importorskip("torch")
    n = 22
    h = S.sv_alloc(n, S.C64)
    try:
        train = [W.random_u3_cx(n, 5, 11), W.qft(n), W.random_cx_blocks(n, 200, 12),
                 W.hea(n, 3, W.hea_params(1, n, 3, 13)[0])]
        F, T = [], []
        for g in train:
            f, t = record_timings(h, n, g)
            F.append(f)
            T.append(t)
        F, T = np.concatenate(F), np.concatenate(T)
        assert len(T) > 200
        loss = S.sv_cost_model_train(F, T, epochs=3000, lr=3e-3, seed=2)
        assert loss < 0.2, loss
        held_out = [W.random_u3_cx(n, 12, 21), W.random_cx_blocks(n, 300, 22)]
        gains = []
        st0 = S.sv_cost_model_stats()
        for g in held_out:
            for _ in range(9):  # the judge times its four trials twice on the first calls
                S.sv_init_basis(h, 0)
                S.sv_apply_circuit(h, g, planner=S.PLAN_MLP, jit=1)
            # the learned plan's results stay within the complex64 bounds
            U.assert_close(S.sv_store_state(h).astype(np.complex128), oracle.apply_circuit(n, g), S.C64, "mlp plan")
            t_mlp = timed(h, g, planner=S.PLAN_MLP)
            t_greedy = timed(h, g)  # greedy fixed width k = 5 (the paper's fusion setting), default tile
            gains.append(t_greedy / t_mlp)
        st = S.sv_cost_model_stats()
        assert st["planned"] - st0["planned"] == len(held_out)
        # the judged plan against the greedy fixed-width plan: the judge keeps
        # greedy unless a trial beat it by more than 1%, so the kept plan is
        # never slower beyond the timings' noise, and faster where the model
        # found a better plan
        assert min(gains) > 0.97 and np.mean(gains) > 0.98, gains
    finally:
        S.sv_free(h)
        S.sv_cost_model_unload()
