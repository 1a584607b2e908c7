"""Pins for the FP64 cost-model reference (CPU only): central finite
differences of the loss, the closed-form gradient of a network reduced to a
linear model, Adam's first step (which moves each parameter by lr in the
direction of -sign(g)), and Adam under a constant gradient, where bias
correction makes the corrected moments exactly g and g^2 at every step, so
every step moves each parameter by lr g / (|g| + eps) (Kingma & Ba 2015,
Sec. 3): a missing, constant or mis-indexed correction fails from step 2."""
import numpy as np
import pytest

from oracle import mlp_ref as M


def _params(rng, scale=0.3):
    return rng.standard_normal(M.NPARAMS) * scale


def test_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    X = rng.uniform(0, 1, size=(17, M.F))
    t = rng.standard_normal(17)
    L, g = M.grad(p, X, t)
    assert abs(L - M.loss(p, X, t)) < 1e-14
    idx = rng.choice(M.NPARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [M.NPARAMS - 1, M.NPARAMS - 2]])  # b3, last of w3
    h = 1e-6
    for i in idx:
        e = np.zeros(M.NPARAMS)
        e[i] = h
        fd = (M.loss(p + e, X, t) - M.loss(p - e, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_linear_closed_form():
    """With W2 = I, biases >= 0 keeping every unit active, the network is
    y = w3 . (W1 x + b1) + b2.w3 + b3 and dL/db3 = 2 mean(y - t),
    dL/dw3 = 2 mean((y - t) h2)."""
    rng = np.random.default_rng(1)
    P = M.unpack(_params(rng))
    P = {k: v.copy() for k, v in P.items()}
    P["W1"] = np.abs(P["W1"])
    P["b1"] = np.abs(P["b1"]) + 1.0
    P["W2"] = np.eye(M.H2, M.H1)
    P["b2"] = np.zeros(M.H2)
    p = M.pack(P)
    X = rng.uniform(0, 1, size=(9, M.F))
    t = rng.standard_normal(9)
    h2 = X @ P["W1"].T + P["b1"]
    y = h2 @ P["w3"] + P["b3"][0]
    _, g = M.grad(p, X, t)
    G = M.unpack(g)
    assert np.allclose(G["b3"][0], 2 * np.mean(y - t), rtol=1e-12)
    assert np.allclose(G["w3"], 2 * (h2.T @ (y - t)) / len(t), rtol=1e-12)
    assert np.allclose(G["b2"], 2 * np.mean(y - t) * P["w3"], rtol=1e-12)


def test_adam_first_step():
    rng = np.random.default_rng(2)
    p = _params(rng)
    g = rng.standard_normal(M.NPARAMS)
    z = np.zeros(M.NPARAMS)
    p1, m, v = M.adam(p, g, z, z, 1, lr=1e-3)
    big = np.abs(g) > 1e-2  # where eps = 1e-8 is negligible against |g|
    assert big.sum() > 100
    assert np.allclose((p1 - p)[big], -1e-3 * np.sign(g[big]), rtol=1e-5, atol=0)
    assert np.all(np.abs(p1 - p) <= 1e-3 * (1 + 1e-12))


def _adam_constant_gradient(adam, steps=12, lr=1e-3):
    rng = np.random.default_rng(4)
    p0 = _params(rng)
    g = rng.standard_normal(M.NPARAMS)
    m = np.zeros(M.NPARAMS)
    v = np.zeros(M.NPARAMS)
    p = p0
    for k in range(1, steps + 1):
        p, m, v = adam(p, g, m, v, k, lr=lr)
        # the moments themselves: m_k = (1 - b1^k) g, v_k = (1 - b2^k) g^2
        assert np.allclose(m, (1 - 0.9 ** k) * g, rtol=1e-12, atol=0), k
        assert np.allclose(v, (1 - 0.999 ** k) * g * g, rtol=1e-12, atol=0), k
        # every step moves by lr g / (|g| + eps)
        assert np.allclose(p, p0 - k * lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15), k


def test_adam_constant_gradient():
    _adam_constant_gradient(M.adam)


def _adam_variant(replace_from, replace_to):
    import inspect
    src = inspect.getsource(M.adam)
    assert src.count(replace_from) == 1
    ns = {"np": np}
    exec(src.replace(replace_from, replace_to), ns)
    return ns["adam"]


@pytest.mark.parametrize("mutant", [
    ("mh = m / (1.0 - b1 ** step)", "mh = m / (1.0 - b1)"),          # constant correction
    ("vh = v / (1.0 - b2 ** step)", "vh = v / (1.0 - b2)"),
    ("mh = m / (1.0 - b1 ** step)", "mh = m"),                       # no correction
    ("mh = m / (1.0 - b1 ** step)", "mh = m / (1.0 - b1 ** (step + 1))"),  # off by one step
])
def test_adam_constant_gradient_catches_planted_mistakes(mutant):
    with pytest.raises(AssertionError):
        _adam_constant_gradient(_adam_variant(*mutant))
