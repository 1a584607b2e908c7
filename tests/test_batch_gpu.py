"""Batched execution (sv_batch_run) against the oracle, circuit by circuit:
uneven sizes spanning the shared-memory path (n <= 13 / 12) and the tile-pass
path, QCrank image-encoding circuits (config-3 shape at reduced size) and
variational-ansatz parameter sets (config-5 shape)."""

import numpy as np
import pytest

import oracle
import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    oracle.set_threads(8)
    yield


def _check_expz(ez, circuits, dtype):
    tol = 1e-5 if dtype == S.C64 else 1e-12
    for c, (n, g) in enumerate(circuits):
        ref = oracle.expect_z(oracle.apply_circuit(n, g))
        assert np.abs(ez[c, :n] - ref).max() <= tol, (c, n)


def _check_samples(samp, circuits, seed, dtype):
    for c, (n, g) in enumerate(circuits):
        psi = oracle.apply_circuit(n, g)
        cref = oracle.cdf(oracle.probs(psi))
        u = oracle.uniforms(seed + c, samp.shape[1])
        band = U.BAND if dtype == S.C128 else 2e-5
        U.compare_samples(samp[c], u, cref, band)


@pytest.mark.parametrize("dtype", [S.C64, S.C128], ids=["c64", "c128"])
def test_batch_uneven_random(dtype):
    rng = np.random.default_rng(7)
    circuits = []
    for c in range(24):
        n = int(rng.integers(3, 17))
        circuits.append((n, W.random_u3_cx(n, 3, 100 + c)))
    circuits.append((1, W.gates_from_list([(W.RY, (0,), (1.1,))])))
    circuits.append((5, np.zeros(0, dtype=W.GATE_DTYPE)))  # empty circuit
    seed = 77
    samp, ez = S.sv_batch_run(circuits, dtype=dtype, shots=2000, seed=seed)
    _check_expz(ez, circuits, dtype)
    _check_samples(samp, circuits, seed, dtype)


def test_batch_qcrank_closed_form():
    """Config-3 shape at reduced size: a ~ U{3..6}, d ~ U{2..4}; the data
    qubits' conditional probabilities from the shots match
    sin^2(pi pixel / 2) (the closed form that pins the generator)."""
    batch = W.qcrank_batch(12, 31, a_range=(3, 6), d_range=(2, 4))
    circuits = [(a + d, W.qcrank(a, d, pix)) for a, d, pix in batch]
    shots = 20000
    samp, ez = S.sv_batch_run(circuits, dtype=S.C64, shots=shots, seed=5)
    _check_expz(ez, circuits, S.C64)
    for (a, d, pix), s in zip(batch, samp):
        s = s.astype(np.int64)
        addr = s & ((1 << a) - 1)
        for k in range(d):
            bit = (s >> (a + k)) & 1
            for j in range(1 << a):
                sel = addr == j
                if sel.sum() > 200:
                    p1 = bit[sel].mean()
                    assert abs(p1 - np.sin(np.pi * pix[j, k] / 2) ** 2) < 5.0 / np.sqrt(sel.sum())


def test_batch_variational_sweep():
    """Config-5 shape at reduced size: HEA, 8 layers, many parameter sets,
    <Z_i> for every qubit."""
    n, layers = 10, 8
    params = W.hea_params(40, n, layers, W.SEED[5])
    circuits = [(n, W.hea(n, layers, params[s])) for s in range(len(params))]
    _, ez = S.sv_batch_run(circuits, dtype=S.C64, shots=0)
    _check_expz(ez, circuits, S.C64)


@pytest.mark.parametrize("count,a_max", [(64, 10), (512, 14)], ids=["64x-a10", "512x-a14"])
def test_batch_qcrank_full_size(count, a_max):
    """Config-3 shape: QCrank circuits with a ~ U{8..a_max}, d ~ U{4..10},
    10^5 shots each, complex64, one call (the full batch: 512 circuits up to
    24 qubits, 37.5 M gates, seconds with the multiplexor passes).  Pinned: every circuit's <Z> of the data qubits against
    the closed form mean_j cos(pi pixel_jk) and of the address qubits against
    0 (uniform addresses), the data marginals from the shots of sampled
    circuits, and exact <Z> against the oracle on the smallest circuits."""
    batch = W.qcrank_batch(count, W.SEED[3], a_range=(8, a_max))
    circuits = [(a + d, W.qcrank(a, d, pix)) for a, d, pix in batch]
    shots = 100000
    samp, ez = S.sv_batch_run(circuits, dtype=S.C64, shots=shots, seed=31)
    assert samp.shape == (count, shots)
    # <Z_data_k> = mean over addresses of cos(pi pixel) for every circuit
    for c, (a, d, pix) in enumerate(batch):
        want = np.cos(np.pi * pix).mean(axis=0)
        assert np.abs(ez[c, a:a + d] - want).max() < 1e-5, c
        assert np.abs(ez[c, :a]).max() < 1e-5, c  # address qubits stay uniform
    # shots of a few circuits against their closed-form data marginals
    for c in range(0, count, max(1, count // 5)):
        a, d, pix = batch[c]
        s = samp[c].astype(np.int64)
        for k in range(d):
            p1 = ((s >> (a + k)) & 1).mean()
            want = (np.sin(np.pi * pix[:, k] / 2) ** 2).mean()
            assert abs(p1 - want) < 5.0 / np.sqrt(shots), (c, k)
    # exact <Z> against the oracle on the smallest circuits
    small = sorted(range(count), key=lambda c: circuits[c][0])[:4]
    _check_expz(ez[small], [circuits[c] for c in small], S.C64)


def test_batch_variational_full_size():
    """Config-5 sizes: hardware-efficient ansatz at n = 20, 8 layers, 4096
    parameter sets in one call (large-circuit path), <Z_i> for every qubit;
    32 sampled sets against the oracle."""
    n, layers = 20, 8
    params = W.hea_params(4096, n, layers, W.SEED[5])
    circuits = [(n, W.hea(n, layers, params[s])) for s in range(len(params))]
    _, ez = S.sv_batch_run(circuits, dtype=S.C64, shots=0)
    assert ez.shape[0] == 4096
    pick = np.random.default_rng(3).choice(4096, 32, replace=False)
    _check_expz(ez[pick], [circuits[c] for c in pick], S.C64)
