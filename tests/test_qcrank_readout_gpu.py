"""QCrank read-out on the device (Sec. 3 image encoding, App. D.3, Table 2) against the oracle's
decoding of the same shots: counts bit-exact, pixels to FP64 rounding; and
against the image itself through the shot-noise law (pixel error variance
1 / (pi^2 s) with s shots per address) and the reconstruction correlation."""
import numpy as np
import pytest

import paper_2504_03967_gb300 as S
import workloads as W
from oracle import qcrank_ref as Q
from paper_2504_03967_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    yield


def _encoded(a, d, dtype, seed, lo=0.1, hi=0.9):
    pix = np.random.default_rng(seed).uniform(lo, hi, size=(1 << a, d))
    h = S.sv_alloc(a + d, dtype)
    S.sv_init_basis(h, 0)
    S.sv_apply_circuit(h, W.qcrank(a, d, pix))
    return h, pix


def _same_pixels(got, want):
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.abs(got[ok] - want[ok]).max(initial=0.0) <= 4e-16


@pytest.mark.parametrize("dtype", [S.C64, S.C128], ids=["c64", "c128"])
@pytest.mark.parametrize("a,d", [(6, 3), (9, 5)])
def test_reconstruct_vs_oracle_decode(dtype, a, d):
    s = 3000
    h, pix = _encoded(a, d, dtype, 50 + a)
    try:
        shots = s << a
        got, counts = S.sv_qcrank_reconstruct(h, a, d, shots, 17)
        samples = S.sv_sample(h, shots, 17)  # the same shots
    finally:
        S.sv_free(h)
    want, wc, _ = Q.decode(samples, a, d)
    assert np.array_equal(counts.astype(np.int64), wc)
    _same_pixels(got, want)
    mse = np.mean((got - pix) ** 2)
    law = 1.0 / (np.pi ** 2 * s)
    assert 0.7 * law < mse < 1.3 * law, (mse, law)
    assert Q.correlation(got, pix) > 0.999


@pytest.mark.parametrize("a,d,shots", [(3, 2, 5), (10, 6, 200000), (13, 12, 300000), (1, 1, 0)],
                         ids=["sparse", "smem-histogram", "global-histogram", "no-shots"])
def test_decode_device_buffers(a, d, shots):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(a * 100 + d)
    x = rng.integers(0, 1 << 62, size=max(shots, 1), dtype=np.int64)[:shots].astype(np.uint64)
    dx = torch.from_numpy(x.view(np.int64)).cuda() if shots else torch.zeros(1, dtype=torch.int64, device="cuda")
    counts = torch.full((1 << a,), 7, dtype=torch.int64, device="cuda")  # overwritten
    ones = torch.full(((1 << a) * d,), 7, dtype=torch.int64, device="cuda")
    pixels = torch.zeros((1 << a) * d, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    S.sv_qcrank_decode_device(dx.data_ptr(), shots, a, d, counts.data_ptr(), ones.data_ptr(), pixels.data_ptr(), st)
    torch.cuda.synchronize()
    want, wc, wo = Q.decode(x, a, d)
    assert np.array_equal(counts.cpu().numpy(), wc)
    assert np.array_equal(ones.cpu().numpy().reshape(1 << a, d), wo)
    _same_pixels(pixels.cpu().numpy().reshape(1 << a, d), want)


def test_decode_rejects_bad_arguments():
    with pytest.raises(S.SVError):
        S.sv_qcrank_decode_device(0, 0, 0, 1, 0, 0, 0)
    h = S.sv_alloc(6, S.C64)
    try:
        S.sv_init_basis(h, 0)
        with pytest.raises(S.SVError):
            S.sv_qcrank_reconstruct(h, 4, 3, 100, 1)  # a + d > n
    finally:
        S.sv_free(h)


def test_table2_zebra_a14_d6():
    """Table 2's largest-shot row at a = 14: 384 x 256 pixels as 2^14 x 6,
    3000 * 2^14 = 49 M shots drawn and decoded on the device (complex64)."""
    a, d, s = 14, 6, 3000
    h, pix = _encoded(a, d, S.C64, 5)
    try:
        got, counts = S.sv_qcrank_reconstruct(h, a, d, s << a, 23)
        samples = S.sv_sample(h, s << a, 23)
    finally:
        S.sv_free(h)
    assert int(counts.sum()) == s << a
    want, wc, _ = Q.decode(samples, a, d)
    assert np.array_equal(counts.astype(np.int64), wc)
    _same_pixels(got, want)
    mse = np.mean((got - pix) ** 2)
    law = 1.0 / (np.pi ** 2 * s)
    assert 0.9 * law < mse < 1.1 * law, (mse, law)
    assert Q.correlation(got, pix) > 0.999
