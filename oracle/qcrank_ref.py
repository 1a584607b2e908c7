"""QCrank read-out in FP64, written out plainly (test infrastructure only:
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use it; the
product never does).

QCrank (Sec. 3 image encoding, App. D.3, Table 2; the encoding of Balewski et al. that the paper
cites) writes data qubit k of address j with a rotation RY(theta_jk) behind
a uniform superposition over the a address qubits.  Hence

    P(data_k = 1 | address = j) = sin^2(theta_jk / 2),

and with theta = pi * pixel (pixels in [0, 1]) the image comes back as

    pixel_jk = (2 / pi) * arcsin(sqrt(P(1 | j))).

From shots, P(1 | j) is the fraction of the shots that landed on address j
with data bit k set.  Table 2 draws s = 3000 shots per address (s * 2^a in
all).  Address qubits are bits 0 .. a-1 of an outcome, data qubit k is bit
a + k.  An address that drew no shot has no estimate (NaN).
"""
from __future__ import annotations

import numpy as np


def decode_counts(samples, a, d):
    """Per address j: shots at j, and per data qubit k the shots at j with
    bit a + k set.  Returns (counts[2^a], ones[2^a, d]) as int64."""
    x = np.asarray(samples, dtype=np.uint64)
    j = (x & np.uint64((1 << a) - 1)).astype(np.int64)
    counts = np.bincount(j, minlength=1 << a).astype(np.int64)
    ones = np.zeros((1 << a, d), dtype=np.int64)
    for k in range(d):
        bit = ((x >> np.uint64(a + k)) & np.uint64(1)).astype(bool)
        ones[:, k] = np.bincount(j[bit], minlength=1 << a)
    return counts, ones


def pixels_from_counts(counts, ones):
    """pixel = (2/pi) arcsin sqrt(ones / counts); NaN where counts == 0."""
    counts = np.asarray(counts, dtype=np.float64)
    ones = np.asarray(ones, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        p = ones / counts[:, None]
    return (2.0 / np.pi) * np.arcsin(np.sqrt(p))


def decode(samples, a, d):
    counts, ones = decode_counts(samples, a, d)
    return pixels_from_counts(counts, ones), counts, ones


def pixels_from_probs(probs, a, d):
    """The same read-out with exact probabilities (infinitely many shots):
    probs is the 2^(a+d) outcome distribution."""
    p = np.asarray(probs, dtype=np.float64).reshape(1 << d, 1 << a)  # [data bits, address]
    addr = p.sum(axis=0)
    out = np.empty((1 << a, d))
    for k in range(d):
        sel = ((np.arange(1 << d) >> k) & 1).astype(bool)
        out[:, k] = (2.0 / np.pi) * np.arcsin(np.sqrt(np.clip(p[sel].sum(axis=0) / addr, 0.0, 1.0)))
    return out


def correlation(x, y):
    """Pearson correlation of two pixel sets (entries where both are finite)."""
    x = np.asarray(x, dtype=np.float64).ravel()
    y = np.asarray(y, dtype=np.float64).ravel()
    ok = np.isfinite(x) & np.isfinite(y)
    x, y = x[ok] - x[ok].mean(), y[ok] - y[ok].mean()
    return float((x * y).sum() / np.sqrt((x * x).sum() * (y * y).sum()))
