"""Helpers for the GPU parity tests: run a circuit through the C ABI and
compare with the FP64 oracle."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2504_03967_gb300 as S

# Bounds (fidelity defect, max amplitude error) per dtype.
TOL = {S.C64: (1e-6, 1e-5), S.C128: (1e-12, 1e-12)}
BAND = 1e-9  # draws this close to a CDF boundary may legitimately differ


def run_gpu(n, gates, dtype, psi0=None, basis=0, **opts):
    h = S.sv_alloc(n, dtype)
    try:
        if psi0 is None:
            S.sv_init_basis(h, basis)
        else:
            S.sv_load_state(h, psi0)
        S.sv_apply_circuit(h, gates, **opts)
        return S.sv_store_state(h).astype(np.complex128)
    finally:
        S.sv_free(h)


def run_oracle(n, gates, psi0=None, basis=0):
    if psi0 is None:
        psi0 = oracle.basis_state(n, basis)
    return oracle.apply_circuit(n, gates, psi0)


def assert_close(got, ref, dtype, what=""):
    fd, ma = TOL[dtype]
    F = oracle.fidelity(got, ref)
    err = oracle.max_abs_err(got, ref)
    assert 1.0 - F <= fd, "%s: 1-F = %.3e > %.1e" % (what, 1.0 - F, fd)
    assert err <= ma, "%s: max |d psi| = %.3e > %.1e" % (what, err, ma)
    return 1.0 - F, err


def compare_samples(got, u, cdf_ref, band):
    """Outcomes must equal min{x : C_x > u S} except for draws within band of
    a CDF boundary.  Returns (compared, skipped)."""
    S_ = cdf_ref[-1]
    t = u * S_
    x0 = np.searchsorted(cdf_ref, t, side="right")
    x0 = np.minimum(x0, len(cdf_ref) - 1)
    hi = cdf_ref[x0] - t
    lo = t - np.where(x0 > 0, cdf_ref[np.maximum(x0 - 1, 0)], -np.inf)
    near = np.minimum(hi, lo) < band
    ok = (got == x0) | near
    bad = np.nonzero(~ok)[0]
    assert len(bad) == 0, "sample mismatch at shots %s: got %s want %s" % (bad[:5], got[bad[:5]], x0[bad[:5]])
    return int((~near).sum()), int(near.sum())
