"""Autotuner: the chosen options are one of the candidates, reproduce the
oracle's state, and are served from the JSON-lines cache on the next call."""
import json

import numpy as np
import pytest

import paper_2504_03967_gb300 as S
import workloads as W
from paper_2504_03967_gb300 import build as B
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    yield


@pytest.mark.parametrize("dtype", [S.C64, S.C128], ids=["c64", "c128"])
def test_autotune_choice_and_cache(dtype, tmp_path):
    n = 16
    g = W.random_u3_cx(n, 4, 31)
    cache = str(tmp_path / "tune.jsonl")
    h = S.sv_alloc(n, dtype)
    try:
        opts, ms = S.sv_autotune(h, g, cache)
        assert 2 <= opts["k_max"] <= 5 and ms > 0
        lo = 11 if dtype == S.C64 else 10
        assert lo <= opts["tile_m"] <= lo + 3
        assert opts["tensor"] in (-1, 1)
        if dtype == S.C128:
            assert opts["tensor"] == -1
        lines = open(cache).read().strip().splitlines()
        assert len(lines) == 1
        rec = json.loads(lines[0])
        assert (rec["k_max"], rec["tile_m"], rec["tensor"], rec["pass_kernel"]) == (
            opts["k_max"], opts["tile_m"], opts["tensor"], opts["pass_kernel"])
        # second call: served from the file, nothing appended
        opts2, ms2 = S.sv_autotune(h, g, cache)
        assert opts2 == opts and abs(ms2 - ms) < 1e-3
        assert len(open(cache).read().strip().splitlines()) == 1
        # the tuned plan is exact
        psi0 = W.random_state(n, 3)
        S.sv_load_state(h, psi0)
        S.sv_apply_circuit(h, g, **opts)
        got = S.sv_store_state(h).astype(np.complex128)
        U.assert_close(got, U.run_oracle(n, g, psi0), dtype, "autotuned plan")
    finally:
        S.sv_free(h)


def test_autotune_rejects_invalid_records():
    h = S.sv_alloc(6, S.C64)
    try:
        bad = W.gates_from_list([(W.H, (7,), ())])
        with pytest.raises(S.SVError):
            S.sv_autotune(h, bad)
    finally:
        S.sv_free(h)
