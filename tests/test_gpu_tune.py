"""The project autotuner: the kernel variants it chooses among give the same results (each
within the parity tolerance against the oracle), its choices are persisted to the JSON file
SC_AUTOTUNE_FILE names, and SC_TUNE_<KERNEL> forces a variant."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1708_07481_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    from paper_1708_07481_gb300 import build, sc as S

    build.build()
    return S


def test_autotuner_persists_choices_and_every_variant_matches_the_oracle(sc, tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("SC_AUTOTUNE_FILE", str(path))
    ctx = sc.sc_ctx_create(0)
    try:
        # a shape no other test uses, so its keys are new to this process
        n, K = 3001, 13
        g = W.dcsbm(n, K, seed=31)
        L = O.laplacian_csr(g.n, g.src, g.dst)
        G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
        X0 = W.start_block(9, g.n, K)
        ref = O.lobpcg(L, X0.astype(np.float32).astype(np.float64), 12)
        lmax = O.lambda_max(L)
        lam, _, X, _ = sc.sc_lobpcg(ctx, G, K, iters=12, prec=sc.SC_PREC_MIXED, X0=X0)
        assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-5
        table = json.loads(path.read_text())
        tall = [k for k in table if k.startswith("tall/f32/n2=12/")]
        spmm = [k for k in table if k.startswith("spmm/f32/n2=12/")]
        assert tall and spmm, table
        assert all(v in (0, 1) for k, v in table.items() if k.startswith("tall/"))
        assert all(0 <= v < 13 for k, v in table.items() if k.startswith("spmm/"))
        # every forced variant computes the same iteration
        for tv in ("0", "1"):
            for sv in ("0", "1", "2"):
                monkeypatch.setenv("SC_TUNE_TALL", tv)
                monkeypatch.setenv("SC_TUNE_SPMM", sv)
                lam, _, X, _ = sc.sc_lobpcg(ctx, G, K, iters=12, prec=sc.SC_PREC_MIXED, X0=X0)
                assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-5, (tv, sv)
                assert O.sin_theta(ref.X, X.astype(np.float64)) <= 1e-3, (tv, sv)
    finally:
        ctx.close()
