"""Failure detection without a GPU fault: injected time-outs, an emulated breakdown of the
direction block, and a rank-deficient start block.  Each failure is made on the host (a
bounded device wait that nothing completes, placed after every copy and MMA has finished; a
flag that the Cholesky-QR would clear; an input), and each test checks the reported status and
that the same context then computes correct results."""
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


@pytest.fixture()
def ctx(sc):
    c = sc.sc_ctx_create(0)
    yield c
    c.close()


def test_gram_wait_timeout_reports_etimeout_and_context_survives(sc, ctx):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((4099, 44)).astype(np.float32)
    B = rng.standard_normal((4099, 132)).astype(np.float32)
    sc.sc_debug_inject(ctx, sc.SC_INJECT_WAIT_TIMEOUT, 1000)
    with pytest.raises(sc.ScError) as e:
        sc.sc_gram(ctx, A, B, sc.SC_PREC_MIXED)
    assert e.value.code == sc.SC_ETIMEOUT
    # a LOBPCG solve on the same context meets the same time-out in its first Gram
    g = W.dcsbm(2000, 6, seed=3)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    with pytest.raises(sc.ScError) as e:
        sc.sc_lobpcg(ctx, G, 6, iters=5, prec=sc.SC_PREC_MIXED, seed=1, cold=1)
    assert e.value.code == sc.SC_ETIMEOUT
    # disarmed: the context computes correct results again
    sc.sc_debug_inject(ctx, sc.SC_INJECT_NONE)
    Cm = sc.sc_gram(ctx, A, B, sc.SC_PREC_MIXED)
    ref = A.astype(np.float64).T @ B.astype(np.float64)
    bound = 1e-6 * np.sqrt(A.shape[0]) * np.outer(np.linalg.norm(A, axis=0), np.linalg.norm(B, axis=0))
    assert np.all(np.abs(Cm - ref) <= bound)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    X0 = W.start_block(1, g.n, 6)
    lam, _, X, info = sc.sc_lobpcg(ctx, G, 6, iters=10, prec=sc.SC_PREC_MIXED, X0=X0)
    ref = O.lobpcg(L, X0.astype(np.float32).astype(np.float64), 10)
    assert np.max(np.abs(lam - ref.lam)) / O.lambda_max(L) <= 1e-5


def test_inject_rejects_bad_arguments(sc, ctx):
    for kind, arg in ((7, 0), (sc.SC_INJECT_WAIT_TIMEOUT, 0)):
        with pytest.raises(sc.ScError) as e:
            sc.sc_debug_inject(ctx, kind, arg)
        assert e.value.code == sc.SC_EINVAL


@pytest.mark.parametrize("K", [11, 24])
@pytest.mark.parametrize("prec", [0, 2])
def test_direction_block_breakdown_falls_back_like_the_oracle(sc, ctx, monkeypatch, prec, K):
    """Pass 5 reports its direction block P as broken down: that pass's Rayleigh-Ritz step runs
    on [X R] (one fallback), the next P is R Y_R, and the iteration carries on.  The oracle with
    the same breakdown planted (its Cholesky-QR of P raises at pass 5) gives the same result.
    K = 24 (m = 72) takes the FP64 Rayleigh-Ritz spread over SMs, whose last kernel re-arms
    the breakdown flag."""
    import oracle.spectral as OS

    g = W.dcsbm(3000, K, seed=5)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    X0 = W.start_block(2, g.n, K)
    sc.sc_debug_inject(ctx, sc.SC_INJECT_P_BREAKDOWN, 4)  # the 5th pass (0-based 4)
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, K, iters=12, prec=prec, X0=X0)
    sc.sc_debug_inject(ctx, sc.SC_INJECT_NONE)
    assert info["fallbacks"] == 1 and info["iters_done"] == 12
    # the Cholesky-QR calls made by lobpcg itself: two for the start block, then one for P in
    # each pass from the second on, so pass 5's is call 6 (cholqr_drop's calls for R are not
    # counted)
    import sys

    real = OS.cholqr
    calls = {"n": 0}

    def planted(V):
        if sys._getframe(1).f_code.co_name == "lobpcg":
            calls["n"] += 1
            if calls["n"] == 6:
                raise OS.BreakdownError("planted")
        return real(V)

    monkeypatch.setattr(OS, "cholqr", planted)
    ref = O.lobpcg(L, X0.astype(np.float32).astype(np.float64), 12)
    monkeypatch.setattr(OS, "cholqr", real)
    assert ref.fallbacks == 1
    lmax = O.lambda_max(L)
    tol = 1e-10 if prec == 2 else 1e-5
    assert np.max(np.abs(lam - ref.lam)) / lmax <= tol
    assert O.sin_theta(ref.X, X.astype(np.float64)) <= (1e-6 if prec == 2 else 1e-3)
    # without the planted breakdown the trajectory differs: the fallback took effect
    clean = O.lobpcg(L, X0.astype(np.float32).astype(np.float64), 12)
    assert np.max(np.abs(clean.lam - ref.lam)) / lmax > 1e-8


def test_rank_deficient_start_block_is_a_breakdown_and_context_survives(sc, ctx):
    g = W.dcsbm(2000, 6, seed=4)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    X0 = W.start_block(3, g.n, 6)
    X0[:, 2] = X0[:, 0]  # two equal columns
    for prec in (0, 2):
        with pytest.raises(sc.ScError) as e:
            sc.sc_lobpcg(ctx, G, 6, iters=5, prec=prec, X0=X0)
        assert e.value.code == sc.SC_EBREAKDOWN
    X0 = W.start_block(3, g.n, 6)
    lam, _, _, _ = sc.sc_lobpcg(ctx, G, 6, iters=8, prec=2, X0=X0)
    ref = O.lobpcg(L, X0.astype(np.float32).astype(np.float64), 8)
    assert np.max(np.abs(lam - ref.lam)) / O.lambda_max(L) <= 1e-10
