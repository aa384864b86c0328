"""Lockstep batches (GPU): FP32 mixed-precision runs with one fixed pass count advance
together, each pass's Cholesky-QR transforms, SpMM and Rayleigh-Ritz solves going out as one
launch per kernel shape for the whole batch, and the batch pass replayed from a CUDA graph.
The sizes cover every batched kernel shape: Rayleigh-Ritz m = 36 (register-resident), 150
(register-slot, global working set), 210 and 360 (cluster tridiagonalization); Cholesky-QR of
24 and 100 columns (register form), 140 (shared memory) and 240 (global memory).  Every run's
results are bitwise its single-run results and the round-robin batch's."""
import numpy as np
import pytest

from paper_1708_07481_gb300 import workload as W

pytestmark = pytest.mark.gpu

SPECS = [(2000, 12, 1), (2600, 50, 2), (3000, 70, 3), (4000, 120, 4)]


@pytest.fixture(scope="module")
def sc():
    from paper_1708_07481_gb300 import build, sc as S

    build.build()
    return S


@pytest.fixture(scope="module")
def ctx(sc):
    c = sc.sc_ctx_create(0)
    yield c
    c.close()


def test_lockstep_batch_is_bitwise_single_and_round_robin(sc, ctx, monkeypatch):
    gs = [W.dcsbm(n, K, seed=s) for n, K, s in SPECS]
    Gs = [sc.sc_build_laplacian(ctx, g.n, g.src, g.dst) for g in gs]
    Ks = [K for _, K, _ in SPECS]
    seeds = [5, 6, 7, 8]
    iters = 20
    # round robin (and the autotuner's measurements of these shapes)
    monkeypatch.setenv("SC_BATCH_LOCKSTEP", "0")
    l0 = ctx.lockstep_passes
    rr = sc.sc_lobpcg_batch(ctx, Gs, Ks, iters=iters, prec=sc.SC_PREC_MIXED, seeds=seeds)
    assert ctx.lockstep_passes == l0
    monkeypatch.delenv("SC_BATCH_LOCKSTEP")
    l0, r0 = ctx.lockstep_passes, ctx.graph_replays
    ls = sc.sc_lobpcg_batch(ctx, Gs, Ks, iters=iters, prec=sc.SC_PREC_MIXED, seeds=seeds)
    # pass 0 run by run, passes 1..19 in lockstep; 2..19 replayed except the re-orthonormalizing
    # pass 15
    assert ctx.lockstep_passes - l0 == iters - 1
    assert ctx.graph_replays - r0 == iters - 3
    for q, (G, K) in enumerate(zip(Gs, Ks)):
        lam, resid, _, info = sc.sc_lobpcg(ctx, G, K, iters=iters, prec=sc.SC_PREC_MIXED,
                                           seed=seeds[q], cold=1, want_X=False)
        for other in (rr[q], ls[q]):
            assert np.array_equal(lam, other["lam"]), q
            assert np.array_equal(resid, other["resid"]), q
            assert other["iters_done"] == iters and other["fallbacks"] == info["fallbacks"]
    # without graphs the lockstep passes are issued eagerly, with the same results
    monkeypatch.setenv("SC_CUDA_GRAPHS", "0")
    r0 = ctx.graph_replays
    ne = sc.sc_lobpcg_batch(ctx, Gs, Ks, iters=iters, prec=sc.SC_PREC_MIXED, seeds=seeds)
    assert ctx.graph_replays == r0
    for a, b in zip(ls, ne):
        assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["resid"], b["resid"])
    for G in Gs:
        G.close()


def test_lockstep_is_not_used_for_mixed_pass_counts_or_tolerances(sc, ctx):
    gs = [W.dcsbm(n, K, seed=s) for n, K, s in SPECS[:2]]
    Gs = [sc.sc_build_laplacian(ctx, g.n, g.src, g.dst) for g in gs]
    Ks = [K for _, K, _ in SPECS[:2]]
    l0 = ctx.lockstep_passes
    with pytest.raises(sc.ScError):  # 6 passes do not reach the tolerance
        sc.sc_lobpcg_batch(ctx, Gs, Ks, iters=6, tol_abs=1e-3, prec=sc.SC_PREC_MIXED)
    sc.sc_lobpcg_batch(ctx, Gs, Ks, iters=6, prec=sc.SC_PREC_FP64)
    assert ctx.lockstep_passes == l0
    for G in Gs:
        G.close()
