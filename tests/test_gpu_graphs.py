"""CUDA-graph replay of fixed-pass LOBPCG solves: the replayed passes are the eager passes'
kernels on the same buffers, so every output is bitwise the same as with SC_CUDA_GRAPHS=0,
in every precision, alone and in a batch; the launch accounting counts replayed kernels."""
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


@pytest.fixture(scope="module")
def ctx(sc):
    c = sc.sc_ctx_create(0)
    yield c
    c.close()


def _solve(sc, ctx, G, K, prec, iters, monkeypatch, graphs, X0):
    if graphs:
        monkeypatch.delenv("SC_CUDA_GRAPHS", raising=False)
    else:
        monkeypatch.setenv("SC_CUDA_GRAPHS", "0")
    r0 = ctx.graph_replays
    lam, res, X, inf = sc.sc_lobpcg(ctx, G, K, iters=iters, prec=prec, X0=X0)
    return lam, res, X, inf, ctx.graph_replays - r0


@pytest.mark.parametrize("prec", ["MIXED", "FP64", "MIXED_DD"])
def test_graph_replay_is_bitwise_the_eager_solve(sc, ctx, prec, monkeypatch):
    p = getattr(sc, "SC_PREC_" + prec)
    g = W.dcsbm(4000, 11, seed=5)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    # 20 passes: pass 0 without P, pass 1 eager, passes 2 and 3 recorded, the re-orthonormalizing
    # pass 15 eager, the rest replayed
    X0 = W.start_block(3, g.n, 11)
    # a first solve lets the autotuner measure this graph's shapes (its timing launches would
    # otherwise count in whichever solve comes first)
    _solve(sc, ctx, G, 11, p, 20, monkeypatch, False, X0)
    a = _solve(sc, ctx, G, 11, p, 20, monkeypatch, False, X0)
    b = _solve(sc, ctx, G, 11, p, 20, monkeypatch, True, X0)
    assert a[4] == 0
    assert b[4] == 17
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v)
    assert a[3]["iters_done"] == b[3]["iters_done"] == 20
    assert a[3]["kernels"] == b[3]["kernels"]
    # and the replayed solve is the oracle's 20-pass solve, to the FP32 / FP64 parity bars
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ref = O.lobpcg(L, X0.astype(np.float32).astype(np.float64), 20)  # the library takes float X0
    tol = 1e-10 if prec == "FP64" else 1e-5
    assert np.max(np.abs(b[0] - ref.lam)) / O.lambda_max(L) <= tol
    G.close()


def test_graph_replay_in_a_batch_is_bitwise_the_eager_batch(sc, ctx, monkeypatch):
    graphs, Ks = [], []
    for i, (n, K) in enumerate([(3000, 9), (6000, 14), (2000, 6)]):
        g = W.dcsbm(n, K, seed=40 + i)
        graphs.append(sc.sc_build_laplacian(ctx, g.n, g.src, g.dst))
        Ks.append(K)
    out = []
    sc.sc_lobpcg_batch(ctx, graphs, Ks, iters=12, prec=sc.SC_PREC_MIXED, seeds=[1, 2, 3])
    # runs issued in turn, eager / each run replaying its own pass graphs; then the lockstep
    # batch, which replays one graph of the whole batch pass
    for lockstep, flag in ((False, False), (False, True), (True, True)):
        monkeypatch.setenv("SC_BATCH_LOCKSTEP", "1" if lockstep else "0")
        if flag:
            monkeypatch.delenv("SC_CUDA_GRAPHS", raising=False)
        else:
            monkeypatch.setenv("SC_CUDA_GRAPHS", "0")
        r0 = ctx.graph_replays
        infos = sc.sc_lobpcg_batch(ctx, graphs, Ks, iters=12, prec=sc.SC_PREC_MIXED,
                                   seeds=[1, 2, 3])
        out.append((infos, ctx.graph_replays - r0))
    assert [o[1] for o in out] == [0, 3 * 10, 10]
    for other in out[1:]:
        for ia, ib in zip(out[0][0], other[0]):
            assert np.array_equal(ia["lam"], ib["lam"])
            assert np.array_equal(ia["resid"], ib["resid"])
    for G in graphs:
        G.close()
