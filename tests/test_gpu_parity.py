"""GPU parity: every step of the CUDA path against the FP64 oracle on the same seeded inputs.

All calls go through the C ABI (ctypes binding).  Tolerances:
  integer / index work (CSR, labels, seeds): bit-exact;
  FP64 form: 1e-10 relative to lambda_max (the check mode);
  FP32 form: |d lambda| / lambda_max <= 1e-5, block sin-theta <= 1e-3 (20 passes), per-element
  SpMM / Gram errors bounded by a few FP32 ulps of the products' magnitudes.
"""
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


def _csr_equal(sc, G, L, algebraic=False):
    rp, ci, val, deg = sc.sc_graph_copy_csr(G)
    assert np.array_equal(rp, L.row_ptr)
    assert np.array_equal(ci, L.col_idx)
    if algebraic:
        np.testing.assert_allclose(val, L.val, rtol=1e-6)
        np.testing.assert_allclose(deg, L.deg, rtol=1e-6)
    else:
        assert np.all(val == 1.0)
        assert np.array_equal(deg, L.deg)


# ------------------------------------------------------------------ a1: Laplacian build


@pytest.mark.parametrize("n,K,seed", [(1000, 11, 0), (5003, 19, 1), (50000, 44, 0)])
def test_laplacian_dcsbm(sc, ctx, n, K, seed):
    g = W.dcsbm(n, K, seed=seed)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    _csr_equal(sc, G, O.laplacian_csr(g.n, g.src, g.dst))


def test_laplacian_multigraph_loops_and_algebraic(sc, ctx):
    rng = np.random.default_rng(3)
    n, m = 257, 5000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    w = rng.uniform(0.25, 2.0, m).astype(np.float32)
    G = sc.sc_build_laplacian(ctx, n, src, dst)
    _csr_equal(sc, G, O.laplacian_csr(n, src, dst))
    Ga = sc.sc_build_laplacian(ctx, n, src, dst, w, sym=sc.SC_SYM_ALGEBRAIC)
    _csr_equal(sc, Ga, O.laplacian_csr(n, src, dst, w.astype(np.float64), sym="algebraic"), True)


def test_laplacian_long_rows_and_edge_cases(sc, ctx):
    # a star: the hub row (9999 entries) exceeds one CTA's shared-memory sort
    n = 10000
    src = np.zeros(n - 1, np.int32)
    dst = np.arange(1, n, dtype=np.int32)
    extra = np.random.default_rng(4).integers(1, n, 3000).astype(np.int32)
    src = np.concatenate([src, extra])
    dst = np.concatenate([dst, np.zeros_like(extra)])  # duplicates of hub edges, reversed
    G = sc.sc_build_laplacian(ctx, n, src, dst)
    _csr_equal(sc, G, O.laplacian_csr(n, src, dst))
    # no edges at all, and only self-loops
    G0 = sc.sc_build_laplacian(ctx, 5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    rp, ci, _, deg = sc.sc_graph_copy_csr(G0)
    assert np.all(rp == 0) and ci.size == 0 and np.all(deg == 0)
    G1 = sc.sc_build_laplacian(ctx, 3, np.array([0, 1, 2], np.int32), np.array([0, 1, 2], np.int32))
    assert sc.sc_graph_info(G1)[1] == 0
    with pytest.raises(sc.ScError) as e:
        sc.sc_build_laplacian(ctx, 4, np.array([0, 4], np.int32), np.array([1, 2], np.int32))
    assert e.value.code == sc.SC_EINVAL


# ------------------------------------------------------------------ a4: SpMM


@pytest.mark.parametrize("k", [1, 3, 11, 44, 160, 300, 512])
def test_spmm_fp32_and_fp64(sc, ctx, k):
    g = W.dcsbm(3001, 7, seed=5)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    V = np.random.default_rng(k).standard_normal((g.n, k))
    ref = O.lap_apply(L, V.astype(np.float32).astype(np.float64))
    Y32 = sc.sc_lap_apply(ctx, G, V.astype(np.float32), sc.SC_PREC_FP32)
    scale = (L.deg[:, None] + 1) * np.abs(V).max()
    assert np.all(np.abs(Y32 - ref) <= 4e-7 * scale * np.sqrt(L.deg.max() + 1))
    Y64 = sc.sc_lap_apply(ctx, G, V, sc.SC_PREC_FP64)
    np.testing.assert_allclose(Y64, O.lap_apply(L, V), rtol=0, atol=1e-12 * scale.max())


def test_spmm_weighted(sc, ctx):
    rng = np.random.default_rng(6)
    n, m = 800, 9000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    w = rng.uniform(0.1, 3.0, m).astype(np.float32)
    G = sc.sc_build_laplacian(ctx, n, src, dst, w, sym=sc.SC_SYM_ALGEBRAIC)
    L = O.laplacian_csr(n, src, dst, w.astype(np.float64), sym="algebraic")
    V = rng.standard_normal((n, 12))
    Y = sc.sc_lap_apply(ctx, G, V, sc.SC_PREC_FP64)
    # W is stored in FP32 on the device: compare with the oracle on the same rounded weights
    Lr = O.laplacian_csr(n, src, dst, w.astype(np.float64), sym="algebraic")
    Lr.val = Lr.val.astype(np.float32).astype(np.float64)
    Lr.deg = np.asarray(Lr.W().sum(axis=1)).ravel()
    np.testing.assert_allclose(Y, O.lap_apply(Lr, V), rtol=0, atol=1e-5 * np.abs(V).max() * L.deg.max())


# ------------------------------------------------------------------ a5: Gram


@pytest.mark.parametrize("n,a,b", [(1, 3, 5), (37, 11, 11), (1000, 44, 132), (50001, 132, 132), (20000, 160, 480)])
@pytest.mark.parametrize("prec", ["mixed", "fp32", "fp64"])
def test_gram(sc, ctx, n, a, b, prec):
    rng = np.random.default_rng(n + a)
    A = rng.standard_normal((n, a))
    B = rng.standard_normal((n, b))
    if prec in ("fp32", "mixed"):
        # mixed: tcgen05 3-term split TF32 (~2^-21 per product); fp32: CUDA cores
        A32, B32 = A.astype(np.float32), B.astype(np.float32)
        Cm = sc.sc_gram(ctx, A32, B32, sc.SC_PREC_MIXED if prec == "mixed" else sc.SC_PREC_FP32)
        ref = A32.astype(np.float64).T @ B32.astype(np.float64)
        bound = 1e-6 * np.sqrt(n) * np.outer(np.linalg.norm(A32, axis=0), np.linalg.norm(B32, axis=0)) + 1e-30
        assert np.all(np.abs(Cm - ref) <= bound)
    else:
        Cm = sc.sc_gram(ctx, A, B, sc.SC_PREC_FP64)
        np.testing.assert_allclose(Cm, A.T @ B, rtol=0, atol=1e-13 * n * 10)


@pytest.mark.parametrize("prec", [0, 1])
def test_gram_empty_rows(sc, ctx, prec):
    Cm = sc.sc_gram(ctx, np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32), prec)
    assert Cm.shape == (4, 6) and np.all(Cm == 0)


def test_gram_tc_ragged_and_structured(sc, ctx):
    # rows not a multiple of the 32-row stage, columns not a multiple of 4, rank-one data
    rng = np.random.default_rng(11)
    for n, a, b in [(33, 5, 7), (4099, 130, 3), (777, 257, 129)]:
        A = rng.standard_normal((n, a)).astype(np.float32)
        B = (rng.standard_normal((n, 1)) @ rng.standard_normal((1, b))).astype(np.float32)
        Cm = sc.sc_gram(ctx, A, B, sc.SC_PREC_MIXED)
        ref = A.astype(np.float64).T @ B.astype(np.float64)
        bound = 2e-6 * np.sqrt(n) * np.outer(np.linalg.norm(A, axis=0), np.linalg.norm(B, axis=0)) + 1e-30
        assert np.all(np.abs(Cm - ref) <= bound), (n, a, b)


# ------------------------------------------------------------------ a7: tall update


@pytest.mark.parametrize("n,a,b", [(1, 3, 5), (33, 5, 7), (777, 44, 44), (50001, 132, 44),
                                   (4099, 88, 96), (3000, 40, 300), (2000, 500, 40),
                                   (100003, 480, 160), (20001, 320, 256)])
@pytest.mark.parametrize("prec", ["mixed", "fp32", "fp64"])
def test_tall_update(sc, ctx, n, a, b, prec):
    """out = beta Cin + A W element by element against the FP64 product of the same (rounded)
    inputs: tcgen05 3xTF32 (mixed; more than 256 output columns fall back to CUDA cores), FP32
    CUDA cores, FP64.  The shapes include the n = 2M workload's widest update (3K = 480 columns
    into K = 160) at a smaller n, and 256 output columns (two staged chunks)."""
    rng = np.random.default_rng(n + a + b)
    A = rng.standard_normal((n, a))
    W = rng.standard_normal((a, b))
    Cin = rng.standard_normal((n, b))
    if prec == "fp64":
        out = sc.sc_tall_update(ctx, A, W, Cin, -0.5, sc.SC_PREC_FP64)
        ref = -0.5 * Cin + A @ W
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13 * (np.abs(A) @ np.abs(W)).max())
        return
    A32, W32, C32 = A.astype(np.float32), W.astype(np.float32), Cin.astype(np.float32)
    p = sc.SC_PREC_MIXED if prec == "mixed" else sc.SC_PREC_FP32
    out = sc.sc_tall_update(ctx, A32, W32, C32, -0.5, p)
    Ad, Wd, Cd = (x.astype(np.float64) for x in (A32, W32, C32))
    ref = -0.5 * Cd + Ad @ Wd
    scale = np.abs(Ad) @ np.abs(Wd) + 0.5 * np.abs(Cd)
    assert np.all(np.abs(out - ref) <= 4e-6 * scale + 1e-30), (n, a, b, prec)
    # no accumulate input
    out0 = sc.sc_tall_update(ctx, A32, W32, None, 0.0, p)
    assert np.all(np.abs(out0 - Ad @ Wd) <= 4e-6 * (np.abs(Ad) @ np.abs(Wd)) + 1e-30)


# ------------------------------------------------------------------ a6: Rayleigh-Ritz solve


def _sym_with_spectrum(m, ev, seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, m)))
    return (Q * ev) @ Q.T


@pytest.mark.parametrize("m,K", [(1, 1), (2, 1), (33, 11), (132, 44), (200, 60), (480, 160), (500, 100)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_rr_solve(sc, ctx, m, K, prec):
    rng = np.random.default_rng(m)
    ev = np.sort(rng.uniform(0, 100, m))
    if m > 4:
        ev[1:4] = ev[1]  # a triple eigenvalue inside the wanted block
        ev = np.sort(ev)
    G = _sym_with_spectrum(m, ev, m + 1)
    p = sc.SC_PREC_FP64 if prec == "fp64" else sc.SC_PREC_FP32
    th, Y = sc.sc_rr_solve(ctx, G, K, p)
    w, V = np.linalg.eigh(G)
    tol = (1e-12 if prec == "fp64" else 2e-5) * max(1.0, np.abs(ev).max())
    assert np.max(np.abs(th - w[:K])) <= tol
    np.testing.assert_allclose(Y.T @ Y, np.eye(K), atol=1e-10 if prec == "fp64" else 1e-4)
    res = np.linalg.norm(G @ Y - Y * th, axis=0)
    assert res.max() <= (1e-9 if prec == "fp64" else 1e-3) * np.abs(ev).max()
    if K < m and w[K] - w[K - 1] > 1e-3:
        assert O.sin_theta(V[:, :K], Y) <= (1e-9 if prec == "fp64" else 1e-3)


# ------------------------------------------------------------------ a2, a3, a7: LOBPCG


def _lobpcg_pair(sc, ctx, n, K, iters, seed=0, prec=None, **kw):
    g = W.dcsbm(n, K, seed=seed)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    X0 = W.start_block(seed, g.n, K)
    p = sc.SC_PREC_MIXED if prec is None else prec
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, K, iters=iters, prec=p, X0=X0, **kw)
    x0 = X0.astype(np.float32).astype(np.float64)  # the library takes a float start block
    ref = O.lobpcg(L, x0, iters, **kw)
    return g, L, lam, resid, X, info, ref


def test_lobpcg_fp64_check_mode_small(sc, ctx):
    g, L, lam, resid, X, info, ref = _lobpcg_pair(sc, ctx, 1000, 11, 20, prec=2)
    lmax = O.lambda_max(L)
    assert info["iters_done"] == ref.iters == 20
    assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-10
    assert O.sin_theta(ref.X, X.astype(np.float64)) <= 1e-6  # sc_lobpcg returns X as float32
    np.testing.assert_allclose(resid, ref.resid, rtol=1e-6, atol=1e-10 * lmax)


@pytest.mark.parametrize("n,K", [(1000, 11), (5003, 19)])
def test_lobpcg_fp64_check_mode_fp64_block(sc, ctx, n, K):
    """The FP64 check mode with an FP64 start block and FP64 result (sc_lobpcg64): Ritz
    values to 1e-10 lambda_max and the block's subspace to sin-theta <= 1e-10 against the
    oracle from the same start block."""
    g = W.dcsbm(n, K, seed=1)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    X0 = W.start_block(3, g.n, K)
    lam, resid, X, info = sc.sc_lobpcg64(ctx, G, K, iters=20, prec=sc.SC_PREC_FP64, X0=X0)
    ref = O.lobpcg(L, X0, 20)
    lmax = O.lambda_max(L)
    assert X.dtype == np.float64 and info["iters_done"] == ref.iters == 20
    assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-10
    assert O.sin_theta(ref.X, X) <= 1e-10
    np.testing.assert_allclose(resid, ref.resid, rtol=1e-6, atol=1e-10 * lmax)
    # the mixed form through the same entry point: FP32 arithmetic, widened result
    lam32, _, X32, _ = sc.sc_lobpcg64(ctx, G, K, iters=20, prec=sc.SC_PREC_MIXED, X0=X0)
    ref32 = O.lobpcg(L, X0.astype(np.float32).astype(np.float64), 20)
    assert np.max(np.abs(lam32 - ref32.lam)) / lmax <= 1e-5
    assert O.sin_theta(ref32.X, X32) <= 1e-3


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_lobpcg_fp32_small(sc, ctx, prec):
    g, L, lam, resid, X, info, ref = _lobpcg_pair(sc, ctx, 1000, 11, 20, prec=prec)
    lmax = O.lambda_max(L)
    assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-5
    assert O.sin_theta(ref.X, X.astype(np.float64)) <= 1e-3
    assert info["fallbacks"] == ref.fallbacks == 0


@pytest.mark.parametrize("prec", [0, 3])
def test_lobpcg_fp32_bench_size(sc, ctx, prec):
    g, L, lam, resid, X, info, ref = _lobpcg_pair(sc, ctx, 50000, 44, 20, prec=prec)
    lmax = O.lambda_max(L)
    assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-5
    assert O.sin_theta(ref.X, X.astype(np.float64)) <= 1e-3


def test_lobpcg_fp64_wide_block(sc, ctx):
    """K = 140 in FP64: the pass's SpMM covers [R P] = 280 columns, wider than one launch of
    the SpMM kernel takes, so it runs in column chunks."""
    g, L, lam, resid, X, info, ref = _lobpcg_pair(sc, ctx, 3000, 140, 4, prec=2)
    lmax = O.lambda_max(L)
    assert info["iters_done"] == ref.iters == 4
    assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-10
    np.testing.assert_allclose(resid, ref.resid, rtol=1e-6, atol=1e-10 * lmax)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_lobpcg_jacobi_matches_oracle(sc, ctx, prec):
    """The Jacobi-preconditioned iteration (T = D^-1 on the residual block, Sec. II.B) against
    the oracle's, 20 passes from the same start block."""
    g = W.dcsbm(3000, 11, seed=23)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    X0 = W.start_block(5, g.n, 11)
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, 11, iters=20, prec=prec, X0=X0,
                                       precond=sc.SC_PRECOND_JACOBI)
    ref = O.lobpcg(L, X0.astype(np.float32).astype(np.float64), 20, precond="jacobi")
    lmax = O.lambda_max(L)
    tol = 1e-10 if prec == 2 else 1e-5
    assert np.max(np.abs(lam - ref.lam)) / lmax <= tol
    assert O.sin_theta(ref.X, X.astype(np.float64)) <= (1e-6 if prec == 2 else 1e-3)
    np.testing.assert_allclose(resid, ref.resid, rtol=1e-3 if prec != 2 else 1e-6,
                               atol=(1e-10 if prec == 2 else 1e-5) * lmax)


def test_lobpcg_jacobi_reaches_tolerance_in_fewer_passes(sc, ctx):
    g = W.dcsbm(20000, 22, seed=24)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    tol = 1e-3 * 2 * sc.sc_graph_info(G)[2]
    runs = {}
    for pc in (sc.SC_PRECOND_NONE, sc.SC_PRECOND_JACOBI):
        _, resid, _, info = sc.sc_lobpcg(ctx, G, 22, iters=400, tol_abs=tol, seed=6, cold=1,
                                         want_X=False, precond=pc)
        assert info["converged"] == 1 and resid.max() <= tol
        runs[pc] = info["iters_done"]
    assert runs[sc.SC_PRECOND_JACOBI] * 2 <= runs[sc.SC_PRECOND_NONE], runs


def test_lobpcg_ragged_sizes(sc, ctx):
    # K = 1, K not a multiple of 4, n = 3K exactly
    for n, K in [(300, 1), (61, 7), (36, 12)]:
        g = W.dcsbm(n, min(K, 4), seed=7, dmin=3, dmax=12)
        L = O.laplacian_csr(g.n, g.src, g.dst)
        G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
        X0 = W.start_block(2, n, K)
        lam, resid, X, info = sc.sc_lobpcg(ctx, G, K, iters=5, prec=2, X0=X0)
        ref = O.lobpcg(L, X0.astype(np.float32).astype(np.float64), 5)
        lmax = O.lambda_max(L)
        assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-9, (n, K)


def test_lobpcg_soft_locking_converges(sc, ctx):
    g = W.dcsbm(2000, 6, seed=8)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    tol = 1e-3 * ev[-1]
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, 6, iters=300, tol_abs=tol, tol_lock=tol,
                                       prec=sc.SC_PREC_FP32, seed=3)
    assert info["converged"] == 1
    assert np.max(np.abs(lam - ev[:6])) <= 1e-4 * ev[-1]
    assert resid.max() <= tol


def test_lobpcg_fp64_far_past_convergence(sc, ctx):
    """400 fixed FP64 passes with no locking: the columns reach roundoff long before the
    end.  Dropped residual/direction columns keep the one-product-per-pass iteration at the
    solution instead of letting normalized noise derail it (Sec. II.B, Sec. IV)."""
    g = W.dcsbm(2000, 6, seed=9)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, 6, iters=400, prec=2, seed=4)
    assert info["iters_done"] == 400 and info["dropped"] > 0
    assert np.max(np.abs(lam - ev[:6])) <= 1e-11 * ev[-1]
    assert resid.max() <= 1e-10 * ev[-1]
    R = O.lap_apply(L, X.astype(np.float64)) - X.astype(np.float64) * lam
    assert np.linalg.norm(R, axis=0).max() <= 1e-6 * ev[-1]  # X returned as float32


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_lobpcg_fp32_far_past_convergence(sc, ctx, prec):
    """400 FP32 passes with no locking: residual columns sink to FP32 rounding noise within
    about 60 passes.  The pass must stay at the solution: exact L-images of the
    orthonormalized trial block, dropped noise columns and the periodic re-orthonormalization
    of X keep Ritz vectors from drifting or merging."""
    g = W.dcsbm(2000, 6, seed=9)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, 6, iters=400, prec=prec, seed=4)
    assert info["iters_done"] == 400
    assert np.max(np.abs(lam - ev[:6])) <= 2e-5 * ev[-1]
    assert resid.max() <= 1e-4 * ev[-1]
    Xd = X.astype(np.float64)
    assert np.max(np.abs(Xd.T @ Xd - np.eye(6))) <= 1e-4
    R = O.lap_apply(L, Xd) - Xd * lam
    assert np.linalg.norm(R, axis=0).max() <= 1e-4 * ev[-1]


@pytest.mark.parametrize("prec", [0, 1])
def test_lobpcg_fp32_soft_locked_long_run(sc, ctx, prec):
    """FP32 run with a 400-pass budget and soft locking at 1e-4 lambda_max (Sec. IV): every
    column locks once it reaches the tolerance, and the result is the converged spectrum."""
    g = W.dcsbm(2000, 6, seed=9)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    tl = 1e-4 * ev[-1]
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, 6, iters=400, tol_lock=tl, prec=prec, seed=4)
    assert info["iters_done"] < 400
    assert np.max(np.abs(lam - ev[:6])) <= 2e-5 * ev[-1]
    assert resid.max() <= tl


@pytest.mark.parametrize("m,K", [(132, 44), (264, 44), (500, 100)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_rr_solve_skips_dropped_columns(sc, ctx, m, K, prec):
    """Zero rows of G beyond the first K (columns the Cholesky-QR dropped) take no part:
    the K smallest eigenpairs are those of G with those rows and columns removed."""
    rng = np.random.default_rng(m + K)
    keep = np.ones(m, bool)
    keep[rng.choice(np.arange(K, m), size=max(3, (m - K) // 5), replace=False)] = False
    mk = int(keep.sum())
    ev = np.sort(rng.uniform(0, 100, mk))
    ev[0] = 0.0  # a zero eigenvalue: must not be confused with the dropped columns
    Gk = _sym_with_spectrum(mk, ev, m)
    G = np.zeros((m, m))
    G[np.ix_(keep, keep)] = Gk
    p = sc.SC_PREC_FP64 if prec == "fp64" else sc.SC_PREC_FP32
    th, Y = sc.sc_rr_solve(ctx, G, K, p)
    tol = (1e-11 if prec == "fp64" else 2e-5) * 100
    assert np.max(np.abs(th - ev[:K])) <= tol
    Yk = Y[keep]
    res = np.linalg.norm(Gk @ Yk - Yk * th, axis=0)
    assert res.max() <= (1e-9 if prec == "fp64" else 1e-3) * 100
    np.testing.assert_allclose(Yk.T @ Yk, np.eye(K), atol=1e-9 if prec == "fp64" else 1e-4)


def test_lobpcg_rejects_bad_sizes(sc, ctx):
    G = sc.sc_build_laplacian(ctx, 10, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(sc.ScError) as e:
        sc.sc_lobpcg(ctx, G, 4, iters=1)
    assert e.value.code == sc.SC_EINVAL
    with pytest.raises(sc.ScError) as e:
        sc.sc_lap_apply(ctx, G, np.zeros((10, 513), np.float32))
    assert e.value.code == sc.SC_EINVAL and "sc_lap_apply" in str(e.value)
    G2 = sc.sc_build_laplacian(ctx, 30, np.arange(29, dtype=np.int32), np.arange(1, 30, dtype=np.int32))
    with pytest.raises(sc.ScError) as e:
        sc.sc_lobpcg(ctx, G2, 4, iters=1, precond=7)
    assert e.value.code == sc.SC_EINVAL and "preconditioner" in str(e.value)


# ------------------------------------------------------------------ a8: embedding


def test_embed_rows(sc, ctx):
    X = np.random.default_rng(9).standard_normal((5000, 44)).astype(np.float32)
    X[7] = 0
    E = sc.sc_embed_rows(ctx, X)
    np.testing.assert_allclose(E, O.embed_rows(X.astype(np.float64)), rtol=0, atol=2e-7)
    assert np.all(E[7] == 0)


# ------------------------------------------------------------------ a9, a10: k-means


def _clustered(n, d, k, seed, spread=0.05):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((k, d))
    lab = rng.integers(0, k, n)
    E = C[lab] + spread * rng.standard_normal((n, d))
    return O.embed_rows(E).astype(np.float32), lab


@pytest.mark.parametrize("assign", ["simt", "tc"])
@pytest.mark.parametrize("n,d,k", [(1000, 11, 11), (50000, 44, 44), (3001, 5, 1), (3000, 100, 70), (3000, 156, 150), (2000, 200, 40)])
def test_kmeans_seeds_and_labels_bit_exact(sc, ctx, n, d, k, assign, monkeypatch):
    # assign = tc: the Lloyd assignment on tensor cores (3-term split TF32 distances, FP64
    # re-decision of near ties) wherever the shape allows it (rows 16-byte aligned: d % 4 == 0)
    monkeypatch.setenv("SC_TUNE_ASSIGN", "1" if assign == "tc" else "0")
    E, _ = _clustered(n, d, max(k, 2), n)
    u = W.kmeans_uniforms(5, k)
    l0 = ctx.launches
    labels, cent, seeds, inertia, ran = sc.sc_kmeans(ctx, E, k, iters=50, seed=5)
    if assign == "tc" and d % 4 == 0 and k > 1:
        # the tensor-core path ran: per round it launches the split of C' and its kernel where
        # the CUDA-core path launches one kernel
        launches_tc = ctx.launches - l0
        monkeypatch.setenv("SC_TUNE_ASSIGN", "0")
        l0 = ctx.launches
        sc.sc_kmeans(ctx, E, k, iters=50, seed=5)
        assert launches_tc > ctx.launches - l0
    Ed = E.astype(np.float64)
    rl, rC, ridx, rin = O.kmeans(Ed, k, u, 50)
    assert np.array_equal(seeds, ridx)
    assert np.array_equal(labels, rl)
    np.testing.assert_allclose(cent, rC, rtol=0, atol=1e-6)
    assert abs(inertia - rin) <= 1e-9 * max(rin, 1.0)


def test_kmeans_given_seeds_and_duplicates(sc, ctx):
    E = np.repeat(np.eye(4, dtype=np.float32), 5, axis=0)  # only 4 distinct rows
    labels, cent, seeds, inertia, ran = sc.sc_kmeans(ctx, E, 6, iters=10, seed=1)
    rl, rC, ridx, rin = O.kmeans(E.astype(np.float64), 6, W.kmeans_uniforms(1, 6), 10)
    assert np.array_equal(seeds, ridx) and np.array_equal(labels, rl) and inertia == 0.0
    init = np.array([0, 5, 10], np.int32)
    labels, cent, seeds, inertia, ran = sc.sc_kmeans(ctx, E, 3, iters=10, init_idx=init)
    rl, _, _ = O.lloyd(E.astype(np.float64), E[init].astype(np.float64), 10)
    assert np.array_equal(labels, rl)


# ------------------------------------------------------------------ end to end


def test_partition_matches_oracle_labels(sc, ctx):
    g = W.dcsbm(1000, 11, seed=0)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    labels, info = sc.sc_partition(ctx, G, 11, 11, iters=20, seed=0)
    X0 = W.start_block(0, g.n, 11).astype(np.float32).astype(np.float64)
    rl, res, E, idx = O.partition(L, X0, 11, W.kmeans_uniforms(0, 11), 20, 50)
    assert O.partition_metrics(rl, labels)[0] == 1.0  # identical up to a permutation
    assert O.partition_metrics(g.truth, labels)[0] == 1.0


@pytest.fixture(scope="module")
def headline_oracle():
    """The oracle's partition of the n = 50,000, K = 44 DC-SBM graph (seed 0): 20 LOBPCG
    passes from the seeded start block, unit rows, k-means++ with the seed-0 uniforms and 50
    Lloyd rounds."""
    g = W.dcsbm(50000, 44, seed=0)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    X0 = W.start_block(0, g.n, 44).astype(np.float32).astype(np.float64)
    rl, res, E, idx = O.partition(L, X0, 44, W.kmeans_uniforms(0, 44), 20, 50)
    return g, L, rl, res, idx


@pytest.mark.parametrize("prec", [0, 3, 2])
def test_partition_labels_match_oracle_at_headline_size(sc, ctx, headline_oracle, prec):
    """sc_partition at n = 50,000, K = 44, seed 0: the labels are identical to the oracle's up to
    a permutation of the cluster ids (matched fraction 1.0), and the k-means++ seeds drawn on the
    library's embedding are the oracle's, in every precision."""
    g, L, rl, res, idx = headline_oracle
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    labels, info = sc.sc_partition(ctx, G, 44, 44, iters=20, seed=0, prec=prec)
    assert info["iters_done"] == 20
    assert O.partition_metrics(rl, labels)[0] == 1.0
    X0 = W.start_block(0, g.n, 44).astype(np.float32).astype(np.float64)
    lam, _, X, _ = sc.sc_lobpcg64(ctx, G, 44, iters=20, prec=prec, X0=X0)
    E = sc.sc_embed_rows(ctx, X.astype(np.float32))
    _, _, seeds, _, _ = sc.sc_kmeans(ctx, E, 44, iters=50, seed=0)
    assert np.array_equal(seeds, idx)
    tol = 1e-10 if prec == 2 else 1e-5
    assert np.max(np.abs(lam - res.lam)) / O.lambda_max(L) <= tol
    G.close()


@pytest.mark.parametrize("n,K", [(3000, 50), (4000, 70), (5000, 140)])
def test_partition_wide_blocks(sc, ctx, n, K):
    # block widths of the serving workload: Rayleigh-Ritz sizes 3K from 150 to 420 and
    # k-means in d = K dimensions with k = K clusters
    g = W.dcsbm(n, K, seed=K)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, K, iters=6, seed=1, cold=1)
    ref = O.lobpcg(L, W.start_block(1, g.n, K).astype(np.float32).astype(np.float64), 6)
    lmax = O.lambda_max(L)
    assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-5
    labels, info = sc.sc_partition(ctx, G, K, K, iters=6, seed=1)
    assert labels.min() >= 0 and labels.max() < K


# ------------------------------------------------------------------ a12: streaming


def test_stream_warm_starts_through_the_component_merge(sc, ctx):
    """Emerging edges at n = 50,000, K = 44: stage 1 cold sets rho*; stages 2-8 run warm to
    max residual <= rho* with soft locking at rho* (Sec. IV), across the stage where the last
    isolated vertices join the graph."""
    n, K = 50000, 44
    g = W.dcsbm(n, K, seed=0)
    deltas = W.emerging_deltas(g, 10)
    G = sc.sc_build_laplacian(ctx, n, g.src[deltas[0]], g.dst[deltas[0]])
    _, resid, _, _ = sc.sc_lobpcg(ctx, G, K, iters=20, seed=0, cold=1, want_X=False)
    rho = float(resid.max())
    for s_ in range(1, 8):
        sc.sc_stream_update(ctx, G, n, g.src[deltas[s_]], g.dst[deltas[s_]])
        lam, resid, _, info = sc.sc_lobpcg(ctx, G, K, iters=300, tol_abs=rho, tol_lock=rho,
                                           seed=0, cold=0, want_X=False)
        assert info["converged"] == 1, s_
        assert resid.max() <= rho
        assert np.all(np.isfinite(lam)) and np.all(np.diff(lam) >= -1e-6 * lam[-1])
        assert lam[0] >= -1e-4 and lam[-1] <= 2 * 205
    G.close()


def test_stream_emerging_matches_rebuild(sc, ctx):
    g = W.dcsbm(5000, 9, seed=10)
    deltas = W.emerging_deltas(g)
    G = sc.sc_build_laplacian(ctx, g.n, g.src[deltas[0]], g.dst[deltas[0]])
    for s in range(1, 10):
        sc.sc_stream_update(ctx, G, g.n, g.src[deltas[s]], g.dst[deltas[s]])
        upto = np.concatenate(deltas[: s + 1])
        _csr_equal(sc, G, O.laplacian_csr(g.n, g.src[upto], g.dst[upto]))


def test_stream_snowball_grows_and_warm_starts(sc, ctx):
    g = W.dcsbm(6000, 8, seed=11)
    st = W.snowball_stages(g)
    G = sc.sc_build_laplacian(ctx, st[0].n, st[0].src, st[0].dst)
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, 8, iters=20, prec=2, seed=1)
    for s in range(1, 4):
        prev = st[s - 1]
        cur = st[s]
        # delta = edges of stage s not in stage s-1 (old vertices keep their ids)
        old = set(zip(prev.src.tolist(), prev.dst.tolist()))
        pairs = [(a, b) for a, b in zip(cur.src.tolist(), cur.dst.tolist())]
        new = np.array([p for p in pairs if p not in old] or [(0, 0)], np.int32)
        sc.sc_stream_update(ctx, G, cur.n, new[:, 0], new[:, 1])
        _csr_equal(sc, G, O.laplacian_csr(cur.n, cur.src, cur.dst))
        # warm start = previous block with zero rows for the new vertices
        Xw = np.zeros((cur.n, 8))
        Xw[: prev.n] = X
        lam, resid, X, info = sc.sc_lobpcg(ctx, G, 8, iters=10, prec=2)
        Lc = O.laplacian_csr(cur.n, cur.src, cur.dst)
        ref = O.lobpcg(Lc, Xw, 10)
        assert np.max(np.abs(lam - ref.lam)) <= 1e-10 * O.lambda_max(Lc)


# ------------------------------------------------------------------ CPQR assignment (f2)


def _planted_block(n, k, seed, noise=0.05):
    rng = np.random.default_rng(seed)
    truth = rng.integers(0, k, n)
    basis, _ = np.linalg.qr(rng.standard_normal((k, k)))
    return truth, (np.eye(k)[truth] @ basis + noise * rng.standard_normal((n, k))).astype(np.float32)


@pytest.mark.parametrize("n,k", [(1, 1), (7, 7), (1000, 5), (20001, 44)])
def test_cpqr_assign_matches_oracle(sc, ctx, n, k):
    truth, Y = _planted_block(n, k, n + k)
    labels, piv = sc.sc_cpqr_assign(ctx, Y)
    ref_labels, ref_piv = O.cpqr_assign(Y.astype(np.float64), k)
    assert list(piv) == list(ref_piv)
    assert np.array_equal(labels, ref_labels)
    if n >= 1000:
        pm, _, _ = O.partition_metrics(truth, labels)
        assert pm == 1.0


def test_cpqr_assign_on_spectral_embedding(sc, ctx):
    """The paper's use: assignment from the LOBPCG eigenvector block of a DC-SBM graph."""
    g = W.dcsbm(5000, 11, seed=1)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    _, _, X, _ = sc.sc_lobpcg(ctx, G, 11, iters=60, prec=sc.SC_PREC_FP64, seed=2,
                              precond=sc.SC_PRECOND_JACOBI)
    labels, piv = sc.sc_cpqr_assign(ctx, X)
    ref_labels, ref_piv = O.cpqr_assign(X.astype(np.float64), 11)
    assert list(piv) == list(ref_piv)
    assert np.mean(labels == ref_labels) >= 0.999
    pm, _, _ = O.partition_metrics(g.truth, labels)
    pm_ref, _, _ = O.partition_metrics(g.truth, ref_labels)
    assert abs(pm - pm_ref) <= 2e-3


# ------------------------------------------------------------------ hard locking (f4)


def test_lobpcg_blocks_matches_oracle_fp64(sc, ctx):
    g = W.dcsbm(2000, 9, seed=51)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    X0 = W.start_block(7, g.n, 9)
    lam, resid, X, info = sc.sc_lobpcg_blocks(ctx, G, 9, 3, iters=20, prec=sc.SC_PREC_FP64,
                                              X0=X0)
    ref = O.lobpcg_blocks(L, X0.astype(np.float32).astype(np.float64), 3, 20)
    lmax = O.lambda_max(L)
    assert info["iters_done"] == ref.iters == 60
    assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-9
    np.testing.assert_allclose(resid, ref.resid, rtol=1e-5, atol=1e-9 * lmax)
    Xd = X.astype(np.float64)
    np.testing.assert_allclose(Xd.T @ Xd, np.eye(9), atol=1e-5)


def test_lobpcg_blocks_converges_and_saves_memory(sc, ctx):
    g = W.dcsbm(3000, 12, seed=52)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    tol = 1e-4 * ev[-1]
    lam, resid, X, info = sc.sc_lobpcg_blocks(ctx, G, 12, 4, iters=400, tol_abs=tol, seed=3,
                                              precond=sc.SC_PRECOND_JACOBI)
    assert info["converged"] == 1 and resid.max() <= tol
    np.testing.assert_allclose(np.sort(lam), ev[:12], rtol=0, atol=2e-5 * ev[-1])
    # one block's workspace instead of the whole block's
    n, K = 200000, 96
    gb = W.dcsbm(n, K, seed=53)
    Gb = sc.sc_build_laplacian(ctx, n, gb.src, gb.dst)
    base = ctx.bytes_in_use
    ctx.bytes_peak()  # reset
    sc.sc_lobpcg(ctx, Gb, K, iters=2, seed=1, cold=1, want_X=False)
    whole = ctx.bytes_peak() - base
    base2 = ctx.bytes_in_use
    sc.sc_lobpcg_blocks(ctx, Gb, K, 24, iters=2, seed=1)
    blocks = ctx.bytes_peak() - base2
    assert blocks < 0.6 * whole, (blocks, whole)


def test_lobpcg_blocks_ragged_last_block_and_device_cpqr(sc, ctx):
    """K = 10 in blocks of 4 (4 + 4 + 2), mixed precision against the FP64 oracle's block
    driver from the same start block; then CPQR on the device-resident copy of the block."""
    torch = pytest.importorskip("torch")
    g = W.dcsbm(2500, 10, seed=54)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    G = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
    X0 = W.start_block(8, g.n, 10)
    lam, resid, X, info = sc.sc_lobpcg_blocks(ctx, G, 10, 4, iters=20, X0=X0)
    ref = O.lobpcg_blocks(L, X0.astype(np.float32).astype(np.float64), 4, 20)
    lmax = O.lambda_max(L)
    assert info["iters_done"] == ref.iters == 60 and len(lam) == 10
    assert np.max(np.abs(lam - ref.lam)) / lmax <= 1e-5
    Xd = torch.from_numpy(X).cuda()
    labels_d, piv_d = sc.sc_cpqr_assign(ctx, Xd)
    labels_h, piv_h = sc.sc_cpqr_assign(ctx, X)
    assert np.array_equal(labels_d, labels_h) and np.array_equal(piv_d, piv_h)


# ------------------------------------------------------------------ eigengap cluster count (f1)


def test_eigengap_on_lobpcg_ritz_values_of_disjoint_cliques(sc, ctx):
    """End to end: 4 disjoint 30-cliques (spectrum 0 x4, then 30), LOBPCG for K = 7, then
    the count read off the Ritz values is 4."""
    c, s = 4, 30
    src, dst = [], []
    for b in range(c):
        for i in range(s):
            for j in range(i + 1, s):
                src.append(b * s + i)
                dst.append(b * s + j)
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    G = sc.sc_build_laplacian(ctx, c * s, src, dst)
    lam, resid, X, info = sc.sc_lobpcg(ctx, G, 7, iters=60, prec=sc.SC_PREC_FP64, seed=3)
    np.testing.assert_allclose(np.sort(lam), [0, 0, 0, 0, s, s, s], atol=1e-6 * s)
    assert sc.sc_eigengap(lam, floor=1e-6 * s) == c
