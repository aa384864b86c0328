"""Pins of the FP64 oracle against facts the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a brute-force
construction, a closed-form spectrum, a special case that reduces to a textbook routine,
an invariant of the method, or a hand-worked example.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_1708_07481_gb300 import workload as W


def _dense_from_edges(n, edges, weights=None, sym="logical"):
    """Brute-force symmetrized adjacency with explicit Python loops (Sec. II.A)."""
    Wd = [[0.0] * n for _ in range(n)]
    for e, (u, v) in enumerate(edges):
        if u == v:
            continue
        w = 1.0 if weights is None else float(weights[e])
        if sym == "logical":
            Wd[u][v] = 1.0
            Wd[v][u] = 1.0
        else:
            Wd[u][v] += w
            Wd[v][u] += w
    return np.array(Wd)


def _rand_graph(n, m, seed, loops=True):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    if not loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    return src, dst


def _run_to_convergence(L, K, seed=0, iters=400, rel=1e-11):
    X0 = W.start_block(seed, L.n, K)
    lmax = np.linalg.eigvalsh(O.laplacian_dense(L))[-1] if L.n <= 400 else 2 * L.deg.max()
    # converged columns are locked at the tolerance, as SciPy's lobpcg does; without it the
    # implicitly updated L*P of a column at rounding level drifts from L times P
    return O.lobpcg(L, X0, iters, tol_abs=rel * lmax, tol_lock=rel * lmax, explicit=True), lmax


# ---------------------------------------------------------------- input generator pins


def test_splitmix64_published_vector():
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")
    want = [int(x) for x in open(path) if x.strip() and not x.startswith("#")]
    got = [int(x) for x in W.sm64(1234567, np.arange(5))]
    assert got == want


# ---------------------------------------------------------------- Laplacian (Sec. II.A)


@pytest.mark.parametrize("sym", ["logical", "algebraic"])
def test_laplacian_matches_bruteforce(sym):
    n = 9
    src, dst = _rand_graph(n, 40, 1)
    w = np.random.default_rng(2).uniform(0.5, 2.0, src.shape[0])
    L = O.laplacian_csr(n, src, dst, w if sym == "algebraic" else None, sym=sym)
    Wd = _dense_from_edges(n, list(zip(src, dst)), w if sym == "algebraic" else None, sym)
    np.testing.assert_allclose(L.W().toarray(), Wd, rtol=0, atol=1e-12)
    np.testing.assert_allclose(L.deg, Wd.sum(axis=1), rtol=0, atol=1e-12)
    # CSR columns sorted and unique within each row
    for i in range(n):
        c = L.col_idx[L.row_ptr[i]:L.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_laplacian_invariants():
    g = W.dcsbm(300, 5, seed=3)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    Ld = O.laplacian_dense(L)
    assert np.array_equal(Ld, Ld.T)
    assert np.all(Ld @ np.ones(g.n) == 0.0)  # exact: integer arithmetic in FP64
    assert L.deg.sum() == L.nnz
    assert np.linalg.eigvalsh(Ld)[0] > -1e-12


def test_algebraic_matches_paper_matrix_free_product():
    """Sec. III: LXfun = diagL.*X - A*X - (X'*A)' with A the nonsymmetric adjacency."""
    n = 12
    src, dst = _rand_graph(n, 60, 4, loops=False)
    w = np.random.default_rng(5).uniform(0.1, 3.0, src.shape[0])
    A = np.zeros((n, n))
    for (u, v, ww) in zip(src, dst, w):
        A[u, v] += ww
    diagL = (A + A.T).sum(axis=1)
    X = np.random.default_rng(6).standard_normal((n, 3))
    want = diagL[:, None] * X - A @ X - (X.T @ A).T
    L = O.laplacian_csr(n, src, dst, w, sym="algebraic")
    np.testing.assert_allclose(O.lap_apply(L, X), want, rtol=1e-13, atol=1e-12)


# ---------------------------------------------------------------- spectra (closed forms)


def _graph_path(n):
    return np.arange(n - 1), np.arange(1, n)


def _graph_cycle(n):
    return np.arange(n), (np.arange(n) + 1) % n


def _graph_complete(n):
    e = [(i, j) for i in range(n) for j in range(i + 1, n)]
    return np.array([a for a, _ in e]), np.array([b for _, b in e])


def _graph_star(n):
    return np.zeros(n - 1, dtype=int), np.arange(1, n)


def _graph_bipartite(a, b):
    e = [(i, a + j) for i in range(a) for j in range(b)]
    return np.array([x for x, _ in e]), np.array([y for _, y in e])


def _graph_hypercube(d):
    n = 1 << d
    e = [(i, i ^ (1 << k)) for i in range(n) for k in range(d) if i < i ^ (1 << k)]
    return np.array([x for x, _ in e]), np.array([y for _, y in e])


CLOSED_FORMS = [
    ("path", 40, _graph_path(40), sorted(2 - 2 * math.cos(math.pi * j / 40) for j in range(40))),
    ("cycle", 40, _graph_cycle(40), sorted(2 - 2 * math.cos(2 * math.pi * j / 40) for j in range(40))),
    ("complete", 15, _graph_complete(15), [0.0] + [15.0] * 14),
    ("star", 20, _graph_star(20), [0.0] + [1.0] * 18 + [20.0]),
    ("bipartite", 21, _graph_bipartite(6, 15), sorted([0.0] + [6.0] * 14 + [15.0] * 5 + [21.0])),
    ("hypercube", 32, _graph_hypercube(5), sorted(2.0 * i for i in range(6) for _ in range(math.comb(5, i)))),
]


@pytest.mark.parametrize("name,n,edges,spec", CLOSED_FORMS, ids=[c[0] for c in CLOSED_FORMS])
def test_closed_form_spectra(name, n, edges, spec):
    L = O.laplacian_csr(n, edges[0], edges[1])
    K = 5 if name != "cycle" else 5  # cycle: 0, then pairs (1,1), (2,2): K = 5 ends a pair
    res, lmax = _run_to_convergence(L, K)
    np.testing.assert_allclose(res.lam, spec[:K], rtol=0, atol=1e-9 * max(lmax, 1.0))
    assert res.resid.max() <= 1e-9 * lmax


def test_zero_eigenvalues_count_components():
    parts = []
    off = 0
    for c, (n_c, K_c, s) in enumerate([(60, 2, 7), (45, 3, 8), (30, 2, 9)]):
        g = W.dcsbm(n_c, K_c, seed=s)
        parts.append((g.src + off, g.dst + off))
        off += n_c
    src = np.concatenate([p[0] for p in parts])
    dst = np.concatenate([p[1] for p in parts])
    L = O.laplacian_csr(off, src, dst)
    # components by BFS, independent of the spectrum
    Ad = O.laplacian_dense(L) != 0
    seen = np.zeros(off, dtype=bool)
    comps = 0
    for s0 in range(off):
        if seen[s0]:
            continue
        comps += 1
        stack = [s0]
        seen[s0] = True
        while stack:
            v = stack.pop()
            for u in np.flatnonzero(Ad[v]):
                if not seen[u]:
                    seen[u] = True
                    stack.append(u)
    assert comps == 3
    res, lmax = _run_to_convergence(L, 5)
    assert np.sum(res.lam < 1e-8 * lmax) == comps
    assert res.lam[comps] > 1e-3


# ---------------------------------------------------------------- LOBPCG vs dense eigh


def test_lobpcg_converges_to_dense_eigenpairs():
    g = W.dcsbm(400, 6, seed=11)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    Ld = O.laplacian_dense(L)
    ev, V = np.linalg.eigh(Ld)
    K = 6
    assert ev[K] - ev[K - 1] > 1e-3  # the K/K+1 gap is open
    res, lmax = _run_to_convergence(L, K)
    assert np.max(np.abs(res.lam - ev[:K])) <= 1e-10 * ev[-1]
    assert O.sin_theta(V[:, :K], res.X) <= 1e-8


def test_first_pass_exact_when_basis_spans_space():
    """n = 2K: span[X R] is all of R^n after one pass, so pass 1 is an exact eigensolve."""
    K = 8
    g = W.dcsbm(2 * K, 2, seed=12, dmin=3, dmax=6)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    res = O.lobpcg(L, W.start_block(1, 2 * K, K), 1)
    np.testing.assert_allclose(res.lam, ev[:K], rtol=0, atol=1e-10 * ev[-1])
    assert res.resid.max() <= 1e-9 * ev[-1]


def test_lobpcg_invariants_per_pass():
    g = W.dcsbm(500, 7, seed=13)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    K = 7
    res = O.lobpcg(L, W.start_block(2, g.n, K), 15, keep_history=True)
    lams = [h[0] for h in res.history] + [res.lam]
    for a, b in zip(lams, lams[1:]):
        assert np.all(b <= a + 1e-10 * ev[-1])  # Ritz values never increase
    for lam in lams:
        assert np.all(lam >= ev[:K] - 1e-10 * ev[-1])  # Cauchy interlacing
    X = res.X
    assert np.max(np.abs(X.T @ X - np.eye(K))) < 1e-12
    G = X.T @ O.lap_apply(L, X)
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 1e-9 * ev[-1]
    np.testing.assert_allclose(np.diag(G), res.lam, rtol=0, atol=1e-9 * ev[-1])
    # residuals reported for the returned pairs
    R = O.lap_apply(L, X) - X * res.lam
    np.testing.assert_allclose(np.linalg.norm(R, axis=0), res.resid, rtol=1e-9, atol=1e-12)


def test_implicit_images_match_explicit_products():
    """One SpMM per pass (implicit LP, LX) is the same iteration as recomputing them."""
    g = W.dcsbm(800, 8, seed=14)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    X0 = W.start_block(3, g.n, 8)
    a = O.lobpcg(L, X0, 15)
    b = O.lobpcg(L, X0, 15, explicit=True)
    lmax = 2 * L.deg.max()
    assert np.max(np.abs(a.lam - b.lam)) <= 1e-10 * lmax
    assert O.sin_theta(a.X, b.X) <= 1e-9
    np.testing.assert_allclose(a.resid, b.resid, rtol=1e-7, atol=1e-10 * lmax)


def test_rayleigh_ritz_matches_generalized_eigh():
    rng = np.random.default_rng(3)
    m, K = 30, 7
    B0 = rng.standard_normal((m, m))
    GB = B0 @ B0.T + m * np.eye(m)
    A0 = rng.standard_normal((m, m))
    GA = A0 + A0.T
    theta, Y = O.rayleigh_ritz(GA, GB, K)
    w, V = sla.eigh(GA, GB)
    np.testing.assert_allclose(theta, w[:K], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Y.T @ GB @ Y, np.eye(K), atol=1e-11)
    np.testing.assert_allclose(GA @ Y, GB @ Y * theta, atol=1e-10)


def test_rayleigh_ritz_breakdown_on_dependent_basis():
    rng = np.random.default_rng(4)
    S = rng.standard_normal((50, 6))
    S = np.concatenate([S, S[:, :1] * 2.0], axis=1)  # a repeated direction
    with pytest.raises(O.BreakdownError):
        O.rayleigh_ritz(np.eye(7), S.T @ S, 3)


def test_cholqr():
    V = np.random.default_rng(5).standard_normal((100, 9))
    Q, C = O.cholqr(V)
    np.testing.assert_allclose(Q.T @ Q, np.eye(9), atol=1e-13)
    np.testing.assert_allclose(Q @ C.T, V, atol=1e-12)


def test_cholqr_drop_keeps_independent_columns_only():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((80, 3))
    V = np.column_stack([A[:, 0], A[:, 1], A[:, 0] - 2.0 * A[:, 1], np.zeros(80), A[:, 2],
                         3.0 * A[:, 2]])
    Q, kept = O.cholqr_drop(V)
    assert kept == [0, 1, 4]
    np.testing.assert_allclose(Q.T @ Q, np.eye(3), atol=1e-13)
    # every column of V lies in span(Q)
    np.testing.assert_allclose(Q @ (Q.T @ V), V, atol=1e-12)
    Q2, kept2 = O.cholqr_drop(A)
    assert kept2 == [0, 1, 2]
    Q3, _ = O.cholqr(A)
    np.testing.assert_allclose(Q2, Q3, atol=1e-13)


def test_lobpcg_stays_at_the_solution_far_past_convergence():
    """400 passes, no locking: columns reach roundoff around pass 150; the direction floor
    keeps the implicitly carried images from derailing the iteration afterwards (without it
    this run ends with Ritz values off by O(lambda_max))."""
    g = W.dcsbm(300, 4, seed=16)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    res = O.lobpcg(L, W.start_block(0, g.n, 4), 400)
    assert res.iters == 400 and res.dropped > 0
    np.testing.assert_allclose(res.lam, ev[:4], rtol=0, atol=1e-13 * ev[-1])
    assert res.resid.max() <= 1e-13 * ev[-1]
    R = O.lap_apply(L, res.X) - res.X * res.lam
    assert np.linalg.norm(R, axis=0).max() <= 1e-13 * ev[-1]


def test_jacobi_first_pass_is_rayleigh_ritz_on_x_and_dinv_r():
    """Pass 1 with precond="jacobi" is Rayleigh-Ritz on span{X, D^-1 R} (T = D^-1), built here
    directly: orthonormal basis by a dense QR, then eigh of the projected L."""
    g = W.dcsbm(400, 5, seed=22)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    Ld = O.laplacian_dense(L)
    K = 5
    X0 = W.start_block(3, g.n, K)
    Q0, _ = np.linalg.qr(X0)
    w0, V0 = np.linalg.eigh(Q0.T @ Ld @ Q0)
    X = Q0 @ V0
    R = Ld @ X - X * w0
    B, _ = np.linalg.qr(np.concatenate([X, R / L.deg[:, None]], axis=1))
    want = np.linalg.eigvalsh(B.T @ Ld @ B)[:K]
    res = O.lobpcg(L, X0, 1, precond="jacobi")
    np.testing.assert_allclose(res.lam, want, rtol=0, atol=1e-10 * 2 * L.deg.max())
    other = O.lobpcg(L, X0, 1)  # T = I gives a different first pass
    assert np.max(np.abs(other.lam - want)) > 1e-6


def test_jacobi_preconditioned_lobpcg_converges_faster_to_dense_eigenpairs():
    g = W.dcsbm(1500, 6, seed=21)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev, V = np.linalg.eigh(O.laplacian_dense(L))
    X0 = W.start_block(0, g.n, 6)
    pre = O.lobpcg(L, X0, 25, precond="jacobi")
    plain = O.lobpcg(L, X0, 25)
    err_pre = np.max(np.abs(pre.lam - ev[:6])) / ev[-1]
    err_plain = np.max(np.abs(plain.lam - ev[:6])) / ev[-1]
    assert err_pre <= 1e-7 and err_pre < 1e-3 * err_plain
    full = O.lobpcg(L, X0, 80, precond="jacobi")
    np.testing.assert_allclose(full.lam, ev[:6], rtol=0, atol=1e-12 * ev[-1])
    assert O.sin_theta(V[:, :6], full.X) <= 1e-8


def test_jacobi_leaves_isolated_vertices_unscaled():
    # two triangles and two isolated vertices: D has zeros, the preconditioned run still
    # reaches the dense eigenpairs (zero eigenvalue of multiplicity 4)
    src = np.array([0, 1, 2, 3, 4, 5], np.int64)
    dst = np.array([1, 2, 0, 4, 5, 3], np.int64)
    n = 12
    rng = np.random.default_rng(7)
    extra_s = rng.integers(6, 10, 12)
    extra_d = rng.integers(6, 10, 12)
    L = O.laplacian_csr(n, np.concatenate([src, extra_s]), np.concatenate([dst, extra_d]))
    assert np.sum(L.deg == 0) == 2
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    res = O.lobpcg(L, W.start_block(1, n, 4), 30, precond="jacobi")
    assert np.all(np.isfinite(res.lam))
    np.testing.assert_allclose(res.lam, ev[:4], rtol=0, atol=1e-10 * max(ev[-1], 1.0))


def test_soft_locking_freezes_converged_columns():
    g = W.dcsbm(400, 4, seed=15)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    res = O.lobpcg(L, W.start_block(0, g.n, 4), 300, tol_abs=1e-8 * ev[-1], tol_lock=1e-6 * ev[-1])
    np.testing.assert_allclose(res.lam, ev[:4], rtol=0, atol=1e-8 * ev[-1])


# ---------------------------------------------------------------- embedding, k-means


def test_embed_rows():
    X = np.array([[3.0, 4.0], [0.0, 0.0], [1e-40, 0.0], [-2.0, 0.0]])
    E = O.embed_rows(X)
    np.testing.assert_allclose(E, [[0.6, 0.8], [0, 0], [0, 0], [-1.0, 0.0]])


def test_kmeanspp_hand_worked():
    E = np.array([[0.0], [1.0], [3.0], [7.0]])
    # u0 = .1 -> floor(.4) = 0; D2 = [0,1,9,49], target .5*59 = 29.5 -> row 3;
    # D2 = [0,1,9,0], target .9*10 = 9 -> cumsum [0,1,10,10] -> row 2
    assert list(O.kmeanspp_seed(E, 3, np.array([0.1, 0.5, 0.9]))) == [0, 3, 2]
    # all points equal: sum D2 = 0 -> lowest unchosen rows
    Z = np.zeros((5, 2))
    assert list(O.kmeanspp_seed(Z, 3, np.array([0.7, 0.2, 0.2]))) == [3, 0, 1]


def test_lloyd_hand_worked_and_ties():
    E = np.array([[0.0], [2.0], [10.0], [12.0]])
    labels, C, it = O.lloyd(E, np.array([[0.0], [2.0]]), 10)
    # pass 1: [0,1,1,1] -> C = [0, 8]; pass 2: [0,0,1,1] -> C = [1, 11]; pass 3 repeats
    assert list(labels) == [0, 0, 1, 1] and it == 2
    np.testing.assert_allclose(C, [[1.0], [11.0]])
    # a point equidistant from two centroids goes to the lower index
    labels, _, _ = O.lloyd(np.array([[1.0]]), np.array([[0.0], [2.0]]), 1)
    assert labels[0] == 0
    # empty cluster keeps its centroid
    _, C, _ = O.lloyd(np.array([[0.0], [0.1]]), np.array([[0.0], [5.0]]), 3)
    assert C[1, 0] == 5.0


def test_lloyd_inertia_monotone():
    rng = np.random.default_rng(7)
    E = rng.standard_normal((300, 4))
    C0 = E[:6].copy()
    prev = np.inf
    for it in range(1, 12):
        labels, C, _ = O.lloyd(E, C0, it)
        # inertia of the assignment that produced C, measured against C
        inert = sum(np.sum((E[labels == j] - C[j]) ** 2) for j in range(6))
        assert inert <= prev + 1e-12
        prev = inert


def test_kmeans_distinct_points_zero_inertia():
    E = np.eye(5)
    labels, C, idx, inertia = O.kmeans(E, 5, np.array([0.3, 0.1, 0.5, 0.7, 0.9]), 10)
    assert inertia == 0.0
    assert len(set(labels.tolist())) == 5


def test_kmeans_bruteforce_optimum_small():
    rng = np.random.default_rng(8)
    E = rng.standard_normal((8, 2))
    k = 3
    best = np.inf
    for lab in itertools.product(range(k), repeat=8):
        lab = np.array(lab)
        if len(set(lab.tolist())) < k:
            continue
        best = min(best, sum(np.sum((E[lab == j] - E[lab == j].mean(0)) ** 2) for j in range(k)))
    got = np.inf
    for init in itertools.combinations(range(8), k):
        labels, C, _ = O.lloyd(E, E[list(init)], 100)
        got = min(got, sum(np.sum((E[labels == j] - C[j]) ** 2) for j in range(k)))
    assert abs(got - best) <= 1e-12


# ---------------------------------------------------------------- metrics, angles


def test_metrics_hand_worked():
    assert O.partition_metrics([0, 0, 1, 1], [5, 5, 7, 7]) == (1.0, 1.0, 1.0)
    pm, pr, pp = O.partition_metrics([0, 0, 1, 1, 1], [0, 0, 0, 0, 0])
    # truth pairs: C(2,2)+C(3,2) = 4; found pairs C(5,2) = 10; both = 4
    assert (pm, pr, pp) == (3 / 5, 1.0, 0.4)
    # contingency [[2,1],[0,3]]: matched 5/6; both = 1 + 3 = 4; truth 3+3=6; found 1+6=7
    pm, pr, pp = O.partition_metrics([0, 0, 0, 1, 1, 1], [0, 0, 1, 1, 1, 1])
    assert pm == 5 / 6 and abs(pr - 4 / 6) < 1e-15 and abs(pp - 4 / 7) < 1e-15


def test_matching_equals_bruteforce_permutations():
    rng = np.random.default_rng(9)
    for k in range(2, 7):
        truth = rng.integers(0, k, 60)
        found = rng.integers(0, k, 60)
        best = 0
        for perm in itertools.permutations(range(k)):
            best = max(best, sum(int(np.sum((truth == t) & (found == perm[t]))) for t in range(k)))
        assert abs(O.partition_metrics(truth, found)[0] - best / 60) < 1e-15


def test_sin_theta_known_angle():
    t = 0.3
    A = np.array([[1.0], [0.0], [0.0]])
    B = np.array([[math.cos(t)], [math.sin(t)], [0.0]])
    assert abs(O.sin_theta(A, B) - math.sin(t)) < 1e-15
    Q = np.linalg.qr(np.random.default_rng(1).standard_normal((20, 4)))[0]
    assert O.sin_theta(Q, Q @ np.diag([1, -2, 3, 5.0])) < 1e-14


def test_planted_partition_fully_recovered():
    """Sec. IV / abstract: well-separated planted blocks are recovered 100%."""
    g = W.dcsbm(600, 4, seed=21, ratio=20.0)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    labels, res, E, idx = O.partition(L, W.start_block(0, g.n, 4), 4, W.kmeans_uniforms(0, 4), 20, 50)
    assert O.partition_metrics(g.truth, labels) == (1.0, 1.0, 1.0)


# ---------------------------------------------------------------- CPQR assignment (Sec. II.A)


def test_cpqr_pivots_match_lapack_on_generic_input():
    import scipy.linalg as sla2

    Y = np.random.default_rng(31).standard_normal((300, 9))
    piv = O.cpqr_pivots(Y, 9)
    _, _, P = sla2.qr(Y.T, pivoting=True, mode="economic")
    assert piv == [int(p) for p in P[:9]]


def test_cpqr_recovers_planted_blocks_and_ignores_column_signs():
    rng = np.random.default_rng(32)
    k, n = 5, 400
    truth = rng.integers(0, k, n)
    basis, _ = np.linalg.qr(rng.standard_normal((k, k)))  # any rotation of the indicators
    Y = np.eye(k)[truth] @ basis + 0.05 * rng.standard_normal((n, k))
    labels, piv = O.cpqr_assign(Y, k)
    assert len(set(truth[piv])) == k  # one pivot per block
    pm, _, _ = O.partition_metrics(truth, labels)
    assert pm == 1.0
    D = np.diag([1.0, -1.0, 1.0, -1.0, -1.0])
    labels2, piv2 = O.cpqr_assign(Y @ D, k)
    assert piv2 == piv and np.array_equal(labels2, labels)


# ---------------------------------------------------------------- hard locking (Sec. IV)


def test_constrained_lobpcg_finds_the_next_eigenpairs():
    g = W.dcsbm(600, 5, seed=41)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev, V = np.linalg.eigh(O.laplacian_dense(L))
    res = O.lobpcg(L, W.start_block(4, g.n, 3), 200, constraint=V[:, :3])
    np.testing.assert_allclose(res.lam, ev[3:6], rtol=0, atol=1e-10 * ev[-1])
    assert np.max(np.abs(V[:, :3].T @ res.X)) <= 1e-8


def test_block_hard_locking_reproduces_dense_eigenpairs():
    g = W.dcsbm(600, 6, seed=42)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    ev, V = np.linalg.eigh(O.laplacian_dense(L))
    X0 = W.start_block(5, g.n, 6)
    res = O.lobpcg_blocks(L, X0, 2, 300)
    np.testing.assert_allclose(res.lam, ev[:6], rtol=0, atol=1e-9 * ev[-1])
    np.testing.assert_allclose(res.X.T @ res.X, np.eye(6), atol=1e-8)
    assert O.sin_theta(V[:, :6], res.X) <= 1e-6


# ------------------------------------------------------------------ eigengap cluster count (f1)


def _clique_union(c, s):
    src, dst = [], []
    for b in range(c):
        for i in range(s):
            for j in range(i + 1, s):
                src.append(b * s + i)
                dst.append(b * s + j)
    return c * s, np.array(src, np.int32), np.array(dst, np.int32)


@pytest.mark.parametrize("c,s", [(2, 4), (3, 5), (5, 7)])
def test_eigengap_counts_disjoint_cliques(c, s):
    """c disjoint cliques K_s: Laplacian spectrum 0 (c times) then s (c(s-1) times)."""
    n, src, dst = _clique_union(c, s)
    ev = np.linalg.eigvalsh(O.laplacian_dense(O.laplacian_csr(n, src, dst)))
    closed = np.array([0.0] * c + [float(s)] * (c * (s - 1)))
    np.testing.assert_allclose(ev, closed, atol=1e-9)
    assert O.eigengap_k(ev[:c + 3], floor=1e-9) == c
    assert O.eigengap_k(closed[:c + 3]) == c


def test_eigengap_none_on_a_path():
    """Path P_n: lam_j = 2 - 2 cos(pi j / n); increments grow by at most 3x (j = 1), so no
    increment is 4x the ones before it."""
    n = 60
    src = np.arange(n - 1, dtype=np.int32)
    dst = src + 1
    ev = np.linalg.eigvalsh(O.laplacian_dense(O.laplacian_csr(n, src, dst)))
    closed = 2 - 2 * np.cos(np.pi * np.arange(n) / n)
    np.testing.assert_allclose(ev, closed, atol=1e-12)
    assert O.eigengap_k(ev[:20], floor=1e-12) == 0
    assert O.eigengap_k(ev[:20], ratio=2.9, floor=1e-12) == 2  # the 3x step at j = 1


def test_eigengap_counts_strong_planted_blocks():
    rng = np.random.default_rng(5)
    K, s = 6, 40
    truth = np.repeat(np.arange(K), s)
    n = K * s
    iu = np.triu_indices(n, 1)
    p = np.where(truth[iu[0]] == truth[iu[1]], 0.5, 0.004)
    keep = rng.random(p.size) < p
    ev = np.linalg.eigvalsh(O.laplacian_dense(
        O.laplacian_csr(n, iu[0][keep].astype(np.int32), iu[1][keep].astype(np.int32))))
    assert O.eigengap_k(ev[:K + 4], floor=1e-9) == K


def test_eigengap_reading_edge_cases():
    # fewer than three values, or no increments: no gap
    assert O.eigengap_k([0.0, 5.0]) == 0
    assert O.eigengap_k(np.zeros(6)) == 0
    # the first increment is never a gap by itself (it has nothing to be compared with)
    assert O.eigengap_k([0.0, 10.0, 10.1, 10.2]) == 0
    # strict comparison: an increment exactly ratio times the largest before it is no gap
    assert O.eigengap_k([0.0, 1.0, 5.0], ratio=4.0) == 0
    assert O.eigengap_k([0.0, 1.0, 5.0 + 1e-9], ratio=4.0) == 2
    # increments at or below the floor count as zero; input order does not matter
    assert O.eigengap_k([3.0, 1e-12, 0.0, 2e-12], floor=1e-9) == 3
    assert O.eigengap_k([3.0, 1e-12, 0.0, 2e-12], floor=0.0) == 3


# ---------------------------------------------------------------- lambda_max (the tolerance scale)


def test_lambda_max_closed_forms_and_lanczos():
    cases = [(_graph_complete(15), 15, 15.0), (_graph_star(20), 20, 20.0),
             (_graph_path(30), 30, 2 + 2 * math.cos(math.pi / 30)),
             (_graph_hypercube(5), 32, 10.0)]
    for (src, dst), n, ref in cases:
        L = O.laplacian_csr(n, src, dst)
        assert abs(O.lambda_max(L) - ref) <= 1e-12 * ref
        assert abs(O.lambda_max(L, dense_below=0) - ref) <= 1e-10 * ref  # Lanczos branch
    g = W.dcsbm(1500, 9, seed=2)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    dense = O.lambda_max(L)
    assert abs(O.lambda_max(L, dense_below=0) - dense) <= 1e-10 * dense
    assert dense <= 2 * L.deg.max()


# ---------------------------------------------------------------- LOBPCG trajectory vs SciPy


def _scipy_history(L, X0, iters, M=None, Y=None):
    """Ritz values of scipy.sparse.linalg.lobpcg (the implementation the paper ran, Sec. II.B)
    before the loop and after each of `iters` passes, every column active (tol = 1e-300)."""
    import warnings

    import scipy.sparse as sp
    import scipy.sparse.linalg as ssla

    A = (sp.diags(L.deg) - L.W()).tocsr()
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        _, _, lh, rh = ssla.lobpcg(A, X0.copy(), M=M, Y=Y, largest=False, tol=1e-300,
                                   maxiter=iters, retLambdaHistory=True,
                                   retResidualNormsHistory=True)
    lams, rhos = [], []
    for i in range(iters + 1):
        o = np.argsort(np.asarray(lh[i]))
        lams.append(np.asarray(lh[i])[o])
        rhos.append(np.asarray(rh[i])[o] if i < iters else None)
    return lams, rhos


def _oracle_history(mod, L, X0, iters, **kw):
    """Ritz values before the loop and after each pass; residual norms before each pass."""
    res = mod.lobpcg(L, X0, iters, keep_history=True, **kw)
    return [h[0] for h in res.history] + [res.lam], [h[1] for h in res.history] + [None]


def _worst(ours, ref):
    (la, ra), (lb, rb) = ours, ref
    w = max(np.max(np.abs(a - b)) for a, b in zip(la, lb))
    return max([w] + [np.max(np.abs(a - b)) for a, b in zip(ra, rb) if a is not None])


def _trajectory_case(kind):
    if kind == "plain":
        g = W.dcsbm(2000, 11, seed=0)
        L = O.laplacian_csr(g.n, g.src, g.dst)
        return L, W.start_block(0, g.n, 11), {}, {}
    g = W.dcsbm(1500, 9, seed=3)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    X0 = W.start_block(4, g.n, 9)
    if kind == "jacobi":
        import scipy.sparse.linalg as ssla

        t = np.where(L.deg > 0, L.deg, 1.0)
        M = ssla.LinearOperator((g.n, g.n), matvec=lambda v: v.reshape(g.n, -1)[:, 0] / t,
                                matmat=lambda V: V / t[:, None], dtype=float)
        return L, X0, {"precond": "jacobi"}, {"M": M}
    Yc = np.linalg.eigh(O.laplacian_dense(L))[1][:, :3]  # hard locking against 3 eigenvectors
    return L, X0[:, 3:], {"constraint": Yc}, {"Y": Yc}


@pytest.mark.parametrize("kind", ["plain", "jacobi", "constraint"])
def test_lobpcg_trajectory_matches_scipy_lobpcg(kind):
    """Pass by pass, the oracle's Ritz values equal those of SciPy's lobpcg from the same
    start block (unpreconditioned, Jacobi-preconditioned, and constrained to the complement
    of exact eigenvectors), while the K/K+1 gap is open and nothing has converged: the
    orthonormal-basis form spans the same trial subspaces as Knyazev's [X W P]."""
    L, X0, kw, skw = _trajectory_case(kind)
    lmax = O.lambda_max(L)
    ev = np.linalg.eigvalsh(O.laplacian_dense(L))
    K = X0.shape[1] + (3 if kind == "constraint" else 0)
    assert ev[K] - ev[K - 1] > 1e-2  # the gap is open
    ours = _oracle_history(O, L, X0, 10, **kw)
    ref = _scipy_history(L, X0, 10, **skw)
    assert len(ours[0]) == len(ref[0]) == 11
    for i, (a, b) in enumerate(zip(ours[0], ref[0])):
        assert np.max(np.abs(a - b)) <= 1e-10 * lmax, (kind, "lambda", i)
    for i, (a, b) in enumerate(zip(ours[1][:10], ref[1][:10])):
        assert np.max(np.abs(a - b)) <= 1e-10 * lmax, (kind, "residual norm", i)
    assert np.max(ours[0][-1] - ev[3 if kind == "constraint" else 0:K]) > 1e-6 * lmax


MUTATIONS = [
    ("P drops P_a Y_P", "Pn = Pn + blocks[2][0] @ Yp", "Pn = Pn"),
    ("X update without P", "X = X @ Yx + Pn", "X = X @ Yx + Ra @ Yr"),
    ("LP image drops LP_a Y_P", "LPn = LPn + blocks[2][1] @ Yp", "LPn = LPn"),
    ("residual sign", "R = LX - X * lam[None, :]\n        rho", "R = LX + X * lam[None, :]\n        rho"),
    ("Y_R taken from the X rows", "Yx, Yr = Y[:K], Y[K:K + ka]", "Yx, Yr = Y[:K], Y[:ka]"),
    ("largest Ritz pairs kept", "return theta[:K], Y", "return theta[-K:], Y"),
    ("image of the unprojected residual", "LRa = lap_apply(L, Ra)",
     "LRa = lap_apply(L, R[:, act]) if True else None"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_trajectory_pin_catches_planted_mistakes(name, old, new):
    """A plausible mistake planted in a copy of the oracle's source (a dropped term, a sign,
    a wrong block of Y, the wrong end of the spectrum, a missing back-transformation) makes
    the pass-by-pass comparison with SciPy fail."""
    import importlib
    import sys
    import types

    src = open(importlib.import_module("oracle.spectral").__file__).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle_mutant")
    sys.modules["oracle_mutant"] = mod  # dataclasses look their module up while being built
    try:
        exec(compile(src.replace(old, new), "oracle_mutant", "exec"), mod.__dict__)
    finally:
        del sys.modules["oracle_mutant"]
    L, X0, kw, skw = _trajectory_case("plain")
    lmax = O.lambda_max(L)
    ref = _scipy_history(L, X0, 10)
    try:
        ours = _oracle_history(mod, L, X0, 10, **kw)
    except Exception:
        return  # the mutant breaks down outright: caught
    assert _worst(ours, ref) > 1e-10 * lmax, name


@pytest.mark.parametrize("n,K", [(1000, 11), (50000, 44)])
def test_rounding_safeguards_do_not_fire_on_the_parity_configs(n, K):
    """The rounding-level safeguards (residual and direction columns at the rounding floor,
    dependent residual columns dropped below PIVOT_TOL, the P block dropped on a Cholesky
    breakdown) fire on no pass of the 20-pass runs the GPU parity tests compare: on these
    inputs the oracle is exactly the textbook iteration."""
    g = W.dcsbm(n, K, seed=0)
    L = O.laplacian_csr(g.n, g.src, g.dst)
    X0 = W.start_block(0, g.n, K).astype(np.float32).astype(np.float64)
    res = O.lobpcg(L, X0, 20)
    assert res.iters == 20 and res.dropped == 0 and res.fallbacks == 0
