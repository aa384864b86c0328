"""FP64 oracle: Laplacian, LOBPCG, row embedding, k-means++ / Lloyd, partition metrics.

TEST INFRASTRUCTURE ONLY.  Plain NumPy/SciPy in float64: every step is written out in the
order the method states it, with library primitives (dense/sparse matmul, Cholesky,
triangular solve, dense symmetric eigendecomposition, cumulative sum, Hungarian
assignment) as the only building blocks.  No blocking, fusion or reordering.

Parity status of each function is stated in its docstring ("pinned by ...").

Paper: Zhuzhunashvili & Knyazev, HPEC 2017 (arXiv 1708.07481).
  Sec. II.A  -- W <- W + W' (logical or algebraic sum), D = row sums, L = D - W; the rows of
                the eigenvector block are clustered (k-means++ or pivoted QR).
  Sec. II.B  -- LOBPCG for the smallest eigenpairs, optionally preconditioned.
  Sec. III   -- random Gaussian start, warm starts (zero fill for new vertices), the
                matrix-free product diagL.*X - A*X - (X'*A)'.
  Sec. IV    -- soft locking; Gram matrices cost n*l^2; PM / PR / PP metrics.
LOBPCG: Knyazev, SIAM J. Sci. Comput. 23(2), 2001 (Rayleigh-Ritz on span{X, W, P}); the
basis handling (residual projected against X, Cholesky-QR of the residual and direction
blocks) is the form of SciPy's lobpcg, which is the implementation the paper ran.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.optimize as sopt
import scipy.sparse as sp

# --------------------------------------------------------------------------------------
# Laplacian (Sec. II.A, Sec. III)
# --------------------------------------------------------------------------------------


@dataclass
class Csr:
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col_idx: np.ndarray  # int64 [nnz]
    val: np.ndarray  # float64 [nnz] entries of the symmetrized W (1 for a logical sum)
    deg: np.ndarray  # float64 [n]   D = row sums of W

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def W(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.n, self.n))


def laplacian_csr(n, src, dst, w=None, sym: str = "logical") -> Csr:
    """Symmetrized adjacency W and degrees D of L = D - W (Sec. II.A).

    ``sym='logical'``: W[u, v] = 1 iff u != v and (u->v or v->u) is an edge (the logical sum
    for unweighted graphs, duplicates merged).  ``sym='algebraic'``: W = A + A' with A[u, v]
    the summed weights of the edges u->v (1 per edge when ``w`` is None).  Self-loops are
    dropped: a loop adds the same amount to D[u, u] and W[u, u], so L is unchanged.

    Pinned by: dense brute-force construction, L*1 = 0, symmetry, sum(deg) = nnz, PSD,
    and (algebraic) the paper's matrix-free product diagL.*X - A*X - (X'*A)'.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("edge endpoint out of range")
    ww = np.ones(src.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    keep = src != dst
    src, dst, ww = src[keep], dst[keep], ww[keep]
    rows = np.concatenate([src, dst])
    cols = np.concatenate([dst, src])
    vals = np.concatenate([ww, ww])
    keys = rows * n + cols
    uk, inv = np.unique(keys, return_inverse=True)
    if sym == "logical":
        v = np.ones(uk.shape[0])
    elif sym == "algebraic":
        v = np.zeros(uk.shape[0])
        np.add.at(v, inv, vals)
    else:
        raise ValueError(sym)
    r = uk // n
    c = uk % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(r, minlength=n))
    deg = np.zeros(n)
    np.add.at(deg, r, v)
    return Csr(n=n, row_ptr=row_ptr, col_idx=c, val=v, deg=deg)


def lap_apply(L: Csr, V: np.ndarray) -> np.ndarray:
    """L V = D V - W V (Sec. II.A), V an n x k block."""
    V = np.asarray(V, dtype=np.float64)
    return L.deg[:, None] * V - L.W() @ V


def laplacian_dense(L: Csr) -> np.ndarray:
    """Dense L = D - W of a small graph."""
    return np.diag(L.deg) - L.W().toarray()


def lambda_max(L: Csr, dense_below: int = 2000) -> float:
    """||L||_2 = the largest eigenvalue of the positive semidefinite L = D - W (Sec. II.A):
    the scale against which eigenvalue errors and residual norms are stated.

    n <= dense_below: dense symmetric eigendecomposition of L.  Larger graphs: Lanczos
    (ARPACK through scipy.sparse.linalg.eigsh) for the largest eigenvalue, to 1e-12 relative.

    Pinned by: closed forms (complete graph K_n and star S_n: n; path P_n: 2 + 2 cos(pi / n);
    hypercube Q_d: 2 d), the Lanczos branch equal to the dense one on a DC-SBM graph, and
    lambda_max <= 2 max_i d_i (Gershgorin).
    """
    if L.n == 0:
        return 0.0
    if L.n <= dense_below:
        return float(np.linalg.eigvalsh(laplacian_dense(L))[-1])
    import scipy.sparse.linalg as ssla

    A = (sp.diags(L.deg) - L.W()).tocsr()
    v0 = np.ones(L.n) + np.arange(L.n) % 7  # fixed start vector: the result is deterministic
    w = ssla.eigsh(A, k=1, which="LA", tol=1e-12, v0=v0, return_eigenvectors=False)
    return float(w[0])


# --------------------------------------------------------------------------------------
# LOBPCG (Sec. II.B, Sec. III, Sec. IV; Knyazev 2001)
# --------------------------------------------------------------------------------------


class BreakdownError(RuntimeError):
    """The Gram matrix of the trial basis is not numerically positive definite."""


# A Cholesky pivot below this (relative to the unit diagonal after scaling) counts as a
# breakdown of the trial basis: a column whose part orthogonal to the columns before it is
# below 1e-5 of its norm would be normalized with its rounding error amplified 1e5-fold.
PIVOT_TOL = 1e-10

# A direction column p_j (X unit) whose norm after projection against X is at or below this
# rounding level is left out of the pass (64 units of roundoff of float64); a residual column
# at or below DIR_FLOOR times the Gershgorin bound 2 max_i d_i on ||L|| likewise.
DIR_FLOOR = 64.0 * 2.0 ** -53


def _chol_lower(G: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor of a symmetric matrix with unit-ish diagonal, or breakdown."""
    try:
        C = np.linalg.cholesky(G)
    except np.linalg.LinAlgError as e:
        raise BreakdownError(str(e)) from None
    if np.min(np.diag(C)) ** 2 <= PIVOT_TOL * np.max(np.diag(G)):
        raise BreakdownError("tiny pivot")
    return C


def cholqr(V: np.ndarray):
    """Cholesky-QR with column scaling: V = Q C' with Q'Q = I, C lower triangular.

    G = V'V; s = diag(G)^-1/2; s G s = Cs Cs'; Q = V diag(s) Cs^-T; C = diag(1/s) Cs.
    The scaling keeps columns of very different norms (converged residuals) from
    tripping the relative pivot test.
    """
    G = V.T @ V
    G = 0.5 * (G + G.T)
    d = np.diag(G)
    if np.any(d <= 0):
        raise BreakdownError("zero column")
    s = 1.0 / np.sqrt(d)
    Cs = _chol_lower(G * s[:, None] * s[None, :])
    Q = sla.solve_triangular(Cs, (V * s[None, :]).T, lower=True).T
    return Q, Cs / s[:, None]


def cholqr_drop(V: np.ndarray, tol: float = PIVOT_TOL):
    """Cholesky-QR of the columns of V that are independent to working accuracy.

    Column k is kept when its pivot in the Cholesky factorization of the scaled Gram
    diag(s) V'V diag(s) restricted to the kept columns before it and k itself exceeds tol,
    i.e. when the part of v_k / ||v_k|| orthogonal to the kept columns has squared norm
    above tol; a zero column is never kept.  Returns (Q, kept) with Q = CholQR(V[:, kept]).
    Used for the residual block, whose converged columns sink to rounding noise that need
    not be independent (the block is rank-deficient to working accuracy).

    Pinned by: exactly dependent columns dropped, independent ones kept, span preserved.
    """
    G = V.T @ V
    G = 0.5 * (G + G.T)
    d = np.diag(G).copy()
    kept = []
    for k in range(V.shape[1]):
        if d[k] <= 0:
            continue
        idx = kept + [k]
        s = 1.0 / np.sqrt(d[idx])
        Gs = G[np.ix_(idx, idx)] * s[:, None] * s[None, :]
        try:
            C = np.linalg.cholesky(Gs)
        except np.linalg.LinAlgError:
            continue
        if C[-1, -1] ** 2 > tol:
            kept.append(k)
    if not kept:
        return V[:, :0].copy(), kept
    Q, _ = cholqr(V[:, kept])
    return Q, kept


def rayleigh_ritz(GA: np.ndarray, GB: np.ndarray, K: int):
    """K smallest eigenpairs of the pencil (GA, GB): GA y = theta GB y, Y' GB Y = I.

    Steps: symmetrize; scale by s = diag(GB)^-1/2; Cholesky  s GB s = C C'; reduce
    M = C^-1 (s GA s) C^-T; eigendecompose M (ascending); Y = diag(s) C^-T V[:, :K].
    Raises BreakdownError if the scaled GB has a pivot <= PIVOT_TOL.

    Pinned by: LOBPCG convergence to dense eigenpairs; exactness when the basis spans R^n.
    """
    GA = 0.5 * (GA + GA.T)
    GB = 0.5 * (GB + GB.T)
    d = np.diag(GB)
    if np.any(d <= 0):
        raise BreakdownError("zero column in the trial basis")
    s = 1.0 / np.sqrt(d)
    Bs = GB * s[:, None] * s[None, :]
    As = GA * s[:, None] * s[None, :]
    C = _chol_lower(Bs)
    T = sla.solve_triangular(C, As, lower=True)  # C^-1 As
    M = sla.solve_triangular(C, T.T, lower=True)  # C^-1 (C^-1 As)' = C^-1 As C^-T
    M = 0.5 * (M + M.T)
    theta, V = np.linalg.eigh(M)
    Y = sla.solve_triangular(C.T, V[:, :K], lower=False)  # C^-T V_K
    Y = Y * s[:, None]
    return theta[:K], Y


@dataclass
class LobpcgResult:
    lam: np.ndarray  # [K] Ritz values, ascending
    X: np.ndarray  # [n, K] Ritz vectors
    resid: np.ndarray  # [K] ||L x_j - lam_j x_j||_2 of the returned pairs
    iters: int  # loop passes performed after the initial Rayleigh-Ritz
    fallbacks: int  # iterations where the direction block P had to be dropped
    history: list = field(default_factory=list)  # per pass: (lam, resid-before-update)
    dropped: int = 0  # residual columns dropped as dependent (cholqr_drop), summed over passes


def lobpcg(L: Csr, X0: np.ndarray, iters: int, tol_abs: float = 0.0, tol_lock: float = 0.0,
           keep_history: bool = False, explicit: bool = False,
           precond: str | None = None, constraint: np.ndarray | None = None) -> LobpcgResult:
    """Unpreconditioned block LOBPCG for the K smallest eigenpairs of L (Sec. II.B, III).

    Start: X = CholQR(CholQR(X0)); LX = L X; Rayleigh-Ritz on span(X).
    Each pass i = 1..iters:
      R = LX - X diag(lam), rho_j = ||r_j||; active = {j : rho_j > tol_lock} (soft locking,
      Sec. IV); stop when nothing is active or max rho <= tol_abs.
      R_a <- R_a - X (X' R_a); columns at the rounding floor (norm <= DIR_FLOOR * 2 max d)
      are left out, which soft-locks pairs that cannot improve; R_a <- CholQR of its
      columns independent to working accuracy (cholqr_drop: residuals of converged columns
      sink to rounding noise, which need not be independent); LR_a = L R_a.
      For i > 1: P_a <- P_a - [X R_a] F with F = [X R_a]' P_a, then CholQR(P_a); LP_a is
      transformed alike (the orthonormal trial basis of Hetmaniuk & Lehoucq 2006).  Columns
      of P_a whose part orthogonal to X is at rounding level (DIR_FLOOR) are left out of
      the pass: past convergence the step sinks to roundoff, and the implicitly carried
      image LP would otherwise be normalized noise that derails the iteration.
      S = [X R_a P_a], LS = [LX LR_a LP_a]; Rayleigh-Ritz on (S' LS, S' S), K smallest.
      With Y = [Y_X; Y_R; Y_P]: P = R_a Y_R + P_a Y_P, X = X Y_X + P (LX, LP alike).
      A breakdown of the Cholesky of P's Gram (P inside span{X, R}) or of the trial basis
      drops P for that pass; a breakdown without P is raised.
    ``precond="jacobi"`` applies the preconditioner T = D^-1 (rows of isolated vertices
    unscaled) to R_a before the projection: the trial basis is [X, T R_a, P_a] (the optional T
    of preconditioned LOBPCG, Sec. II.B); the rounding floor for R_a is divided by max d.
    Residual norms, the tolerance and locking refer to the unpreconditioned R.
    ``constraint`` (n x c, orthonormal columns) runs the iteration in its orthogonal
    complement (hard locking, Sec. IV): the start block and every (preconditioned) residual
    block are projected off it before anything else, so X and P stay in the complement.
    One multiplication by L per pass (Sec. III): LP and LX are carried along implicitly.
    ``explicit=True`` recomputes LX, LR_a and LP_a as products with L instead -- the same
    iteration in exact arithmetic, stable when a direction column sinks to rounding level
    in runs driven to tight tolerances.
    When every column is active this spans the same trial subspaces as Knyazev's basis
    [X R P] (span{X_new, P_new} = span{X_new, X_old}), so the iterates agree in exact
    arithmetic with SciPy's lobpcg, which the paper used.
    Returns the final Ritz values, vectors, and residual norms of the returned pairs.

    Pinned by: dense eigendecomposition (converged runs), closed-form Laplacian spectra,
    exactness when [X R] spans R^n, monotone Ritz values, orthonormality.
    """
    X0 = np.asarray(X0, dtype=np.float64)
    n, K = X0.shape
    Yc = None
    if constraint is not None and np.asarray(constraint).shape[1] > 0:
        Yc = np.asarray(constraint, dtype=np.float64)
        X0 = X0 - Yc @ (Yc.T @ X0)
    X, _ = cholqr(X0)
    X, _ = cholqr(X)
    LX = lap_apply(L, X)
    G = X.T @ LX
    G = 0.5 * (G + G.T)
    lam, Q = np.linalg.eigh(G)
    X = X @ Q
    LX = LX @ Q
    P = LP = None
    hist = []
    fallbacks = 0
    dropped = 0
    done = 0
    dmax = float(np.max(L.deg, initial=0.0))
    res_floor = DIR_FLOOR * 2.0 * dmax
    if precond not in (None, "jacobi"):
        raise ValueError(precond)
    tinv = None
    if precond == "jacobi":
        tinv = np.where(L.deg > 0, L.deg, 1.0)
        if dmax > 0:
            res_floor /= dmax
    for _ in range(iters):
        R = LX - X * lam[None, :]
        rho = np.linalg.norm(R, axis=0)
        act = rho > tol_lock
        if keep_history:
            hist.append((lam.copy(), rho.copy()))
        if not act.any() or rho.max() <= tol_abs:
            break
        Ra = R[:, act]
        if tinv is not None:
            Ra = Ra / tinv[:, None]
        if Yc is not None:
            Ra = Ra - Yc @ (Yc.T @ Ra)
        Ra = Ra - X @ (X.T @ Ra)
        # a residual at the rounding floor cannot improve its Ritz pair: leave it out (this
        # soft-locks the pair at the accuracy the arithmetic allows)
        Ra = Ra[:, np.linalg.norm(Ra, axis=0) > res_floor]
        Ra, kept_r = cholqr_drop(Ra)
        dropped += int(act.sum()) - len(kept_r)
        LRa = lap_apply(L, Ra)
        blocks = [(X, LX), (Ra, LRa)]
        if P is not None:
            Pa, LPa = P[:, act], LP[:, act]
            # against X first; a column whose part orthogonal to X has sunk to rounding
            # level (norm <= DIR_FLOOR, X unit) is left out: it carries no step, and its
            # implicitly updated image would be amplified noise once normalized
            F = X.T @ Pa
            Pa = Pa - X @ F
            LPa = LPa - LX @ F
            live = np.linalg.norm(Pa, axis=0) > DIR_FLOOR
            dropped += int((~live).sum())
            Pa, LPa = Pa[:, live], LPa[:, live]
            # then against R_a (orthogonal to X, so the two steps project against [X R_a])
            F = Ra.T @ Pa
            Pa = Pa - Ra @ F
            LPa = LPa - LRa @ F
            if Pa.shape[1] > 0:
                try:
                    Pa, Cp = cholqr(Pa)
                    if explicit:
                        LPa = lap_apply(L, Pa)
                    else:
                        LPa = sla.solve_triangular(Cp, LPa.T, lower=True).T
                    blocks.append((Pa, LPa))
                except BreakdownError:
                    fallbacks += 1
        try:
            theta, Y = _rr_blocks(blocks, K)
        except BreakdownError:
            if len(blocks) < 3:
                raise
            fallbacks += 1
            blocks = blocks[:2]
            theta, Y = _rr_blocks(blocks, K)
        ka = Ra.shape[1]
        Yx, Yr = Y[:K], Y[K:K + ka]
        Pn = Ra @ Yr
        LPn = LRa @ Yr
        if len(blocks) == 3:
            Yp = Y[K + ka:]
            Pn = Pn + blocks[2][0] @ Yp
            LPn = LPn + blocks[2][1] @ Yp
        X = X @ Yx + Pn
        LX = lap_apply(L, X) if explicit else LX @ Yx + LPn
        P, LP = Pn, LPn
        lam = theta
        done += 1
    R = LX - X * lam[None, :]
    return LobpcgResult(lam=lam, X=X, resid=np.linalg.norm(R, axis=0), iters=done,
                        fallbacks=fallbacks, history=hist, dropped=dropped)


def lobpcg_blocks(L: Csr, X0: np.ndarray, nb: int, iters: int, tol_abs: float = 0.0,
                  precond: str | None = None) -> LobpcgResult:
    """Hard locking (Sec. IV): the K = X0.shape[1] smallest eigenpairs computed nb columns at a
    time.  Block b starts from columns [b nb, (b + 1) nb) of X0 and runs lobpcg in the
    orthogonal complement of the Ritz vectors of the blocks before it; the blocks' Ritz
    vectors, values and residual norms are concatenated in order.

    Pinned by: converged block runs reproduce the dense eigenpairs; a block constrained by
    exact eigenvectors finds the next eigenvalues.
    """
    X0 = np.asarray(X0, dtype=np.float64)
    n, K = X0.shape
    Yc = np.zeros((n, 0))
    lams, res = [], []
    done = fb = drop = 0
    for b0 in range(0, K, nb):
        r = lobpcg(L, X0[:, b0:b0 + nb], iters, tol_abs=tol_abs, precond=precond,
                   constraint=Yc)
        Yc = np.concatenate([Yc, r.X], axis=1)
        lams.extend(r.lam.tolist())
        res.extend(r.resid.tolist())
        done += r.iters
        fb += r.fallbacks
        drop += r.dropped
    return LobpcgResult(lam=np.array(lams), X=Yc, resid=np.array(res), iters=done,
                        fallbacks=fb, dropped=drop)


def _rr_blocks(blocks, K):
    S = np.concatenate([b[0] for b in blocks], axis=1)
    LS = np.concatenate([b[1] for b in blocks], axis=1)
    return rayleigh_ritz(S.T @ LS, S.T @ S, K)


# --------------------------------------------------------------------------------------
# Embedding and k-means (Sec. II.A)
# --------------------------------------------------------------------------------------


def embed_rows(X: np.ndarray) -> np.ndarray:
    """Rows of the eigenvector block scaled to unit 2-norm; rows of norm < 1e-30 stay 0."""
    X = np.asarray(X, dtype=np.float64)
    nr = np.sqrt(np.sum(X * X, axis=1))
    E = np.zeros_like(X)
    ok = nr >= 1e-30
    E[ok] = X[ok] / nr[ok, None]
    return E


def _sqdist_to(E: np.ndarray, c: np.ndarray) -> np.ndarray:
    diff = E - c[None, :]
    return np.sum(diff * diff, axis=1)


def kmeanspp_seed(E: np.ndarray, k: int, u: np.ndarray) -> np.ndarray:
    """k-means++ seeding (Arthur & Vassilvitskii 2007), driven by the uniforms u[0..k-1].

    First seed: floor(u_0 n).  Seed t: with D2_i the squared distance of row i to its
    nearest chosen seed, take the first i whose cumulative sum of D2 exceeds u_t sum(D2)
    (clamped to the last row with D2 > 0); when sum(D2) = 0, the lowest unchosen row.

    Pinned by: hand-worked small cases in the tests.
    """
    E = np.asarray(E, dtype=np.float64)
    n = E.shape[0]
    idx = [min(int(np.floor(u[0] * n)), n - 1)]
    D2 = _sqdist_to(E, E[idx[0]])
    for t in range(1, k):
        total = float(np.sum(D2))
        if total > 0.0:
            c = np.cumsum(D2)
            i = int(np.searchsorted(c, u[t] * total, side="right"))
            if i >= n:
                i = int(np.flatnonzero(D2 > 0)[-1])
        else:
            chosen = set(idx)
            i = next(j for j in range(n) if j not in chosen)
        idx.append(i)
        D2 = np.minimum(D2, _sqdist_to(E, E[i]))
    return np.asarray(idx, dtype=np.int64)


def _assign(E: np.ndarray, C: np.ndarray) -> np.ndarray:
    d = np.stack([_sqdist_to(E, C[j]) for j in range(C.shape[0])], axis=1)
    return np.argmin(d, axis=1)  # first minimum = lowest cluster index on ties


def lloyd(E: np.ndarray, C0: np.ndarray, iters: int):
    """Lloyd iterations: assign every row to its nearest centroid (squared Euclidean,
    ties to the lowest index), then move each centroid to the mean of its rows (an empty
    cluster keeps its centroid); stop early when an assignment repeats the previous one.

    Returns (labels, centroids, iterations_run).  Pinned by: monotone inertia, brute-force
    optimum on tiny sets, zero inertia on k distinct points.
    """
    E = np.asarray(E, dtype=np.float64)
    C = np.array(C0, dtype=np.float64, copy=True)
    prev = None
    done = 0
    labels = _assign(E, C)
    for _ in range(iters):
        labels = _assign(E, C)
        if prev is not None and np.array_equal(labels, prev):
            break
        done += 1
        for j in range(C.shape[0]):
            mask = labels == j
            if mask.any():
                C[j] = E[mask].mean(axis=0)
        prev = labels
    return labels.astype(np.int64), C, done


def kmeans(E: np.ndarray, k: int, u: np.ndarray, iters: int = 50, init_idx=None):
    """k-means++ seeding followed by Lloyd; returns (labels, centroids, seed_idx, inertia)."""
    E = np.asarray(E, dtype=np.float64)
    idx = kmeanspp_seed(E, k, u) if init_idx is None else np.asarray(init_idx, dtype=np.int64)
    labels, C, _ = lloyd(E, E[idx], iters)
    inertia = float(sum(np.sum((E[labels == j] - C[j]) ** 2) for j in range(k)))
    return labels, C, idx, inertia


def partition(L: Csr, X0: np.ndarray, k: int, u: np.ndarray, iters: int = 20,
              kmeans_iters: int = 50, tol_abs: float = 0.0, tol_lock: float = 0.0,
              precond: str | None = None):
    """Spectral partition: LOBPCG block -> unit rows -> k-means (Sec. II.A)."""
    res = lobpcg(L, X0, iters, tol_abs=tol_abs, tol_lock=tol_lock, precond=precond)
    E = embed_rows(res.X)
    labels, C, idx, inertia = kmeans(E, k, u, kmeans_iters)
    return labels, res, E, idx


# --------------------------------------------------------------------------------------
# Metrics (Sec. IV) and subspace comparison
# --------------------------------------------------------------------------------------


# --------------------------------------------------------------------------------------
# Assignment by QR with column pivoting (Sec. II.A; Damle, Minden & Ying, arXiv 1609.08251)
# --------------------------------------------------------------------------------------


def cpqr_pivots(Y: np.ndarray, k: int) -> list:
    """The first k column pivots of a QR factorization with column pivoting of Y' (K x n).

    Greedy rule: at step t the column of the current residual with the largest 2-norm is
    chosen (the lowest index on ties); the residual is then projected off its direction
    (Gram-Schmidt: A <- A - q (q' A) with q the chosen column normalized).

    Pinned by: agreement with LAPACK's pivoted QR on generic inputs; one pivot per planted
    block on block-indicator inputs.
    """
    A = np.asarray(Y, dtype=np.float64).T.copy()
    piv = []
    for _ in range(k):
        norms = np.einsum("ij,ij->j", A, A)
        norms[piv] = -1.0
        j = int(np.argmax(norms))
        piv.append(j)
        nj = np.sqrt(norms[j])
        if nj == 0.0:  # the remaining columns are zero: nothing left to project off
            continue
        q = A[:, j] / nj
        A -= np.outer(q, q @ A)
    return piv


def cpqr_assign(Y: np.ndarray, k: int):
    """Cluster labels from the eigenvector block Y (n x K, K = k) by the CPQR method.

    Steps: C = Y'[:, pivots] (K x k) from cpqr_pivots; its polar factor Q = U V' (the SVD
    C = U S V'); label_i = argmax_j |(Y Q)_ij| (the lowest j on ties).  Returns
    (labels, pivots).

    Pinned by: exact recovery of planted blocks; invariance under sign flips of Y's columns
    (Y -> Y D leaves Y Q unchanged).
    """
    Y = np.asarray(Y, dtype=np.float64)
    piv = cpqr_pivots(Y, k)
    C = Y[piv, :].T
    U, _, Vt = np.linalg.svd(C)
    Q = U @ Vt
    scores = np.abs(Y @ Q)
    return np.argmax(scores, axis=1).astype(np.int64), piv


def eigengap_k(lam, ratio: float = 4.0, floor: float = 0.0) -> int:
    """Number of clusters from the gap in the smallest Laplacian eigenvalues (Sec. II.A).

    The paper compares the increments of the ascending eigenvalues and takes the first
    significantly large one; the eigenvalues below it count the clusters, and no such
    increment means no reliable multi-way partition.  Reading used here: with
    d_i = lam_{i+1} - lam_i (ascending lam, i = 0 .. l-2), increments at or below ``floor``
    (the accuracy of the eigenvalues) count as zero; the first i >= 1 with
    d_i > ratio * max(d_0 .. d_{i-1}) and d_i > 0 gives k = i + 1.  The first increment has no
    earlier one to be compared with, so k = 1 is never returned; 0 means no gap.

    Pinned by: disjoint cliques (closed-form spectrum: c zeros, then the clique size) give
    k = c; a path graph's smooth spectrum gives no gap; planted blocks with a strong
    within/between contrast give k = number of blocks (dense spectrum).
    """
    lam = np.sort(np.asarray(lam, dtype=np.float64))
    if lam.size < 3:
        return 0
    d = np.diff(lam)
    d = np.where(d > floor, d, 0.0)
    prev = d[0]
    for i in range(1, d.size):
        if d[i] > 0.0 and d[i] > ratio * prev:
            return i + 1
        prev = max(prev, d[i])
    return 0


def partition_metrics(truth, found):
    """(PM, PR, PP): optimal partition matching, pairwise recall, pairwise precision.

    PM = best one-to-one matching of truth and found blocks (Hungarian) / n;
    PR = sum_ij C(c_ij, 2) / sum_t C(n_t, 2); PP = sum_ij C(c_ij, 2) / sum_f C(n_f, 2),
    c_ij the contingency counts.  Pinned by hand-worked contingency tables.
    """
    truth = np.asarray(truth, dtype=np.int64)
    found = np.asarray(found, dtype=np.int64)
    n = truth.shape[0]
    _, ti = np.unique(truth, return_inverse=True)
    _, fi = np.unique(found, return_inverse=True)
    Cm = np.zeros((ti.max() + 1, fi.max() + 1), dtype=np.int64)
    np.add.at(Cm, (ti, fi), 1)
    r, c = sopt.linear_sum_assignment(-Cm)
    pm = Cm[r, c].sum() / n

    def pairs(x):
        return (x * (x - 1) // 2).sum()

    both = pairs(Cm)
    pt = pairs(Cm.sum(axis=1))
    pf = pairs(Cm.sum(axis=0))
    pr = both / pt if pt else 1.0
    pp = both / pf if pf else 1.0
    return float(pm), float(pr), float(pp)


def sin_theta(A: np.ndarray, B: np.ndarray) -> float:
    """Largest principal angle sine between span(A) and span(B) (same column count).

    Q_A, Q_B orthonormal bases; E = Q_B - Q_A (Q_A' Q_B) formed explicitly; sin = ||E||_2.
    """
    Qa, _ = np.linalg.qr(np.asarray(A, dtype=np.float64))
    Qb, _ = np.linalg.qr(np.asarray(B, dtype=np.float64))
    Em = Qb - Qa @ (Qa.T @ Qb)
    return float(np.linalg.norm(Em, 2))
