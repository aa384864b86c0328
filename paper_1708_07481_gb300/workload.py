"""Seeded synthetic inputs: DC-SBM graphs, streaming stages, start blocks, k-means uniforms.

This module is shared by the tests, the bench and the smoke check; it holds none of the
spectral-clustering arithmetic (no Laplacian, no eigensolver, no k-means), only the
random inputs both the CUDA path and the FP64 oracle consume.

The paper measures on the HPEC Graph Challenge stochastic-block-partition datasets
(Sec. III), which are not available here; a degree-corrected stochastic block model
with the same shapes stands in for them:

1. Block proportions ~ Dirichlet(alpha * 1_K) from Gamma(alpha) draws (Marsaglia-Tsang);
   integer sizes by largest remainder (each >= 1); vertices go to blocks through a
   seeded random permutation, so vertex ids carry no block order.
2. Out-degree d_v from the discrete power law P(d) ~ d^-2.5 on {dmin..dmax} by inverse CDF.
3. Each out-edge of v stays in block b(v) with probability r/(r+1) (r = within:between
   ratio, read as a count ratio), else goes to another block chosen in proportion to its
   size; the target inside the chosen block is drawn in proportion to d (the degree
   correction theta_v = d_v / sum_{u in b(v)} d_u).  Self-loops are redrawn; multi-edges
   stay in the list (the Laplacian build merges them).
4. Streaming: "emerging edges" reveals a seeded permutation of the edge list in 10
   slices; "snowball" relabels vertices in BFS order and reveals 10% of them per stage
   together with the edges among them (old vertices first, in the same order, Sec. III).

Random numbers come from SplitMix64 used as a counter-based generator:
``x_i = mix64(key + (i + 1) * 0x9E3779B97F4A7C15)`` (Steele, Lea & Flood, OOPSLA 2014;
the output function is Stafford's "Mix13" variant as used in Vigna's splitmix64.c),
``key(seed, purpose) = x_0`` of a generator started at ``seed ^ purpose``, and a uniform
in [0, 1) is ``(x >> 11) * 2**-53``.  The C library implements the same published
generator for its own seeded start blocks and k-means++ draws.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# purpose ids for key(seed, purpose)
PURPOSE_GRAPH = 0
PURPOSE_X0 = 1
PURPOSE_KMEANS = 2
PURPOSE_STREAM = 3
PURPOSE_ARRIVALS = 4


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def sm64(state: int, idx) -> np.ndarray:
    """idx-th output (0-based) of a SplitMix64 generator whose state starts at ``state``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GOLDEN
    return mix64(z)


def key(seed: int, purpose: int, sub: int = 0) -> int:
    """Stream key for (seed, purpose[, sub-stream])."""
    k = int(sm64((seed ^ purpose) & 0xFFFFFFFFFFFFFFFF, 0))
    if sub:
        k = int(sm64(k, sub))
    return k


def uniforms(k: int, idx) -> np.ndarray:
    """Uniforms in [0, 1) at counters ``idx`` of stream ``k``."""
    return (sm64(k, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussians(k: int, count: int) -> np.ndarray:
    """``count`` N(0,1) draws by Box-Muller on consecutive uniform pairs of stream ``k``.

    Element e uses pair e // 2: u1 = U[2p], u2 = U[2p + 1]; radius sqrt(-2 ln(1 - u1));
    even e takes the cosine, odd e the sine.
    """
    npair = (count + 1) // 2
    u = uniforms(k, np.arange(2 * npair, dtype=np.uint64))
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    out = np.empty(2 * npair)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:count]


def start_block(seed: int, n: int, K: int, stage: int = 0) -> np.ndarray:
    """Seeded Gaussian start block X0 (n x K, row-major, float64), Sec. III random init."""
    return gaussians(key(seed, PURPOSE_X0, stage), n * K).reshape(n, K)


def kmeans_uniforms(seed: int, k: int) -> np.ndarray:
    """The k uniforms u_0..u_{k-1} that drive k-means++ seeding."""
    return uniforms(key(seed, PURPOSE_KMEANS), np.arange(k, dtype=np.uint64))


def _gamma_mt(k: int, alpha: float) -> float:
    """One Gamma(alpha, 1) draw (alpha >= 1) by Marsaglia & Tsang (2000) on stream k."""
    d = alpha - 1.0 / 3.0
    c = 1.0 / math.sqrt(9.0 * d)
    i = 0
    while True:
        g = gaussians(key(k, 0, i + 1), 1)[0]
        u = float(uniforms(k, np.array([i], dtype=np.uint64))[0])
        i += 1
        v = (1.0 + c * g) ** 3
        if v <= 0.0:
            continue
        if math.log(max(u, 1e-300)) < 0.5 * g * g + d - d * v + d * math.log(v):
            return d * v


def block_sizes(seed: int, n: int, K: int, alpha: float = 10.0) -> np.ndarray:
    """Dirichlet(alpha) proportions -> integer sizes by largest remainder, each >= 1."""
    kg = key(seed, PURPOSE_GRAPH, 1)
    g = np.array([_gamma_mt(key(kg, 0, b + 1), alpha) for b in range(K)])
    p = g / g.sum()
    raw = p * n
    s = np.floor(raw).astype(np.int64)
    rem = n - int(s.sum())
    frac = raw - s
    order = sorted(range(K), key=lambda b: (-frac[b], b))
    for b in order[:rem]:
        s[b] += 1
    while (s == 0).any():
        z = int(np.flatnonzero(s == 0)[0])
        big = int(np.argmax(s))
        s[z] += 1
        s[big] -= 1
    return s


def _perm(k: int, n: int) -> np.ndarray:
    """Seeded permutation of range(n): stable argsort of n stream outputs."""
    return np.argsort(sm64(k, np.arange(n, dtype=np.uint64)), kind="stable")


@dataclass
class Graph:
    """A directed multigraph edge list with its planted partition."""

    n: int
    src: np.ndarray  # int32 [m]
    dst: np.ndarray  # int32 [m]
    truth: np.ndarray  # int32 [n] planted block of every vertex
    K: int
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def dcsbm(
    n: int,
    K: int,
    seed: int = 0,
    alpha: float = 10.0,
    dmin: int = 10,
    dmax: int = 100,
    exponent: float = 2.5,
    ratio: float = 2.5,
) -> Graph:
    """Directed degree-corrected SBM edge list (see module docstring for the recipe)."""
    if n < K or K < 1:
        raise ValueError("need n >= K >= 1")
    kg = key(seed, PURPOSE_GRAPH)
    sizes = block_sizes(seed, n, K, alpha)
    perm = _perm(key(kg, 0, 2), n)
    block_of = np.empty(n, dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    for b in range(K):
        block_of[perm[starts[b] : starts[b + 1]]] = b

    # out-degrees: inverse CDF of P(d) ~ d^-exponent on {dmin..dmax}
    dv = np.arange(dmin, dmax + 1, dtype=np.float64)
    w = dv ** (-exponent)
    cdf = np.cumsum(w) / w.sum()
    u = uniforms(key(kg, 0, 3), np.arange(n, dtype=np.uint64))
    deg_out = (dmin + np.searchsorted(cdf, u, side="right")).clip(dmin, dmax).astype(np.int64)

    # members of each block sorted by id, with integer cumulative out-degree (theta weights)
    order = np.lexsort((np.arange(n), block_of))  # by block, then id
    members = order  # members[starts[b]:starts[b+1]] are block b's vertices, ascending id
    dcum = np.cumsum(deg_out[members])  # global cumulative over the block-ordered list
    dcum_start = np.concatenate([[0], dcum])[starts[:-1]]  # cum before each block
    dtot = np.array([dcum[starts[b + 1] - 1] - dcum_start[b] for b in range(K)], dtype=np.int64)

    m = int(deg_out.sum())
    src = np.repeat(np.arange(n, dtype=np.int64), deg_out)
    bsrc = block_of[src]
    eidx = np.arange(m, dtype=np.uint64)
    ke = key(kg, 0, 4)
    MSTR = np.uint64(1 << 40)

    def u_at(slot: int, rnd: int, idx: np.ndarray) -> np.ndarray:
        return uniforms(ke, np.uint64(rnd * 4 + slot) * MSTR + idx)

    within = (u_at(0, 0, eidx) < ratio / (ratio + 1.0)) | (K == 1)
    # between: block != b(src) chosen proportional to size
    t = np.floor(u_at(1, 0, eidx) * np.maximum(n - sizes[bsrc], 1)).astype(np.int64)
    t = np.where(t >= starts[bsrc], t + sizes[bsrc], t)
    bb = np.minimum(np.searchsorted(starts[1:], t, side="right"), K - 1)
    tblock = np.where(within, bsrc, bb)

    def draw_target(blk: np.ndarray, uu: np.ndarray) -> np.ndarray:
        tt = np.floor(uu * dtot[blk]).astype(np.int64)
        pos = np.searchsorted(dcum, dcum_start[blk] + tt, side="right")
        pos = np.minimum(pos, starts[blk + 1] - 1)
        return members[pos]

    dst = draw_target(tblock, u_at(2, 0, eidx))
    rnd = 0
    while True:
        bad = np.flatnonzero(dst == src)
        if bad.size == 0:
            break
        rnd += 1
        if rnd > 64:  # only possible for a single-vertex block with a within-edge
            keep = dst != src
            src, dst, tblock = src[keep], dst[keep], tblock[keep]
            break
        dst[bad] = draw_target(tblock[bad], u_at(2, rnd, bad.astype(np.uint64)))
    return Graph(
        n=n,
        src=src.astype(np.int32),
        dst=dst.astype(np.int32),
        truth=block_of.astype(np.int32),
        K=K,
        meta=dict(seed=seed, alpha=alpha, dmin=dmin, dmax=dmax, exponent=exponent, ratio=ratio),
    )


def emerging_stages(g: Graph, stages: int = 10, seed: int = 0) -> list[np.ndarray]:
    """Edge-index sets revealed by each 'emerging edges' stage (cumulative)."""
    p = _perm(key(seed, PURPOSE_STREAM, 1), g.m)
    cuts = [(s * g.m) // stages for s in range(stages + 1)]
    return [np.sort(p[: cuts[s + 1]]) for s in range(stages)]


def emerging_deltas(g: Graph, stages: int = 10, seed: int = 0) -> list[np.ndarray]:
    """Edge-index slices added at each 'emerging edges' stage."""
    p = _perm(key(seed, PURPOSE_STREAM, 1), g.m)
    cuts = [(s * g.m) // stages for s in range(stages + 1)]
    return [np.sort(p[cuts[s] : cuts[s + 1]]) for s in range(stages)]


def bfs_order(g: Graph, seed: int = 0) -> np.ndarray:
    """Snowball order: BFS over the undirected graph from a seeded start vertex,
    neighbours in ascending id; unreached parts restart at the lowest unvisited id.
    Returns order[new_id] = old_id."""
    n = g.n
    a = np.concatenate([g.src, g.dst]).astype(np.int64)
    b = np.concatenate([g.dst, g.src]).astype(np.int64)
    keys = np.unique(a * n + b)
    rows, cols = keys // n, keys % n
    ptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))])
    start = int(sm64(key(seed, PURPOSE_STREAM, 2), 0) % np.uint64(n))
    seen = np.zeros(n, dtype=bool)
    order = np.empty(n, dtype=np.int64)
    head = tail = 0
    nxt_unvisited = 0
    cur = start
    while tail < n:
        if head == tail:
            if seen[cur]:
                while seen[nxt_unvisited]:
                    nxt_unvisited += 1
                cur = nxt_unvisited
            seen[cur] = True
            order[tail] = cur
            tail += 1
        v = order[head]
        head += 1
        nb = cols[ptr[v] : ptr[v + 1]]
        nb = nb[~seen[nb]]
        seen[nb] = True
        order[tail : tail + nb.size] = nb
        tail += nb.size
    return order


def snowball_stages(g: Graph, stages: int = 10, seed: int = 0) -> list[Graph]:
    """Snowball stages: relabel in BFS order; stage s keeps the first ceil(s n / stages)
    vertices and the edges among them."""
    order = bfs_order(g, seed)
    newid = np.empty(g.n, dtype=np.int64)
    newid[order] = np.arange(g.n)
    s_new, d_new = newid[g.src], newid[g.dst]
    out = []
    for s in range(1, stages + 1):
        ns = -(-s * g.n // stages)
        keep = (s_new < ns) & (d_new < ns)
        out.append(
            Graph(
                n=int(ns),
                src=s_new[keep].astype(np.int32),
                dst=d_new[keep].astype(np.int32),
                truth=g.truth[order[:ns]].astype(np.int32),
                K=g.K,
                meta=dict(g.meta, stage=s),
            )
        )
    return out


def serving_requests(count: int = 512, rate: float = 200.0, seed: int = 0):
    """Poisson arrivals of partition requests with n log-uniform in [1e3, 2e5] and
    K = round(4 n^0.3); even-numbered requests are cold graphs, odd ones are streaming
    deltas (emerging edges) of the most recent cold graph."""
    ka = key(seed, PURPOSE_ARRIVALS)
    u = uniforms(ka, np.arange(3 * count, dtype=np.uint64))
    gaps = -np.log1p(-u[0::3]) / rate
    t = np.cumsum(gaps)
    ns = np.exp(np.log(1e3) + u[1::3] * (np.log(2e5) - np.log(1e3))).astype(np.int64)
    reqs = []
    for i in range(count):
        n = int(ns[i])
        reqs.append(dict(t=float(t[i]), n=n, K=int(round(4 * n ** 0.3)), cold=(i % 2 == 0), seed=int(seed * 1000003 + i)))
    return reqs
