"""Properties of the seeded synthetic inputs (the DC-SBM stand-in for the Challenge data)."""
import numpy as np

from paper_1708_07481_gb300 import workload as W


def test_dcsbm_shape_and_recipe():
    g = W.dcsbm(5000, 19, seed=1)
    sizes = np.bincount(g.truth, minlength=19)
    assert sizes.sum() == 5000 and sizes.min() >= 1
    assert np.array_equal(sizes, W.block_sizes(1, 5000, 19))
    assert np.all(g.src != g.dst)
    outdeg = np.bincount(g.src, minlength=5000)
    assert outdeg.min() >= 10 and outdeg.max() <= 100
    within = np.mean(g.truth[g.src] == g.truth[g.dst])
    assert abs(within - 2.5 / 3.5) < 0.02
    assert 15 < g.m / g.n < 30


def test_dcsbm_deterministic():
    a = W.dcsbm(2000, 7, seed=5)
    b = W.dcsbm(2000, 7, seed=5)
    c = W.dcsbm(2000, 7, seed=6)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
    assert not np.array_equal(a.dst, c.dst)


def test_start_block_and_uniforms():
    X = W.start_block(0, 1000, 8)
    assert X.shape == (1000, 8)
    assert abs(X.mean()) < 0.05 and abs(X.std() - 1) < 0.05
    u = W.kmeans_uniforms(0, 1000)
    assert u.min() >= 0 and u.max() < 1


def test_streams():
    g = W.dcsbm(3000, 6, seed=2)
    st = W.emerging_stages(g)
    assert len(st) == 10 and st[-1].size == g.m
    assert all(np.all(np.isin(st[i], st[i + 1])) for i in range(9))
    deltas = W.emerging_deltas(g)
    assert sum(d.size for d in deltas) == g.m
    sb = W.snowball_stages(g)
    assert [s.n for s in sb] == [-(-k * 3000 // 10) for k in range(1, 11)]
    assert sb[-1].m == g.m
    for s in sb:
        assert s.src.max() < s.n and s.dst.max() < s.n
    order = W.bfs_order(g)
    assert np.array_equal(np.sort(order), np.arange(g.n))
