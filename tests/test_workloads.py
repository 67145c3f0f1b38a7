"""Checks of the seeded input generator against brute force on small inputs."""
import math

import numpy as np
import pytest

from paper_2003_04920_gb300 import workloads as W


def test_knn_symmetrised_union_matches_brute_force():
    rng = np.random.default_rng(0)
    pts = rng.uniform(0, 1, (300, 3))
    k = 7
    u, v = W._knn_edges(pts, k)
    d = np.linalg.norm(pts[:, None] - pts[None], axis=2)
    np.fill_diagonal(d, np.inf)
    nn = np.argsort(d, axis=1)[:, :k]
    want = {(min(i, j), max(i, j)) for i in range(300) for j in nn[i]}
    got = set(zip(u.tolist(), v.tolist()))
    assert got == want
    assert len(got) == len(u)  # no duplicates
    assert np.all(u < v)


def test_rdisc_edges_match_brute_force():
    rng = np.random.default_rng(1)
    pts = rng.uniform(0, 1, (200, 2))
    u, v = W._rdisc_edges(pts, 0.1)
    d = np.linalg.norm(pts[:, None] - pts[None], axis=2)
    iu, iv = np.nonzero(np.triu(d < 0.1, 1))
    assert set(zip(u.tolist(), v.tolist())) == set(zip(iu.tolist(), iv.tolist()))


def test_exact_segment_test_against_dense_sampling():
    rm = W.roadmap_c1(trial=3, n_samples=400)
    sc = rm.scene
    t = np.linspace(0, 1, 257)
    a, b = rm.points[rm.u], rm.points[rm.v]
    for tt in t[::8]:
        p = a + tt * (b - a)
        assert not sc.inside(p).any(), "kept edge passes through an obstacle"


def test_sixteen_point_rule():
    rm = W.roadmap_nd_knn("t", 7, 3000, 6, 64, 0.3, 0.8, 10, 3000)
    sc = rm.scene
    a, b = rm.points[rm.u], rm.points[rm.v]
    for i in range(16):
        p = a + (i / 15.0) * (b - a)
        assert not sc.inside(p).any()
    assert np.all(rm.cost > 0) and rm.cost.dtype == np.float32


def test_blocks_slice_edges_by_larger_endpoint():
    rm = W.roadmap_c2(n=5000, block=700, companion=True)
    seen = 0
    for v0, v1, e0, e1 in rm.blocks():
        assert np.all((rm.v[e0:e1] >= v0) & (rm.v[e0:e1] < v1))
        assert np.all(rm.u[e0:e1] < rm.v[e0:e1])
        seen += e1 - e0
    assert seen == rm.m
    assert rm.n_blocks() == math.ceil(5000 / 700)


def test_generator_is_seeded():
    a = W.roadmap_c2(n=3000, block=500, companion=True)
    b = W.roadmap_c2(n=3000, block=500, companion=True)
    np.testing.assert_array_equal(a.u, b.u)
    np.testing.assert_array_equal(a.cost, b.cost)


def test_c1_matches_config():
    rm = W.roadmap_c1()
    assert rm.n == 2001 and rm.cost.dtype == np.float64
    np.testing.assert_array_equal(rm.points[0], [0.05, 0.05])
    assert len(rm.scene.radii) == 20
    assert np.all((rm.scene.radii >= 0.02) & (rm.scene.radii <= 0.08))
    assert 0.04 < rm.meta["radius"] < 0.08
    assert not rm.scene.inside(rm.points).any()


def test_bfs_tree_parents_is_first_discoverer():
    rm = W.random_graph(5, 30, 60)
    p = W.bfs_tree_parents(rm)
    assert p[0] == -1
    # every parent is adjacent and has a smaller BFS level
    adj = {(int(a), int(b)) for a, b in zip(rm.u, rm.v)}
    adj |= {(b, a) for a, b in adj}
    for x in range(1, 30):
        if p[x] >= 0:
            assert (int(p[x]), x) in adj
