"""The GPU roadmap generator (workloads/gpu.py, roadgen_gpu.cu) against a plain
CPU reference of the same definitions (roadgen_gpu.h): Philox4x32-10 samples
of the free space, FP32 k-nearest neighbours by brute force, union-symmetrised
collision-checked edges with FP64 lengths ordered by the larger endpoint.

The generator is input tooling (no policy-iteration arithmetic).  The CPU
reference below is written from the definitions, shares no code with the
CUDA generator, and is itself pinned on the CPU: its Philox stream against
its own scalar form and basic uniformity, its k-NN against scipy's k-d tree,
its symmetrisation against the host generator's.  A roadmap built on the GPU
then goes through the exploitation path and must match the oracle's Dijkstra.
"""
import math

import numpy as np
import pytest

from paper_2003_04920_gb300 import workloads as W

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


# ---------------------------------------------------------------- CPU reference

def philox_np(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32-10 of counters ctr (N x 4 uint32) under key (k0, k1)."""
    x = [ctr[:, i].astype(np.uint64) for i in range(4)]
    k0, k1 = np.uint64(key[0]), np.uint64(key[1])
    for _ in range(10):
        p0 = x[0] * np.uint64(M0)
        p1 = x[2] * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
        k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
        k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
    return np.stack(x, axis=1).astype(np.uint32)


def philox_scalar(ctr, key):
    """The same rounds on Python integers (one counter)."""
    x0, x1, x2, x3 = ctr
    k0, k1 = key
    for _ in range(10):
        p0, p1 = x0 * M0, x2 * M1
        x0, x1, x2, x3 = ((p1 >> 32) ^ x1 ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ x3 ^ k1) & MASK, p0 & MASK
        k0, k1 = (k0 + W0) & MASK, (k1 + W1) & MASK
    return x0, x1, x2, x3


def candidates_np(lo, hi, dim, seed, i0, count):
    i = np.arange(i0, i0 + count, dtype=np.uint64)
    key = (seed & MASK, (seed >> 32) & MASK)
    words = []
    for blk in range((dim + 3) // 4):
        ctr = np.stack([i & np.uint64(MASK), i >> np.uint64(32),
                        np.full_like(i, blk), np.zeros_like(i)], axis=1).astype(np.uint32)
        words.append(philox_np(ctr, key))
    x = np.concatenate(words, axis=1)[:, :dim]
    u = (x >> np.uint32(8)).astype(np.float64) * (1.0 / 16777216.0)
    span = np.float64(hi) - np.float64(lo)
    return np.float64(lo) + span * u


def d2_seq(a, b):
    """Sum over coordinates in order of (a - b)^2, in the arrays' dtype."""
    s = np.zeros(np.broadcast_shapes(a.shape[:-1], b.shape[:-1]), dtype=a.dtype)
    for d in range(a.shape[-1]):
        t = a[..., d] - b[..., d]
        s = s + t * t
    return s


def sample_np(scene, n, seed):
    out, i0 = [], 0
    while sum(len(o) for o in out) < n:
        c = candidates_np(scene.lo, scene.hi, scene.dim, seed, i0, 1 << 14)
        free = np.ones(len(c), dtype=bool)
        for cc, r in zip(scene.centers, scene.radii):
            free &= d2_seq(c, cc[None, :]) >= np.float64(r) * np.float64(r)
        out.append(c[free])
        i0 += 1 << 14
    return np.concatenate(out)[:n]


def knn_np(pts, k):
    p32 = pts.astype(np.float32)
    n = len(p32)
    ids = np.arange(n)
    out = np.empty((n, k), dtype=np.int32)
    for i in range(n):
        d = d2_seq(p32[i][None, :], p32)
        d[i] = np.inf
        order = np.lexsort((ids, d))
        out[i] = order[:k]
    return out


def segment_free_np(a, b, centers, radii, exact, n_check):
    """Every ball at once (elementwise IEEE arithmetic, coordinates in order)."""
    c = np.asarray(centers, dtype=np.float64)
    r2 = np.asarray(radii, dtype=np.float64) * np.asarray(radii, dtype=np.float64)
    if exact:
        ab2 = 0.0
        t = np.zeros(len(c))
        for d in range(len(a)):
            e = b[d] - a[d]
            ab2 = ab2 + e * e
            t = t + (c[:, d] - a[d]) * e
        t = t / ab2 if ab2 > 0.0 else np.zeros(len(c))
        t = np.minimum(np.maximum(t, 0.0), 1.0)
        s2 = np.zeros(len(c))
        for d in range(len(a)):
            p = (a[d] + t * (b[d] - a[d])) - c[:, d]
            s2 = s2 + p * p
        return not np.any(s2 < r2)
    for i in range(n_check):
        t = i / (n_check - 1) if n_check > 1 else 0.0
        s2 = np.zeros(len(c))
        for d in range(len(a)):
            p = (a[d] + t * (b[d] - a[d])) - c[:, d]
            s2 = s2 + p * p
        if np.any(s2 < r2):
            return False
    return True


def edges_np(pts, nbr, scene, exact, n_check, cost_dtype):
    n, k = nbr.shape
    rows = [set(r.tolist()) for r in nbr]
    out = []
    for i in range(n):
        for j in nbr[i].tolist():
            if j == i or (j < i and i in rows[j]):
                continue
            u, v = min(i, j), max(i, j)
            a, b = pts[u], pts[v]
            s = 0.0
            for d in range(len(a)):
                t = a[d] - b[d]
                s = s + t * t
            if s > 0.0 and segment_free_np(a, b, scene.centers, scene.radii, exact, n_check):
                out.append((v, u, math.sqrt(s)))
    out.sort()
    u = np.array([e[1] for e in out], dtype=np.int32)
    v = np.array([e[0] for e in out], dtype=np.int32)
    cost = np.array([e[2] for e in out], dtype=np.float64).astype(cost_dtype)
    start = np.searchsorted(v, np.arange(n + 1)).astype(np.int64)
    return u, v, cost, start


# ------------------------------------------------------- pins of the reference

def test_philox_vectorised_equals_scalar_and_is_uniform():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, (64, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9ABCDEF0)
    got = philox_np(ctr, key)
    for r in range(len(ctr)):
        assert tuple(int(x) for x in got[r]) == philox_scalar(tuple(int(x) for x in ctr[r]), key)
    # consecutive counters: every output bit fair, words uncorrelated
    big = candidates_np(0.0, 1.0, 4, 7, 0, 200_000)
    assert np.all(np.abs(big.mean(axis=0) - 0.5) < 0.005)
    assert np.all(np.abs(big.var(axis=0) - 1.0 / 12.0) < 0.002)
    cc = np.corrcoef(big.T)
    assert np.max(np.abs(cc - np.eye(4))) < 0.01
    hist = np.histogram(big[:, 0], bins=64, range=(0.0, 1.0))[0]
    chi2 = np.sum((hist - len(big) / 64) ** 2 / (len(big) / 64))
    assert chi2 < 120  # 63 degrees of freedom
    # a different seed or counter gives a different stream
    assert not np.array_equal(candidates_np(0, 1, 4, 8, 0, 16), candidates_np(0, 1, 4, 7, 0, 16))


def test_knn_reference_equals_kdtree_on_distinct_points():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1, 1, (700, 3))
    k = 12
    ref = knn_np(pts, k)
    _, idx = spatial.cKDTree(pts.astype(np.float32).astype(np.float64)).query(pts.astype(np.float32).astype(np.float64), k=k + 1)
    # ties in FP32 are tie-broken by id in the reference; compare as sets where distinct
    for i in range(len(pts)):
        assert set(ref[i].tolist()) == set(idx[i, 1:].tolist())


def test_symmetrisation_reference_equals_host_generator():
    rng = np.random.default_rng(5)
    pts = rng.uniform(0, 1, (400, 2))
    nbr = knn_np(pts, 8)
    empty = W.Scene(2, 0.0, 1.0, np.zeros((0, 2)), np.zeros(0))
    u, v, _, _ = edges_np(pts, nbr, empty, True, 16, np.float64)
    hu, hv = W._knn_edges(pts.astype(np.float32).astype(np.float64), 8)
    got = set(zip(u.tolist(), v.tolist()))
    want = set(zip(hu.tolist(), hv.tolist()))
    assert got == want


# ------------------------------------------------------------- GPU generator

def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_04920_gb300.workloads import gpu as G
    G.load()
    return torch, G


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["6d-points", "2d-exact", "2d-large-k"])
def test_gpu_generator_matches_cpu_reference(case):
    torch, G = _gpu()
    if case == "6d-points":
        scene = W._draw_scene(np.random.default_rng(31), 6, -math.pi, math.pi, 64, 0.3, 0.8, [])
        n, k, exact, seed, cost_dtype = 1500, 24, False, 0x1234_5678_9ABC, np.float32
    elif case == "2d-large-k":
        # k = ceil(2e ln N) at N = 10^6 (the 2-D and learned-proposal roadmaps)
        scene = W._draw_scene(np.random.default_rng(33), 2, 0.0, 1.0, 200, 0.01, 0.04, [])
        n, k, exact, seed, cost_dtype = 2500, 76, True, 5005, np.float32
    else:
        scene = W._draw_scene(np.random.default_rng(32), 2, 0.0, 1.0, 60, 0.01, 0.05, [])
        n, k, exact, seed, cost_dtype = 3000, 16, True, 77, np.float64
    pts, tried = G.sample(scene, n, seed)
    want_pts = sample_np(scene, n, seed)
    np.testing.assert_array_equal(pts.cpu().numpy(), want_pts)
    nbr = G.knn(pts, scene.lo, scene.hi, k)
    want_nbr = knn_np(want_pts, k)
    np.testing.assert_array_equal(nbr.cpu().numpy(), want_nbr)
    u, v, cost, start = G.edges(pts, nbr, scene, exact, 16, cost_dtype)
    wu, wv, wc, ws = edges_np(want_pts, want_nbr, scene, exact, 16, cost_dtype)
    np.testing.assert_array_equal(u.cpu().numpy(), wu)
    np.testing.assert_array_equal(v.cpu().numpy(), wv)
    np.testing.assert_array_equal(cost.cpu().numpy(), wc)
    np.testing.assert_array_equal(start, ws)
    assert len(wu) > n  # obstacles remove some edges, not most


@pytest.mark.gpu
def test_gpu_roadmap_schedule_matches_dijkstra():
    """A 6-D roadmap built on the device, exploited block by block straight from
    device memory, reaches the oracle's shortest-path tree."""
    torch, G = _gpu()
    import oracle as O
    import paper_2003_04920_gb300 as P
    from tests.gpu_util import assert_parity
    rm = G.roadmap_nd("t", 901, 20_000, 6, 64, 0.3, 0.8, 30, 2_000)
    with P.Graph(rm.n, rm.m, 0, np.float32) as D:
        for v0, v1, e0, e1 in rm.blocks():
            D.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            assert D.exploit()["converged"] == 1
        g, p = D.get_costs(), D.get_parents()
    host = rm.to_host()
    d, _ = O.dijkstra(host.n, host.u, host.v, host.cost.astype(np.float64))
    assert_parity(host, g, p, d)


# ------------------------------------------------------------- exploration

def pred_knn_np(pts, k):
    """Vertex i's k nearest among vertices 0 .. i-1 (FP32, ties by id)."""
    p32 = pts.astype(np.float32)
    out = np.full((len(p32), k), -1, dtype=np.int32)
    for i in range(1, len(p32)):
        d = d2_seq(p32[i][None, :], p32[:i])
        order = np.lexsort((np.arange(i), d))[:k]
        out[i, :len(order)] = order
    return out


def pred_edges_np(pts, nbr, scene, exact, n_check, cost_dtype):
    out_u, out_v, out_c = [], [], []
    for i in range(len(pts)):
        for j in nbr[i].tolist():
            if j < 0:
                continue
            a, b = pts[j], pts[i]
            s = 0.0
            for d in range(len(a)):
                t = a[d] - b[d]
                s = s + t * t
            if s > 0.0 and segment_free_np(a, b, scene.centers, scene.radii, exact, n_check):
                out_u.append(j)
                out_v.append(i)
                out_c.append(math.sqrt(s))
    return (np.array(out_u, dtype=np.int32), np.array(out_v, dtype=np.int32),
            np.array(out_c, dtype=np.float64).astype(cost_dtype))


def _explore_all(G, scene, n, k, seed, S, exact=False):
    import torch
    x = G.Explorer(scene, n, k, seed, S, exact_segment=exact)
    us, vs, cs = [], [], []
    for b, v0 in enumerate(range(0, n, S)):
        v1 = min(n, v0 + S)
        u, v, c, cnt = x.extend(v0, v1, b & 1)
        torch.cuda.synchronize()
        m = int(cnt.item())
        us.append(u[:m].cpu().numpy())
        vs.append(v[:m].cpu().numpy())
        cs.append(c[:m].cpu().numpy())
    pts = x.points().cpu().numpy()
    x.close()
    return pts, np.concatenate(us), np.concatenate(vs), np.concatenate(cs)


@pytest.mark.gpu
def test_gpu_exploration_matches_cpu_reference_and_block_size():
    torch, G = _gpu()
    scene = W._draw_scene(np.random.default_rng(41), 6, -math.pi, math.pi, 64, 0.3, 0.8, [])
    n, k, seed = 1800, 20, 4242
    pts, u, v, c = _explore_all(G, scene, n, k, seed, 500)
    np.testing.assert_array_equal(pts, sample_np(scene, n, seed))
    wu, wv, wc = pred_edges_np(pts, pred_knn_np(pts, k), scene, False, 16, np.float32)
    np.testing.assert_array_equal(u, wu)
    np.testing.assert_array_equal(v, wv)
    np.testing.assert_array_equal(c, wc)
    # the roadmap does not depend on the block size (Alg. 3)
    _, u2, v2, c2 = _explore_all(G, scene, n, k, seed, 1800)
    np.testing.assert_array_equal(u2, u)
    np.testing.assert_array_equal(v2, v)
    np.testing.assert_array_equal(c2, c)
