"""Seeded synthetic roadmaps shaped like the PI-RRT# planning workloads.

Input generation only: this module builds the graph G = (V, E) with cached
edge costs c (Sec. III; Sec. IV-A "the cost of an edge ... is cached") that
both the CUDA path and the CPU oracle consume.  It holds none of the
policy-iteration arithmetic (Improve / Evaluate, Alg. 2).  The paper's own
scene (a 2-D query with polygonal obstacles, Sec. V) is not given, so seeded
circle / hypersphere scenes stand in for it:

* ``roadmap_c1``  -- 2-D unit square, 20 circles, 2000 samples + x_init,
  r-disc connection, FP64 costs, BFS-tree initial policy.
* ``roadmap_c2``  -- 2-D, 200 circles, N = 10^6, k = ceil(2e ln N) nearest
  neighbours, FP32 costs, Batched-Extension blocks of 10^4 vertices
  (``companion=True`` draws radii from [0.01, 0.04] so x_init is not sealed
  in a pocket).
* ``roadmap_c3``  -- 6-D [-pi, pi]^6, 64 hyperspheres, N = 4*10^6, k = 30,
  16-point edge check, FP32 costs, blocks of 5*10^4 vertices.
* ``roadmap_batch`` -- many independent roadmaps of log-uniform size and
  dimension in {2, 3, 4, 6, 7} for the batched form.

Every roadmap lists each undirected edge once (u < v) ordered by its larger
endpoint, so Batched-Extension block b (vertices [b*S, (b+1)*S), Alg. 3)
inserts the contiguous edge slice ``edge_start[b*S] : edge_start[(b+1)*S]``:
each block brings its vertices plus every edge whose other endpoint is
already present.  The final graph is therefore independent of S.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "roadgen.c")
_LIB_PATH = os.path.join(_HERE, "libroadgen.so")
_lib = None


def build_roadgen(force: bool = False) -> str:
    """Compile the generator's host helper (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off"]
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _roadgen():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_roadgen())
        i64, i32p, f64p, i64p, u8p = (ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p)
        lib.rg_symmetrize_knn.restype = ctypes.c_int64
        lib.rg_symmetrize_knn.argtypes = [i64, i64, i64p, i32p, i32p, i64]
        lib.rg_filter_collisions.restype = None
        lib.rg_filter_collisions.argtypes = [i64, ctypes.c_int, f64p, i32p, i32p, i64,
                                             f64p, f64p, ctypes.c_int, ctypes.c_int, u8p]
        lib.rg_edge_lengths.restype = None
        lib.rg_edge_lengths.argtypes = [i64, ctypes.c_int, f64p, i32p, i32p, f64p]
        lib.rg_order_by_max.restype = ctypes.c_int
        lib.rg_order_by_max.argtypes = [i64, i64, i32p, i64p, i64p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


@dataclass
class Scene:
    """Ball obstacles in a box [lo, hi]^dim; free space is outside every ball."""
    dim: int
    lo: float
    hi: float
    centers: np.ndarray  # (n_obs, dim) float64
    radii: np.ndarray    # (n_obs,) float64

    def inside(self, pts: np.ndarray) -> np.ndarray:
        """Boolean mask of points lying strictly inside some obstacle."""
        hit = np.zeros(len(pts), dtype=bool)
        for c, r in zip(self.centers, self.radii):
            d2 = np.sum((pts - c) ** 2, axis=1)
            hit |= d2 < r * r
        return hit


@dataclass
class Roadmap:
    """Undirected roadmap, vertex 0 = x_init, edges u < v ordered by v."""
    name: str
    points: np.ndarray        # (n, dim) float64
    u: np.ndarray             # (m,) int32, smaller endpoint
    v: np.ndarray             # (m,) int32, larger endpoint
    cost: np.ndarray          # (m,) float32 or float64 (the cached c)
    edge_start: np.ndarray    # (n + 1,) int64: edges with larger endpoint x start here
    block: int                # Batched-Extension block size S
    scene: Scene | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def m(self) -> int:
        return int(self.u.shape[0])

    def blocks(self, block: int | None = None):
        """Yield (v0, v1, e0, e1): block vertices [v0, v1) and edge slice [e0, e1)."""
        s = self.block if block is None else int(block)
        for v0 in range(0, self.n, s):
            v1 = min(self.n, v0 + s)
            yield v0, v1, int(self.edge_start[v0]), int(self.edge_start[v1])

    def n_blocks(self, block: int | None = None) -> int:
        s = self.block if block is None else int(block)
        return (self.n + s - 1) // s


def _draw_scene(rng: np.random.Generator, dim: int, lo: float, hi: float, n_obs: int,
                rmin: float, rmax: float, keep_free: list[np.ndarray]) -> Scene:
    """Obstacles drawn one at a time; one that covers a kept point is redrawn
    from the same stream."""
    centers = np.empty((n_obs, dim))
    radii = np.empty(n_obs)
    for i in range(n_obs):
        while True:
            c = rng.uniform(lo, hi, dim)
            r = rng.uniform(rmin, rmax)
            if all(np.sum((p - c) ** 2) >= r * r for p in keep_free):
                break
        centers[i] = c
        radii[i] = r
    return Scene(dim, lo, hi, centers, radii)


def _free_samples(rng: np.random.Generator, scene: Scene, count: int) -> np.ndarray:
    """`count` uniform samples outside every obstacle (rejection sampling)."""
    out = []
    have = 0
    chunk = max(1024, min(1 << 20, 2 * count))
    while have < count:
        p = rng.uniform(scene.lo, scene.hi, (chunk, scene.dim))
        p = p[~scene.inside(p)]
        out.append(p)
        have += len(p)
    return np.concatenate(out)[:count]


def free_fraction(scene: Scene, seed: int, n_mc: int = 1_000_000) -> float:
    """Monte-Carlo estimate of the free fraction of the box (seeded)."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(scene.lo, scene.hi, (n_mc, scene.dim))
    return float(1.0 - scene.inside(p).mean())


def _finish(name: str, pts: np.ndarray, u: np.ndarray, v: np.ndarray, scene: Scene,
            cost_dtype, block: int, exact_segment: bool, n_check: int, meta: dict) -> Roadmap:
    lib = _roadgen()
    m = len(u)
    keep = np.empty(m, dtype=np.uint8)
    lib.rg_filter_collisions(m, scene.dim, _ptr(pts), _ptr(u), _ptr(v), len(scene.radii),
                             _ptr(np.ascontiguousarray(scene.centers)),
                             _ptr(np.ascontiguousarray(scene.radii)),
                             0 if exact_segment else 1, n_check, _ptr(keep))
    sel = keep.astype(bool)
    u = np.ascontiguousarray(u[sel])
    v = np.ascontiguousarray(v[sel])
    m = len(u)
    length = np.empty(m, dtype=np.float64)
    lib.rg_edge_lengths(m, scene.dim, _ptr(pts), _ptr(u), _ptr(v), _ptr(length))
    cost = length.astype(cost_dtype)
    ok = cost > 0  # a zero-length edge would be a duplicate sample
    if not ok.all():
        u, v, cost = u[ok], v[ok], cost[ok]
        m = len(u)
    n = len(pts)
    perm = np.empty(m, dtype=np.int64)
    start = np.empty(n + 1, dtype=np.int64)
    if lib.rg_order_by_max(m, n, _ptr(v), _ptr(perm), _ptr(start)) != 0:
        raise MemoryError("rg_order_by_max")
    u = np.ascontiguousarray(u[perm])
    v = np.ascontiguousarray(v[perm])
    cost = np.ascontiguousarray(cost[perm])
    meta = dict(meta)
    meta.update(n=n, m_undirected=m, directed_entries=2 * m, dim=scene.dim,
                cost_dtype=np.dtype(cost_dtype).name)
    return Roadmap(name, pts, u, v, cost, start, block, scene, meta)


def _knn_edges(pts: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    from scipy.spatial import cKDTree
    n = len(pts)
    kk = min(k, n - 1)
    tree = cKDTree(pts, leafsize=16, balanced_tree=False, compact_nodes=False)
    _, idx = tree.query(pts, k=kk + 1, workers=-1)
    idx = np.ascontiguousarray(idx[:, 1:].astype(np.int64))
    # the query may list self among equidistant hits; the helper skips self
    cap = n * kk
    u = np.empty(cap, dtype=np.int32)
    v = np.empty(cap, dtype=np.int32)
    m = _roadgen().rg_symmetrize_knn(n, kk, _ptr(idx), _ptr(u), _ptr(v), cap)
    if m < 0:
        raise MemoryError("rg_symmetrize_knn")
    return u[:m].copy(), v[:m].copy()


def _rdisc_edges(pts: np.ndarray, r: float) -> tuple[np.ndarray, np.ndarray]:
    from scipy.spatial import cKDTree
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    pairs = np.sort(pairs, axis=1)
    order = np.lexsort((pairs[:, 0], pairs[:, 1]))
    pairs = pairs[order]
    return (np.ascontiguousarray(pairs[:, 0].astype(np.int32)),
            np.ascontiguousarray(pairs[:, 1].astype(np.int32)))


def knn_k(n: int) -> int:
    """k = ceil(2e ln N), the k-nearest connection rule of the configs."""
    return int(math.ceil(2.0 * math.e * math.log(n)))


def roadmap_c1(trial: int = 0, n_samples: int = 2000, n_obs: int = 20) -> Roadmap:
    """2-D unit square, circles r ~ U[0.02, 0.08], x_init = (0.05, 0.05) as
    vertex 0, r-disc radius r = 1.1 sqrt(2 (1 + 1/2) A_free / pi) sqrt(ln N / N),
    exact segment-circle rejection, FP64 costs."""
    seed = 1 * 1000 + trial
    rng = np.random.default_rng(seed)
    x_init = np.array([0.05, 0.05])
    scene = _draw_scene(rng, 2, 0.0, 1.0, n_obs, 0.02, 0.08, [x_init])
    samples = _free_samples(rng, scene, n_samples)
    pts = np.ascontiguousarray(np.vstack([x_init[None, :], samples]))
    n = len(pts)
    a_free = free_fraction(scene, seed + 500_000)
    r = 1.1 * math.sqrt(2.0 * 1.5 * a_free / math.pi) * math.sqrt(math.log(n) / n)
    u, v = _rdisc_edges(pts, r)
    return _finish("c1", pts, u, v, scene, np.float64, n, True, 16,
                   dict(seed=seed, radius=r, free_fraction=a_free))


def roadmap_2d_knn(name: str, seed: int, n: int, n_obs: int, rmin: float, rmax: float,
                   block: int, k: int | None = None, cost_dtype=np.float32) -> Roadmap:
    rng = np.random.default_rng(seed)
    x_init = np.array([0.05, 0.05])
    scene = _draw_scene(rng, 2, 0.0, 1.0, n_obs, rmin, rmax, [x_init])
    samples = _free_samples(rng, scene, n - 1)
    pts = np.ascontiguousarray(np.vstack([x_init[None, :], samples]))
    kk = knn_k(n) if k is None else k
    u, v = _knn_edges(pts, kk)
    return _finish(name, pts, u, v, scene, cost_dtype, block, True, 16,
                   dict(seed=seed, k=kk, radii=(rmin, rmax), n_obs=n_obs))


def roadmap_c2(trial: int = 0, n: int = 1_000_000, block: int = 10_000,
               companion: bool = False) -> Roadmap:
    """2-D, 200 circles, k = ceil(2e ln N), FP32 costs, blocks of 10^4."""
    rmin, rmax = (0.01, 0.04) if companion else (0.02, 0.08)
    return roadmap_2d_knn("c2-companion" if companion else "c2", 2 * 1000 + trial, n, 200,
                          rmin, rmax, block)


def roadmap_nd_knn(name: str, seed: int, n: int, dim: int, n_obs: int, rmin: float,
                   rmax: float, k: int, block: int, cost_dtype=np.float32,
                   n_check: int = 16) -> Roadmap:
    """[-pi, pi]^dim with ball obstacles; x_init is the first free sample."""
    rng = np.random.default_rng(seed)
    scene = _draw_scene(rng, dim, -math.pi, math.pi, n_obs, rmin, rmax, [])
    pts = np.ascontiguousarray(_free_samples(rng, scene, n))
    u, v = _knn_edges(pts, k)
    return _finish(name, pts, u, v, scene, cost_dtype, block, False, n_check,
                   dict(seed=seed, k=k, radii=(rmin, rmax), n_obs=n_obs))


def roadmap_c3(trial: int = 0, n: int = 4_000_000, block: int = 50_000) -> Roadmap:
    """6-D [-pi, pi]^6, 64 hyperspheres r ~ U[0.3, 0.8], k = 30, 16 points per
    segment (t = i/15), FP32 costs, blocks of 5*10^4."""
    return roadmap_nd_knn("c3", 3 * 1000 + trial, n, 6, 64, 0.3, 0.8, 30, block)


C5_X_INIT = (0.05, 0.05)
C5_X_GOAL = (0.95, 0.95)


def c5_scene(seed: int) -> Scene:
    """Learned-proposal scene: 200 circles, r ~ U[0.01, 0.04], in the unit
    square; an obstacle covering x_init = (0.05, 0.05) or x_goal = (0.95, 0.95)
    is redrawn."""
    rng = np.random.default_rng(5 * 1000 + int(seed))
    return _draw_scene(rng, 2, 0.0, 1.0, 200, 0.01, 0.04,
                       [np.array(C5_X_INIT), np.array(C5_X_GOAL)])


def occupancy_grid(scene: Scene, res: int = 64) -> np.ndarray:
    """res x res occupancy of a 2-D scene, row-major (row = y cell, column =
    x cell): 1 where the cell centre lies inside an obstacle, else 0."""
    c = (np.arange(res) + 0.5) / res
    xx, yy = np.meshgrid(c, c)
    pts = np.stack([xx.ravel(), yy.ravel()], axis=1) * (scene.hi - scene.lo) + scene.lo
    return scene.inside(pts).astype(np.float32)


def free_uniform(rng: np.random.Generator, scene: Scene, count: int) -> np.ndarray:
    """``count`` uniform samples of the free space (rejection sampling)."""
    return _free_samples(rng, scene, count)


def roadmap_from_points(name: str, pts: np.ndarray, scene: Scene, k: int | None = None,
                        cost_dtype=np.float32, exact_segment: bool = True,
                        n_check: int = 16) -> Roadmap:
    """Roadmap over given free points (vertex i = pts[i]): symmetrised k-NN,
    k = ceil(2e ln N) unless given, collision-checked edges, Euclidean costs,
    one block holding every vertex."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    n = len(pts)
    kk = knn_k(n) if k is None else int(k)
    u, v = _knn_edges(pts, kk)
    return _finish(name, pts, u, v, scene, cost_dtype, n, exact_segment, n_check,
                   dict(k=kk, n_obs=len(scene.radii)))


def _batch_member(args):
    i, n, d, s = args
    if d == 2:
        return roadmap_2d_knn(f"b{i}", s, n, 20, 0.02, 0.08, n)
    return roadmap_nd_knn(f"b{i}", s, n, d, 64, 0.3, 0.8, knn_k(n), n)


def roadmap_batch(n_graphs: int = 512, trial: int = 0, n_min: int = 1_000,
                  n_max: int = 200_000, dims=(2, 3, 4, 6, 7), workers: int = 1) -> list[Roadmap]:
    """Independent roadmaps: N_g log-uniform in [n_min, n_max], dimension
    uniform in ``dims``, k = ceil(2e ln N_g), each with its own obstacles.
    2-D scenes use 20 circles r ~ U[0.02, 0.08] in the unit square with an
    exact segment test; higher dimensions use 64 balls r ~ U[0.3, 0.8] in
    [-pi, pi]^d with the 16-point check."""
    rng = np.random.default_rng(4 * 1000 + trial)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_graphs)).round().astype(int)
    dim_pick = rng.choice(np.asarray(dims), n_graphs)
    seeds = rng.integers(0, 2**31 - 1, n_graphs)
    jobs = [(i, int(sizes[i]), int(dim_pick[i]), int(seeds[i])) for i in range(n_graphs)]
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        build_roadgen()
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_batch_member, jobs, chunksize=4))
    return [_batch_member(j) for j in jobs]


def bfs_tree_parents(rm: Roadmap, root: int = 0) -> np.ndarray:
    """Initial policy of the oracle-sized config: a breadth-first tree from
    x_init over G, neighbours visited in ascending id, parent = first
    discoverer; -1 for the root and for vertices outside its component."""
    n = rm.n
    uu = np.concatenate([rm.u, rm.v]).astype(np.int64)
    vv = np.concatenate([rm.v, rm.u]).astype(np.int64)
    order = np.lexsort((vv, uu))
    uu, vv = uu[order], vv[order]
    off = np.searchsorted(uu, np.arange(n + 1))
    parent = np.full(n, -1, dtype=np.int32)
    seen = np.zeros(n, dtype=bool)
    seen[root] = True
    queue = [root]
    head = 0
    while head < len(queue):
        x = queue[head]
        head += 1
        for y in vv[off[x]:off[x + 1]]:
            if not seen[y]:
                seen[y] = True
                parent[y] = x
                queue.append(int(y))
    return parent


def random_graph(seed: int, n: int, m: int, cost_dtype=np.float64, connected: bool = True,
                 cmin: float = 0.1, cmax: float = 1.0) -> Roadmap:
    """Small random weighted graph (no geometry) for hand-checkable tests.
    With ``connected`` a random spanning tree is laid down first."""
    rng = np.random.default_rng(seed)
    pairs = set()
    if connected:
        for x in range(1, n):
            y = int(rng.integers(0, x))
            pairs.add((y, x))
    tries = 0
    while len(pairs) < m and tries < 50 * m:
        a, b = sorted(int(t) for t in rng.integers(0, n, 2))
        tries += 1
        if a != b:
            pairs.add((a, b))
    pairs = sorted(pairs, key=lambda p: (p[1], p[0]))
    u = np.array([p[0] for p in pairs], dtype=np.int32)
    v = np.array([p[1] for p in pairs], dtype=np.int32)
    cost = rng.uniform(cmin, cmax, len(u)).astype(cost_dtype)
    start = np.searchsorted(v, np.arange(n + 1)).astype(np.int64)
    pts = np.zeros((n, 1))
    return Roadmap(f"random{seed}", pts, u, v, cost, start, n, None,
                   dict(seed=seed, n=n, m_undirected=len(u)))


def cached(name: str, fn, **kw) -> Roadmap:
    """``fn(**kw)`` memoised on disk (``$PIRRT_CACHE`` or /tmp/pirrt_cache), so
    several processes of one session share an expensive generation."""
    import hashlib
    import json
    import tempfile
    root = os.environ.get("PIRRT_CACHE", os.path.join(tempfile.gettempdir(), "pirrt_cache"))
    os.makedirs(root, exist_ok=True)
    key = hashlib.sha1(json.dumps([name, sorted(kw.items())], default=str).encode()).hexdigest()[:16]
    path = os.path.join(root, f"{name}-{key}.npz")
    if os.path.exists(path):
        d = np.load(path, allow_pickle=False)
        meta = json.loads(str(d["meta"]))
        sc = Scene(int(d["dim"]), float(d["lo"]), float(d["hi"]), d["centers"], d["radii"])
        return Roadmap(str(d["name"]), d["points"], d["u"], d["v"], d["cost"], d["edge_start"],
                       int(d["block"]), sc, meta)
    rm = fn(**kw)
    tmp = f"{path}.{os.getpid()}.tmp.npz"
    sc = rm.scene
    np.savez(tmp, name=rm.name, points=rm.points, u=rm.u, v=rm.v, cost=rm.cost,
             edge_start=rm.edge_start, block=rm.block, meta=json.dumps(rm.meta, default=str),
             dim=sc.dim, lo=sc.lo, hi=sc.hi, centers=sc.centers, radii=sc.radii)
    os.replace(tmp, path)
    return rm


def cached_batch(n_graphs: int = 512, trial: int = 0, n_min: int = 1_000, n_max: int = 200_000,
                 workers: int = 1) -> list[Roadmap]:
    """roadmap_batch memoised on disk as one archive (members concatenated)."""
    import json
    import tempfile
    root = os.environ.get("PIRRT_CACHE", os.path.join(tempfile.gettempdir(), "pirrt_cache"))
    os.makedirs(root, exist_ok=True)
    path = os.path.join(root, f"batch-{n_graphs}-{trial}-{n_min}-{n_max}.npz")
    if os.path.exists(path):
        d = np.load(path, allow_pickle=False)
        out = []
        nv, ne = d["nv"], d["ne"]
        ov, oe = np.r_[0, np.cumsum(nv)], np.r_[0, np.cumsum(ne)]
        metas = json.loads(str(d["metas"]))
        for i in range(len(nv)):
            u = d["u"][oe[i]:oe[i + 1]]
            v = d["v"][oe[i]:oe[i + 1]]
            n = int(nv[i])
            out.append(Roadmap(f"b{i}", np.zeros((n, 1)), u, v, d["cost"][oe[i]:oe[i + 1]],
                               np.searchsorted(v, np.arange(n + 1)).astype(np.int64), n, None,
                               metas[i]))
        return out
    rms = roadmap_batch(n_graphs, trial, n_min, n_max, workers=workers)
    tmp = f"{path}.{os.getpid()}.tmp.npz"
    np.savez(tmp, nv=np.array([r.n for r in rms]), ne=np.array([r.m for r in rms]),
             u=np.concatenate([r.u for r in rms]), v=np.concatenate([r.v for r in rms]),
             cost=np.concatenate([r.cost for r in rms]),
             metas=json.dumps([r.meta for r in rms], default=str))
    os.replace(tmp, path)
    return rms

