"""GPU-resident roadmap generator (input generation only).

A ctypes binding over ``libroadgen_gpu.so`` (``roadgen_gpu.cu``, definitions
in ``roadgen_gpu.h``): seeded free-space samples (Philox4x32-10), grid
k-nearest neighbours, union-symmetrised collision-checked edges ordered by the
larger endpoint -- the same kind of sampling-based roadmap as the host
generator in this package (Sec. III; Sec. IV-A cached edge costs), built on
the device in seconds for 10^7 samples and more.  It holds none of the
policy-iteration arithmetic.  Obstacle scenes are drawn on the host exactly as
the host generator draws them.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

from . import Roadmap, Scene, _draw_scene

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "roadgen_gpu.cu")
LIB_PATH = os.path.join(_HERE, "libroadgen_gpu.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator for sm_103a in place (nvcc)."""
    deps = [_SRC, os.path.join(_HERE, "roadgen_gpu.h")]
    if not force and os.path.exists(LIB_PATH) and \
            all(os.path.getmtime(LIB_PATH) >= os.path.getmtime(d) for d in deps):
        return LIB_PATH
    tmp = f"{LIB_PATH}.{os.getpid()}.tmp"
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
           "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "-cudart", "static", _SRC, "-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode:
        raise RuntimeError("nvcc failed for the GPU roadmap generator:\n" + res.stderr)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def load():
    """Load the generator (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with workloads.gpu.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.rgg_sample.restype = ctypes.c_int
    lib.rgg_sample.argtypes = [i32, f64, f64, i32, vp, vp, ctypes.c_uint64, i64, vp, vp, vp]
    lib.rgg_knn.restype = ctypes.c_int
    lib.rgg_knn.argtypes = [i32, f64, f64, i64, vp, i32, f64, vp, vp]
    lib.rgg_explore_create.restype = ctypes.c_int
    lib.rgg_explore_create.argtypes = [i32, f64, f64, i32, vp, vp, ctypes.c_uint64, i64, i32, i32,
                                       i32, i32, i64, vp, ctypes.POINTER(vp)]
    lib.rgg_explore_block.restype = ctypes.c_int
    lib.rgg_explore_block.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp]
    lib.rgg_explore_points.restype = vp
    lib.rgg_explore_points.argtypes = [vp]
    lib.rgg_explore_size.restype = i64
    lib.rgg_explore_size.argtypes = [vp]
    lib.rgg_explore_copy_points.restype = ctypes.c_int
    lib.rgg_explore_copy_points.argtypes = [vp, vp, vp]
    lib.rgg_explore_destroy.restype = None
    lib.rgg_explore_destroy.argtypes = [vp]
    lib.rgg_edges.restype = ctypes.c_int
    lib.rgg_edges.argtypes = [i32, i64, vp, i32, vp, i32, vp, vp, i32, i32, i32, vp, vp, vp, vp,
                              i64, vp, vp]
    _lib = lib
    return lib


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(name: str, rc: int):
    if rc:
        raise RuntimeError(f"{name} failed with code {rc}")


def _scene_dev(scene: Scene):
    import torch
    c = torch.from_numpy(np.ascontiguousarray(scene.centers, dtype=np.float64)).cuda()
    r = torch.from_numpy(np.ascontiguousarray(scene.radii, dtype=np.float64)).cuda()
    return c, r


def sample(scene: Scene, n: int, seed: int):
    """n free samples of the scene's box (float64 CUDA tensor n x dim) and the
    number of candidates drawn."""
    import torch
    lib = load()
    c, r = _scene_dev(scene)
    pts = torch.empty((n, scene.dim), dtype=torch.float64, device="cuda")
    tried = ctypes.c_int64(0)
    _check("rgg_sample", lib.rgg_sample(scene.dim, float(scene.lo), float(scene.hi),
                                        len(scene.radii), c.data_ptr(), r.data_ptr(),
                                        int(seed) & 0xFFFFFFFFFFFFFFFF, n, pts.data_ptr(),
                                        ctypes.byref(tried), _stream()))
    return pts, int(tried.value)


def knn(points, lo: float, hi: float, k: int, cell: float = 0.0):
    """k nearest neighbours (int32 CUDA tensor n x k, nearest first)."""
    import torch
    lib = load()
    n, dim = points.shape
    out = torch.empty((n, k), dtype=torch.int32, device="cuda")
    _check("rgg_knn", lib.rgg_knn(dim, float(lo), float(hi), n, points.data_ptr(), k,
                                  float(cell), out.data_ptr(), _stream()))
    return out


def edges(points, nbr, scene: Scene, exact_segment: bool, n_check: int = 16,
          cost_dtype=np.float32):
    """Union-symmetrised, collision-checked edges of the k-NN table ordered by
    the larger endpoint: u, v, cost (CUDA tensors) and edge_start (host int64)."""
    import torch
    lib = load()
    n, dim = points.shape
    k = nbr.shape[1]
    c, r = _scene_dev(scene)
    f64 = np.dtype(cost_dtype) == np.float64
    tdt = torch.float64 if f64 else torch.float32
    start = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    m = ctypes.c_int64(0)
    args = (dim, n, points.data_ptr(), k, nbr.data_ptr(), len(scene.radii), c.data_ptr(),
            r.data_ptr(), 0 if exact_segment else 1, int(n_check), 1 if f64 else 0)
    rc = lib.rgg_edges(*args, None, None, None, start.data_ptr(), 0, ctypes.byref(m), _stream())
    if rc not in (0, 3):
        _check("rgg_edges", rc)
    cap = int(m.value)
    u = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    v = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    cost = torch.empty(max(cap, 1), dtype=tdt, device="cuda")
    _check("rgg_edges", lib.rgg_edges(*args, u.data_ptr(), v.data_ptr(), cost.data_ptr(),
                                      start.data_ptr(), cap, ctypes.byref(m), _stream()))
    mm = int(m.value)
    return u[:mm], v[:mm], cost[:mm], start.cpu().numpy()


@dataclass
class DeviceRoadmap:
    """A roadmap whose points and edge arrays live on the GPU (the Roadmap
    layout: edges u < v ordered by v; edge_start on the host)."""
    name: str
    points: object       # CUDA float64 n x dim
    u: object            # CUDA int32
    v: object            # CUDA int32
    cost: object         # CUDA float32 / float64
    edge_start: np.ndarray
    block: int
    scene: Scene | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def m(self) -> int:
        return int(self.u.shape[0])

    def blocks(self, block: int | None = None):
        s = self.block if block is None else int(block)
        for v0 in range(0, self.n, s):
            v1 = min(self.n, v0 + s)
            yield v0, v1, int(self.edge_start[v0]), int(self.edge_start[v1])

    def n_blocks(self, block: int | None = None) -> int:
        s = self.block if block is None else int(block)
        return (self.n + s - 1) // s

    def to_host(self) -> Roadmap:
        return Roadmap(self.name, self.points.cpu().numpy(), self.u.cpu().numpy(),
                       self.v.cpu().numpy(), self.cost.cpu().numpy(), self.edge_start.copy(),
                       self.block, self.scene, dict(self.meta))


def roadmap_nd(name: str, seed: int, n: int, dim: int, n_obs: int, rmin: float, rmax: float,
               k: int, block: int, lo: float = -math.pi, hi: float = math.pi,
               cost_dtype=np.float32, exact_segment: bool = False, n_check: int = 16,
               cell: float = 0.0) -> DeviceRoadmap:
    """A [lo, hi]^dim roadmap built on the GPU: ball obstacles drawn on the host
    (numpy, seed), n free Philox samples (vertex 0 = the first, x_init), k-NN
    union edges, collision checks, Euclidean costs, blocks of `block`."""
    import time
    import torch
    t0 = time.perf_counter()
    scene = _draw_scene(np.random.default_rng(seed), dim, lo, hi, n_obs, rmin, rmax, [])
    pts, tried = sample(scene, n, seed)
    t1 = time.perf_counter()
    nbr = knn(pts, lo, hi, k, cell)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    u, v, cost, start = edges(pts, nbr, scene, exact_segment, n_check, cost_dtype)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    del nbr
    meta = dict(seed=seed, k=k, radii=(rmin, rmax), n_obs=n_obs, n=n, dim=dim,
                m_undirected=int(u.shape[0]), candidates=tried, generator="gpu",
                seconds=dict(sample=round(t1 - t0, 3), knn=round(t2 - t1, 3),
                             edges=round(t3 - t2, 3)))
    return DeviceRoadmap(name, pts, u, v, cost, start, block, scene, meta)


def roadmap_c3_gpu(trial: int = 0, n: int = 4_000_000, block: int = 50_000) -> DeviceRoadmap:
    """The 6-D workload built on the GPU: [-pi, pi]^6, 64 hyperspheres
    r ~ U[0.3, 0.8], k = 30, 16 points per segment, FP32 costs, blocks of 5e4
    (same scene law and seed as the host generator's; Philox samples)."""
    return roadmap_nd("c3-gpu", 3 * 1000 + trial, n, 6, 64, 0.3, 0.8, 30, block)


class Explorer:
    """Incremental exploration, one Batched-Extension block at a time (the
    Extend step of RRT#, Alg. 3): vertex i is joined to its k nearest
    predecessors by collision-free edges.  ``extend(v0, v1, slot, stream)``
    enqueues the block's edge construction on `stream` into one of two
    device buffers (`slot` 0 or 1) and returns (u, v, cost, count), count being
    a page-locked host tensor filled when the stream gets there: the work of
    the next block can run on its own stream while the current one is
    exploited (Sec. VII).  The graph does not depend on the block size."""

    def __init__(self, scene: Scene, n: int, k: int, seed: int, max_block: int,
                 exact_segment: bool = False, n_check: int = 16, cost_dtype=np.float32,
                 stream=None):
        import torch
        self._lib = load()
        self.scene, self.n, self.k = scene, int(n), int(k)
        self.cost_dtype = np.dtype(cost_dtype)
        c, r = _scene_dev(scene)
        h = ctypes.c_void_p()
        st = stream if stream is not None else _stream()
        _check("rgg_explore_create", self._lib.rgg_explore_create(
            scene.dim, float(scene.lo), float(scene.hi), len(scene.radii), c.data_ptr(),
            r.data_ptr(), int(seed) & 0xFFFFFFFFFFFFFFFF, self.n, self.k,
            0 if exact_segment else 1, int(n_check), 1 if self.cost_dtype == np.float64 else 0,
            int(max_block), st, ctypes.byref(h)))
        self._h = h
        torch.cuda.synchronize()
        tdt = torch.float64 if self.cost_dtype == np.float64 else torch.float32
        cap = int(max_block) * self.k
        self.bufs = [(torch.empty(cap, dtype=torch.int32, device="cuda"),
                      torch.empty(cap, dtype=torch.int32, device="cuda"),
                      torch.empty(cap, dtype=tdt, device="cuda")) for _ in range(2)]
        self.counts = [torch.zeros(1, dtype=torch.int64).pin_memory() for _ in range(2)]

    def extend(self, v0: int, v1: int, slot: int, stream=None):
        u, v, c = self.bufs[slot]
        cnt = self.counts[slot]
        st = stream if stream is not None else _stream()
        _check("rgg_explore_block", self._lib.rgg_explore_block(
            self._h, int(v0), int(v1), u.data_ptr(), v.data_ptr(), c.data_ptr(),
            cnt.data_ptr(), st))
        return u, v, c, cnt

    def points(self):
        """The samples as a CUDA float64 tensor (n x dim), copied."""
        import torch
        out = torch.empty((self.n, self.scene.dim), dtype=torch.float64, device="cuda")
        _check("rgg_explore_copy_points",
               self._lib.rgg_explore_copy_points(self._h, out.data_ptr(), _stream()))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rgg_explore_destroy(self._h)
            self._h = None

    __del__ = close
