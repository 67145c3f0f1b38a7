"""CPU oracle for the PI-RRT# exploitation path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the C source ``pirrt_oracle.c`` is compiled with gcc into
``liboracle.so`` and driven through ctypes.

* :class:`OracleGraph` -- O1, serial policy iteration following Alg. 2
  (Replan = loop of Improve and Evaluate) on an adjacency-list graph, in the
  goal-free form or, after ``set_goal``, the goal-directed form that prunes
  the walk to the promising set (Sec. IV-C).
* :func:`dijkstra` -- O2, FP64 Dijkstra (binary heap keyed (distance, id)).
  The correctness argument for Batched-Extension PI-RRT# (Sec. IV,
  "Correctness") says Replan reaches the optimal policy from any initial
  policy, so O1's fixpoint equals single-source shortest paths.
* checkers -- Bellman inequality, tree consistency, acyclic rooted parent
  tree, reachable set, and the unambiguous-parent mask used for parity.

Parity status: O2 is pinned to ``scipy.sparse.csgraph.dijkstra`` and to
brute-force path enumeration; O1 is pinned to O2 (theorem), to hand-solved
graphs and to closed forms (see ``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "pirrt_oracle.c")
LIB_PATH = os.path.join(_HERE, "liboracle.so")
LIB_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")

OK, ERR_ARG, ERR_CAPACITY, ERR_OOM, ERR_BAD_INPUT, ERR_NOT_CONVERGED = range(6)

_lib = None


def compile_oracle(source: str = SOURCE, out: str = LIB_PATH, extra=()) -> str:
    """gcc -O2 the oracle into a shared library (atomic replace)."""
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           *extra, source, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB_PATH) or \
            os.path.getmtime(LIB_PATH) < os.path.getmtime(SOURCE):
        compile_oracle()
    return LIB_PATH


def build_parallel(force: bool = False) -> str | None:
    """The same source built with OpenMP: the Jacobi Improve sweep shared
    over the host's cores, results identical to the plain build.  None if
    the compiler has no OpenMP (nothing else depends on it)."""
    try:
        if force or not os.path.exists(LIB_OMP_PATH) or \
                os.path.getmtime(LIB_OMP_PATH) < os.path.getmtime(SOURCE):
            compile_oracle(out=LIB_OMP_PATH, extra=("-fopenmp",))
    except (subprocess.CalledProcessError, OSError):
        return None
    return LIB_OMP_PATH


_lib_omp = None


def load_parallel():
    """The OpenMP build (built first if needed), or None without OpenMP."""
    global _lib_omp
    if _lib_omp is None:
        path = build_parallel()
        if path is None:
            return None
        _lib_omp = _declare(ctypes.CDLL(path))
    return _lib_omp


def threads(lib) -> int:
    """Threads a build's Improve sweep runs on (1 for the plain build)."""
    return int(lib.or_threads())


def _declare(lib):
    vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "or_create": (vp, [i64, i32]),
        "or_destroy": (None, [vp]),
        "or_num_vertices": (i64, [vp]),
        "or_insert": (ctypes.c_int, [vp, i64, i64, vp, vp, vp]),
        "or_set_policy": (ctypes.c_int, [vp, vp]),
        "or_replan": (ctypes.c_int, [vp, f64, i64, vp]),
        "or_get": (None, [vp, vp, vp]),
        "or_set_goal": (ctypes.c_int, [vp, i32, vp, i64]),
        "or_get_promising": (None, [vp, vp]),
        "or_csr_build": (vp, [i64, i64, vp, vp, vp]),
        "or_csr_destroy": (None, [vp]),
        "or_csr_entries": (i64, [vp]),
        "or_dijkstra": (ctypes.c_int, [vp, i32, vp, vp]),
        "or_component": (i64, [vp, i32, vp]),
        "or_check_tree": (i64, [vp, i32, vp, vp]),
        "or_check_bellman": (i64, [vp, vp, f64, vp]),
        "or_check_consistency": (i64, [vp, i32, vp, vp, f64, vp]),
        "or_unambiguous": (i64, [vp, i32, vp, f64, vp, vp]),
        "or_threads": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path: str | None = None):
    """Load the oracle library (building it first if needed).  A ``path``
    loads a separate copy, e.g. a deliberately mutated build in a test."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous"
    return a.ctypes.data


def _edges(u, v, c):
    return (np.ascontiguousarray(u, dtype=np.int32), np.ascontiguousarray(v, dtype=np.int32),
            np.ascontiguousarray(c, dtype=np.float64))


class OracleError(RuntimeError):
    def __init__(self, what: str, code: int):
        super().__init__(f"{what} failed with oracle status {code}")
        self.code = code


class OracleGraph:
    """O1: serial policy iteration (Alg. 2) on an adjacency-list graph."""

    def __init__(self, cap_n: int, root: int = 0, lib=None):
        self._lib = lib or load()
        self._h = self._lib.or_create(int(cap_n), int(root))
        if not self._h:
            raise MemoryError("or_create")
        self.root = int(root)

    def close(self):
        if self._h:
            self._lib.or_destroy(self._h)
            self._h = None

    __del__ = close

    @property
    def n(self) -> int:
        return int(self._lib.or_num_vertices(self._h))

    def insert(self, n_new: int, u, v, c) -> None:
        u, v, c = _edges(u, v, c)
        rc = self._lib.or_insert(self._h, int(n_new), len(u), _p(u), _p(v), _p(c))
        if rc:
            raise OracleError("or_insert", rc)

    def set_policy(self, parent) -> None:
        parent = np.ascontiguousarray(parent, dtype=np.int32)
        assert len(parent) == self.n
        rc = self._lib.or_set_policy(self._h, _p(parent))
        if rc:
            raise OracleError("or_set_policy", rc)

    def replan(self, eps: float = 0.0, max_iters: int = 0, check: bool = True) -> dict:
        st = np.zeros(5, dtype=np.int64)
        rc = self._lib.or_replan(self._h, float(eps), int(max_iters), _p(st))
        if rc and check:
            raise OracleError("or_replan", rc)
        return dict(iterations=int(st[0]), relaxations=int(st[1]), evaluated=int(st[2]),
                    switches=int(st[3]), converged=bool(st[4]), status=int(rc))

    def get(self):
        g = np.empty(self.n, dtype=np.float64)
        p = np.empty(self.n, dtype=np.int32)
        self._lib.or_get(self._h, _p(g), _p(p))
        return g, p

    def set_goal(self, goal: int, h=None) -> None:
        """Goal-directed form (Sec. IV-C): x_goal and h(v) for v < len(h)
        (0 beyond); goal = -1 switches it off."""
        h = np.ascontiguousarray(np.zeros(0) if h is None else h, dtype=np.float64)
        rc = self._lib.or_set_goal(self._h, int(goal), _p(h), len(h))
        if rc:
            raise OracleError("or_set_goal", rc)

    def promising(self) -> np.ndarray:
        """b(v) of the last Evaluate (the promising set B)."""
        b = np.empty(self.n, dtype=np.uint8)
        self._lib.or_get_promising(self._h, _p(b))
        return b.astype(bool)


class CSR:
    """Static merged adjacency for O2 and the checkers."""

    def __init__(self, n: int, u, v, c, lib=None):
        self._lib = lib or load()
        u, v, c = _edges(u, v, c)
        self.n = int(n)
        self._h = self._lib.or_csr_build(self.n, len(u), _p(u), _p(v), _p(c))
        if not self._h:
            raise MemoryError("or_csr_build")

    def close(self):
        if self._h:
            self._lib.or_csr_destroy(self._h)
            self._h = None

    __del__ = close

    @property
    def entries(self) -> int:
        return int(self._lib.or_csr_entries(self._h))

    def dijkstra(self, root: int = 0):
        d = np.empty(self.n, dtype=np.float64)
        p = np.empty(self.n, dtype=np.int32)
        rc = self._lib.or_dijkstra(self._h, int(root), _p(d), _p(p))
        if rc:
            raise OracleError("or_dijkstra", rc)
        return d, p

    def component(self, root: int = 0) -> np.ndarray:
        r = np.empty(self.n, dtype=np.uint8)
        self._lib.or_component(self._h, int(root), _p(r))
        return r.astype(bool)

    def check_tree(self, parent, root: int = 0):
        parent = np.ascontiguousarray(parent, dtype=np.int32)
        first = ctypes.c_int64(-1)
        bad = self._lib.or_check_tree(self._h, int(root), _p(parent), ctypes.byref(first))
        return int(bad), int(first.value)

    def check_bellman(self, g, rel: float = 1e-12):
        g = np.ascontiguousarray(g, dtype=np.float64)
        worst = ctypes.c_int64(-1)
        bad = self._lib.or_check_bellman(self._h, _p(g), float(rel), ctypes.byref(worst))
        return int(bad), int(worst.value)

    def check_consistency(self, parent, g, rel: float = 1e-12, root: int = 0):
        parent = np.ascontiguousarray(parent, dtype=np.int32)
        g = np.ascontiguousarray(g, dtype=np.float64)
        first = ctypes.c_int64(-1)
        bad = self._lib.or_check_consistency(self._h, int(root), _p(parent), _p(g),
                                             float(rel), ctypes.byref(first))
        return int(bad), int(first.value)

    def unambiguous(self, g, rel: float = 1e-6, root: int = 0):
        g = np.ascontiguousarray(g, dtype=np.float64)
        mask = np.empty(self.n, dtype=np.uint8)
        arg = np.empty(self.n, dtype=np.int32)
        self._lib.or_unambiguous(self._h, int(root), _p(g), float(rel), _p(mask), _p(arg))
        return mask.astype(bool), arg


def dijkstra(n: int, u, v, c, root: int = 0):
    """O2 on the undirected graph given as an edge list."""
    A = CSR(n, u, v, c)
    try:
        return A.dijkstra(root)
    finally:
        A.close()


def replan_schedule(rm, block: int | None = None, init_parent=None, eps: float = 0.0,
                    lib=None, n_blocks: int | None = None, goal: int | None = None, h=None):
    """Batched-Extension schedule (Alg. 3) on O1: insert block b (its vertices
    and the edges whose larger endpoint lies in it), then Replan.  With
    ``init_parent`` (one block holding every vertex) the policy is set to it
    before the single Replan.  With ``goal`` the Replan is goal-directed
    (Sec. IV-C) with heuristic ``h``.  Returns (g, parent, per-block stats)."""
    G = OracleGraph(rm.n, 0, lib=lib)
    stats = []
    try:
        if goal is not None:
            G.set_goal(goal, h)
        for i, (v0, v1, e0, e1) in enumerate(rm.blocks(block)):
            if n_blocks is not None and i >= n_blocks:
                break
            G.insert(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1].astype(np.float64))
            if init_parent is not None:
                G.set_policy(init_parent[:v1])
            stats.append(G.replan(eps=eps))
        g, p = G.get()
    finally:
        G.close()
    return g, p, stats
