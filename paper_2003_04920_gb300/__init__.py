"""GB300 exploitation path of PI-RRT# (Policy Iteration RRT#).

A thin ctypes binding over the C ABI declared in ``include/pirrt.h``
(``libpirrt.so``, hand-written sm_103a CUDA kernels).  The functions keep the
C names (``pirrt_graph_create`` ... ``pirrt_graph_get_parents``) and only
marshal arguments: every step of insertion, Improve and Evaluate runs in the
library's kernels.  There is no CPU fallback: if the library is not built,
loading fails loudly.

:class:`Graph` wraps a handle for Python callers.  Device buffers may be
PyTorch CUDA tensors (PyTorch supplies device memory and the stream); host
buffers are NumPy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpirrt.so")

PIRRT_OK = 0
PIRRT_ERR_INVALID_ARG = 1
PIRRT_ERR_CAPACITY = 2
PIRRT_ERR_OOM = 3
PIRRT_ERR_CUDA = 4
PIRRT_ERR_NOT_CONVERGED = 5
PIRRT_ERR_DEVICE_TIMEOUT = 6
PIRRT_ERR_BAD_INPUT = 7
PIRRT_ERR_BAD_TREE = 8
PIRRT_COST_F32 = 0
PIRRT_COST_F64 = 1
PIRRT_EVAL_AUTO = 0
PIRRT_EVAL_WAVE = 1
PIRRT_EVAL_JUMP = 2
PIRRT_EVAL_ASYNC = 3
PIRRT_SELFTEST_GRID_BARRIER = 0
PIRRT_SELFTEST_MBARRIER = 1
EVALUATE_MODES = {"auto": PIRRT_EVAL_AUTO, "wave": PIRRT_EVAL_WAVE, "jump": PIRRT_EVAL_JUMP,
                  "async": PIRRT_EVAL_ASYNC}


class pirrt_config(ctypes.Structure):
    _fields_ = [("max_vertices", ctypes.c_int64), ("max_edges", ctypes.c_int64),
                ("root", ctypes.c_int32), ("cost_dtype", ctypes.c_int32),
                ("device", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class pirrt_exploit_opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("group", ctypes.c_int32), ("tile", ctypes.c_int32), ("evaluate", ctypes.c_int32),
                ("wave_levels", ctypes.c_int32), ("host_loop", ctypes.c_int32),
                ("dense_fraction", ctypes.c_double), ("wave_tail", ctypes.c_int32),
                ("wave_ctas", ctypes.c_int32), ("wave_local", ctypes.c_int32),
                ("wave_local_max", ctypes.c_int32), ("wave_local_step", ctypes.c_int32)]


class pirrt_exploit_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("relaxations", ctypes.c_int64), ("improved", ctypes.c_int64),
                ("switches", ctypes.c_int64), ("evaluated", ctypes.c_int64),
                ("jump_rounds", ctypes.c_int32), ("dense_sweeps", ctypes.c_int32),
                ("wave_levels", ctypes.c_int32), ("jump_evaluates", ctypes.c_int32),
                ("ms_exploit", ctypes.c_float), ("graph_launch", ctypes.c_int32),
                ("improve_entries", ctypes.c_int64), ("offers", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class pirrt_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("improve_launches", ctypes.c_int64),
                ("evaluate_launches", ctypes.c_int64), ("mark_launches", ctypes.c_int64),
                ("insert_calls", ctypes.c_int64), ("improve_ms", ctypes.c_double),
                ("evaluate_ms", ctypes.c_double), ("mark_ms", ctypes.c_double),
                ("insert_ms", ctypes.c_double), ("improve_entries", ctypes.c_int64),
                ("improve_vertices", ctypes.c_int64), ("improve_dense_vertices", ctypes.c_int64),
                ("improve_switches", ctypes.c_int64), ("evaluate_vertices", ctypes.c_int64),
                ("evaluate_visits", ctypes.c_int64), ("mark_vertices", ctypes.c_int64),
                ("insert_new_entries", ctypes.c_int64), ("insert_copied_entries", ctypes.c_int64),
                ("evaluate_offers", ctypes.c_int64),
                ("level_count", ctypes.c_int64 * 24), ("level_vertices", ctypes.c_int64 * 24),
                ("level_cycles", ctypes.c_int64 * 24), ("wave_pre_cycles", ctypes.c_int64),
                ("wave_post_cycles", ctypes.c_int64), ("wave_jump_cycles", ctypes.c_int64),
                ("wave_calls", ctypes.c_int64),
                ("share_tiles", ctypes.c_int64 * 24), ("share_vertices", ctypes.c_int64 * 24),
                ("share_cycles", ctypes.c_int64 * 24), ("local_tiles", ctypes.c_int64 * 24),
                ("local_vertices", ctypes.c_int64 * 24), ("local_cycles", ctypes.c_int64 * 24),
                ("wave_span_ns", ctypes.c_int64), ("wave_spans", ctypes.c_int64),
                ("wave_gap_ns", ctypes.c_int64), ("wave_gaps", ctypes.c_int64)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class pirrt_trace_record(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int32), ("dense", ctypes.c_int32),
                ("improve_vertices", ctypes.c_int64), ("improve_entries", ctypes.c_int64),
                ("switches", ctypes.c_int32), ("changed", ctypes.c_int32),
                ("wave_levels", ctypes.c_int32), ("next_frontier", ctypes.c_int32),
                ("improve_ms", ctypes.c_float), ("evaluate_ms", ctypes.c_float),
                ("mark_ms", ctypes.c_float), ("iteration_ms", ctypes.c_float),
                ("offers", ctypes.c_int64)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpirrt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library {path} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    st = ctypes.c_int
    sig = {
        "pirrt_graph_create": (st, [ctypes.POINTER(pirrt_config), ctypes.POINTER(vp)]),
        "pirrt_graph_destroy": (None, [vp]),
        "pirrt_graph_reset": (st, [vp]),
        "pirrt_graph_insert_batch": (st, [vp, i64, i64, vp, vp, vp, i32]),
        "pirrt_graph_set_policy": (st, [vp, vp, i64, i32]),
        "pirrt_graph_exploit": (st, [vp, ctypes.POINTER(pirrt_exploit_opts),
                                     ctypes.POINTER(pirrt_exploit_stats)]),
        "pirrt_graph_get_costs": (st, [vp, vp, i64, i32]),
        "pirrt_graph_get_parents": (st, [vp, vp, i64, i32]),
        "pirrt_graph_get_adjacency": (st, [vp, vp, vp, vp, i32]),
        "pirrt_graph_save": (st, [vp, ctypes.c_char_p]),
        "pirrt_graph_prefetch_batch": (st, [vp, i64, vp, vp, vp]),
        "pirrt_graph_set_goal": (st, [vp, ctypes.c_int32, vp, i64]),
        "pirrt_graph_load": (st, [vp, ctypes.c_char_p]),
        "pirrt_graph_set_profiling": (st, [vp, i32]),
        "pirrt_graph_get_profile": (st, [vp, ctypes.POINTER(pirrt_profile)]),
        "pirrt_graph_get_trace": (i64, [vp, ctypes.POINTER(pirrt_trace_record), i64]),
        "pirrt_graph_num_vertices": (i64, [vp]),
        "pirrt_graph_num_entries": (i64, [vp]),
        "pirrt_graph_last_error": (ctypes.c_char_p, [vp]),
        "pirrt_status_string": (ctypes.c_char_p, [st]),
        "pirrt_evaluate_noalloc": (st, [i64, ctypes.c_int32, vp, vp, vp, vp]),
        "pirrt_selftest_wait": (st, [ctypes.c_int32, i64, vp]),
        "pirrt_batch_create": (st, [ctypes.c_int32, vp, vp, vp, ctypes.c_int32, ctypes.c_int32, vp,
                                    ctypes.POINTER(vp)]),
        "pirrt_batch_destroy": (None, [vp]),
        "pirrt_batch_reset": (st, [vp]),
        "pirrt_batch_insert": (st, [vp, ctypes.c_int32, i64, vp, vp, vp, i32]),
        "pirrt_batch_exploit": (st, [vp, ctypes.POINTER(pirrt_exploit_opts),
                                     ctypes.POINTER(pirrt_exploit_stats)]),
        "pirrt_batch_autotune": (st, [vp, ctypes.POINTER(pirrt_exploit_opts), ctypes.c_int32,
                                      ctypes.POINTER(pirrt_exploit_opts),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
        "pirrt_batch_autotune_search": (st, [vp, ctypes.POINTER(pirrt_exploit_opts), ctypes.c_int32,
                                             ctypes.POINTER(pirrt_exploit_opts),
                                             ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(ctypes.c_int32)]),
        "pirrt_batch_get_costs": (st, [vp, ctypes.c_int32, vp, i64, i32]),
        "pirrt_batch_get_parents": (st, [vp, ctypes.c_int32, vp, i64, i32]),
        "pirrt_batch_graph": (vp, [vp]),
        "pirrt_proposal_num_params": (i64, []),
        "pirrt_proposal_create": (st, [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                       ctypes.c_int32, vp, ctypes.POINTER(vp)]),
        "pirrt_proposal_destroy": (None, [vp]),
        "pirrt_proposal_set_weights": (st, [vp, vp, i64]),
        "pirrt_proposal_get_weights": (st, [vp, vp, i64]),
        "pirrt_proposal_forward": (st, [vp, ctypes.c_int32, vp, ctypes.c_int32, vp, vp, vp]),
        "pirrt_proposal_sample": (st, [vp, ctypes.c_int32, vp, ctypes.c_int32, vp, vp, vp, vp,
                                       ctypes.c_float, vp]),
        "pirrt_proposal_imle_select": (st, [vp, ctypes.c_int32, vp, ctypes.c_int32, vp, vp,
                                            ctypes.c_int32, vp, vp]),
        "pirrt_proposal_backward": (st, [vp, ctypes.c_int32, vp, ctypes.c_int32, vp, vp, vp,
                                         ctypes.POINTER(ctypes.c_float)]),
        "pirrt_proposal_get_grads": (st, [vp, vp, i64]),
        "pirrt_proposal_zero_grads": (st, [vp]),
        "pirrt_proposal_set_options": (st, [vp, ctypes.c_int32, ctypes.c_int32]),
        "pirrt_proposal_get_activations": (st, [vp, ctypes.c_int32, vp, vp]),
        "pirrt_proposal_kernel_ms": (st, [vp, ctypes.POINTER(ctypes.c_float)]),
        "pirrt_proposal_train_step": (st, [vp, ctypes.c_int32, vp, ctypes.c_int32, vp, vp,
                                           ctypes.c_int32, vp, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_float)]),
        "pirrt_proposal_adam": (st, [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PirrtError(RuntimeError):
    def __init__(self, call: str, status: int, detail: str = ""):
        lib = load_library()
        name = lib.pirrt_status_string(status).decode()
        super().__init__(f"{call}: {name}" + (f" ({detail})" if detail else ""))
        self.status = status


def _buf(x, dtype):
    """(pointer, on_device, keepalive) for a torch tensor or array-like."""
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        assert x.is_contiguous(), "tensor must be contiguous"
        if x.is_cuda:
            return x.data_ptr(), 1, x
        x = x.numpy()
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, 0, a


def _current_stream_ptr(device: int):
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except ImportError:
        pass
    return None


class Graph:
    """One planning graph resident on a GPU (wraps a ``pirrt_graph*``)."""

    def __init__(self, max_vertices: int, max_edges: int, root: int = 0,
                 cost_dtype=np.float32, device: int = 0, stream=None):
        self._lib = load_library()
        self.cost_dtype = np.dtype(cost_dtype)
        if self.cost_dtype not in (np.float32, np.float64):
            raise ValueError("cost_dtype must be float32 or float64")
        if stream is None:
            stream = _current_stream_ptr(device)
        cfg = pirrt_config(int(max_vertices), int(max_edges), int(root),
                           PIRRT_COST_F32 if self.cost_dtype == np.float32 else PIRRT_COST_F64,
                           int(device), 0, stream)
        h = ctypes.c_void_p()
        rc = self._lib.pirrt_graph_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc:
            raise PirrtError("pirrt_graph_create", rc)
        self._h = h
        self.root = int(root)
        self.device = int(device)

    def _check(self, call: str, rc: int):
        if rc:
            detail = self._lib.pirrt_graph_last_error(self._h).decode()
            raise PirrtError(call, rc, detail)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pirrt_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n(self) -> int:
        return int(self._lib.pirrt_graph_num_vertices(self._h))

    @property
    def m(self) -> int:
        return int(self._lib.pirrt_graph_num_entries(self._h))

    def reset(self):
        self._check("pirrt_graph_reset", self._lib.pirrt_graph_reset(self._h))

    def insert_batch(self, n_new: int, src, dst, cost):
        ps, ds, ks = _buf(src, np.int32)
        pd, dd, kd = _buf(dst, np.int32)
        pc, dc, kc = _buf(cost, self.cost_dtype)
        if not (ds == dd == dc):
            raise ValueError("src, dst and cost must all be host or all be device buffers")
        n_edges = len(ks) if ds == 0 else ks.numel()
        rc = self._lib.pirrt_graph_insert_batch(self._h, int(n_new), int(n_edges), ps, pd, pc, ds)
        self._check("pirrt_graph_insert_batch", rc)

    def prefetch_batch(self, src, dst, cost):
        """Copy the next block's host edge list on the graph's copy stream while
        the current exploit runs; the next insert_batch with the same arrays
        uses it.  Keep the arrays unchanged until then (page-locked memory lets
        the copy overlap)."""
        ps, ds, ks = _buf(src, np.int32)
        pd, dd, kd = _buf(dst, np.int32)
        pc, dc, kc = _buf(cost, self.cost_dtype)
        if ds or dd or dc:
            raise ValueError("prefetch_batch takes host arrays")
        self._pre_keep = (ks, kd, kc)
        self._check("pirrt_graph_prefetch_batch",
                    self._lib.pirrt_graph_prefetch_batch(self._h, int(len(ks)), ps, pd, pc))

    def set_goal(self, goal: int, h=None):
        """Goal-directed Replan (Sec. IV-C): x_goal and the heuristic h(v) for
        v < len(h) (host, FP32; 0 beyond).  goal = -1 returns to the goal-free
        form."""
        h = np.ascontiguousarray(np.zeros(0) if h is None else h, dtype=np.float32)
        self._check("pirrt_graph_set_goal",
                    self._lib.pirrt_graph_set_goal(self._h, int(goal), h.ctypes.data, int(len(h))))

    def set_policy(self, parent):
        pp, dev, keep = _buf(parent, np.int32)
        n = len(keep) if dev == 0 else keep.numel()
        self._check("pirrt_graph_set_policy",
                    self._lib.pirrt_graph_set_policy(self._h, pp, int(n), dev))

    def exploit(self, eps: float = 0.0, max_iters: int = 0, group: int = 0, tile: int = 0,
                dense_fraction: float = 0.0, evaluate: str = "auto", wave_levels: int = 0,
                host_loop: bool = False, wave_tail: int = 0, wave_ctas: int = 0,
                wave_local: int = 0, wave_local_max: int = 0, wave_local_step: int = 0,
                check: bool = True) -> dict:
        opts = exploit_opts(eps, max_iters, group, tile, dense_fraction, evaluate, wave_levels,
                            host_loop, wave_tail, wave_ctas, wave_local, wave_local_max,
                            wave_local_step)
        st = pirrt_exploit_stats()
        rc = self._lib.pirrt_graph_exploit(self._h, ctypes.byref(opts), ctypes.byref(st))
        out = st.as_dict()
        out["status"] = int(rc)
        if check:
            self._check("pirrt_graph_exploit", rc)
        return out

    def set_profiling(self, enable=True):
        """True: event timing (host loop); False: off; 2: the device-side wave
        trace alone, every exploit still one CUDA-graph launch."""
        mode = 2 if enable == 2 else (1 if enable else 0)
        self._check("pirrt_graph_set_profiling",
                    self._lib.pirrt_graph_set_profiling(self._h, mode))

    def get_profile(self) -> dict:
        pr = pirrt_profile()
        self._check("pirrt_graph_get_profile",
                    self._lib.pirrt_graph_get_profile(self._h, ctypes.byref(pr)))
        return pr.as_dict()

    def get_trace(self) -> np.ndarray:
        """Per-iteration trace recorded while profiling (structured array)."""
        n = int(self._lib.pirrt_graph_get_trace(self._h, None, 0))
        buf = (pirrt_trace_record * max(n, 1))()
        self._lib.pirrt_graph_get_trace(self._h, buf, n)
        names = [f for f, _ in pirrt_trace_record._fields_]
        arr = np.ctypeslib.as_array(buf)[:n]
        return np.array([tuple(r) for r in arr.tolist()], dtype=[(nm, arr.dtype[nm]) for nm in names]) \
            if n else np.zeros(0, dtype=arr.dtype)

    def get_costs(self, out=None) -> np.ndarray:
        n = self.n
        if out is None:
            out = np.empty(n, dtype=np.float64)
        p, dev, keep = _buf(out, np.float64)
        self._check("pirrt_graph_get_costs", self._lib.pirrt_graph_get_costs(self._h, p, n, dev))
        return out

    def get_parents(self, out=None) -> np.ndarray:
        n = self.n
        if out is None:
            out = np.empty(n, dtype=np.int32)
        p, dev, keep = _buf(out, np.int32)
        self._check("pirrt_graph_get_parents",
                    self._lib.pirrt_graph_get_parents(self._h, p, n, dev))
        return out

    def get_adjacency(self):
        n, m = self.n, self.m
        off = np.empty(n + 1, dtype=np.int64)
        col = np.empty(m, dtype=np.int32)
        cost = np.empty(m, dtype=self.cost_dtype)
        self._check("pirrt_graph_get_adjacency",
                    self._lib.pirrt_graph_get_adjacency(self._h, off.ctypes.data, col.ctypes.data,
                                                        cost.ctypes.data, 0))
        return off, col, cost

    def save(self, path: str):
        """Checkpoint the graph (CSR, g, policy) to a file."""
        self._check("pirrt_graph_save", self._lib.pirrt_graph_save(self._h, os.fsencode(path)))

    def load(self, path: str):
        """Replace this graph's contents with a checkpoint."""
        self._check("pirrt_graph_load", self._lib.pirrt_graph_load(self._h, os.fsencode(path)))


def pirrt_status_string(status: int) -> str:
    return load_library().pirrt_status_string(int(status)).decode()


def run_schedule(graph: Graph, roadmap, block: int | None = None, on_device_inputs=None,
                 **exploit_kw) -> list[dict]:
    """Batched-Extension schedule (Alg. 3): for each block, insert its
    vertices and edges, then exploit to convergence.  ``on_device_inputs``
    may hold (u, v, cost) device tensors of the whole roadmap."""
    stats = []
    for v0, v1, e0, e1 in roadmap.blocks(block):
        if on_device_inputs is not None:
            u, v, c = on_device_inputs
            graph.insert_batch(v1 - v0, u[e0:e1], v[e0:e1], c[e0:e1])
        else:
            graph.insert_batch(v1 - v0, roadmap.u[e0:e1], roadmap.v[e0:e1], roadmap.cost[e0:e1])
        stats.append(graph.exploit(**exploit_kw))
    return stats


def pirrt_evaluate_noalloc(parent, parent_cost, g_out, root: int = 0, stream=None) -> int:
    """Evaluate g from device tensors without any allocation by the library
    (scratch in a static device array, at most 262,144 vertices).  ``parent``
    is int32, ``parent_cost`` and ``g_out`` are float64, all three contiguous
    CUDA tensors of one length on one device.  Returns the pirrt_status code."""
    import torch
    lib = load_library()
    for name, t, dt in (("parent", parent, torch.int32), ("parent_cost", parent_cost, torch.float64),
                        ("g_out", g_out, torch.float64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise TypeError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    n = int(parent.numel())
    if parent_cost.numel() != n or g_out.numel() != n:
        raise ValueError("parent, parent_cost and g_out must have the same length")
    if parent_cost.device != parent.device or g_out.device != parent.device:
        raise ValueError("parent, parent_cost and g_out must be on one device")
    dev = parent.device.index or 0
    with torch.cuda.device(dev):
        if stream is None:
            stream = _current_stream_ptr(dev)
        return int(lib.pirrt_evaluate_noalloc(n, int(root), parent.data_ptr(),
                                              parent_cost.data_ptr(), g_out.data_ptr(), stream))


def pirrt_selftest_wait(which: int, limit: int, stream=None) -> int:
    """Run one bounded device wait that nothing will end (failure detection
    self-test): ``which`` = PIRRT_SELFTEST_GRID_BARRIER (limit in polls) or
    PIRRT_SELFTEST_MBARRIER (limit in ns).  Returns the pirrt_status code,
    PIRRT_ERR_DEVICE_TIMEOUT when the wait gave up as designed."""
    lib = load_library()
    if stream is None:
        stream = _current_stream_ptr(0)
    return int(lib.pirrt_selftest_wait(int(which), int(limit), stream))


def opts_dict(o: pirrt_exploit_opts) -> dict:
    """The keyword arguments of exploit_opts that give `o`."""
    modes = {v: k for k, v in EVALUATE_MODES.items()}
    return {"eps": o.eps, "max_iters": o.max_iters, "group": o.group, "tile": o.tile,
            "dense_fraction": o.dense_fraction, "evaluate": modes[o.evaluate],
            "wave_levels": o.wave_levels, "host_loop": bool(o.host_loop),
            "wave_tail": o.wave_tail, "wave_ctas": o.wave_ctas, "wave_local": o.wave_local,
            "wave_local_max": o.wave_local_max, "wave_local_step": o.wave_local_step}


def exploit_opts(eps: float = 0.0, max_iters: int = 0, group: int = 0, tile: int = 0,
                 dense_fraction: float = 0.0, evaluate: str = "auto", wave_levels: int = 0,
                 host_loop: bool = False, wave_tail: int = 0,
                 wave_ctas: int = 0, wave_local: int = 0,
                 wave_local_max: int = 0, wave_local_step: int = 0) -> pirrt_exploit_opts:
    return pirrt_exploit_opts(float(eps), int(max_iters), int(group), int(tile),
                              EVALUATE_MODES[evaluate], int(wave_levels), int(bool(host_loop)),
                              float(dense_fraction), int(wave_tail), int(wave_ctas),
                              int(wave_local), int(wave_local_max), int(wave_local_step))


class Batch:
    """Many independent planning graphs exploited together (wraps a
    ``pirrt_batch*``): the disjoint union of the members in one device graph,
    one CUDA-graph launch per exploit."""

    def __init__(self, max_vertices, max_edges, roots=None, cost_dtype=np.float32,
                 device: int = 0, stream=None):
        self._lib = load_library()
        mv = np.ascontiguousarray(max_vertices, dtype=np.int64)
        me = np.ascontiguousarray(max_edges, dtype=np.int64)
        rt = np.ascontiguousarray(np.zeros(len(mv)) if roots is None else roots, dtype=np.int32)
        self.cost_dtype = np.dtype(cost_dtype)
        if stream is None:
            stream = _current_stream_ptr(device)
        h = ctypes.c_void_p()
        rc = self._lib.pirrt_batch_create(len(mv), mv.ctypes.data, me.ctypes.data, rt.ctypes.data,
                                          PIRRT_COST_F32 if self.cost_dtype == np.float32
                                          else PIRRT_COST_F64, int(device), stream,
                                          ctypes.byref(h))
        if rc:
            raise PirrtError("pirrt_batch_create", rc)
        self._h = h
        self.n_graphs = len(mv)
        self.max_vertices = mv

    def _graph_handle(self):
        return self._lib.pirrt_batch_graph(self._h)

    def _check(self, call: str, rc: int):
        if rc:
            detail = self._lib.pirrt_graph_last_error(self._graph_handle()).decode()
            raise PirrtError(call, rc, detail)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pirrt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def reset(self):
        self._check("pirrt_batch_reset", self._lib.pirrt_batch_reset(self._h))

    def insert(self, graph: int, src, dst, cost):
        ps, ds, ks = _buf(src, np.int32)
        pd, dd, kd = _buf(dst, np.int32)
        pc, dc, kc = _buf(cost, self.cost_dtype)
        if not (ds == dd == dc):
            raise ValueError("src, dst and cost must all be host or all be device buffers")
        n_edges = len(ks) if ds == 0 else ks.numel()
        self._check("pirrt_batch_insert",
                    self._lib.pirrt_batch_insert(self._h, int(graph), int(n_edges), ps, pd, pc, ds))

    def exploit(self, check: bool = True, **kw) -> dict:
        opts = exploit_opts(**kw)
        st = pirrt_exploit_stats()
        rc = self._lib.pirrt_batch_exploit(self._h, ctypes.byref(opts), ctypes.byref(st))
        out = st.as_dict()
        out["status"] = int(rc)
        if check:
            self._check("pirrt_batch_exploit", rc)
        return out

    def autotune(self, candidates: list[dict]):
        """Time every candidate option set from the current state (restored
        after each trial); returns (best options dict, index, ms)."""
        arr = (pirrt_exploit_opts * len(candidates))(*[exploit_opts(**c) for c in candidates])
        best = pirrt_exploit_opts()
        idx = ctypes.c_int32(-1)
        ms = ctypes.c_float(0)
        self._check("pirrt_batch_autotune",
                    self._lib.pirrt_batch_autotune(self._h, arr, len(candidates), ctypes.byref(best),
                                                   ctypes.byref(idx), ctypes.byref(ms)))
        return candidates[idx.value], idx.value, ms.value

    def autotune_search(self, max_trials: int = 40, start: dict | None = None):
        """Coordinate-descent search of the exploit options from the current
        state (restored after each trial); returns (best options dict, ms,
        trials run)."""
        st = exploit_opts(**start) if start else None
        best = pirrt_exploit_opts()
        ms = ctypes.c_float(0)
        n = ctypes.c_int32(0)
        self._check("pirrt_batch_autotune_search",
                    self._lib.pirrt_batch_autotune_search(
                        self._h, ctypes.byref(st) if st is not None else None, int(max_trials),
                        ctypes.byref(best), ctypes.byref(ms), ctypes.byref(n)))
        return opts_dict(best), ms.value, n.value

    def get_costs(self, graph: int, n: int, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(n, dtype=np.float64)
        p, dev, keep = _buf(out, np.float64)
        self._check("pirrt_batch_get_costs",
                    self._lib.pirrt_batch_get_costs(self._h, int(graph), p, int(n), dev))
        return out

    def get_parents(self, graph: int, n: int, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(n, dtype=np.int32)
        p, dev, keep = _buf(out, np.int32)
        self._check("pirrt_batch_get_parents",
                    self._lib.pirrt_batch_get_parents(self._h, int(graph), p, int(n), dev))
        return out

    def set_profiling(self, enable: bool = True):
        self._check("pirrt_graph_set_profiling",
                    self._lib.pirrt_graph_set_profiling(self._graph_handle(), 1 if enable else 0))

    def get_profile(self) -> dict:
        pr = pirrt_profile()
        self._check("pirrt_graph_get_profile",
                    self._lib.pirrt_graph_get_profile(self._graph_handle(), ctypes.byref(pr)))
        return pr.as_dict()


class Proposal:
    """Learned sampling proposal (wraps a ``pirrt_proposal*``).  Arrays are
    PyTorch CUDA tensors: grids [S, 4096] float32 in {0, 1}, scene int32 [R],
    noise float32 [R, 8], targets float32 [R, 2]."""

    def __init__(self, max_scenes: int, max_rows: int, seed: int = 0, device: int = 0,
                 stream=None):
        self._lib = load_library()
        if stream is None:
            stream = _current_stream_ptr(device)
        h = ctypes.c_void_p()
        rc = self._lib.pirrt_proposal_create(int(max_scenes), int(max_rows), int(seed),
                                             int(device), stream, ctypes.byref(h))
        if rc:
            raise PirrtError("pirrt_proposal_create", rc)
        self._h = h
        self.max_scenes, self.max_rows = int(max_scenes), int(max_rows)
        self.n_params = int(self._lib.pirrt_proposal_num_params())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pirrt_proposal_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, call, rc):
        if rc:
            raise PirrtError(call, rc)

    @staticmethod
    def _dev(x, dtype: str = "float32"):
        """Device pointer of a contiguous CUDA tensor of the given dtype."""
        import torch
        want = {"float32": torch.float32, "int32": torch.int32}[dtype]
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.is_contiguous()):
            raise ValueError("expected a contiguous CUDA tensor")
        if x.dtype != want:
            raise TypeError(f"expected a {dtype} tensor, got {x.dtype}")
        return x.data_ptr()

    def get_weights(self):
        import torch
        w = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        self._check("pirrt_proposal_get_weights",
                    self._lib.pirrt_proposal_get_weights(self._h, w.data_ptr(), self.n_params))
        return w

    def set_weights(self, w):
        self._check("pirrt_proposal_set_weights",
                    self._lib.pirrt_proposal_set_weights(self._h, self._dev(w), self.n_params))

    def get_grads(self):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        self._check("pirrt_proposal_get_grads",
                    self._lib.pirrt_proposal_get_grads(self._h, g.data_ptr(), self.n_params))
        return g

    def zero_grads(self):
        self._check("pirrt_proposal_zero_grads", self._lib.pirrt_proposal_zero_grads(self._h))

    FORWARD_KERNELS = {"tcgen05": 0, "layered": 1}

    def set_options(self, forward_kernel: str = "tcgen05", keep_activations: bool = False):
        """Forward kernel of forward / sample / imle_select / train_step's
        draws ("tcgen05": the fused tensor-core kernel, "layered": GEMM per
        layer) and whether forward passes leave h1, h2 for get_activations."""
        if forward_kernel not in self.FORWARD_KERNELS:
            raise ValueError(f"forward_kernel must be one of {sorted(self.FORWARD_KERNELS)}")
        self._check("pirrt_proposal_set_options",
                    self._lib.pirrt_proposal_set_options(self._h,
                                                         self.FORWARD_KERNELS[forward_kernel],
                                                         1 if keep_activations else 0))

    def kernel_ms(self) -> float:
        """Device time of the last fused forward kernel (CUDA events), ms."""
        ms = ctypes.c_float(0)
        self._check("pirrt_proposal_kernel_ms",
                    self._lib.pirrt_proposal_kernel_ms(self._h, ctypes.byref(ms)))
        return float(ms.value)

    def get_activations(self, rows: int):
        """h1, h2 of the last forward pass's first `rows` rows as BF16 bit
        patterns (int16 CUDA tensors [rows, 256])."""
        import torch
        h1 = torch.empty((int(rows), 256), dtype=torch.int16, device="cuda")
        h2 = torch.empty((int(rows), 256), dtype=torch.int16, device="cuda")
        self._check("pirrt_proposal_get_activations",
                    self._lib.pirrt_proposal_get_activations(self._h, int(rows), h1.data_ptr(),
                                                             h2.data_ptr()))
        return h1, h2

    def forward(self, grids, scene, noise):
        import torch
        out = torch.empty((scene.numel(), 2), dtype=torch.float32, device="cuda")
        self._check("pirrt_proposal_forward",
                    self._lib.pirrt_proposal_forward(self._h, grids.shape[0], self._dev(grids),
                                                     scene.numel(), self._dev(scene, "int32"),
                                                     self._dev(noise), out.data_ptr()))
        return out

    def sample(self, grids, scene, noise, uniform_xy, coin, learned_fraction: float = 0.5):
        """Mixture of the network's samples and the caller's uniform ones:
        row r is learned when coin[r] < learned_fraction."""
        import torch
        out = torch.empty((scene.numel(), 2), dtype=torch.float32, device="cuda")
        self._check("pirrt_proposal_sample",
                    self._lib.pirrt_proposal_sample(self._h, grids.shape[0], self._dev(grids),
                                                    scene.numel(), self._dev(scene, "int32"),
                                                    self._dev(noise), self._dev(uniform_xy),
                                                    self._dev(coin), float(learned_fraction),
                                                    out.data_ptr()))
        return out

    def imle_select(self, grids, draw_scene, targets, K: int, noise):
        import torch
        pick = torch.empty(targets.shape[0], dtype=torch.int32, device="cuda")
        self._check("pirrt_proposal_imle_select",
                    self._lib.pirrt_proposal_imle_select(self._h, grids.shape[0], self._dev(grids),
                                                         targets.shape[0], self._dev(draw_scene, "int32"),
                                                         self._dev(targets), int(K),
                                                         self._dev(noise), pick.data_ptr()))
        return pick

    def backward(self, grids, scene, noise, targets) -> float:
        loss = ctypes.c_float(0)
        self._check("pirrt_proposal_backward",
                    self._lib.pirrt_proposal_backward(self._h, grids.shape[0], self._dev(grids),
                                                      scene.numel(), self._dev(scene, "int32"),
                                                      self._dev(noise), self._dev(targets),
                                                      ctypes.byref(loss)))
        return float(loss.value)

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self._check("pirrt_proposal_adam",
                    self._lib.pirrt_proposal_adam(self._h, float(lr), float(beta1), float(beta2),
                                                  float(eps)))

    def train_step(self, grids, target_scene, targets, K: int, noise, lr: float) -> float:
        """One IMLE step in the library: K draws per target, the nearest is
        pulled to it, then Adam.  Returns the loss before the step."""
        loss = ctypes.c_float(0)
        self._check("pirrt_proposal_train_step",
                    self._lib.pirrt_proposal_train_step(self._h, grids.shape[0], self._dev(grids),
                                                        targets.shape[0], self._dev(target_scene, "int32"),
                                                        self._dev(targets), int(K),
                                                        self._dev(noise), float(lr),
                                                        ctypes.byref(loss)))
        return float(loss.value)
