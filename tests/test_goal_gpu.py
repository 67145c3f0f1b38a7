"""Goal-directed Replan (Sec. IV-C) on the GPU against the oracle.

With a goal x_goal and an admissible heuristic h, a vertex is promising when
g(v) + h(v) < g(x_goal); Improve takes only switches that make a vertex
promising and the top-down Evaluate expands only promising vertices.  What
the method fixes: g(x_goal) is the shortest-path cost, and with a consistent h
so is g(v) of every v with d(v) + h(v) < d(x_goal).  Values below pruned
vertices depend on the order of work and are checked for validity only (a
rooted tree; a stored g never below its parent's g plus the edge cost).

With a consistent h and the wave Evaluate only (no pointer jumping, which
does not prune), the GPU's pruning decisions are the oracle's: the whole
(g, parent) state is compared bit for bit.
"""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle as O
import paper_2003_04920_gb300 as P
from paper_2003_04920_gb300 import workloads as W
from tests import golden_io
from tests.gpu_util import G_RTOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()


def _goal_case(rm, target):
    """x_goal = the reachable vertex nearest to `target`; h = 0.99 x the
    Euclidean distance to it, rounded to FP32 (consistent: the edge costs are
    Euclidean lengths and the factor leaves room for the rounding)."""
    d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    reach = np.flatnonzero(np.isfinite(d))
    near = np.linalg.norm(rm.points[reach] - np.asarray(target), axis=1)
    goal = int(reach[np.argmin(near)])
    h = (0.99 * np.linalg.norm(rm.points - rm.points[goal], axis=1)).astype(np.float32)
    return d, goal, h


def _fixed(d, h, goal, rel=1e-9):
    sel = np.isfinite(d) & (d + h.astype(np.float64) < d[goal] * (1.0 - rel))
    sel[goal] = True
    return sel


def _edge_costs(rm):
    best = {}
    for a, b, c in zip(rm.u.tolist(), rm.v.tolist(), rm.cost.astype(np.float64).tolist()):
        k = (min(a, b), max(a, b))
        best[k] = min(best.get(k, math.inf), c)
    return best


def _check_valid(rm, g, p, d):
    """A rooted parent tree; g >= d; g(v) >= g(p(v)) + c(p(v), v)."""
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    try:
        bad, first = A.check_tree(p)
        assert bad == 0, f"parent tree broken at {first}"
    finally:
        A.close()
    fin = np.isfinite(g)
    assert np.all(g[fin] >= d[fin] * (1 - 1e-9))
    best = _edge_costs(rm)
    kids = np.flatnonzero(p >= 0)
    pc = np.array([best[(min(v, int(p[v])), max(v, int(p[v])))] for v in kids])
    assert np.all(g[kids] >= (g[p[kids]] + pc) * (1 - 1e-12))
    assert np.all(np.isinf(g[p < 0][1:]))


def _gpu_schedule(rm, goal, h, block=None, **kw):
    with P.Graph(rm.n, rm.m, 0, rm.cost.dtype) as G:
        if goal is not None:
            G.set_goal(goal, h)
        stats = []
        for v0, v1, e0, e1 in rm.blocks(block):
            G.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            stats.append(G.exploit(**kw))
        return G.get_costs(), G.get_parents(), stats


# ------------------------------------------------------------ golden ---

@pytest.mark.parametrize("name", [n for n in golden_io.names() if n.startswith("goal_")])
@pytest.mark.parametrize("evaluate", ["auto", "wave", "jump"])
def test_goal_golden_evaluate_forms(name, evaluate):
    gd = golden_io.load(name)
    with P.Graph(gd["n"], len(gd["u"]), gd["root"], np.float64) as G:
        G.insert_batch(gd["n"], gd["u"], gd["v"], gd["c"])
        G.set_goal(gd["goal"], gd["h"])
        if gd["init"] is not None:
            G.set_policy(gd["init"])
        st = G.exploit(evaluate=evaluate)
        g, p = G.get_costs(), G.get_parents()
    assert st["converged"] == 1
    d, _ = O.dijkstra(gd["n"], gd["u"], gd["v"], gd["c"], gd["root"])
    sel = _fixed(d, gd["h"].astype(np.float32), gd["goal"])
    np.testing.assert_array_equal(g[sel], gd["g"][sel])
    if evaluate != "jump":  # pointer jumping does not prune
        np.testing.assert_array_equal(g, gd["g"])
        np.testing.assert_array_equal(p, gd["parent"])
        assert st["iterations"] == gd["iterations"]


# ------------------------------------------------- 2-D roadmaps (C1) ---

def _c1(trial, dtype, block):
    rm = W.roadmap_c1(trial=trial)
    return W.Roadmap(rm.name, rm.points, rm.u, rm.v, rm.cost.astype(dtype), rm.edge_start,
                     block or rm.n)


@pytest.mark.parametrize("trial,block", [(0, None), (1, None), (0, 200), (2, 200)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_goal_wave_matches_oracle_bitwise(trial, block, dtype):
    """One insertion of the whole roadmap, or Batched-Extension blocks of 200
    (where ancestors improve after their subtrees were pruned, leaving values
    above their policy paths)."""
    rm = _c1(trial, dtype, block)
    d, goal, h = _goal_case(rm, (0.6, 0.6))
    g_ref, p_ref, st_ref = O.replan_schedule(rm, goal=goal, h=h.astype(np.float64))
    g, p, st = _gpu_schedule(rm, goal, h, evaluate="wave")
    np.testing.assert_array_equal(g, g_ref)
    np.testing.assert_array_equal(p, p_ref)
    assert [s["iterations"] for s in st] == [s["iterations"] for s in st_ref]
    assert [s["switches"] for s in st] == [s["switches"] for s in st_ref]
    sel = _fixed(d, h, goal)
    np.testing.assert_allclose(g[sel], d[sel], rtol=1e-12, atol=0)


@pytest.mark.parametrize("evaluate", ["auto", "jump", "async"])
def test_goal_other_evaluate_forms_fix_the_same_values(evaluate):
    rm = W.roadmap_c1(trial=2)
    d, goal, h = _goal_case(rm, (0.6, 0.6))
    g, p, st = _gpu_schedule(rm, goal, h, evaluate=evaluate)
    assert st[0]["converged"] == 1
    sel = _fixed(d, h, goal)
    np.testing.assert_allclose(g[sel], d[sel], rtol=G_RTOL, atol=0)
    _check_valid(rm, g, p, d)


# --------------------------------------- Batched-Extension (Alg. 3) ---

def test_goal_schedule_c2_small_and_pruning_saves_work():
    rm = W.roadmap_c2(n=30_000, block=1_000, companion=True)
    d, goal, h = _goal_case(rm, (0.7, 0.7))
    g, p, st = _gpu_schedule(rm, goal, h)
    assert all(s["converged"] == 1 for s in st)
    sel = _fixed(d, h, goal)
    assert sel.sum() > 100
    np.testing.assert_allclose(g[sel], d[sel], rtol=G_RTOL, atol=0)
    _check_valid(rm, g, p, d)
    g0, _, st0 = _gpu_schedule(rm, None, None)
    assert sum(s["relaxations"] for s in st) < sum(s["relaxations"] for s in st0)
    assert sum(s["evaluated"] for s in st) < sum(s["evaluated"] for s in st0)
    # the goal-free schedule fixes every vertex; the goal-directed one agrees on its set
    np.testing.assert_allclose(g[sel], g0[sel], rtol=G_RTOL, atol=0)


# ------------------------------------------ switching the goal around ---

def test_goal_off_or_unreachable_is_goal_free():
    rm = W.roadmap_c1(trial=0)
    n = rm.n
    u, v, c = rm.u, rm.v, rm.cost
    h = np.random.default_rng(3).random(n + 1).astype(np.float32)
    runs = []
    for goal in (None, n, -1):  # no goal; an isolated goal; a goal switched off
        with P.Graph(n + 1, len(u), 0, np.float64) as G:
            if goal is not None:
                G.set_goal(3 if goal == -1 else goal, h)
                if goal == -1:
                    G.set_goal(-1)
            G.insert_batch(n + 1, u, v, c)
            st = G.exploit()
            runs.append((G.get_costs(), G.get_parents(), st["iterations"], st["switches"]))
    for g, p, it, sw in runs[1:]:
        np.testing.assert_array_equal(g, runs[0][0])
        np.testing.assert_array_equal(p, runs[0][1])
        assert (it, sw) == runs[0][2:]


def test_goal_change_brings_pruned_subtrees_up_to_date():
    rm = W.roadmap_c2(n=20_000, block=2_000, companion=True)
    d, goal_a, h_a = _goal_case(rm, (0.3, 0.3))
    _, goal_b, h_b = _goal_case(rm, (0.9, 0.2))
    with P.Graph(rm.n, rm.m, 0, rm.cost.dtype) as G:
        G.set_goal(goal_a, h_a)
        for v0, v1, e0, e1 in rm.blocks():
            G.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            G.exploit()
        g_a = G.get_costs()
        G.set_goal(goal_b, h_b)
        assert G.exploit()["converged"] == 1
        g_b, p_b = G.get_costs(), G.get_parents()
        G.set_goal(-1)
        assert G.exploit()["converged"] == 1
        g_f, p_f = G.get_costs(), G.get_parents()
    sel_a = _fixed(d, h_a, goal_a)
    np.testing.assert_allclose(g_a[sel_a], d[sel_a], rtol=G_RTOL, atol=0)
    sel_b = _fixed(d, h_b, goal_b)
    np.testing.assert_allclose(g_b[sel_b], d[sel_b], rtol=G_RTOL, atol=0)
    _check_valid(rm, g_b, p_b, d)
    # back to the goal-free form: every vertex at its shortest-path cost
    np.testing.assert_allclose(g_f, d, rtol=G_RTOL, atol=0)
    assert O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64)).check_tree(p_f)[0] == 0


def test_goal_checkpoint_holds_the_whole_tree():
    rm = _c1(1, np.float64, 200)
    d, goal, h = _goal_case(rm, (0.6, 0.6))
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "g.ckpt")
        with P.Graph(rm.n, rm.m, 0, np.float64) as G:
            G.set_goal(goal, h)
            for v0, v1, e0, e1 in rm.blocks():
                G.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
                G.exploit(evaluate="wave")
            g_pruned, p_pruned = G.get_costs(), G.get_parents()
            G.save(path)
        with P.Graph(rm.n, rm.m, 0, np.float64) as H:
            H.load(path)
            g, p = H.get_costs(), H.get_parents()
    # the pruned state held values above their policy path; the file does not
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost)
    try:
        assert A.check_consistency(p, g, 1e-9)[0] == 0
        assert A.check_consistency(p_pruned, g_pruned, 1e-9)[0] > 0
        np.testing.assert_array_equal(p, p_pruned)
    finally:
        A.close()
    sel = _fixed(d, h, goal)
    np.testing.assert_allclose(g[sel], d[sel], rtol=G_RTOL, atol=0)


def test_goal_at_the_root_attaches_nothing():
    gd = golden_io.load("path5.txt")
    with P.Graph(gd["n"], len(gd["u"]), 0, np.float64) as G:
        G.set_goal(0, np.zeros(gd["n"], np.float32))
        G.insert_batch(gd["n"], gd["u"], gd["v"], gd["c"])
        st = G.exploit()
        g, p = G.get_costs(), G.get_parents()
    assert g[0] == 0.0 and np.all(np.isinf(g[1:])) and np.all(p == -1)
    assert st["iterations"] == 1 and st["switches"] == 0


def test_goal_argument_errors():
    with P.Graph(4, 4, 0, np.float64) as G:
        for goal, h, status in [(4, None, P.PIRRT_ERR_INVALID_ARG),
                                (-2, None, P.PIRRT_ERR_INVALID_ARG),
                                (1, np.ones(5, np.float32), P.PIRRT_ERR_INVALID_ARG),
                                (1, np.array([0, -1], np.float32), P.PIRRT_ERR_BAD_INPUT),
                                (1, np.array([np.nan], np.float32), P.PIRRT_ERR_BAD_INPUT),
                                (1, np.array([np.inf], np.float32), P.PIRRT_ERR_BAD_INPUT)]:
            with pytest.raises(P.PirrtError) as e:
                G.set_goal(goal, h)
            assert e.value.status == status
