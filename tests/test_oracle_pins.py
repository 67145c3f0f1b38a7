"""Pins for the CPU oracle: each check ties it to something other than itself.

* O2 (Dijkstra) against scipy.sparse.csgraph.dijkstra (a library routine) and
  against brute-force enumeration of every simple path on tiny graphs.
* O1 (serial policy iteration, Alg. 2) against O2: by the correctness
  argument of Sec. IV ("Correctness"), Replan reaches the optimal policy from
  any initial policy, so its fixpoint is the shortest-path tree.
* Hand-solved graphs (tests/golden/) for g, parents and iteration counts,
  including the tie rule of Alg. 2's strict comparison.
* Closed form: on a complete Euclidean graph the triangle inequality makes
  the direct edge optimal, g(v) = |x_v - x_0| and parent 0.
* Lower bound g(v) >= |x_v - x_0| on any Euclidean roadmap.
* Batched-Extension (Alg. 3): the final policy does not depend on S.
* Iteration bound (Sec. IV): at most (optimal path length in edges) + 2.
* Goal-directed form (Sec. IV-C): hand-solved pruning cases; g(x_goal) is
  the shortest-path cost (admissible h), and so is g(v) of every v with
  d(v) + h(v) < d(x_goal) (consistent h); no goal, an unreachable goal and
  h = 0 reduce to the goal-free Replan or to Dijkstra's settled set.
* Checkers flag planted violations; planted mistakes in a copy of the oracle
  source fail the pins above.
"""
import itertools
import math
import os
import re
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import dijkstra as scipy_dijkstra

import oracle as O
from paper_2003_04920_gb300 import workloads as W
from tests import golden_io


def _scipy_sp(n, u, v, c, root=0):
    # scipy keeps duplicate COO entries summed; merge to the minimum first
    key = np.minimum(u, v).astype(np.int64) * n + np.maximum(u, v)
    order = np.lexsort((c, key))
    key, c2 = key[order], np.asarray(c, dtype=np.float64)[order]
    first = np.r_[True, key[1:] != key[:-1]]
    key, c2 = key[first], c2[first]
    a, b = key // n, key % n
    M = coo_matrix((np.r_[c2, c2], (np.r_[a, b], np.r_[b, a])), shape=(n, n)).tocsr()
    return scipy_dijkstra(M, directed=True, indices=root)


def _o1(n, u, v, c, init=None, root=0, eps=0.0, goal=None, h=None, lib=None):
    G = O.OracleGraph(n, root, lib=lib)
    G.insert(n, u, v, c)
    if goal is not None:
        G.set_goal(goal, h)
    if init is not None:
        G.set_policy(init)
    st = G.replan(eps=eps)
    g, p = G.get()
    G.close()
    return g, p, st


# ---------------------------------------------------------------- golden ---

@pytest.mark.parametrize("name", golden_io.names())
def test_golden_o1(name):
    gd = golden_io.load(name)
    g, p, st = _o1(gd["n"], gd["u"], gd["v"], gd["c"], gd["init"], gd["root"],
                   goal=gd["goal"], h=gd["h"])
    np.testing.assert_array_equal(g, gd["g"])
    np.testing.assert_array_equal(p, gd["parent"])
    assert st["converged"]
    assert st["iterations"] == gd["iterations"]


@pytest.mark.parametrize("name", golden_io.names())
def test_golden_o2(name):
    gd = golden_io.load(name)
    d, _ = O.dijkstra(gd["n"], gd["u"], gd["v"], gd["c"], gd["root"])
    if gd["goal"] is None:
        np.testing.assert_array_equal(d, gd["g"])
    else:  # only x_goal and the vertices promising at the optimum are fixed
        sel = _goal_fixed(d, gd["h"], gd["goal"])
        assert sel[gd["goal"]] and sel.sum() >= 2
        np.testing.assert_array_equal(d[sel], gd["g"][sel])


# ------------------------------------------------------- O2 vs library ---

@pytest.mark.parametrize("seed", range(6))
def test_dijkstra_matches_scipy_random(seed):
    n = 50 + 37 * seed
    rm = W.random_graph(seed, n, 4 * n, connected=seed % 2 == 0)
    d, _ = O.dijkstra(n, rm.u, rm.v, rm.cost)
    ref = _scipy_sp(n, rm.u, rm.v, rm.cost)
    np.testing.assert_array_equal(np.isinf(d), np.isinf(ref))
    fin = np.isfinite(ref)
    np.testing.assert_allclose(d[fin], ref[fin], rtol=1e-13, atol=0)


def test_dijkstra_matches_scipy_roadmap_c1():
    rm = W.roadmap_c1()
    d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost)
    ref = _scipy_sp(rm.n, rm.u, rm.v, rm.cost)
    np.testing.assert_allclose(d, ref, rtol=1e-13, atol=0)


# ------------------------------------------------------- brute force ---

def _all_simple_paths_min(n, u, v, c, root=0):
    adj = {x: {} for x in range(n)}
    for a, b, w in zip(u.tolist(), v.tolist(), c.tolist()):
        for x, y in ((a, b), (b, a)):
            adj[x][y] = min(w, adj[x].get(y, math.inf))
    best = [math.inf] * n
    best_paths = [[] for _ in range(n)]
    stack = [(root, 0.0, (root,))]
    while stack:
        x, dist, path = stack.pop()
        if dist < best[x]:
            best[x] = dist
            best_paths[x] = [path]
        elif dist == best[x]:
            best_paths[x].append(path)
        for y, w in adj[x].items():
            if y not in path:
                stack.append((y, dist + w, path + (y,)))
    return np.array(best), best_paths


@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_tiny(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 9))
    m = int(rng.integers(n - 1, n * (n - 1) // 2 + 1))
    rm = W.random_graph(100 + seed, n, m, connected=bool(seed % 3))
    ref, paths = _all_simple_paths_min(n, rm.u, rm.v, rm.cost)
    d, _ = O.dijkstra(n, rm.u, rm.v, rm.cost)
    g, p, st = _o1(n, rm.u, rm.v, rm.cost)
    for got in (d, g):
        np.testing.assert_array_equal(np.isinf(got), np.isinf(ref))
        fin = np.isfinite(ref)
        np.testing.assert_allclose(got[fin], ref[fin], rtol=1e-12)
    # where exactly one optimal path exists, its last hop is O1's parent
    for x in range(1, n):
        if len(paths[x]) == 1 and np.isfinite(ref[x]):
            assert p[x] == paths[x][0][-2]
        if not np.isfinite(ref[x]):
            assert p[x] == -1


# ------------------------------------------------ O1 vs O2 (theorem) ---

def test_o1_fixpoint_equals_dijkstra_c1_bfs_start():
    rm = W.roadmap_c1()
    init = W.bfs_tree_parents(rm)
    g, p, st = _o1(rm.n, rm.u, rm.v, rm.cost, init)
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost)
    d, _ = A.dijkstra()
    np.testing.assert_allclose(g, d, rtol=1e-12, atol=0)
    mask, arg = A.unambiguous(d)
    assert mask.sum() > 0.9 * rm.n
    np.testing.assert_array_equal(p[mask], arg[mask])
    assert A.check_tree(p) == (0, -1)
    assert A.check_bellman(g)[0] == 0
    assert A.check_consistency(p, g, 0.0)[0] == 0


@pytest.mark.parametrize("seed", range(5))
def test_o1_fixpoint_equals_dijkstra_random(seed):
    n = 300
    rm = W.random_graph(200 + seed, n, 5 * n, cost_dtype=np.float32, connected=seed != 2)
    c = rm.cost.astype(np.float64)
    g, p, _ = _o1(n, rm.u, rm.v, c)
    A = O.CSR(n, rm.u, rm.v, c)
    d, _ = A.dijkstra()
    np.testing.assert_array_equal(np.isinf(g), np.isinf(d))
    fin = np.isfinite(d)
    np.testing.assert_allclose(g[fin], d[fin], rtol=1e-12)
    mask, arg = A.unambiguous(d)
    np.testing.assert_array_equal(p[mask], arg[mask])
    reach = A.component()
    np.testing.assert_array_equal(p >= 0, reach & (np.arange(n) != 0))


def test_o1_schedule_equals_dijkstra_fp32_knn():
    rm = W.roadmap_c2(n=8000, block=500, companion=True)
    g, p, stats = O.replan_schedule(rm)
    assert all(s["converged"] for s in stats)
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    d, _ = A.dijkstra()
    np.testing.assert_allclose(g, d, rtol=1e-12)
    mask, arg = A.unambiguous(d)
    np.testing.assert_array_equal(p[mask], arg[mask])


# ------------------------------------------------------- closed forms ---

@pytest.mark.parametrize("dim", [2, 3, 6])
def test_closed_form_complete_euclidean_graph(dim):
    rng = np.random.default_rng(dim)
    n = 60
    x = rng.uniform(-1, 1, (n, dim))
    u, v = np.triu_indices(n, 1)
    c = np.linalg.norm(x[u] - x[v], axis=1)
    g, p, _ = _o1(n, u.astype(np.int32), v.astype(np.int32), c)
    want = np.linalg.norm(x - x[0], axis=1)
    np.testing.assert_allclose(g, want, rtol=1e-13, atol=0)
    assert (p[1:] == 0).mean() > 0.95  # near-collinear triples may tie in rounding
    np.testing.assert_allclose(g[p == 0], want[p == 0], rtol=0, atol=0)


def test_lower_bound_euclidean_c1():
    rm = W.roadmap_c1()
    g, _, _ = _o1(rm.n, rm.u, rm.v, rm.cost)
    lb = np.linalg.norm(rm.points - rm.points[0], axis=1)
    fin = np.isfinite(g)
    assert np.all(g[fin] >= lb[fin] * (1 - 1e-12))


# ------------------------------------------- Batched-Extension (Alg. 3) ---

def test_s_independence():
    rm = W.roadmap_c2(n=1500, block=1500, companion=True)
    runs = {}
    for s in (1, 7, 100, rm.n):
        g, p, stats = O.replan_schedule(rm, block=s)
        assert all(st["converged"] for st in stats)
        runs[s] = (g, p)
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    d, _ = A.dijkstra()
    mask, _ = A.unambiguous(d)
    for s, (g, p) in runs.items():
        np.testing.assert_allclose(g, d, rtol=1e-12)
        np.testing.assert_array_equal(p[mask], runs[rm.n][1][mask])


def test_iteration_bound():
    rm = W.roadmap_c1()
    init = W.bfs_tree_parents(rm)
    g, p, st = _o1(rm.n, rm.u, rm.v, rm.cost, init)
    depth = np.zeros(rm.n, dtype=np.int64)
    order = np.argsort(g)
    for x in order:
        if p[x] >= 0:
            depth[x] = depth[p[x]] + 1
    assert st["iterations"] <= depth.max() + 2


# ---------------------------------------- goal-directed form (Sec. IV-C) ---

def _goal_fixed(d, h, goal, rel=1e-9):
    """The vertices whose g a goal-directed Replan fixes: x_goal, and every v
    with d(v) + h(v) < d(x_goal), by a relative margin so that rounding
    cannot move a vertex across the boundary."""
    sel = np.isfinite(d) & (d + h < d[goal] * (1.0 - rel))
    sel[goal] = True
    return sel


def _goal_case(seed, target=(0.6, 0.6), scale=0.99):
    """A 2-D roadmap of the C1 recipe, x_goal = the reachable vertex nearest to
    ``target`` and h = scale x the Euclidean distance to x_goal, which is
    consistent because every edge cost is a Euclidean length."""
    rm = W.roadmap_c1(trial=seed)
    d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost)
    reach = np.flatnonzero(np.isfinite(d))
    near = np.linalg.norm(rm.points[reach] - np.asarray(target), axis=1)
    goal = int(reach[np.argmin(near)])
    h = scale * np.linalg.norm(rm.points - rm.points[goal], axis=1)
    return rm, d, goal, h


def _goal_theorem_holds(seed, lib=None) -> bool:
    rm, d, goal, h = _goal_case(seed)
    g, _, st = _o1(rm.n, rm.u, rm.v, rm.cost, goal=goal, h=h, lib=lib)
    sel = _goal_fixed(d, h, goal)
    return bool(st["converged"] and np.allclose(g[sel], d[sel], rtol=1e-12, atol=0))


def _parent_cost(rm, p):
    """c(p(v), v) of the cheapest parallel edge, +inf where p(v) < 0."""
    best = {}
    for a, b, c in zip(rm.u.tolist(), rm.v.tolist(), np.asarray(rm.cost, np.float64).tolist()):
        k = (min(a, b), max(a, b))
        best[k] = min(best.get(k, math.inf), c)
    return np.array([best[(min(v, int(q)), max(v, int(q)))] if q >= 0 else math.inf
                     for v, q in enumerate(p)])


@pytest.mark.parametrize("seed", range(3))
def test_goal_directed_reaches_the_optimum_c1(seed):
    rm, d, goal, h = _goal_case(seed)
    g, p, st = _o1(rm.n, rm.u, rm.v, rm.cost, goal=goal, h=h)
    _, _, st_free = _o1(rm.n, rm.u, rm.v, rm.cost)
    assert st["converged"]
    sel = _goal_fixed(d, h, goal)
    np.testing.assert_allclose(g[sel], d[sel], rtol=1e-12, atol=0)
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost)
    assert A.check_tree(p) == (0, -1)
    # a stored g is never below the cost of its policy path
    fin = np.isfinite(g)
    assert np.all(g[fin] >= d[fin] * (1 - 1e-12))
    kid = p >= 0
    assert np.all(g[kid] >= g[p[kid]] + _parent_cost(rm, p)[kid])
    # the pruning took effect: fewer values assigned, some vertices left
    # above their shortest-path cost or unreached
    assert st["evaluated"] < st_free["evaluated"]
    assert np.sum(~np.isfinite(g) | (g > d * (1 + 1e-12))) > 0


def test_goal_with_zero_heuristic_fixes_the_dijkstra_ball():
    rm, d, goal, _ = _goal_case(1)
    g, _, _ = _o1(rm.n, rm.u, rm.v, rm.cost, goal=goal, h=np.zeros(rm.n))
    sel = _goal_fixed(d, np.zeros(rm.n), goal)
    assert sel.sum() > 10
    np.testing.assert_allclose(g[sel], d[sel], rtol=1e-12, atol=0)


def test_goal_off_or_unreachable_is_the_goal_free_replan():
    n = 300
    rm = W.random_graph(77, n, 5 * n)
    c = rm.cost.astype(np.float64)
    h = np.random.default_rng(5).random(n + 1)
    g0, p0, st0 = _o1(n + 1, rm.u, rm.v, c)
    # x_goal = vertex n, which no edge reaches: g(x_goal) stays +inf
    g1, p1, st1 = _o1(n + 1, rm.u, rm.v, c, goal=n, h=h)
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(p0, p1)
    assert st0 == st1
    G = O.OracleGraph(n + 1)
    G.insert(n + 1, rm.u, rm.v, c)
    G.set_goal(3, h)
    G.set_goal(-1, h)
    st2 = G.replan()
    g2, p2 = G.get()
    G.close()
    np.testing.assert_array_equal(g0, g2)
    np.testing.assert_array_equal(p0, p2)
    assert st0 == st2


def test_goal_at_the_root_attaches_nothing():
    n = 50
    rm = W.random_graph(9, n, 4 * n)
    g, p, st = _o1(n, rm.u, rm.v, rm.cost, goal=0, h=np.zeros(n))
    assert g[0] == 0.0 and np.all(np.isinf(g[1:])) and np.all(p == -1)
    assert st["iterations"] == 1 and st["switches"] == 0


def test_goal_directed_schedule_fp32_knn():
    rm = W.roadmap_c2(n=8000, block=500, companion=True)
    c = rm.cost.astype(np.float64)
    d, _ = O.dijkstra(rm.n, rm.u, rm.v, c)
    reach = np.flatnonzero(np.isfinite(d))
    goal = int(reach[np.argmin(np.linalg.norm(rm.points[reach] - 0.9, axis=1))])
    h = 0.99 * np.linalg.norm(rm.points - rm.points[goal], axis=1)
    sel = _goal_fixed(d, h, goal)
    for block in (500, rm.n):
        g, _, stats = O.replan_schedule(rm, block=block, goal=goal, h=h)
        assert all(s["converged"] for s in stats)
        np.testing.assert_allclose(g[sel], d[sel], rtol=1e-12, atol=0)


@pytest.mark.parametrize("seed", range(40))
def test_goal_directed_bruteforce_tiny(seed):
    """Points in the plane, edge costs at least the Euclidean distance, so
    h(v) = |x_v - x_goal| is consistent; every simple path is enumerated."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(3, 9))
    x = rng.random((n, 2))
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.6]
    if not pairs:
        pairs = [(0, 1)]
    u = np.array([a for a, _ in pairs], dtype=np.int32)
    v = np.array([b for _, b in pairs], dtype=np.int32)
    c = np.linalg.norm(x[u] - x[v], axis=1) * (1.0 + rng.random(len(u)))
    ref, _ = _all_simple_paths_min(n, u, v, c)
    goal = int(rng.integers(1, n))
    h = np.linalg.norm(x - x[goal], axis=1) * rng.choice([0.0, 0.5, 1.0])
    g, p, st = _o1(n, u, v, c, goal=goal, h=h)
    assert st["converged"]
    if math.isinf(ref[goal]):  # no goal cost ever: the goal-free result
        g0, p0, _ = _o1(n, u, v, c)
        np.testing.assert_array_equal(g, g0)
        np.testing.assert_array_equal(p, p0)
        return
    np.testing.assert_allclose(g[goal], ref[goal], rtol=1e-12, atol=0)
    sel = np.isfinite(ref) & (ref + h < ref[goal] * (1 - 1e-9))
    np.testing.assert_allclose(g[sel], ref[sel], rtol=1e-12, atol=0)
    fin = np.isfinite(g)
    assert np.all(g[fin] >= ref[fin] * (1 - 1e-12))


def test_goal_rejects_bad_heuristic():
    G = O.OracleGraph(4)
    for bad in ([0.0, -1.0], [0.0, np.nan], [np.inf]):
        with pytest.raises(O.OracleError):
            G.set_goal(1, np.array(bad))
    with pytest.raises(O.OracleError):
        G.set_goal(4, None)
    G.close()


# ------------------------------------------------------------ checkers ---

def test_checkers_flag_planted_violations():
    gd = golden_io.load("chain_shortcut.txt")
    A = O.CSR(gd["n"], gd["u"], gd["v"], gd["c"])
    g, p = gd["g"].copy(), gd["parent"].copy()
    assert A.check_tree(p) == (0, -1)
    assert A.check_bellman(g)[0] == 0
    assert A.check_consistency(p, g, 0.0)[0] == 0
    cyc = p.copy(); cyc[4], cyc[5] = 5, 4          # 4 <-> 5 cycle
    assert A.check_tree(cyc)[0] == 2
    far = p.copy(); far[3] = 0                      # 0-3 is not an edge
    assert A.check_tree(far)[0] >= 1
    rooted = p.copy(); rooted[0] = 1
    assert A.check_tree(rooted)[0] >= 1
    worse = g.copy(); worse[3] = 9.0                # g(3) > g(2) + 1
    assert A.check_bellman(worse)[0] >= 1
    off = g.copy(); off[5] += 1e-6
    assert A.check_consistency(p, off, 1e-9)[0] >= 1
    mask, arg = A.unambiguous(g)
    assert arg[4] == 5 and mask[4]


def test_oracle_rejects_bad_input():
    G = O.OracleGraph(4)
    for u, v, c in (([0], [4], [1.0]), ([1], [1], [1.0]), ([0], [1], [0.0]),
                    ([0], [1], [-1.0]), ([0], [1], [np.nan]), ([0], [1], [np.inf])):
        with pytest.raises(O.OracleError):
            G.insert(4, u, v, c)
    with pytest.raises(O.OracleError):
        G.insert(5, [], [], [])
    G.close()


# ------------------------------------------------ planted mistakes ---

MUTANTS = {
    "strict_to_nonstrict": ("if (cand < ghat) {", "if (cand <= ghat) {"),
    "dropped_parent_cost": ("G->g[y] = G->pc[y] + G->g[x];", "G->g[y] = G->g[x];"),
    "wrong_index_in_evaluate": ("G->g[y] = G->pc[y] + G->g[x];", "G->g[y] = G->pc[x] + G->g[x];"),
    "stale_policy_cost": ("G->pc[x] = best_c;\n", "\n"),
    "wrong_sign_delta": ("double d = cur - ghat;", "double d = ghat - cur;"),
    "parallel_edge_max": ("(L->nbr[j] == w && L->c[j] > c)", "(L->nbr[j] == w && L->c[j] < c)"),
    "dijkstra_dropped_cost": ("double nd = dist[x] + A->c[i];", "double nd = dist[x] + 1.0;"),
    "promising_nonstrict": ("if (G->g[y] + G->h[y] < bound) {", "if (G->g[y] + G->h[y] <= bound) {"),
    "promising_tests_parent": ("if (G->g[y] + G->h[y] < bound) {",
                               "if (G->g[x] + G->h[x] < bound) {"),
    "evaluate_ignores_h": ("if (G->g[y] + G->h[y] < bound) {", "if (G->g[y] < bound) {"),
    "lookahead_nonstrict": ("ghat + G->h[x] < bound", "ghat + G->h[x] <= bound"),
    "no_lookahead": ("if (best >= 0 && ghat + G->h[x] < bound) {", "if (best >= 0) {"),
    "improve_ignores_h": ("ghat + G->h[x] < bound", "ghat < bound"),
}


def _pins_pass(lib) -> bool:
    try:
        for name in golden_io.names():
            gd = golden_io.load(name)
            g, p, st = _o1(gd["n"], gd["u"], gd["v"], gd["c"], gd["init"], gd["root"],
                           goal=gd["goal"], h=gd["h"], lib=lib)
            if not (np.array_equal(g, gd["g"]) and np.array_equal(p, gd["parent"])
                    and st["iterations"] == gd["iterations"]):
                return False
            A = O.CSR(gd["n"], gd["u"], gd["v"], gd["c"], lib=lib)
            d, _ = A.dijkstra()
            A.close()
            sel = (np.ones(gd["n"], dtype=bool) if gd["goal"] is None
                   else _goal_fixed(d, gd["h"], gd["goal"]))
            if not np.array_equal(d[sel], gd["g"][sel]):
                return False
        if not _goal_theorem_holds(0, lib):
            return False
        for seed in range(3):
            rm = W.random_graph(300 + seed, 40, 120)
            A = O.CSR(40, rm.u, rm.v, rm.cost, lib=lib)
            d, _ = A.dijkstra()
            A.close()
            if not np.allclose(d, _scipy_sp(40, rm.u, rm.v, rm.cost), rtol=1e-13):
                return False
    except O.OracleError:
        return False
    return True


def test_pins_pass_on_the_real_oracle():
    assert _pins_pass(O.load())


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant, tmp_path):
    src = open(O.SOURCE).read()
    old, new = MUTANTS[mutant]
    assert src.count(old) >= 1, f"mutation anchor missing: {old!r}"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new, 1))
    lib_path = O.compile_oracle(str(mutated), str(tmp_path / "libmutant.so"))
    assert not _pins_pass(O.load(lib_path)), f"mutant {mutant} survived the pins"
