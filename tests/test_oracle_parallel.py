"""The oracle built with OpenMP (the Jacobi Improve sweep shared over the
host's cores, a CPU baseline on all cores) gives the plain build's results
bit for bit: g, parents and every statistic of every Replan, on a
Batched-Extension schedule and on the goal-directed form."""
import numpy as np
import pytest

import oracle as O
from paper_2003_04920_gb300 import workloads as W


@pytest.fixture(scope="module")
def par():
    lib = O.load_parallel()
    if lib is None:
        pytest.skip("no OpenMP in this compiler")
    return lib


def _schedule(rm, lib, goal=None, h=None):
    G = O.OracleGraph(rm.n, lib=lib)
    if goal is not None:
        G.set_goal(goal, h)
    stats = []
    for v0, v1, e0, e1 in rm.blocks():
        G.insert(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1].astype(np.float64))
        stats.append(G.replan())
    g, p = G.get()
    G.close()
    return g, p, stats


@pytest.mark.parametrize("goal", [False, True])
def test_parallel_build_matches_the_plain_build(par, goal):
    rm = W.roadmap_c3(n=6_000, block=500)
    h = target = None
    if goal:
        target = rm.n - 1
        h = 0.99 * np.linalg.norm(rm.points - rm.points[target], axis=1)
    g0, p0, s0 = _schedule(rm, O.load(), target, h)
    g1, p1, s1 = _schedule(rm, par, target, h)
    assert np.array_equal(g0.view(np.int64), g1.view(np.int64))
    assert np.array_equal(p0, p1)
    assert s0 == s1
    assert O.threads(O.load()) == 1 and O.threads(par) >= 1
