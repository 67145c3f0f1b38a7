"""Batched form: many independent graphs exploited together in one device
graph (the disjoint union) with one CUDA-graph launch per exploit.

Policy iteration on a disjoint union is policy iteration on each member at
once, so every member must equal its own solo run bit for bit (with the
top-down Evaluate, whose sums do not depend on the batch)."""
import numpy as np
import pytest

import oracle as O
import paper_2003_04920_gb300 as P
from paper_2003_04920_gb300 import workloads as W
from tests.gpu_util import assert_parity, gpu_schedule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()


@pytest.fixture(scope="module")
def members():
    return W.roadmap_batch(n_graphs=24, trial=1, n_min=300, n_max=8000)


def _batch_run(members, **kw):
    with P.Batch([rm.n for rm in members], [rm.m for rm in members]) as B:
        for i, rm in enumerate(members):
            B.insert(i, rm.u, rm.v, rm.cost)
        st = B.exploit(**kw)
        res = [(B.get_costs(i, rm.n), B.get_parents(i, rm.n)) for i, rm in enumerate(members)]
    return res, st


def test_batch_equals_solo_runs_bitwise(members):
    res, st = _batch_run(members, evaluate="wave")
    assert st["converged"] == 1 and st["graph_launch"] == 1
    for (g, p), rm in zip(res, members):
        g1, p1, _ = gpu_schedule(rm, block=rm.n, evaluate="wave")
        np.testing.assert_array_equal(g, g1)
        np.testing.assert_array_equal(p, p1)


def test_batch_matches_oracle(members):
    # every member against the oracle's Dijkstra on its own graph
    res, _ = _batch_run(members)
    assert len(res) == len(members)
    for (g, p), rm in zip(res, members):
        d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
        assert_parity(rm, g, p, d)


def test_batch_host_loop_and_jump_agree(members):
    a, _ = _batch_run(members, evaluate="wave")
    b, _ = _batch_run(members, evaluate="wave", host_loop=True)
    c, _ = _batch_run(members, evaluate="jump")
    for (ga, pa), (gb, pb), (gc, pc), rm in zip(a, b, c, members):
        np.testing.assert_array_equal(ga, gb)
        np.testing.assert_array_equal(pa, pb)
        np.testing.assert_allclose(gc, ga, rtol=1e-12)
        A = O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
        mask, _ = A.unambiguous(ga)
        np.testing.assert_array_equal(pc[mask], pa[mask])


def test_autotune_restores_state_and_picks_a_candidate(members):
    cands = [dict(group=2), dict(group=4), dict(group=8, dense_fraction=0.1),
             dict(evaluate="jump")]
    with P.Batch([rm.n for rm in members], [rm.m for rm in members]) as B:
        for i, rm in enumerate(members):
            B.insert(i, rm.u, rm.v, rm.cost)
        best, idx, ms = B.autotune(cands)
        assert best in cands and ms > 0
        st = B.exploit(evaluate="wave")
        got = [(B.get_costs(i, rm.n), B.get_parents(i, rm.n)) for i, rm in enumerate(members)]
    ref, _ = _batch_run(members, evaluate="wave")
    for (g, p), (g0, p0) in zip(got, ref):
        np.testing.assert_array_equal(g, g0)
        np.testing.assert_array_equal(p, p0)


def test_autotune_search_restores_state_and_keeps_results(members):
    """The searching autotuner runs at most max_trials exploits from the same
    state, returns a complete option set no slower than where it started, and
    leaves the batch as it found it; exploiting with the options it picked gives
    the wave's trees (bit for bit when it picked the wave; when AUTO hands deep
    changes to pointer jumping, whose sums are reassociated, g within 1e-12 and
    the unambiguous parents equal)."""
    with P.Batch([rm.n for rm in members], [rm.m for rm in members]) as B:
        for i, rm in enumerate(members):
            B.insert(i, rm.u, rm.v, rm.cost)
        best, ms, trials = B.autotune_search(max_trials=12)
        assert 1 <= trials <= 12 and ms > 0
        assert best["tile"] in (0, 2) and best["group"] in (2, 4, 8)
        assert 0.1 <= best["dense_fraction"] <= 0.8 and best["wave_ctas"] in (1, 2)
        assert best["evaluate"] in ("auto", "wave")
        st = B.exploit(**best)
        got = [(B.get_costs(i, rm.n), B.get_parents(i, rm.n)) for i, rm in enumerate(members)]
    assert st["converged"] == 1
    ref, _ = _batch_run(members, evaluate="wave")
    for (g, p), (g0, p0), rm in zip(got, ref, members):
        if best["evaluate"] == "wave":
            np.testing.assert_array_equal(g, g0)
            np.testing.assert_array_equal(p, p0)
        else:
            np.testing.assert_allclose(g, g0, rtol=1e-12)
            A = O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
            mask, _ = A.unambiguous(g0)
            np.testing.assert_array_equal(p[mask], p0[mask])


def test_batch_incremental_inserts_and_errors():
    rms = [W.random_graph(900 + i, 40 + 10 * i, 120) for i in range(5)]
    with P.Batch([rm.n for rm in rms], [rm.m + 8 for rm in rms], cost_dtype=np.float64) as B:
        # first half of every member, exploit, then the rest
        for i, rm in enumerate(rms):
            h = rm.m // 2
            B.insert(i, rm.u[:h], rm.v[:h], rm.cost[:h])
        B.exploit()
        for i, rm in enumerate(rms):
            h = rm.m // 2
            B.insert(i, rm.u[h:], rm.v[h:], rm.cost[h:])
        B.exploit()
        for i, rm in enumerate(rms):
            d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost)
            np.testing.assert_array_equal(B.get_costs(i, rm.n), d)
        with pytest.raises(P.PirrtError) as e:
            B.insert(2, [0], [rms[2].n], [1.0])   # id past the member's capacity
        assert e.value.status == P.PIRRT_ERR_BAD_INPUT
        with pytest.raises(P.PirrtError) as e:
            B.insert(0, np.zeros(500, np.int32), np.ones(500, np.int32), np.ones(500))
        assert e.value.status == P.PIRRT_ERR_CAPACITY
