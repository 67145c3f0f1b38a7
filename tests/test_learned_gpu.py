"""The learned-proposal workflow end to end at a small scale: planner
solutions on the GPU (one pirrt_batch per chunk of scenes) against the
oracle's Dijkstra, the near-path targets, IMLE training and the paired
mixed-vs-uniform comparison."""
import math

import numpy as np
import pytest

from paper_2003_04920_gb300 import learned as L
from paper_2003_04920_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_planner_solutions_match_dijkstra(torch):
    import oracle
    rms = L.roadmaps([(s, ("uniform", 3000, 0)) for s in range(6)])
    sols = L.solve(rms, max_entries=40_000)  # several chunks
    assert len(sols) == 6
    for rm, (g, p) in zip(rms, sols):
        d, _ = oracle.dijkstra(rm[3], rm[0], rm[1], rm[2].astype(np.float64))
        fin = np.isfinite(d)
        np.testing.assert_array_equal(np.isfinite(g), fin)
        np.testing.assert_allclose(g[fin], d[fin], rtol=1e-5)
        if fin[L.GOAL]:
            path = L.path_to_root(p, L.GOAL)
            assert path[-1] == 0
            # the path's edge lengths add up to g(x_goal)
            pts = rm[4]
            length = np.sum(np.linalg.norm(np.diff(pts[path], axis=0), axis=1))
            assert math.isclose(length, g[L.GOAL], rel_tol=1e-5)


def test_training_set_targets_lie_in_the_band(torch):
    grids, targets, costs, kept = L.training_set(range(6), 3000, band=0.02, chunk=4)
    assert grids.shape == (len(kept), 4096) and len(targets) == len(kept) > 0
    for s, t in zip(kept, targets):
        assert len(t) > 0
        assert not W.c5_scene(s).inside(t.astype(np.float64)).any()
    # costs are at least the straight-line distance
    assert np.all(costs >= np.linalg.norm(L.X_GOAL - L.X_INIT) - 1e-9)


def test_train_and_compare_small(torch):
    from paper_2003_04920_gb300 import Proposal
    grids, targets, costs, kept = L.training_set(range(8), 3000, chunk=8)
    prop = Proposal(4, 4 * 16 * 8, seed=1)
    losses, secs = L.train(prop, grids, targets, 60, scenes_per_step=4, targets_per_scene=16, K=8,
                           lr=3e-4)
    assert np.all(np.isfinite(losses)) and losses[-10:].mean() < losses[:10].mean()
    ev = Proposal(1, 4096, seed=1)
    ev.set_weights(prop.get_weights())
    pts = L.learned_points(ev, 123, 2000, 0.5, chunk=4096)
    assert pts.shape == (2000, 2) and not W.c5_scene(123).inside(pts).any()
    res = L.compare(ev, [100, 101, 102], [2000], pool_=None)
    cu, cl = res[2000]
    assert cu.shape == cl.shape == (3,)
    summ = L.summarize(res)[2000]
    assert summ["scenes"] == 3
    prop.close(); ev.close()


def test_device_pipeline_comparison_reports_signs(torch, record_property):
    """The device-resident workflow at a small scale: GPU-built roadmaps,
    near-path targets, IMLE training, reference paths, the four arms
    (uniform, learned mixture, ideal mixture, fixed corridor) paired by
    scene, the spread check, and the sign of each arm's paired difference.
    A proposal that puts half of the samples near the optimal path (the
    ideal arm) must make the start-goal path cheaper than uniform sampling;
    the learned arm's sign is reported, not asserted."""
    from paper_2003_04920_gb300 import Proposal
    grids, targets, costs, kept = L.dev_training_set(range(12), 6000, band=0.02, chunk=6)
    assert len(kept) > 0 and grids.shape == (len(kept), 4096)
    for s, t in zip(kept, targets):
        assert t.shape[1] == 2 and t.shape[0] > 0
        assert not W.c5_scene(s).inside(t.cpu().numpy().astype(np.float64)).any()
    assert np.all(costs >= np.linalg.norm(L.X_GOAL - L.X_INIT) - 1e-9)
    prop = Proposal(4, 4 * 32 * 8, seed=1)
    losses, _ = L.train(prop, grids, targets, 200, scenes_per_step=4, targets_per_scene=32, K=8)
    assert np.all(np.isfinite(losses)) and losses[-20:].mean() < losses[:20].mean()
    ev = Proposal(1, 1 << 16, seed=1)
    ev.set_weights(prop.get_weights())
    seeds = list(range(2000, 2016))
    refs = L.reference_paths(seeds, 40_000)
    res = L.dev_compare(ev, seeds, [8000], refs, chunk=8)
    table = L.paired_table(res)["8000"]
    for arm in ("learned", "ideal", "corridor"):
        assert table[arm]["both_solved"] > 0
        assert table[arm]["sign"] in ("cheaper", "costlier", "no difference")
        record_property(f"{arm}_sign", table[arm]["sign"])
        record_property(f"{arm}_paired_diff", table[arm]["paired_diff"])
    assert table["ideal"]["paired_diff"] < 0, table["ideal"]
    sp = L.spread(ev, seeds, refs, m=4000)
    assert 0.0 <= sp["within_band"] <= 1.0 and 0.0 <= sp["path_coverage"] <= 1.0
    print({arm: (table[arm]["sign"], table[arm]["paired_diff"]) for arm in
           ("learned", "ideal", "corridor")}, sp)
    prop.close(); ev.close()
