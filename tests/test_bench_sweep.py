"""The block-size sweep of bench.py (Sec. VI) on the CPU: its query keeps
x_init and x_goal as vertices 0 and 1 (Alg. 1), and its oracle leg reaches
the shortest-path cost of x_goal for every block size S."""
import importlib.util
import os

import numpy as np

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sweep_query_and_oracle_leg():
    b = _bench()
    rm, goal, h = b.sweep_case(2000, 1, True)
    assert goal == 1
    np.testing.assert_allclose(rm.points[0], (0.05, 0.05))
    np.testing.assert_allclose(rm.points[1], (0.95, 0.95))
    np.testing.assert_allclose(h, 0.99 * np.linalg.norm(rm.points - rm.points[1], axis=1),
                               rtol=1e-6)
    d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    assert np.isfinite(d[1])
    out = b.sweep_oracle(rm, goal, h, [1, 50, rm.n], seconds=60.0)
    for S, r in out.items():
        assert r["complete"] and r["blocks"] == -(-rm.n // S)
        np.testing.assert_allclose(r["g_goal"], d[1], rtol=1e-12, atol=0)
    # fewer, larger blocks: fewer Replan rounds in all
    assert out[1]["iterations"] > out[50]["iterations"] > out[rm.n]["iterations"]
    rm0, goal0, h0 = b.sweep_case(2000, 1, False)
    assert goal0 is None and h0 is None
    np.testing.assert_array_equal(rm0.u, rm.u)
