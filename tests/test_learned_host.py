"""Host-side pieces of the learned-proposal workflow (no GPU): scenes, grids,
path extraction and the near-path band that selects training targets."""
import numpy as np

from paper_2003_04920_gb300 import learned as L
from paper_2003_04920_gb300 import workloads as W


def test_scene_keeps_start_and_goal_free():
    for s in range(20):
        sc = W.c5_scene(s)
        assert len(sc.radii) == 200
        assert np.all((sc.radii >= 0.01) & (sc.radii <= 0.04))
        assert not sc.inside(np.array([W.C5_X_INIT, W.C5_X_GOAL])).any()


def test_occupancy_grid_layout():
    # one obstacle in the lower-right corner: only cells with large x, small y
    sc = W.Scene(2, 0.0, 1.0, np.array([[0.9, 0.1]]), np.array([0.05]))
    g = W.occupancy_grid(sc, 64).reshape(64, 64)  # [y, x]
    ys, xs = np.nonzero(g)
    assert len(ys) > 0
    assert xs.min() > 48 and ys.max() < 16
    # cell (iy, ix) is occupied exactly when its centre lies within the circle
    cx, cy = (xs + 0.5) / 64, (ys + 0.5) / 64
    assert np.all((cx - 0.9) ** 2 + (cy - 0.1) ** 2 < 0.05 ** 2)


def test_path_to_root():
    parent = np.array([-1, 3, 0, 2, -1], dtype=np.int32)
    np.testing.assert_array_equal(L.path_to_root(parent, 1), [1, 3, 2, 0])
    np.testing.assert_array_equal(L.path_to_root(parent, 4), [4])


def test_near_path_band():
    path = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0]])
    pts = np.array([[0.5, 0.019], [0.5, 0.021], [1.019, 0.5], [1.021, 0.5],
                    [-0.01, 0.0], [-0.03, 0.0], [1.014, -0.014], [1.015, -0.015]])
    np.testing.assert_array_equal(L.near_path(pts, path, 0.02),
                                  [True, False, True, False, True, False, True, False])


def test_uniform_points_are_free_and_seeded():
    a = L.uniform_points(7, 500)
    b = L.uniform_points(7, 500)
    np.testing.assert_array_equal(a, b)
    assert a.shape == (500, 2)
    np.testing.assert_array_equal(a[0], W.C5_X_INIT)
    np.testing.assert_array_equal(a[1], W.C5_X_GOAL)
    assert not W.c5_scene(7).inside(a).any()


def test_roadmap_from_points_edges_are_free():
    pts = L.uniform_points(3, 1500)
    rm = W.roadmap_from_points("t", pts, W.c5_scene(3))
    assert rm.n == 1500 and rm.m > 0
    assert np.all(rm.u < rm.v)
    # every kept edge misses every circle (dense sampling along the segment)
    t = np.linspace(0, 1, 33)[:, None, None]
    seg = pts[rm.u][None] * (1 - t) + pts[rm.v][None] * t
    sc = W.c5_scene(3)
    assert not sc.inside(seg.reshape(-1, 2)).any()
