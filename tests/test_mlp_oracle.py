"""Pins for the MLP oracle: its backward pass against central finite
differences of its own forward pass in exact FP64, its BF16 rounding against
hand-worked values, and the IMLE pick / Adam step against their definitions."""
import numpy as np
import pytest

from oracle import mlp as M


def _instance(seed=0, S=3, R=11):
    rng = np.random.default_rng(seed)
    params = {}
    for name, shape in M.SHAPES:
        scale = 0.05 if name.startswith("W1") else 0.2
        params[name] = rng.normal(0, scale, shape)
    grids = (rng.random((S, M.GRID)) < 0.3).astype(np.float64)
    scene = rng.integers(0, S, R)
    z = rng.normal(size=(R, M.NOISE))
    target = rng.random((R, 2))
    return params, grids, scene, z, target


def test_bf16_rounding_hand_values():
    x = np.array([1.0, 1 + 2 ** -7, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -2.5, 0.0, 3.0e38, 1e-40])
    want = np.array([1.0, 1 + 2 ** -7, 1.0, 1 + 2 ** -7, -2.5, 0.0, None, None], dtype=object)
    got = M.bf16(x)
    for g, w in zip(got[:6], want[:6]):
        assert g == w
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: nearest even keeps 1
    assert M.bf16(np.array([1 + 2 ** -8]))[0] == 1.0
    assert M.bf16(np.array([1 + 2 ** -8 + 2 ** -12]))[0] == 1 + 2 ** -7


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    params, grids, scene, z, target = _instance(seed)
    _, g = M.backward(params, grids, scene, z, target, rounded=False)
    rng = np.random.default_rng(100 + seed)
    h = 1e-6
    for name, shape in M.SHAPES:
        flat = params[name].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            keep = flat[idx]
            flat[idx] = keep + h
            lp = M.loss(params, grids, scene, z, target, rounded=False)
            flat[idx] = keep - h
            lm = M.loss(params, grids, scene, z, target, rounded=False)
            flat[idx] = keep
            fd = (lp - lm) / (2 * h)
            an = g[name].ravel()[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, an)


def test_rounded_network_stays_close_to_exact():
    params, grids, scene, z, target = _instance(2)
    y0 = M.forward(params, grids, scene, z, rounded=False)["y"]
    y1 = M.forward(params, grids, scene, z, rounded=True)["y"]
    assert np.max(np.abs(y0 - y1)) < 2e-2


def test_imle_pick_and_adam_definitions():
    y = np.array([[0.1, 0.1], [0.5, 0.5], [0.5, 0.5], [0.9, 0.2]])
    t = np.array([[0.45, 0.5], [0.9, 0.25]])
    np.testing.assert_array_equal(M.imle_pick(y, t, 2), [1, 1])
    w, m, v = M.adam(np.array([1.0]), np.zeros(1), np.zeros(1), np.array([0.5]), 1, 0.1)
    # first step of bias-corrected Adam moves by lr * sign(grad)
    assert abs(w[0] - (1.0 - 0.1)) < 1e-7


def test_pack_roundtrip_and_count():
    params, *_ = _instance(3)
    flat = M.pack(params)
    assert flat.size == M.N_PARAMS == 1_117_186
    back = M.unpack(flat)
    for name, _ in M.SHAPES:
        np.testing.assert_array_equal(back[name], params[name])
