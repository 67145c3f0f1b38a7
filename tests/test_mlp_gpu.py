"""The proposal's CUDA forward / backward / IMLE / Adam kernels against the
CPU oracle (oracle/mlp.py, FP64 with BF16 rounding where the kernels round).

Forward and backward are compared element by element.  The inputs of those
two tests are chosen so that every value the kernels round to BF16 in the
forward pass is exact in FP32 on both sides: weights are small multiples of
2^-10, biases of 2^-14, the noise of 2^-4, the grid is 0/1, and every partial
sum of layers 1 and 2 stays below the magnitude at which FP32 could drop one
of those bits (checked).  The forward pass then rounds identically on the GPU
and in the oracle up to the output layer, whose 256-term FP32 sum and FP32
sigmoid give the only difference in y.

In the backward pass the kernels round da2 and the per-scene sums D to BF16
from FP32 values that carry the FP32 rounding of the output layer.  Where the
oracle's FP64 value lies within that FP32 error of a BF16 rounding midpoint,
the two sides may round to neighbouring BF16 values (one BF16 ulp apart); the
test finds those ambiguous elements from the oracle's values and adds each
one's one-ulp effect, propagated linearly through the later sums, to the
tolerance of the gradient elements it reaches.  Every element must satisfy
|gpu - ref| <= RTOL * |ref| + atol, atol = ACC * (sum of |terms| of the
element's FP32 sums) + the ambiguity allowance; RTOL = 1e-3 is the relative
bar of the learned part's parity rule and ACC = 2^-13 covers FP32
accumulation over up to a few hundred terms (n * 2^-24 * sum |terms|)."""
import numpy as np
import pytest

import paper_2003_04920_gb300 as P
from oracle import mlp as M

pytestmark = pytest.mark.gpu

RTOL = 1e-3
ACC = 2.0 ** -13      # FP32 accumulation error per unit of sum |terms|
AMBIG = 2.0 ** -14    # relative FP32 error of da2 and D before their BF16 rounding


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()
    return t


def _data(torch, seed=0, S=5, R=300):
    rng = np.random.default_rng(seed)
    grids = (rng.random((S, M.GRID)) < 0.25).astype(np.float32)
    scene = rng.integers(0, S, R).astype(np.int32)
    z = rng.normal(size=(R, M.NOISE)).astype(np.float32)
    target = rng.random((R, 2)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return (grids, scene, z, target), (dev(grids), dev(scene), dev(z), dev(target))


def _dyadic(seed, S=5, R=300):
    """Weights and inputs whose forward pass is exact in FP32 (see above)."""
    rng = np.random.default_rng(seed)
    q = lambda lo, hi, shape, e: rng.integers(lo, hi + 1, shape).astype(np.float64) * 2.0 ** e
    params = {"W1g": q(-8, 8, (M.HIDDEN, M.GRID), -10), "W1n": q(-24, 24, (M.HIDDEN, M.NOISE), -10),
              "b1": q(-800, 800, (M.HIDDEN,), -14), "W2": q(-8, 8, (M.HIDDEN, M.HIDDEN), -10),
              "b2": q(-160, 160, (M.HIDDEN,), -14), "W3": q(1, 32, (M.OUT, M.HIDDEN), -10),
              "b3": np.zeros(M.OUT)}
    grids = (rng.random((S, M.GRID)) < 0.25).astype(np.float64)
    scene = rng.integers(0, S, R).astype(np.int32)
    z = q(-32, 32, (R, M.NOISE), -4)
    target = np.full((R, 2), 0.1)  # y is near 0.5: y - target keeps one sign, no cancellation
    f = M.forward(params, grids, scene, z, rounded=True)
    # exactness: every partial sum of layers 1 and 2 below 2^10 and 1 (their
    # granularities are 2^-14 and 2^-24), so FP32 adds them without rounding
    s1 = np.abs(grids) @ np.abs(params["W1g"]).T
    s1 = s1[scene] + np.abs(z) @ np.abs(params["W1n"]).T + np.abs(params["b1"])
    s2 = f["h1"] @ np.abs(params["W2"]).T + np.abs(params["b2"])
    assert s1.max() < 2.0 ** 10 and s2.max() < 1.0, (s1.max(), s2.max())
    return params, grids.astype(np.float32), scene, z.astype(np.float32), target.astype(np.float32)


def _mid_dist_ulp(x):
    """Distance of each FP64 value to the nearest BF16 rounding midpoint (as
    seen from FP32), and the BF16 ulp at the value."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.int64)
    hi = b & ~0xFFFF
    cands = [(hi | 0x8000), ((hi - 0x10000) | 0x8000), ((hi + 0x10000) | 0x8000)]
    d = np.full(f.shape, np.inf)
    for c in cands:
        c = np.clip(c, 0, 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
        d = np.minimum(d, np.abs(np.asarray(x, dtype=np.float64) - c))
    lo = hi.astype(np.uint32).view(np.float32).astype(np.float64)
    up = np.clip(hi + 0x10000, 0, 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    return d, np.abs(up - lo)


def _check(name, got, ref, atol):
    bad = np.abs(got - ref) > RTOL * np.abs(ref) + atol
    assert not bad.any(), (name, int(bad.sum()), float(np.max(np.abs(got - ref)[bad])))


def _upload(torch, prop, params, grids, scene, z, target):
    prop.set_weights(torch.from_numpy(M.pack(params).astype(np.float32)).cuda())
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dev(grids), dev(scene), dev(z), dev(target)


@pytest.mark.parametrize("kernel", ["tcgen05", "layered"])
def test_forward_matches_oracle_elementwise(torch, kernel):
    params, grids, scene, z, target = _dyadic(seed=0)
    prop = P.Proposal(8, 1024, seed=3)
    prop.set_options(kernel)
    gd, sd, zd, _ = _upload(torch, prop, params, grids, scene, z, target)
    y = prop.forward(gd, sd, zd).cpu().numpy().astype(np.float64)
    f = M.forward(params, grids, scene, z.astype(np.float64), rounded=True)
    # only the output layer differs: its FP32 sum and sigmoid
    atol = 0.25 * ACC * (f["h2"] @ np.abs(params["W3"]).T) + 2.0 ** -21
    bad = np.abs(y - f["y"]) > 1e-5 * np.abs(f["y"]) + atol
    assert not bad.any(), float(np.max(np.abs(y - f["y"])))
    prop.close()


def test_backward_matches_oracle_elementwise(torch):
    params, grids, scene, z, target = _dyadic(seed=1)
    R, S = len(scene), grids.shape[0]
    prop = P.Proposal(8, 1024, seed=4)
    gd, sd, zd, td = _upload(torch, prop, params, grids, scene, z, target)
    prop.zero_grads()
    loss = prop.backward(gd, sd, zd, td)
    got = M.unpack(prop.get_grads().cpu().numpy().astype(np.float64))
    z64, t64, G = z.astype(np.float64), target.astype(np.float64), grids.astype(np.float64)
    L, ref = M.backward(params, G, scene, z64, t64, rounded=True)
    assert abs(loss - L) <= 1e-5 * L
    f = M.forward(params, G, scene, z64, rounded=True)
    y = f["y"]
    da3 = (2.0 / R) * (y - t64) * y * (1.0 - y)
    W2b, W3b, zb = M.bf16(params["W2"]), M.bf16(params["W3"]), M.bf16(z64)
    da2 = (da3 @ W3b) * (f["a2"] > 0)
    da2r = M.bf16(da2)
    m1 = (f["a1"] > 0).astype(np.float64)
    # ambiguous BF16 roundings of da2: a one-ulp difference there, propagated
    dist, ulp = _mid_dist_ulp(da2)
    A = np.where((da2 != 0) & (dist <= AMBIG * np.abs(da2)), ulp, 0.0)
    _check("W3", got["W3"], ref["W3"], ACC * (np.abs(da3).T @ f["h2"]))
    _check("b3", got["b3"], ref["b3"], ACC * np.abs(da3).sum(0))
    _check("b2", got["b2"], ref["b2"], ACC * np.abs(da2).sum(0))
    _check("W2", got["W2"], ref["W2"], ACC * (np.abs(da2r).T @ f["h1"]) + A.T @ f["h1"])
    # bound on the GPU's dh1 error (FP32 GEMM, ambiguous da2), masked by relu(a1)
    E = (ACC * (np.abs(da2r) @ np.abs(W2b)) + A @ np.abs(W2b)) * m1
    da1 = (da2r @ W2b) * m1
    _check("b1", got["b1"], ref["b1"], E.sum(0) + ACC * np.abs(da1).sum(0))
    _check("W1n", got["W1n"], ref["W1n"], E.T @ np.abs(zb) + ACC * (np.abs(da1).T @ np.abs(zb)))
    D = np.zeros((S, M.HIDDEN))
    dD = np.zeros((S, M.HIDDEN))
    np.add.at(D, scene, da1)
    np.add.at(dD, scene, E + ACC * np.abs(da1))
    dist_d, ulp_d = _mid_dist_ulp(D)
    dDr = np.where(dist_d <= dD + AMBIG * np.abs(D), dD + ulp_d, 0.0)
    _check("W1g", got["W1g"], ref["W1g"], dDr.T @ G + ACC * (np.abs(M.bf16(D)).T @ G))
    n_amb = int((A > 0).sum())
    assert n_amb < 0.05 * A.size  # the allowance stays targeted
    prop.close()


def test_imle_select_matches_oracle(torch):
    (g, s, z, t), _ = _data(torch, seed=2, R=64)
    K = 16
    rng = np.random.default_rng(7)
    zk = rng.normal(size=(64 * K, M.NOISE)).astype(np.float32)
    draw_scene = np.repeat(s, K).astype(np.int32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    prop = P.Proposal(8, 64 * K, seed=5)
    pick = prop.imle_select(dev(g), dev(draw_scene), dev(t), K, dev(zk)).cpu().numpy()
    y = prop.forward(dev(g), dev(draw_scene), dev(zk)).cpu().numpy()
    np.testing.assert_array_equal(pick, M.imle_pick(y.astype(np.float64), t.astype(np.float64), K))
    params = M.unpack(prop.get_weights().cpu().numpy().astype(np.float64))
    yref = M.forward(params, g, draw_scene, zk.astype(np.float64), rounded=True)["y"]
    d = np.sum((yref.reshape(64, K, 2) - t[:, None, :]) ** 2, axis=2)
    srt = np.sort(d, axis=1)
    clear = (srt[:, 1] - srt[:, 0]) > 1e-3
    np.testing.assert_array_equal(pick[clear], np.argmin(d, axis=1)[clear])
    prop.close()


def test_adam_step_matches_definition(torch):
    (g, s, z, t), (gd, sd, zd, td) = _data(torch, seed=3)
    prop = P.Proposal(8, 1024, seed=6)
    w0 = prop.get_weights().cpu().numpy().astype(np.float64)
    prop.zero_grads()
    prop.backward(gd, sd, zd, td)
    grad = prop.get_grads().cpu().numpy().astype(np.float64)
    prop.adam(1e-3)
    w1 = prop.get_weights().cpu().numpy().astype(np.float64)
    want, _, _ = M.adam(w0, np.zeros_like(w0), np.zeros_like(w0), grad, 1, 1e-3)
    np.testing.assert_allclose(w1, want, rtol=1e-5, atol=1e-6)
    assert np.all(prop.get_grads().cpu().numpy() == 0)  # the step clears the gradient
    prop.close()


def test_imle_training_reduces_loss(torch):
    """Targets cluster around a scene-dependent point; IMLE training pulls the
    nearest draws onto them.  The learning rate is one at which the exact FP64
    network trained by the oracle's rule also converges on this data (at 3e-3
    it saturates the sigmoid, on the CPU as well)."""
    rng = np.random.default_rng(11)
    S, T, K = 6, 128, 8
    grids = (rng.random((S, M.GRID)) < 0.2).astype(np.float32)
    centers = rng.uniform(0.2, 0.8, (S, 2)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    prop = P.Proposal(S, T * K, seed=8)
    losses = []
    for it in range(150):
        sc = rng.integers(0, S, T).astype(np.int32)
        tg = (centers[sc] + rng.normal(0, 0.03, (T, 2))).astype(np.float32)
        nz = rng.normal(size=(T * K, M.NOISE)).astype(np.float32)
        losses.append(prop.train_step(dev(grids), dev(sc), dev(tg), K, dev(nz), 3e-4))
    assert np.mean(losses[-10:]) < 0.1 * np.mean(losses[:10])
    prop.close()


def test_train_step_is_the_composition_of_its_parts(torch):
    """train_step == forward of K draws, nearest-draw pick, backward on the
    picked noise, Adam: run both ways from the same initial weights."""
    rng = np.random.default_rng(12)
    S, T, K = 4, 96, 6
    grids = (rng.random((S, M.GRID)) < 0.3).astype(np.float32)
    sc = rng.integers(0, S, T).astype(np.int32)
    tg = rng.uniform(0.1, 0.9, (T, 2)).astype(np.float32)
    nz = rng.normal(size=(T * K, M.NOISE)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    a = P.Proposal(S, T * K, seed=21)
    b = P.Proposal(S, T * K, seed=21)
    la = a.train_step(dev(grids), dev(sc), dev(tg), K, dev(nz), 1e-3)
    pick = b.imle_select(dev(grids), dev(np.repeat(sc, K)), dev(tg), K, dev(nz)).cpu().numpy()
    zs = nz.reshape(T, K, -1)[np.arange(T), pick]
    b.zero_grads()
    lb = b.backward(dev(grids), dev(sc), dev(zs), dev(tg))
    b.adam(1e-3)
    assert abs(la - lb) <= 1e-6 * max(1.0, lb)
    np.testing.assert_allclose(a.get_weights().cpu().numpy(), b.get_weights().cpu().numpy(),
                               rtol=0, atol=1e-6)
    a.close(); b.close()


def test_sample_mixture(torch):
    rng = np.random.default_rng(13)
    S, R = 3, 500
    grids = (rng.random((S, M.GRID)) < 0.3).astype(np.float32)
    sc = rng.integers(0, S, R).astype(np.int32)
    nz = rng.normal(size=(R, M.NOISE)).astype(np.float32)
    uni = rng.random((R, 2)).astype(np.float32)
    coin = rng.random(R).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    prop = P.Proposal(S, R, seed=2)
    y = prop.forward(dev(grids), dev(sc), dev(nz)).cpu().numpy()
    for frac in (0.0, 0.5, 1.0):
        out = prop.sample(dev(grids), dev(sc), dev(nz), dev(uni), dev(coin), frac).cpu().numpy()
        learned = coin < frac
        np.testing.assert_array_equal(out[learned], y[learned])
        np.testing.assert_array_equal(out[~learned], uni[~learned])
    prop.close()


def _bf16_ulps(a, b):
    """Distance in BF16 steps between two arrays of BF16 bit patterns (int16)."""
    def key(x):
        x = x.astype(np.int32) & 0xFFFF
        return np.where(x & 0x8000, -(x & 0x7FFF), x)
    return np.abs(key(a) - key(b))


def _bf16_value(bits):
    """FP64 values of BF16 bit patterns (int16)."""
    u = (bits.astype(np.int32) & 0xFFFF).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def _bf16_step(x):
    """One BF16 step at |x| (0 at 0)."""
    ax = np.abs(x)
    e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    return np.where(ax > 0, 2.0 ** (e - 7), 0.0)


@pytest.mark.parametrize("rows", [1, 128, 152 * 128 * 2 + 77])
def test_fused_forward_matches_layered(torch, rows):
    """The fused tcgen05 kernel against the layer-by-layer path on the same
    weights (He-uniform, not dyadic), element by element.  Both round h1,
    h2 to BF16 after FP32 sums taken in different orders, so an activation
    near a BF16 rounding midpoint may land one step apart; such a step then
    moves every later sum of its row.  The bounds follow that propagation:
    h1 at most one BF16 step apart (and rarely); h2 within the h1 differences
    carried through |W2| plus FP32 accumulation (ACC per unit of sum |terms|)
    plus one BF16 step; y within a quarter (the sigmoid's slope bound) of
    the h2 differences carried through |W3| plus accumulation.  The largest
    case spans more than two passes of the persistent grid, scenes mixed
    within tiles, and a ragged last tile."""
    rng = np.random.default_rng(rows)
    S = 5
    grids = (rng.random((S, M.GRID)) < 0.25).astype(np.float32)
    scene = rng.integers(0, S, rows).astype(np.int32)
    z = rng.normal(size=(rows, M.NOISE)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    prop = P.Proposal(S, rows, seed=31)
    out = {}
    for kernel in ("layered", "tcgen05"):
        prop.set_options(kernel, keep_activations=True)
        y = prop.forward(dev(grids), dev(scene), dev(z)).cpu().numpy().astype(np.float64)
        h1, h2 = (t.cpu().numpy() for t in prop.get_activations(rows))
        out[kernel] = (y, h1, h2)
    w = M.unpack(prop.get_weights().cpu().numpy().astype(np.float64))
    W2b, W3b = np.abs(M.bf16(w["W2"])), np.abs(M.bf16(w["W3"]))
    (yl, h1l, h2l), (yf, h1f, h2f) = out["layered"], out["tcgen05"]
    d1 = _bf16_ulps(h1f, h1l)
    assert d1.max() <= 1 and (d1 > 0).mean() < 1e-3, (d1.max(), (d1 > 0).mean())
    v1l, v1f = _bf16_value(h1l), _bf16_value(h1f)
    v2l, v2f = _bf16_value(h2l), _bf16_value(h2f)
    bound2 = (np.abs(v1f - v1l) @ W2b.T + ACC * (np.abs(v1l) @ W2b.T)
              + np.maximum(_bf16_step(v2l), _bf16_step(v2f)))
    bad = np.abs(v2f - v2l) > bound2
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(v2f - v2l) - bound2)))
    assert (_bf16_ulps(h2f, h2l) > 0).mean() < 0.05
    bound3 = 0.25 * (np.abs(v2f - v2l) @ W3b.T + ACC * (np.abs(v2l) @ W3b.T)) + 2.0 ** -21
    bad = np.abs(yf - yl) > bound3
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(yf - yl) - bound3)))
    assert np.all(np.isfinite(yf)) and np.all((yf >= 0) & (yf <= 1))
    prop.close()


def test_fused_forward_rejects_scene_out_of_range(torch):
    rng = np.random.default_rng(5)
    grids = (rng.random((3, M.GRID)) < 0.25).astype(np.float32)
    scene = np.array([0, 1, 2, 7] * 40, dtype=np.int32)
    z = rng.normal(size=(len(scene), M.NOISE)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    prop = P.Proposal(3, 256, seed=1)
    with pytest.raises(P.PirrtError) as e:
        prop.forward(dev(grids), dev(scene), dev(z))
    assert e.value.status == P.PIRRT_ERR_BAD_INPUT
    # the handle stays usable
    y = prop.forward(dev(grids), dev(scene % 3), dev(z)).cpu().numpy()
    assert np.all((y >= 0) & (y <= 1))
    prop.close()
