"""CPU oracle of the learned sampling proposal (test infrastructure only).

Plain NumPy in FP64.  With ``rounded=True`` the weights and the layer inputs
are rounded to BF16 (round to nearest even, through FP32) exactly where the
CUDA kernels round them, so the GPU forward / backward can be compared
element by element; with ``rounded=False`` it is the exact network, whose
backward pass is pinned to central finite differences of its forward pass
(tests/test_mlp_oracle.py).

Network (3 weight matrices, 256 hidden units, ReLU, sigmoid output):
    a1 = W1g grid + W1n z + b1, h1 = relu(a1)
    a2 = W2 h1 + b2,            h2 = relu(a2)
    y  = sigmoid(W3 h2 + b3)
Loss: mean over rows of |y - target|^2.  Training rule (IMLE): for each
target, the draw (of K noise vectors) whose output is nearest the target is
the one pulled towards it.  Adam on FP32 master weights.
"""
from __future__ import annotations

import numpy as np

GRID, NOISE, HIDDEN, OUT = 4096, 8, 256, 2
SHAPES = [("W1g", (HIDDEN, GRID)), ("W1n", (HIDDEN, NOISE)), ("b1", (HIDDEN,)),
          ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)), ("W3", (OUT, HIDDEN)), ("b3", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[n], dtype=np.float64).ravel() for n, _ in SHAPES])


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to BF16 (nearest even) through FP32, returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(x, rounded):
    return bf16(x) if rounded else np.asarray(x, dtype=np.float64)


def forward(params: dict, grids, scene, z, rounded: bool = True) -> dict:
    """Activations of the network for rows (scene[r], z[r])."""
    G = np.asarray(grids, dtype=np.float64)
    hg = G @ _r(params["W1g"], rounded).T
    a1 = hg[scene] + _r(z, rounded) @ _r(params["W1n"], rounded).T + params["b1"]
    h1 = _r(np.maximum(a1, 0.0), rounded)
    a2 = h1 @ _r(params["W2"], rounded).T + params["b2"]
    h2 = _r(np.maximum(a2, 0.0), rounded)
    a3 = h2 @ _r(params["W3"], rounded).T + params["b3"]
    y = 1.0 / (1.0 + np.exp(-a3))
    return dict(G=G, a1=a1, h1=h1, a2=a2, h2=h2, a3=a3, y=y)


def loss(params, grids, scene, z, target, rounded: bool = True) -> float:
    y = forward(params, grids, scene, z, rounded)["y"]
    return float(np.mean(np.sum((y - target) ** 2, axis=1)))


def backward(params: dict, grids, scene, z, target, rounded: bool = True) -> tuple[float, dict]:
    """Loss and its gradient with respect to every parameter (chain rule)."""
    f = forward(params, grids, scene, z, rounded)
    y, R = f["y"], len(scene)
    e = y - target
    L = float(np.mean(np.sum(e ** 2, axis=1)))
    da3 = (2.0 / R) * e * y * (1.0 - y)
    g = {"W3": da3.T @ f["h2"], "b3": da3.sum(0)}
    dh2 = da3 @ _r(params["W3"], rounded)
    da2 = dh2 * (f["a2"] > 0)
    g["b2"] = da2.sum(0)
    da2r = _r(da2, rounded)
    g["W2"] = da2r.T @ f["h1"]
    dh1 = da2r @ _r(params["W2"], rounded)
    da1 = dh1 * (f["a1"] > 0)
    g["b1"] = da1.sum(0)
    g["W1n"] = da1.T @ _r(z, rounded)
    D = np.zeros((f["G"].shape[0], HIDDEN))
    np.add.at(D, scene, da1)
    g["W1g"] = _r(D, rounded).T @ f["G"]
    return L, g


def imle_pick(y_draws: np.ndarray, target: np.ndarray, K: int) -> np.ndarray:
    """Index (0..K-1) of the draw nearest each target, lowest on ties."""
    d = np.sum((y_draws.reshape(len(target), K, 2) - target[:, None, :]) ** 2, axis=2)
    return np.argmin(d, axis=1)


def adam(w, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (bias-corrected); returns new (w, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    w = w - lr * (m / (1 - beta1 ** t)) / (np.sqrt(v / (1 - beta2 ** t)) + eps)
    return w, m, v
