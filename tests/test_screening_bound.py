"""Host check of the FP32 screening bound used by the Improve kernel.

The kernel screens a candidate g(u) + c(u, v) with a = fl32(fl32(g) + c)
and computes fl64(g + c) exactly only when a <= min(a) * (1 + 2^-20) + 2^-125.
This is sound if |a - fl64(g + c)| <= 2^-22 * a for every g in [0, 2^100]
and every positive finite FP32 cost; numpy's float32 / float64 arithmetic is
IEEE round-to-nearest, the same as the device's.
"""
import numpy as np


def _screen(g, c):
    g32 = g.astype(np.float32)
    return (g32 + c).astype(np.float32)


def test_relative_error_bound_random():
    rng = np.random.default_rng(0)
    for scale in (1e-30, 1e-3, 1.0, 37.0, 1e6, 1e20, 1e29):
        g = rng.uniform(0, scale, 200_000)
        c = rng.uniform(1e-6, 1.0, 200_000).astype(np.float32) * np.float32(max(scale, 1e-30))
        c = np.maximum(c, np.float32(1e-38))
        a = _screen(g, c).astype(np.float64)
        v = g + c.astype(np.float64)
        assert np.all(np.abs(a - v) <= 2.0 ** -22 * a + 2.0 ** -140)


def test_keep_rule_keeps_exact_minimum():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        k = rng.integers(1, 60)
        base = rng.uniform(0.1, 50.0)
        g = base + rng.uniform(0, 1e-5, k) * base   # many near ties
        c = rng.uniform(0.01, 0.02, k).astype(np.float32)
        v = g + c.astype(np.float64)
        a = _screen(g, c)
        tau = np.float32(a.min() * np.float32(1.0 + 2.0 ** -20)) + np.float32(2.0 ** -125)
        keep = a <= tau
        best = v.min()
        assert keep[v == best].all()
