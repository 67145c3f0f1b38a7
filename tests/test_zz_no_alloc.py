"""The allocation-free Evaluate (pirrt_evaluate_noalloc) against the oracle.

Some callers cannot allocate device memory when they need g: a planning loop
that fixes all of its memory at start-up and must not stall on the allocator
in the middle of a control cycle.  They pass their own parent array,
parent-edge costs and output buffer; the library keeps its scratch in a
static device array.  Its g must be the oracle's Evaluate of the same policy
(Alg. 2, a breadth-first walk of the policy tree, FP64) within the parity
tolerance, on two calls in a row (the calls share the static scratch).  A
policy with an id outside [0, n) is rejected before any kernel follows it, and
a cycle ends through the pointer-jumping round limit.  This file is collected
last so a failure here never hides the other GPU tests.
"""
import numpy as np
import pytest

import oracle
import paper_2003_04920_gb300 as P
from paper_2003_04920_gb300 import workloads as W
from tests.gpu_util import G_RTOL

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _parent_costs(rm, parent):
    """Cost of the edge (parent[v], v), cheapest parallel edge, FP64."""
    best = {}
    for a, b, c in zip(rm.u.tolist(), rm.v.tolist(), rm.cost.astype(np.float64).tolist()):
        key = (min(a, b), max(a, b))
        if c < best.get(key, np.inf):
            best[key] = c
    pc = np.zeros(rm.n, dtype=np.float64)
    for v, q in enumerate(parent.tolist()):
        if q >= 0:
            pc[v] = best[(min(q, v), max(q, v))]
    return pc


def _oracle_g(rm, parent):
    """The oracle's Evaluate (Alg. 2) of the policy `parent`."""
    G = oracle.OracleGraph(rm.n)
    try:
        G.insert(rm.n, rm.u, rm.v, rm.cost)
        G.set_policy(parent)
        g, _ = G.get()
    finally:
        G.close()
    return g


def test_noalloc_evaluate_matches_oracle_twice():
    torch = _torch()
    rm = W.roadmap_c2(n=60_000, block=60_000, companion=True)
    rm64 = W.Roadmap(rm.name, rm.points, rm.u, rm.v, rm.cost.astype(np.float64), rm.edge_start,
                     rm.block)
    init = W.bfs_tree_parents(rm64)
    # a second policy: the oracle's converged one (the shortest-path tree)
    O = oracle.OracleGraph(rm64.n)
    try:
        O.insert(rm64.n, rm64.u, rm64.v, rm64.cost)
        O.set_policy(init)
        O.replan()
        _, p_opt = O.get()
    finally:
        O.close()
    for parent in (init, p_opt):
        want = _oracle_g(rm64, parent)
        assert np.isfinite(want).sum() > rm64.n // 2
        pt = torch.from_numpy(np.ascontiguousarray(parent, dtype=np.int32)).cuda()
        ct = torch.from_numpy(_parent_costs(rm64, parent)).cuda()
        for _ in range(2):  # two calls in a row share the static scratch
            out = torch.full((rm64.n,), -7.0, dtype=torch.float64, device="cuda")
            rc = P.pirrt_evaluate_noalloc(pt, ct, out, root=0)
            assert rc == P.PIRRT_OK, P.pirrt_status_string(rc)
            g = out.cpu().numpy()
            np.testing.assert_array_equal(np.isinf(g), np.isinf(want))
            fin = np.isfinite(want)
            np.testing.assert_allclose(g[fin], want[fin], rtol=G_RTOL, atol=0)


def test_noalloc_rejects_oversize_and_bad_args():
    torch = _torch()
    n = (1 << 18) + 1
    pt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ct = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    assert P.pirrt_evaluate_noalloc(pt, ct, out) == P.PIRRT_ERR_CAPACITY
    small = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    assert P.pirrt_evaluate_noalloc(small, ct[:4], out[:4], root=9) == P.PIRRT_ERR_INVALID_ARG
    with pytest.raises(TypeError):
        P.pirrt_evaluate_noalloc(small, ct[:4].float(), out[:4])
    with pytest.raises(ValueError):
        P.pirrt_evaluate_noalloc(small, ct[:4], out[:3])


def test_noalloc_rejects_parent_out_of_range_then_works():
    torch = _torch()
    # vertex 3's parent is n = 4: rejected on the device before any kernel follows it
    pt = torch.tensor([-1, 0, 1, 4], dtype=torch.int32, device="cuda")
    ct = torch.tensor([0.0, 1.0, 2.0, 3.0], dtype=torch.float64, device="cuda")
    out = torch.full((4,), -7.0, dtype=torch.float64, device="cuda")
    assert P.pirrt_evaluate_noalloc(pt, ct, out, root=0) == P.PIRRT_ERR_BAD_INPUT
    g = out.cpu().numpy()
    assert g[0] == 0.0 and np.all(np.isinf(g[1:]))
    # a negative cost on a used parent edge is rejected too
    pt_ok = torch.tensor([-1, 0, 1, 2], dtype=torch.int32, device="cuda")
    bad_c = torch.tensor([0.0, 1.0, -2.0, 3.0], dtype=torch.float64, device="cuda")
    assert P.pirrt_evaluate_noalloc(pt_ok, bad_c, out, root=0) == P.PIRRT_ERR_BAD_INPUT
    # the next call with a valid path 0 - 1 - 2 - 3 succeeds (no state carried over)
    assert P.pirrt_evaluate_noalloc(pt_ok, ct, out, root=0) == P.PIRRT_OK
    np.testing.assert_array_equal(out.cpu().numpy(), [0.0, 1.0, 3.0, 6.0])


def test_noalloc_cycle_is_a_bad_tree():
    torch = _torch()
    # 1 -> 2 -> 3 -> 1 never reaches the root: the round limit ends pointer jumping
    pt = torch.tensor([-1, 3, 1, 2, 0], dtype=torch.int32, device="cuda")
    ct = torch.tensor([0.0, 1.0, 1.0, 1.0, 0.5], dtype=torch.float64, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    assert P.pirrt_evaluate_noalloc(pt, ct, out, root=0) == P.PIRRT_ERR_BAD_TREE
    # and the scratch is usable again afterwards
    pt2 = torch.tensor([-1, 0, 1, 2, 0], dtype=torch.int32, device="cuda")
    assert P.pirrt_evaluate_noalloc(pt2, ct, out, root=0) == P.PIRRT_OK
    np.testing.assert_array_equal(out.cpu().numpy(), [0.0, 1.0, 2.0, 3.0, 0.5])
