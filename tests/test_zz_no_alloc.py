"""The allocation-free Evaluate (pirrt_evaluate_noalloc) agrees with the graph
handle's Evaluate.

Callers that cannot allocate device memory when they need g -- a planning
loop that fixes its memory at start-up, or code recording into a stream
capture -- pass their own parent array, parent-edge costs and output buffer;
the library keeps its scratch in a static device array.  This file is
collected last so a failure here never hides the other GPU tests.
"""
import numpy as np
import pytest

import paper_2003_04920_gb300 as P
from paper_2003_04920_gb300 import workloads as W
from tests.gpu_util import G_RTOL

pytestmark = pytest.mark.gpu


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


def test_noalloc_evaluate_matches_graph_evaluate_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rm = W.roadmap_c2(n=60_000, block=60_000, companion=True)
    rm64 = W.Roadmap(rm.name, rm.points, rm.u, rm.v, rm.cost.astype(np.float64), rm.edge_start,
                     rm.block)
    init = W.bfs_tree_parents(rm64)
    # reference: the graph handle's Evaluate of the same policy
    with P.Graph(rm64.n, rm64.m, 0, np.float64) as G:
        G.insert_batch(rm64.n, rm64.u, rm64.v, rm64.cost)
        G.set_policy(init)
        g_ref = G.get_costs()
        # and of the converged policy
        G.exploit()
        p_opt = G.get_parents()
        g_opt = G.get_costs()
    for parent, want in ((init, g_ref), (p_opt, g_opt)):
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
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = (1 << 18) + 1
    pt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ct = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    assert P.pirrt_evaluate_noalloc(pt, ct, out) == P.PIRRT_ERR_CAPACITY
    small = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    assert P.pirrt_evaluate_noalloc(small, ct[:4], out[:4], root=9) == P.PIRRT_ERR_INVALID_ARG
