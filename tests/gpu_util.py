"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare with the parity rule:
parents bit-exact wherever the best and second-best candidates differ by more
than 1e-6 relative, g within 1e-5 relative of FP64."""
import numpy as np

import oracle as O
import paper_2003_04920_gb300 as P

G_RTOL = 1e-5       # g vs FP64 oracle
AMBIG_REL = 1e-6    # parents compared where the runner-up is this much worse


def gpu_schedule(rm, block=None, init_parent=None, device_inputs=False, graph=None, **kw):
    """Run the Batched-Extension schedule on the GPU; returns (g, p, stats)."""
    import torch
    own = graph is None
    if own:
        graph = P.Graph(rm.n, rm.m, 0, rm.cost.dtype)
    stats = []
    try:
        dev = None
        if device_inputs:
            dev = (torch.from_numpy(rm.u).cuda(), torch.from_numpy(rm.v).cuda(),
                   torch.from_numpy(rm.cost).cuda())
        for v0, v1, e0, e1 in rm.blocks(block):
            if dev is not None:
                graph.insert_batch(v1 - v0, dev[0][e0:e1], dev[1][e0:e1], dev[2][e0:e1])
            else:
                graph.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            if init_parent is not None:
                graph.set_policy(init_parent[:v1])
            stats.append(graph.exploit(**kw))
        g, p = graph.get_costs(), graph.get_parents()
    finally:
        if own:
            graph.close()
    return g, p, stats


def assert_parity(rm, g, p, g_ref, p_ref=None, csr=None, rtol=G_RTOL):
    """g vs reference within rtol; parents equal on the unambiguous mask
    (computed from the reference g); the tree and Bellman checks pass."""
    A = csr or O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    np.testing.assert_array_equal(np.isinf(g), np.isinf(g_ref))
    fin = np.isfinite(g_ref)
    np.testing.assert_allclose(g[fin], g_ref[fin], rtol=rtol, atol=0)
    mask, arg = A.unambiguous(g_ref, AMBIG_REL)
    np.testing.assert_array_equal(p[mask], arg[mask])
    if p_ref is not None:
        np.testing.assert_array_equal(p[mask], p_ref[mask])
    bad, first = A.check_tree(p)
    assert bad == 0, f"parent tree broken at {first}"
    bad, worst = A.check_bellman(g, 1e-9)
    assert bad == 0, f"Bellman inequality violated at {worst}"
    bad, first = A.check_consistency(p, g, 1e-9)
    assert bad == 0, f"g inconsistent with parents at {first}"
    np.testing.assert_array_equal(p == -1, ~fin | (np.arange(rm.n) == 0))
    return mask
