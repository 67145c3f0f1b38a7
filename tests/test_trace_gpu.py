"""The wave trace (pirrt_profile's level_*, share_*, local_*, wave_* fields)
agrees with the exploit statistics it describes, in the host-driven profiled
loop and in the trace-only mode that keeps every exploit one graph launch, and
turning it on changes no result."""
import numpy as np
import pytest

import paper_2003_04920_gb300 as P
from paper_2003_04920_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()


@pytest.fixture(scope="module")
def c3_small():
    return W.roadmap_c3(n=40_000, block=5_000)


def _schedule(rm, mode):
    with P.Graph(rm.n, rm.m, 0, np.float32) as G:
        G.set_profiling(mode)
        stats = []
        for v0, v1, e0, e1 in rm.blocks():
            G.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            stats.append(G.exploit(evaluate="wave"))
        prof = G.get_profile()
        g, p = G.get_costs(), G.get_parents()
    return g, p, stats, prof


def test_level_trace_matches_statistics(c3_small):
    g0, p0, s0, _ = _schedule(c3_small, False)
    for mode in (True, 2):
        g, p, st, prof = _schedule(c3_small, mode)
        np.testing.assert_array_equal(g, g0)
        np.testing.assert_array_equal(p, p0)
        steps = sum(s["wave_levels"] for s in st)
        assert steps > 0
        # one bucket entry per grid step; the buckets hold the step sizes
        assert sum(prof["level_count"]) == steps
        for b, (n, items) in enumerate(zip(prof["level_count"], prof["level_vertices"])):
            if n and 0 < b < 23:
                assert n * (1 << (b - 1)) <= items <= n * ((1 << b) - 1)
        # every wave launch is traced once, and CTA 0's share tiles cover at
        # most the vertices of the steps
        launches = sum(s["iterations"] for s in st)
        assert prof["wave_calls"] == launches > 0
        assert sum(prof["share_vertices"]) <= sum(prof["level_vertices"])
        assert all(c >= 0 for c in prof["level_cycles"])
        if mode == 2:
            # graph mode: spans of the launches, gaps between them within exploits
            assert prof["wave_spans"] == prof["wave_calls"]
            assert prof["wave_span_ns"] > 0
            # the first launch of each exploit has no predecessor to measure from
            assert prof["wave_gaps"] == prof["wave_spans"] - len(st)
            assert all(s["graph_launch"] == 1 for s in st)
        else:
            assert all(s["graph_launch"] == 0 for s in st)
