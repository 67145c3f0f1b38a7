"""Failure detection on the device without a fault.

Every wait in the exploitation kernels is bounded and ends in a status bit
instead of a hang.  pirrt_selftest_wait runs one such wait -- the grid
barrier of the cooperative kernels, or the mbarrier wait of the staged
Improve -- where nothing will ever end it (a CTA that never arrives, a phase
nothing completes), under a short limit.  The wait must give up, the host
must see PIRRT_ERR_DEVICE_TIMEOUT, and the device must stay usable: an
exploit run right after it still matches the oracle."""
import numpy as np
import pytest

import oracle as O
import paper_2003_04920_gb300 as P
from paper_2003_04920_gb300 import workloads as W
from tests.gpu_util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()


def _exploit_matches_oracle():
    rm = W.roadmap_c1()
    with P.Graph(rm.n, rm.m, 0, np.float64) as G:
        G.insert_batch(rm.n, rm.u, rm.v, rm.cost)
        st = G.exploit()
        g, p = G.get_costs(), G.get_parents()
    assert st["converged"] == 1
    d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost)
    assert_parity(rm, g, p, d)


@pytest.mark.parametrize("which,limit", [(P.PIRRT_SELFTEST_GRID_BARRIER, 4096),
                                         (P.PIRRT_SELFTEST_MBARRIER, 2_000_000)])
def test_bounded_wait_expires_and_device_stays_usable(which, limit):
    for _ in range(2):
        assert P.pirrt_selftest_wait(which, limit) == P.PIRRT_ERR_DEVICE_TIMEOUT
    _exploit_matches_oracle()


def test_selftest_rejects_bad_arguments():
    assert P.pirrt_selftest_wait(7, 10) == P.PIRRT_ERR_INVALID_ARG
    assert P.pirrt_selftest_wait(P.PIRRT_SELFTEST_GRID_BARRIER, 0) == P.PIRRT_ERR_INVALID_ARG
    assert P.pirrt_selftest_wait(P.PIRRT_SELFTEST_GRID_BARRIER, 1 << 21) == P.PIRRT_ERR_INVALID_ARG
