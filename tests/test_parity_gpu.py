"""Parity of the CUDA exploitation path (through the C ABI) with the CPU oracle.

Sizes here finish on the oracle in seconds yet span many CUDA blocks, several
Improve groups per row, multi-round pointer jumping and ragged tails.
"""
import numpy as np
import pytest

import oracle as O
import paper_2003_04920_gb300 as P
from paper_2003_04920_gb300 import workloads as W
from tests import golden_io
from tests.gpu_util import assert_parity, gpu_schedule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load_library()


# ------------------------------------------------------------ golden ---

@pytest.mark.parametrize("name", golden_io.names())
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_golden(name, dtype):
    gd = golden_io.load(name)
    with P.Graph(gd["n"], len(gd["u"]), gd["root"], dtype) as G:
        G.insert_batch(gd["n"], gd["u"], gd["v"], gd["c"].astype(dtype))
        if gd["goal"] is not None:
            G.set_goal(gd["goal"], gd["h"])
        if gd["init"] is not None:
            G.set_policy(gd["init"])
        st = G.exploit()
        np.testing.assert_array_equal(G.get_costs(), gd["g"])
        np.testing.assert_array_equal(G.get_parents(), gd["parent"])
        assert st["converged"] == 1
        assert st["iterations"] == gd["iterations"]


# ------------------------------------------- oracle-sized roadmap (C1) ---

def _o1(rm, init=None, block=None):
    return O.replan_schedule(rm, block=block, init_parent=init)


def test_c1_bfs_start_matches_oracle():
    rm = W.roadmap_c1()
    init = W.bfs_tree_parents(rm)
    g_ref, p_ref, st_ref = _o1(rm, init)
    g, p, st = gpu_schedule(rm, init_parent=init)
    assert_parity(rm, g, p, g_ref, p_ref)
    assert st[0]["iterations"] == st_ref[0]["iterations"]
    assert st[0]["switches"] == st_ref[0]["switches"]


@pytest.mark.parametrize("trial", [0, 1, 2])
def test_c1_unreached_start_matches_oracle(trial):
    rm = W.roadmap_c1(trial=trial)
    g_ref, p_ref, st_ref = _o1(rm)
    g, p, st = gpu_schedule(rm)
    assert_parity(rm, g, p, g_ref, p_ref)
    assert st[0]["iterations"] == st_ref[0]["iterations"]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_random_graphs(seed, dtype):
    n = [1, 2, 17, 300, 2049, 5000][seed]
    rm = W.random_graph(500 + seed, n, 3 * n, cost_dtype=dtype, connected=seed % 2 == 0)
    g_ref, p_ref, _ = _o1(rm)
    g, p, _ = gpu_schedule(rm)
    assert_parity(rm, g, p, g_ref, p_ref)


def test_high_degree_rows_span_chunks():
    """A hub joined to thousands of vertices: its row spans several
    2048-entry chunks of the tiled Improve; plus a long path hanging off it."""
    n = 6000
    rng = np.random.default_rng(11)
    hub_u = np.r_[0, np.ones(4998)].astype(np.int32)      # vertex 1 is the hub
    hub_v = np.r_[1, np.arange(2, 5000)].astype(np.int32)
    hub_c = np.r_[0.5, rng.uniform(1.0, 2.0, 4998)]
    path_u = np.arange(4999, n - 1, dtype=np.int32)
    path_v = path_u + 1
    path_c = rng.uniform(0.1, 0.2, len(path_u))
    extra_u = rng.integers(2, 5000, 3000).astype(np.int32)
    extra_v = rng.integers(5000, n, 3000).astype(np.int32)
    extra_c = rng.uniform(0.5, 3.0, 3000)
    u = np.r_[hub_u, path_u, extra_u]
    v = np.r_[hub_v, path_v, extra_v]
    c = np.r_[hub_c, path_c, extra_c]
    order = np.argsort(np.maximum(u, v), kind="stable")
    u, v, c = u[order], v[order], c[order]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    rm = W.Roadmap("hub", np.zeros((n, 1)), lo, hi, c,
                   np.searchsorted(hi, np.arange(n + 1)).astype(np.int64), n)
    for dtype in (np.float64, np.float32):
        rmd = W.Roadmap(rm.name, rm.points, rm.u, rm.v, rm.cost.astype(dtype), rm.edge_start, n)
        g_ref, p_ref, _ = _o1(rmd)
        g, p, _ = gpu_schedule(rmd)
        assert_parity(rmd, g, p, g_ref, p_ref)


# ------------------------------------ Batched-Extension schedules (C2/C3) ---

@pytest.fixture(scope="module")
def c2_small():
    return W.roadmap_c2(n=30_000, block=1_000, companion=True)


@pytest.fixture(scope="module")
def c3_small():
    return W.roadmap_c3(n=40_000, block=5_000)


def test_c2_schedule_matches_oracle_every_block(c2_small):
    rm = c2_small
    G = O.OracleGraph(rm.n)
    with P.Graph(rm.n, rm.m, 0, np.float32) as D:
        for v0, v1, e0, e1 in rm.blocks():
            G.insert(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1].astype(np.float64))
            st_ref = G.replan()
            D.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            st = D.exploit()
            g_ref, p_ref = G.get()
            g, p = D.get_costs(), D.get_parents()
            sub = W.Roadmap(rm.name, rm.points[:v1], rm.u[:e1], rm.v[:e1], rm.cost[:e1],
                            rm.edge_start[:v1 + 1], rm.block)
            assert_parity(sub, g, p, g_ref, p_ref)
            assert st["converged"] == 1
    G.close()


def test_c3_schedule_matches_dijkstra(c3_small):
    rm = c3_small
    g, p, stats = gpu_schedule(rm)
    assert all(s["converged"] for s in stats)
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    d, _ = A.dijkstra()
    assert_parity(rm, g, p, d, csr=A)


def test_c2_as_specified_small_reachable_set():
    rm = W.roadmap_c2(n=20_000, block=2_000)
    g, p, _ = gpu_schedule(rm)
    d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    assert_parity(rm, g, p, d)


# ------------------------------------------------------ invariances ---

@pytest.mark.parametrize("group,tile", [(2, 0), (8, 0), (16, 0), (32, 0), (0, 1), (2, 2),
                                        (4, 2), (8, 2), (4, 3), (8, 3), (32, 3)])
def test_improve_kernels_agree(c3_small, group, tile):
    """Every Improve kernel -- from candidate offers (tile 0, the default),
    full screened scans (2), staged scans (1) and exact scans (3) -- takes the
    same lexicographic argmin, so whole schedules agree bit for bit."""
    rm = c3_small
    g0, p0, _ = gpu_schedule(rm)
    g, p, _ = gpu_schedule(rm, group=group, tile=tile)
    np.testing.assert_array_equal(g, g0)
    np.testing.assert_array_equal(p, p0)


@pytest.mark.parametrize("evaluate", ["wave", "jump", "async", "auto"])
@pytest.mark.parametrize("which", ["c2", "c3"])
def test_offers_match_full_scans(c2_small, c3_small, evaluate, which):
    """Improve from candidate offers (a listed vertex reads its row only when
    the best offer beats its parent) reaches the policy of full scans bit for
    bit, iteration for iteration, with every Evaluate form making the offers;
    it forms far fewer candidates."""
    rm = c2_small if which == "c2" else c3_small
    g0, p0, s0 = gpu_schedule(rm, evaluate=evaluate, tile=2)
    g1, p1, s1 = gpu_schedule(rm, evaluate=evaluate, tile=0)
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(p0, p1)
    assert [s["iterations"] for s in s0] == [s["iterations"] for s in s1]
    assert [s["switches"] for s in s0] == [s["switches"] for s in s1]
    assert sum(s["relaxations"] for s in s1) < sum(s["relaxations"] for s in s0)


@pytest.mark.parametrize("frac", [1e-9, 0.05, 1.0])
def test_dense_threshold_does_not_change_results(c2_small, frac):
    rm = c2_small
    g0, p0, _ = gpu_schedule(rm)
    g, p, st = gpu_schedule(rm, dense_fraction=frac)
    np.testing.assert_array_equal(g, g0)
    np.testing.assert_array_equal(p, p0)
    if frac == 1e-9:
        assert sum(s["dense_sweeps"] for s in st) > 0


def test_block_size_does_not_change_results(c3_small):
    """Alg. 3: the final policy is independent of S (Sec. IV "Correctness")."""
    rm = c3_small
    g1, p1, _ = gpu_schedule(rm, block=rm.n)
    g2, p2, _ = gpu_schedule(rm, block=997)
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    d, _ = A.dijkstra()
    m1 = assert_parity(rm, g1, p1, d, csr=A)
    assert_parity(rm, g2, p2, d, csr=A)
    np.testing.assert_array_equal(p1[m1], p2[m1])


def test_prefetched_blocks_match_plain_inserts(c2_small):
    """Host blocks copied on the copy stream during the previous exploit (and a
    prefetch that does not match the next insertion, which is discarded) give
    the schedule of plain host inserts, bit for bit."""
    rm = c2_small
    u = np.ascontiguousarray(rm.u)
    v = np.ascontiguousarray(rm.v)
    c = np.ascontiguousarray(rm.cost)
    blocks = list(rm.blocks())
    g0, p0, _ = gpu_schedule(rm)
    with P.Graph(rm.n, rm.m, 0, np.float32) as D:
        for b, (v0, v1, e0, e1) in enumerate(blocks):
            D.insert_batch(v1 - v0, u[e0:e1], v[e0:e1], c[e0:e1])
            if b + 1 < len(blocks):
                k = b + 1 if b % 3 else min(b + 2, len(blocks) - 1)  # every third one misses
                _, _, f0, f1 = blocks[k]
                D.prefetch_batch(u[f0:f1], v[f0:f1], c[f0:f1])
            D.exploit()
        g1, p1 = D.get_costs(), D.get_parents()
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(p0, p1)


def test_device_and_host_inputs_agree(c2_small):
    rm = c2_small
    g0, p0, _ = gpu_schedule(rm)
    g1, p1, _ = gpu_schedule(rm, device_inputs=True)
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(p0, p1)


def test_runs_are_deterministic(c3_small):
    a = gpu_schedule(c3_small)
    b = gpu_schedule(c3_small)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


# ---------------------------------------------------------- insertion ---

def test_csr_equals_host_sort_of_union(c2_small):
    rm = c2_small
    with P.Graph(rm.n, rm.m, 0, np.float32) as D:
        for k, (v0, v1, e0, e1) in enumerate(rm.blocks()):
            D.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            if k in (0, 3):
                off, col, cost = D.get_adjacency()
                uu = np.r_[rm.u[:e1], rm.v[:e1]].astype(np.int64)
                vv = np.r_[rm.v[:e1], rm.u[:e1]].astype(np.int64)
                cc = np.r_[rm.cost[:e1], rm.cost[:e1]]
                o = np.lexsort((cc, vv, uu))
                want_off = np.searchsorted(uu[o], np.arange(v1 + 1))
                np.testing.assert_array_equal(off, want_off)
                rows = np.repeat(np.arange(v1), np.diff(off))
                o2 = np.lexsort((cost, col, rows))
                np.testing.assert_array_equal(col[o2], vv[o])
                np.testing.assert_array_equal(cost[o2], cc[o])


def _csr_matches(off, col, cost, uu, vv, cc, n):
    """Packed export equals a host sort of both directions of the edge list."""
    U = np.r_[uu, vv].astype(np.int64)
    V = np.r_[vv, uu].astype(np.int64)
    C = np.r_[cc, cc]
    o = np.lexsort((C, V, U))
    np.testing.assert_array_equal(off, np.searchsorted(U[o], np.arange(n + 1)))
    rows = np.repeat(np.arange(n), np.diff(off))
    o2 = np.lexsort((cost, col, rows))
    np.testing.assert_array_equal(col[o2], V[o])
    np.testing.assert_array_equal(cost[o2], C[o])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_rows_that_outgrow_their_room_move_and_repack(dtype):
    """Every row grows by two entries per block for 30 blocks: rows outgrow
    their room again and again, move to the end of the pool, and the pool
    runs out, so every row is repacked into the second pool (more than once).
    After every few blocks the packed CSR equals a host sort of the union, and
    the exploited tree equals Dijkstra on it."""
    n, blocks = 3000, 30
    rng = np.random.default_rng(5)
    w = rng.uniform(1.0, 3.0, (blocks, n))
    us, vs, cs = [], [], []
    with P.Graph(n, n * blocks, 0, dtype) as D:
        D.insert_batch(n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, dtype))
        D.set_profiling(True)
        for b in range(blocks):
            u = np.arange(n, dtype=np.int32)
            v = ((u + b + 1) % n).astype(np.int32)
            c = w[b].astype(dtype)
            D.insert_batch(0, u, v, c)
            us.append(u)
            vs.append(v)
            cs.append(c)
            if b % 7 == 3 or b == blocks - 1:
                uu, vv, cc = np.concatenate(us), np.concatenate(vs), np.concatenate(cs)
                off, col, cost = D.get_adjacency()
                _csr_matches(off, col, cost, uu, vv, cc, n)
                D.exploit()
                g, p = D.get_costs(), D.get_parents()
                rm = W.Roadmap("grow", np.zeros((n, 2)), uu, vv, cc, np.zeros(n + 1, np.int64), n)
                d, _ = O.dijkstra(n, uu, vv, cc.astype(np.float64))
                assert_parity(rm, g, p, d)
        prof = D.get_profile()
    # moves and repacks copied old entries many times over
    assert prof["insert_copied_entries"] > 2 * n * blocks


# --------------------------------------------------------- edge cases ---

def test_empty_and_vertex_only_batches():
    with P.Graph(10, 10, 0, np.float64) as D:
        D.insert_batch(0, [], [], [])
        assert D.exploit()["converged"] == 1
        D.insert_batch(1, [], [], [])          # the root alone
        D.exploit()
        np.testing.assert_array_equal(D.get_costs(), [0.0])
        D.insert_batch(3, [], [], [])          # isolated vertices
        D.exploit()
        np.testing.assert_array_equal(D.get_costs(), [0, np.inf, np.inf, np.inf])
        np.testing.assert_array_equal(D.get_parents(), [-1, -1, -1, -1])
        D.insert_batch(0, [0, 2], [2, 3], [1.5, 0.25])   # edges between old vertices
        D.exploit()
        np.testing.assert_array_equal(D.get_costs(), [0, np.inf, 1.5, 1.75])
        np.testing.assert_array_equal(D.get_parents(), [-1, -1, 0, 2])
        D.insert_batch(0, [3], [0], [1.0])     # a cheaper route to 3 (and via 3 to 2)
        D.exploit()
        np.testing.assert_array_equal(D.get_costs(), [0, np.inf, 1.25, 1.0])
        np.testing.assert_array_equal(D.get_parents(), [-1, -1, 3, 0])


def test_nonzero_root():
    gd = golden_io.load("chain_shortcut.txt")
    # relabel: root becomes vertex 6
    perm = np.array([6, 5, 4, 3, 2, 1, 0])
    u, v = perm[gd["u"]], perm[gd["v"]]
    with P.Graph(7, 7, 6, np.float64) as D:
        D.insert_batch(7, u, v, gd["c"])
        D.exploit()
        g = D.get_costs()
    d, _ = O.dijkstra(7, u, v, gd["c"], root=6)
    np.testing.assert_array_equal(g, d)


@pytest.mark.parametrize("bad", ["range", "negative", "self", "zero", "neg_cost", "nan", "inf"])
def test_bad_input_rejected_graph_unchanged(bad):
    u, v, c = [0, 1], [1, 2], [1.0, 1.0]
    if bad == "range":
        v = [1, 3]
    elif bad == "negative":
        u = [-1, 1]
    elif bad == "self":
        v = [1, 1]
    elif bad == "zero":
        c = [1.0, 0.0]
    elif bad == "neg_cost":
        c = [1.0, -2.0]
    elif bad == "nan":
        c = [np.nan, 1.0]
    elif bad == "inf":
        c = [1.0, np.inf]
    with P.Graph(8, 8, 0, np.float32) as D:
        D.insert_batch(2, [0], [1], [0.5])
        D.exploit()
        with pytest.raises(P.PirrtError) as e:
            D.insert_batch(1, u, v, c)
        assert e.value.status == P.PIRRT_ERR_BAD_INPUT
        assert D.n == 2 and D.m == 2
        D.exploit()
        np.testing.assert_array_equal(D.get_costs(), [0.0, 0.5])


def test_capacity_errors():
    with P.Graph(3, 2, 0, np.float32) as D:
        with pytest.raises(P.PirrtError) as e:
            D.insert_batch(4, [], [], [])
        assert e.value.status == P.PIRRT_ERR_CAPACITY
        with pytest.raises(P.PirrtError) as e:
            D.insert_batch(3, [0, 1, 0], [1, 2, 2], [1, 1, 1])
        assert e.value.status == P.PIRRT_ERR_CAPACITY
        D.insert_batch(3, [0, 1], [1, 2], [1, 1])
        D.exploit()
        np.testing.assert_array_equal(D.get_costs(), [0, 1, 2])


def test_set_policy_rejects_missing_edge_and_root_parent():
    gd = golden_io.load("triangle_switch.txt")
    with P.Graph(3, 3, 0, np.float64) as D:
        D.insert_batch(3, gd["u"], gd["v"], gd["c"])
        with pytest.raises(P.PirrtError) as e:
            D.set_policy([1, 0, 0])
        assert e.value.status == P.PIRRT_ERR_BAD_INPUT
        with pytest.raises(P.PirrtError) as e:
            D.set_policy([-1, 0, 5])
        assert e.value.status == P.PIRRT_ERR_BAD_INPUT
        with pytest.raises(P.PirrtError) as e:
            D.set_policy([-1, 0])
        assert e.value.status == P.PIRRT_ERR_INVALID_ARG


def test_set_policy_cycle_is_reported():
    # 1 <-> 2 point at each other: no chain reaches the root
    with P.Graph(3, 3, 0, np.float64) as D:
        D.insert_batch(3, [0, 1, 0], [1, 2, 2], [1.0, 1.0, 1.0])
        with pytest.raises(P.PirrtError) as e:
            D.set_policy([-1, 2, 1])
        assert e.value.status == P.PIRRT_ERR_BAD_TREE


def test_max_iters_then_resume():
    gd = golden_io.load("path5.txt")
    with P.Graph(5, 4, 0, np.float64) as D:
        D.insert_batch(5, gd["u"], gd["v"], gd["c"])
        st = D.exploit(max_iters=2, check=False)
        assert st["status"] == P.PIRRT_ERR_NOT_CONVERGED and st["converged"] == 0
        st = D.exploit()
        assert st["converged"] == 1
        np.testing.assert_array_equal(D.get_costs(), gd["g"])
        np.testing.assert_array_equal(D.get_parents(), gd["parent"])


def test_reset_reuses_allocations(c3_small):
    rm = c3_small
    with P.Graph(rm.n, rm.m, 0, np.float32) as D:
        g0, p0, _ = gpu_schedule(rm, graph=D)
        D.reset()
        assert D.n == 0
        g1, p1, _ = gpu_schedule(rm, graph=D)
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(p0, p1)


def test_outputs_into_device_tensors(c2_small):
    import torch
    rm = c2_small
    with P.Graph(rm.n, rm.m, 0, np.float32) as D:
        gpu_schedule(rm, graph=D)
        gt = torch.empty(rm.n, dtype=torch.float64, device="cuda")
        pt = torch.empty(rm.n, dtype=torch.int32, device="cuda")
        D.get_costs(gt)
        D.get_parents(pt)
        np.testing.assert_array_equal(gt.cpu().numpy(), D.get_costs())
        np.testing.assert_array_equal(pt.cpu().numpy(), D.get_parents())


# ------------------------------------------------- Evaluate strategies ---

@pytest.mark.parametrize("mode,levels", [("wave", 0), ("jump", 0), ("async", 0), ("auto", 0),
                                         ("auto", 1), ("auto", 3)])
def test_evaluate_strategies_agree(c2_small, mode, levels):
    """Top-down waves, pointer jumping, the barrier-free walk and a walk
    handing over to pointer jumping past depth `levels` reach the same policy
    (Alg. 2 Evaluate)."""
    rm = c2_small
    g_ref, p_ref, _ = O.replan_schedule(rm)
    g, p, st = gpu_schedule(rm, evaluate=mode, wave_levels=levels)
    assert_parity(rm, g, p, g_ref, p_ref)
    if mode == "jump" or (mode == "auto" and levels == 1):
        assert sum(s["jump_evaluates"] for s in st) > 0
    if mode in ("wave", "async"):
        assert sum(s["jump_evaluates"] for s in st) == 0


@pytest.mark.parametrize("mode", ["wave", "async"])
def test_wave_sums_match_oracle_bitwise(mode):
    """The top-down Evaluates add one edge cost per level from the root, the
    order of Alg. 2's breadth-first Evaluate, so with the same tree g agrees
    with the oracle to the last bit."""
    rm = W.roadmap_c1(trial=4)
    g_ref, p_ref, _ = O.replan_schedule(rm)
    g, p, _ = gpu_schedule(rm, evaluate=mode)
    same = p == p_ref
    assert same.mean() > 0.99
    # vertices whose whole root path agrees
    ok = np.zeros(rm.n, dtype=bool)
    ok[0] = True
    for x in np.argsort(g_ref):
        if x != 0 and p_ref[x] >= 0:
            ok[x] = same[x] and ok[p_ref[x]]
    np.testing.assert_array_equal(g[ok], g_ref[ok])
    assert ok.mean() > 0.9


def test_c3_wave_and_jump_identical_parents(c3_small):
    rm = c3_small
    gw, pw, _ = gpu_schedule(rm, evaluate="wave")
    gj, pj, _ = gpu_schedule(rm, evaluate="jump")
    np.testing.assert_allclose(gw, gj, rtol=1e-12)
    d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    mask, _ = A.unambiguous(d)
    np.testing.assert_array_equal(pw[mask], pj[mask])


@pytest.mark.parametrize("tail", [-1, 1, 512, 1_000_000])
@pytest.mark.parametrize("which", ["c2", "c3"])
def test_wave_tail_walk_is_bitwise_neutral(c2_small, c3_small, which, tail):
    """Levels walked by one CTA without grid barriers (none, single-vertex
    levels, levels up to a tile, every level) give the same schedule bit for
    bit."""
    rm = c2_small if which == "c2" else c3_small
    g0, p0, s0 = gpu_schedule(rm, evaluate="wave", wave_tail=-1)
    g1, p1, s1 = gpu_schedule(rm, evaluate="wave", wave_tail=tail)
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(p0, p1)
    assert [s["iterations"] for s in s0] == [s["iterations"] for s in s1]
    assert [s["dense_sweeps"] for s in s0] == [s["dense_sweeps"] for s in s1]


@pytest.mark.parametrize("ctas", [1, 2])
def test_wave_grid_size_is_bitwise_neutral(c3_small, ctas):
    """One or two wave CTAs per SM: the same schedule bit for bit."""
    rm = c3_small
    g0, p0, s0 = gpu_schedule(rm)
    g1, p1, s1 = gpu_schedule(rm, wave_ctas=ctas)
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(p0, p1)
    assert [s["iterations"] for s in s0] == [s["iterations"] for s in s1]


@pytest.mark.parametrize("which", ["c2", "c3"])
def test_async_walk_equals_wave_bitwise(c2_small, c3_small, which):
    """The barrier-free walk and the level-synchronous wave compute the same
    sums, so whole schedules agree bit for bit, iteration for iteration.  (The
    wave counts a vertex recomputed on two levels twice when it decides on a
    dense next sweep, the walk once, so their Improve sweeps may differ in
    shape, not in result.)"""
    rm = c2_small if which == "c2" else c3_small
    gw, pw, sw = gpu_schedule(rm, evaluate="wave")
    ga, pa, sa = gpu_schedule(rm, evaluate="async")
    np.testing.assert_array_equal(gw, ga)
    np.testing.assert_array_equal(pw, pa)
    assert [s["iterations"] for s in sw] == [s["iterations"] for s in sa]
    assert [s["switches"] for s in sw] == [s["switches"] for s in sa]


@pytest.mark.parametrize("mode,n", [("async", 30_000), ("wave", 2_000), ("auto", 30_000)])
def test_long_chain_with_nested_switches(mode, n):
    """A path whose vertices first hang off the root by long direct edges
    (cost 10^6 + 10k), so that the second Improve re-parents every path vertex
    at once onto its predecessor: one Evaluate then walks an n-level tree in
    which every vertex switched.  g is the exact prefix sum (one FP64 addition
    per level, as Alg. 2's Evaluate).  The level-synchronous wave recomputes
    every stale vertex on every level, so it runs a shorter path; AUTO hands
    the deep walk over to pointer jumping.  A hub joined to the root and to
    every 7th vertex then re-parents thousands of nested vertices again."""
    rng = np.random.default_rng(11)
    c = rng.uniform(1.0, 2.0, n - 1)
    ks = np.arange(2, n, dtype=np.int32)
    u1 = np.r_[np.arange(n - 1, dtype=np.int32), np.zeros(len(ks), np.int32)].astype(np.int32)
    v1 = np.r_[np.arange(1, n, dtype=np.int32), ks].astype(np.int32)
    c1 = np.r_[c, 1e6 + 10.0 * ks]
    hub = n
    far = np.arange(7, n, 7, dtype=np.int32)
    u2 = np.r_[np.int32(0), far].astype(np.int32)
    v2 = np.full(len(u2), hub, dtype=np.int32)
    c2 = np.r_[0.5, rng.uniform(0.5, 1.0, len(far))]
    with P.Graph(n + 1, len(u1) + len(u2), 0, np.float64) as D:
        D.insert_batch(n, u1, v1, c1)
        st1 = D.exploit(evaluate=mode)
        g1 = D.get_costs()
        assert st1["switches"] >= 2 * (n - 2)
        if mode == "auto":  # the walk passes its depth cap; pointer jumping finishes
            assert st1["jump_evaluates"] > 0
            np.testing.assert_allclose(g1[1:], np.cumsum(c), rtol=1e-12)
        else:
            assert st1["jump_evaluates"] == 0
            np.testing.assert_array_equal(g1[1:], np.cumsum(c))
        D.insert_batch(1, u2, v2, c2)
        st2 = D.exploit(evaluate=mode)
        g, p = D.get_costs(), D.get_parents()
    assert st2["switches"] > 100
    uu, vv, cc = np.r_[u1, u2], np.r_[v1, v2], np.r_[c1, c2]
    rm = W.Roadmap("chain", np.zeros((n + 1, 2)), uu, vv, cc, np.zeros(n + 2, np.int64), n + 1)
    d, _ = O.dijkstra(n + 1, uu, vv, cc)
    assert_parity(rm, g, p, d)


@pytest.mark.parametrize("scale", [1e-39, 1e29, 1e36])
def test_extreme_cost_scales(scale):
    """Costs in the FP32 subnormal range, and costs whose path sums exceed
    2^100 (the Improve kernel's FP32 screen then defers to exact FP64)."""
    rm = W.random_graph(700, 3000, 12000, cost_dtype=np.float64, cmin=1.0, cmax=4.0)
    c = (rm.cost * scale).astype(np.float32)
    rmd = W.Roadmap(rm.name, rm.points, rm.u, rm.v, c, rm.edge_start, rm.n)
    g_ref, p_ref, _ = _o1(rmd)
    g, p, _ = gpu_schedule(rmd)
    assert_parity(rmd, g, p, g_ref, p_ref)


@pytest.mark.parametrize("evaluate", ["auto", "wave", "jump", "async"])
def test_graph_launch_matches_host_loop(c2_small, evaluate):
    """The Replan loop captured as one CUDA graph (WHILE node) and the host-driven
    loop run the same kernels and reach the same policy, bit for bit."""
    rm = c2_small
    g0, p0, st0 = gpu_schedule(rm, evaluate=evaluate, host_loop=True)
    g1, p1, st1 = gpu_schedule(rm, evaluate=evaluate)
    assert all(s["graph_launch"] == 0 for s in st0)
    assert all(s["graph_launch"] == 1 for s in st1)
    assert [s["iterations"] for s in st0] == [s["iterations"] for s in st1]
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(p0, p1)


def test_graph_launch_max_iters_then_resume():
    gd = golden_io.load("path5.txt")
    with P.Graph(5, 4, 0, np.float64) as D:
        D.insert_batch(5, gd["u"], gd["v"], gd["c"])
        st = D.exploit(max_iters=2, check=False)
        assert st["graph_launch"] == 1 and st["iterations"] == 2
        assert st["status"] == P.PIRRT_ERR_NOT_CONVERGED
        st = D.exploit()
        assert st["converged"] == 1
        np.testing.assert_array_equal(D.get_costs(), gd["g"])

