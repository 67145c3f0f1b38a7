"""Checkpoint and resume of a graph (pirrt_graph_save / pirrt_graph_load).

Not in the paper: it keeps a roadmap and its converged policy across
processes.  A graph saved in the middle of a Batched-Extension schedule
(Alg. 3) and loaded into a fresh handle carries on to exactly the tree the
uninterrupted schedule reaches (and both equal Dijkstra on the final graph);
bad files and mismatched graphs are rejected with the graph left usable.
"""
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


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_save_load_resume_equals_uninterrupted(tmp_path, dtype):
    rm = W.roadmap_c3(n=30_000, block=3_000)
    rm = W.Roadmap(rm.name, rm.points, rm.u, rm.v, rm.cost.astype(dtype), rm.edge_start, rm.block)
    blocks = list(rm.blocks())
    path = str(tmp_path / "graph.ckpt")
    with P.Graph(rm.n, rm.m, 0, dtype) as A:
        for v0, v1, e0, e1 in blocks[:5]:
            A.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            A.exploit(evaluate="wave")
        A.save(path)
        g_mid, p_mid = A.get_costs(), A.get_parents()
        off_mid = A.get_adjacency()
        for v0, v1, e0, e1 in blocks[5:]:
            A.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            A.exploit(evaluate="wave")
        g_a, p_a = A.get_costs(), A.get_parents()
    with P.Graph(rm.n, rm.m, 0, dtype) as B:
        B.load(path)
        assert B.n == blocks[4][1] and B.m == 2 * blocks[4][3]
        np.testing.assert_array_equal(B.get_costs(), g_mid)
        np.testing.assert_array_equal(B.get_parents(), p_mid)
        for x, y in zip(B.get_adjacency(), off_mid):
            np.testing.assert_array_equal(x, y)
        st = B.exploit(evaluate="wave")  # a stable policy: one full sweep, no switch
        assert st["converged"] == 1 and st["switches"] == 0 and st["iterations"] == 1
        for v0, v1, e0, e1 in blocks[5:]:
            B.insert_batch(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1])
            B.exploit(evaluate="wave")
        g_b, p_b = B.get_costs(), B.get_parents()
    np.testing.assert_array_equal(g_a, g_b)
    np.testing.assert_array_equal(p_a, p_b)
    d, _ = O.dijkstra(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    assert_parity(rm, g_b, p_b, d)


def test_load_rejects_bad_files_and_mismatches(tmp_path):
    rm = W.roadmap_c1()
    path = str(tmp_path / "c1.ckpt")
    with P.Graph(rm.n, rm.m, 0, np.float64) as A:
        A.insert_batch(rm.n, rm.u, rm.v, rm.cost)
        A.exploit()
        A.save(path)
        g = A.get_costs()
    junk = tmp_path / "junk.ckpt"
    junk.write_bytes(b"not a checkpoint at all")
    short = tmp_path / "short.ckpt"
    short.write_bytes(open(path, "rb").read()[:1000])
    with P.Graph(rm.n, rm.m, 0, np.float64) as B:
        B.insert_batch(rm.n, rm.u, rm.v, rm.cost)
        for bad, status in ((str(junk), P.PIRRT_ERR_BAD_INPUT),
                            (str(short), P.PIRRT_ERR_BAD_INPUT),
                            (str(tmp_path / "missing.ckpt"), P.PIRRT_ERR_INVALID_ARG)):
            with pytest.raises(P.PirrtError) as e:
                B.load(bad)
            assert e.value.status == status
        # the graph is untouched and still works
        assert B.exploit()["converged"] == 1
        np.testing.assert_array_equal(B.get_costs(), g)
    with P.Graph(rm.n, rm.m, 0, np.float32) as C:  # other cost type
        with pytest.raises(P.PirrtError) as e:
            C.load(path)
        assert e.value.status == P.PIRRT_ERR_INVALID_ARG
    with P.Graph(rm.n // 2, rm.m, 0, np.float64) as D:  # too small
        with pytest.raises(P.PirrtError) as e:
            D.load(path)
        assert e.value.status == P.PIRRT_ERR_CAPACITY


def _corrupt(src, dst, field, value):
    """Copy checkpoint `src` to `dst` with one value replaced: the first
    adjacency entry's column ("col"), or a non-root vertex's parent ("parent")."""
    import struct
    raw = bytearray(open(src, "rb").read())
    magic, dtype, root, n, m = struct.unpack_from("<8siiqq", raw, 0)
    hdr = 32
    ent = 8 if dtype == P.PIRRT_COST_F32 else 16
    if field == "col":
        struct.pack_into("<i", raw, hdr + 8 * (n + 1), value)
    else:
        v = 1 if root != 1 else 2
        off_p = hdr + 8 * (n + 1) + ent * m + 8 * n
        struct.pack_into("<i", raw, off_p + 4 * v, value)
    open(dst, "wb").write(bytes(raw))
    return n


def test_load_rejects_out_of_range_ids_before_any_copy(tmp_path):
    """A column id equal to n, or the root marker on a vertex other than the
    root, is caught on the host before anything reaches the device; the graph
    keeps its contents and still exploits."""
    rm = W.roadmap_c1()
    path = str(tmp_path / "c1.ckpt")
    with P.Graph(rm.n, rm.m, 0, np.float64) as A:
        A.insert_batch(rm.n, rm.u, rm.v, rm.cost)
        A.exploit()
        A.save(path)
        g = A.get_costs()
    n = _corrupt(path, str(tmp_path / "col.ckpt"), "col", rm.n)
    assert n == rm.n
    _corrupt(path, str(tmp_path / "mark.ckpt"), "parent", -2)
    _corrupt(path, str(tmp_path / "par.ckpt"), "parent", rm.n + 5)
    with P.Graph(rm.n, rm.m, 0, np.float64) as B:
        B.insert_batch(rm.n, rm.u, rm.v, rm.cost)
        for name in ("col", "mark", "par"):
            with pytest.raises(P.PirrtError) as e:
                B.load(str(tmp_path / f"{name}.ckpt"))
            assert e.value.status == P.PIRRT_ERR_BAD_INPUT, name
        assert B.n == rm.n
        assert B.exploit()["converged"] == 1
        np.testing.assert_array_equal(B.get_costs(), g)
