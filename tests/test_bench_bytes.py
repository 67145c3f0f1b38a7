"""The roofline numerator of bench.py: the algorithmic bytes per unit of work
(per CSR entry, listed vertex, dense-sweep vertex, switch, recomputed vertex
and offer), each one fixed by the arrays the method must read or write once."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _improve(b, offers, cost_bytes=4, **kw):
    prof = dict(improve_entries=0, improve_vertices=0, improve_dense_vertices=0,
                improve_switches=0)
    prof.update(kw)
    if "improve_dense_vertices" in kw:
        prof["improve_vertices"] += kw["improve_dense_vertices"]
    entry = 8 if cost_bytes == 4 else 16
    return b.improve_bytes(prof, entry, cost_bytes, offers)


def test_improve_bytes_per_unit():
    b = _bench()
    for offers in (True, False):
        # a CSR entry: column id + FP32 cost (FP64: padded 16-byte entry)
        assert _improve(b, offers, improve_entries=1) == 8
        assert _improve(b, offers, 8, improve_entries=1) == 16
        # a dense-sweep vertex: row extent 8, parent 4, parent cost 4, g(p) 8, g(v) 8
        assert _improve(b, offers, improve_dense_vertices=1) == 32
    # a listed vertex: list id 4, parent 4, parent cost 4, g(p) 8, and its best
    # offer 8 (offers) or its row extent 8 (full scans)
    assert _improve(b, True, improve_vertices=1) == 28
    assert _improve(b, False, improve_vertices=1) == 28
    # a switch: parent 4 + cost 4 written, switch-list id 4; with offers also
    # the row extent of the deciding vertex 8
    assert _improve(b, False, improve_switches=1) == 12
    assert _improve(b, True, improve_switches=1) == 20


def test_evaluate_bytes_per_unit():
    b = _bench()
    # a recomputed vertex: parent 4, parent cost 4, g(p) 8, g written 8
    assert b.evaluate_bytes(dict(evaluate_vertices=1), 8, 4) == 24
    assert b.evaluate_bytes(dict(evaluate_vertices=1), 16, 8) == 28
    # an offer: the CSR entry it is formed from
    assert b.evaluate_bytes(dict(evaluate_vertices=0, evaluate_offers=1), 8, 4) == 8
    # linear in the counts
    assert b.evaluate_bytes(dict(evaluate_vertices=1000, evaluate_offers=300), 8, 4) == \
        1000 * 24 + 300 * 8


def test_step_roofline_counts_one_step():
    """The whole-step roofline divides one step's algorithmic bytes (the
    profiled steps' total over their number) by the timed step time."""
    b = _bench()
    kb = {"improve": 2e9, "evaluate": 6e9, "insert": 2e9, "mark_frontier": None}
    r = b.step_roofline(kb, 2, 100.0, 5000.0)
    assert r["algorithmic_bytes"] == 5_000_000_000
    assert abs(r["achieved"] - 50.0) < 1e-9 and abs(r["frac"] - 0.01) < 1e-9


def test_level_profile_buckets():
    """Bucket b of the level trace holds steps of 2^(b-1) .. 2^b - 1 vertices;
    cycles become microseconds at the sampled SM clock."""
    b = _bench()
    z = [0] * 24
    prof = {"level_count": list(z), "level_vertices": list(z), "level_cycles": list(z),
            "share_tiles": list(z), "share_vertices": list(z), "share_cycles": list(z),
            "local_tiles": list(z), "local_vertices": list(z), "local_cycles": list(z),
            "wave_calls": 3, "wave_pre_cycles": 2000, "wave_post_cycles": 4000,
            "wave_jump_cycles": 0}
    prof["level_count"][1], prof["level_vertices"][1], prof["level_cycles"][1] = 5, 5, 10000
    prof["level_count"][4], prof["level_vertices"][4], prof["level_cycles"][4] = 2, 20, 8000
    prof["local_tiles"][3], prof["local_vertices"][3], prof["local_cycles"][3] = 4, 20, 4000
    out = b.level_profile(prof, {"sm_mhz": 2000.0})
    rows = {r["vertices_lo"]: r for r in out["buckets"]}
    assert set(rows) == {1, 8}
    assert rows[1]["vertices_hi"] == 1 and rows[8]["vertices_hi"] == 15
    assert rows[1]["us_per_level"] == 1.0 and rows[8]["us_per_level"] == 2.0
    assert out["levels_us_total"] == 9.0 and out["pre_us_total"] == 1.0
    assert out["cta0_local_tiles"] == [{"vertices_lo": 4, "tiles": 4, "vertices": 20,
                                        "us_per_tile": 0.5}]
