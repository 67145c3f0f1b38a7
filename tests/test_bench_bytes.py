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
