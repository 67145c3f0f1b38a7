"""The host C code under AddressSanitizer and UndefinedBehaviorSanitizer.

The oracle (oracle/pirrt_oracle.c) and the roadmap generator's helper
(workloads/roadgen.c) are rebuilt with -fsanitize=address,undefined and
exercised in a child Python process that preloads the ASan runtime: the
hand-solved graphs in both forms, random graphs, the checkers, the rejection
of bad input, and a 2-D roadmap generated, replanned and checked.  Any
sanitizer report fails the child (UBSan is made fatal; leaks are not checked,
Python itself keeps memory to the end).
"""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle as O
from paper_2003_04920_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLAGS = ["-O1", "-g", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
         "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
         "-fno-omit-frame-pointer"]


def _asan_runtime():
    try:
        out = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                             text=True, check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return out if os.path.isabs(out) and os.path.exists(out) else None


CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import oracle as O
    from paper_2003_04920_gb300 import workloads as W
    from tests import golden_io

    lib = O.load({oracle_lib!r})
    W._LIB_PATH = {roadgen_lib!r}
    W._lib = None

    def o1(n, u, v, c, init=None, root=0, goal=None, h=None):
        G = O.OracleGraph(n, root, lib=lib)
        G.insert(n, u, v, c)
        if goal is not None:
            G.set_goal(goal, h)
        if init is not None:
            G.set_policy(init)
        st = G.replan()
        g, p = G.get()
        G.promising()
        G.close()
        return g, p, st

    for name in golden_io.names():
        gd = golden_io.load(name)
        g, p, st = o1(gd["n"], gd["u"], gd["v"], gd["c"], gd["init"], gd["root"],
                      gd["goal"], gd["h"])
        assert np.array_equal(g, gd["g"]) and np.array_equal(p, gd["parent"]), name

    for seed in range(4):
        rm = W.random_graph(500 + seed, 200, 900, connected=seed != 1)
        c = rm.cost.astype(np.float64)
        A = O.CSR(200, rm.u, rm.v, c, lib=lib)
        d, _ = A.dijkstra()
        g, p, _ = o1(200, rm.u, rm.v, c)
        assert A.check_tree(p)[0] == 0 and A.check_bellman(g)[0] == 0
        assert A.check_consistency(p, g)[0] == 0
        A.unambiguous(d)
        A.component()
        o1(200, rm.u, rm.v, c, goal=7, h=np.random.default_rng(seed).random(200))
        A.close()

    G = O.OracleGraph(4, 0, lib=lib)
    for bad in (([0], [0], [1.0]), ([0], [9], [1.0]), ([0], [1], [-1.0]), ([0], [1], [np.nan])):
        try:
            G.insert(2, *bad)
            raise SystemExit("bad input accepted")
        except O.OracleError:
            pass
    G.close()

    rm = W.roadmap_c1(n_samples=600)
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost, lib=lib)
    d, _ = A.dijkstra()
    g, p, _ = o1(rm.n, rm.u, rm.v, rm.cost, init=W.bfs_tree_parents(rm))
    assert np.allclose(g[np.isfinite(d)], d[np.isfinite(d)], rtol=1e-12)
    h = 0.99 * np.linalg.norm(rm.points - rm.points[5], axis=1)
    o1(rm.n, rm.u, rm.v, rm.cost, goal=5, h=h)
    A.close()
    rm6 = W.roadmap_nd_knn("t", 77, 3000, 6, 8, 0.3, 0.8, 12, 3000)
    assert rm6.m > 0
    print("sanitized run ok")
""")


def _run_child(tmp_path, oracle_src):
    """Build the oracle from `oracle_src` and the generator helper with the
    sanitizers, run the child script; returns the finished process."""
    runtime = _asan_runtime()
    if runtime is None:
        pytest.skip("gcc has no AddressSanitizer runtime here")
    oracle_lib = str(tmp_path / "liboracle_asan.so")
    roadgen_lib = str(tmp_path / "libroadgen_asan.so")
    subprocess.run(["gcc", *FLAGS, oracle_src, "-o", oracle_lib, "-lm"], check=True)
    subprocess.run(["gcc", *FLAGS, W._SRC, "-o", roadgen_lib, "-lm"], check=True)
    script = tmp_path / "child.py"
    script.write_text(CHILD.format(root=ROOT, oracle_lib=oracle_lib, roadgen_lib=roadgen_lib))
    env = dict(os.environ, LD_PRELOAD=runtime, ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    return subprocess.run([sys.executable, str(script)], capture_output=True, text=True,
                          env=env, timeout=600)


def test_oracle_and_generator_under_asan_and_ubsan(tmp_path):
    r = _run_child(tmp_path, O.SOURCE)
    report = r.stdout[-2000:] + r.stderr[-4000:]
    assert r.returncode == 0, report
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, report
    assert "sanitized run ok" in r.stdout


def test_the_harness_catches_a_planted_overflow(tmp_path):
    """A copy of the oracle with an out-of-bounds write must fail the child."""
    src = open(O.SOURCE).read()
    anchor = "G->b[G->root] = 1;"
    assert src.count(anchor) == 1
    bad = tmp_path / "planted.c"
    bad.write_text(src.replace(anchor, "G->b[G->cap_n + 64] = 1;"))
    r = _run_child(tmp_path, str(bad))
    assert r.returncode != 0
    assert "heap-buffer-overflow" in r.stderr
