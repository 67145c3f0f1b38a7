"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/pirrt.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2003_04920_gb300 import build as B

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared_symbols():
    names = set()
    for f in os.listdir(HEADER_DIR):
        if f.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(pirrt_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for want in ("pirrt_graph_create", "pirrt_graph_insert_batch", "pirrt_graph_exploit",
                 "pirrt_graph_get_costs", "pirrt_graph_get_parents", "pirrt_graph_destroy",
                 "pirrt_status_string"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_status_strings(lib):
    lib.pirrt_status_string.restype = ctypes.c_char_p
    assert lib.pirrt_status_string(0) == b"PIRRT_OK"
    assert lib.pirrt_status_string(8) == b"PIRRT_ERR_BAD_TREE"
    assert lib.pirrt_status_string(99) == b"PIRRT_UNKNOWN_STATUS"


def test_null_handles_are_rejected(lib):
    lib.pirrt_graph_num_vertices.restype = ctypes.c_int64
    assert lib.pirrt_graph_num_vertices(None) == -1
    assert lib.pirrt_graph_exploit(None, None, None) == 1
    assert lib.pirrt_graph_create(None, None) == 1
    lib.pirrt_graph_destroy(None)


def test_null_handles_are_rejected_by_every_graph_call(lib):
    """Each graph entry point answers PIRRT_ERR_INVALID_ARG to a NULL handle
    before touching the device (no GPU here)."""
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    calls = {
        "pirrt_graph_reset": ([vp], (None,)),
        "pirrt_graph_insert_batch": ([vp, i64, i64, vp, vp, vp, ctypes.c_int],
                                     (None, 0, 0, None, None, None, 0)),
        "pirrt_graph_prefetch_batch": ([vp, i64, vp, vp, vp], (None, 0, None, None, None)),
        "pirrt_graph_set_goal": ([vp, i32, vp, i64], (None, 0, None, 0)),
        "pirrt_graph_set_policy": ([vp, vp, i64, ctypes.c_int], (None, None, 0, 0)),
        "pirrt_graph_get_costs": ([vp, vp, i64, ctypes.c_int], (None, None, 0, 0)),
        "pirrt_graph_get_parents": ([vp, vp, i64, ctypes.c_int], (None, None, 0, 0)),
        "pirrt_graph_save": ([vp, ctypes.c_char_p], (None, b"x")),
        "pirrt_graph_load": ([vp, ctypes.c_char_p], (None, b"x")),
    }
    for name, (argtypes, args) in calls.items():
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = argtypes
        assert fn(*args) == 1, name


C_CALLER = r"""
#include <stddef.h>
#include <stdint.h>
#include "pirrt.h"
int main(void) {
    float h[4] = {0};
    int32_t src[3] = {0, 1, 2}, dst[3] = {1, 2, 3};
    float cost[3] = {1, 1, 1};
    double g_out[4];
    int32_t p_out[4];
    pirrt_config cfg = {.max_vertices = 4, .max_edges = 3, .root = 0,
                        .cost_dtype = PIRRT_COST_F32, .device = 0, .stream = NULL};
    pirrt_graph *g = NULL;
    if (pirrt_graph_create(&cfg, &g) != PIRRT_OK) return 1;
    pirrt_graph_set_goal(g, 3, h, 4);
    pirrt_graph_insert_batch(g, 4, 3, src, dst, cost, 0);
    pirrt_exploit_stats st;
    pirrt_graph_exploit(g, NULL, &st);
    pirrt_graph_get_costs(g, g_out, 4, 0);
    pirrt_graph_get_parents(g, p_out, 4, 0);
    pirrt_graph_destroy(g);
    return 0;
}
"""


def test_header_is_c11_and_a_c_caller_links(tmp_path):
    """include/pirrt.h compiles as C11 with warnings as errors, and a C caller
    links against the library (it is not run: that needs a GPU)."""
    import subprocess
    path = B.build()
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", f"-I{HEADER_DIR}",
                    str(src), "-o", str(exe), path, f"-Wl,-rpath,{os.path.dirname(path)}"],
                   check=True)
    assert exe.exists()


def test_library_links_no_driver_library():
    path = B.build()
    import subprocess
    out = subprocess.run(["ldd", path], capture_output=True, text=True).stdout
    assert "libcuda.so" not in out


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout: the same
    size and the same offset for every field (a C program compiled against
    include/pirrt.h prints them; nothing calls the library)."""
    import subprocess
    import paper_2003_04920_gb300 as P
    structs = {"pirrt_config": P.pirrt_config, "pirrt_exploit_opts": P.pirrt_exploit_opts,
               "pirrt_exploit_stats": P.pirrt_exploit_stats, "pirrt_profile": P.pirrt_profile,
               "pirrt_trace_record": P.pirrt_trace_record}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pirrt.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", f"-I{HEADER_DIR}", str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_option_dicts_round_trip():
    """The searching autotuner's result comes back as exploit() keywords that
    rebuild the same option struct."""
    import paper_2003_04920_gb300 as P
    o = P.exploit_opts(eps=0.5, max_iters=7, group=8, tile=2, dense_fraction=0.2,
                       evaluate="wave", wave_levels=40, host_loop=True, wave_tail=-1,
                       wave_ctas=1, wave_local=4, wave_local_max=32, wave_local_step=1024)
    back = P.exploit_opts(**P.opts_dict(o))
    assert bytes(back) == bytes(o)
