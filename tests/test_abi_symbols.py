"""The C-ABI library loads on a machine without a GPU and exports every symbol
that include/*.h declares (no compute calls)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pycool_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_core_calls():
    names = declared_symbols()
    for core in ("pycool_create", "pycool_set_initial", "pycool_evolve", "pycool_energies",
                 "pycool_field_stats", "pycool_get_fields", "pycool_destroy", "pycool_sync"):
        assert core in names


def test_library_exports_every_declared_symbol():
    import paper_1201_5029_gb300 as P
    lib = ctypes.CDLL(P.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_work_without_gpu():
    import paper_1201_5029_gb300 as P
    assert [P.pycool_stages_per_step(o) for o in (2, 4, 6, 8)] == [1, 3, 7, 15]
    assert P.pycool_stages_per_step(5) == -1
    w = P.pycool_stage_weights(8)
    assert w == w[::-1] and abs(sum(w) - 1.0) < 1e-14
    cfg = P.make_config(32, 10.0, "chaotic2", (1.0, 1e4), 0.005, order=2)
    state, ws = P.pycool_query_bytes(cfg)
    assert state >= 4 * 2 * 32 ** 3 * 8 and ws > 0
    split = P.make_config(32, 10.0, "chaotic2", (1.0, 1e4), 0.005, order=2, precision="split_fp32")
    assert P.pycool_query_bytes(split)[0] < state
    bad = P.make_config(32, 10.0, "chaotic2", (1.0, 1e4), 0.5, order=8)
    try:
        P.pycool_query_bytes(bad)
        raise AssertionError("unstable dt accepted")
    except P.PycoolError as e:
        assert e.status == P.E_UNSTABLE_DT
    assert "stability" in P.pycool_strerror(P.E_UNSTABLE_DT)


def test_fault_injection_calls_check_their_arguments_without_gpu():
    import paper_1201_5029_gb300 as P
    assert P.pycool_debug_fail_alloc(-1) == P.E_INVALID
    assert P.pycool_debug_barrier_stall(None, 1000) == P.E_INVALID
    assert P.pycool_server_cancel(None, 1) == P.E_INVALID
    assert P.pycool_strerror(P.E_CANCELLED) == "request cancelled"


def test_fourth_order_stencil_needs_four_sites_per_axis():
    import paper_1201_5029_gb300 as P
    for n, want in ((3, P.E_INVALID), (4, P.OK)):
        cfg = P.make_config(n, 4.0, "chaotic2", (1.0, 1.0), 0.01, order=2, stencil="4th")
        assert P.lib.pycool_query_bytes(ctypes.byref(cfg), None, None) == want
