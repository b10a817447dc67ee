"""Potentials given at run time: CPU checks (no GPU needed).

pycool_model_define compiles C expressions with NVRTC before it needs the
GPU, so a malformed expression is refused with E_INVALID on any machine,
and arguments are checked first."""
import ctypes as C

import pytest

P = pytest.importorskip("paper_1201_5029_gb300")


def test_bad_expressions_and_arguments_are_refused():
    mid = C.c_int32()
    bad = (C.c_char_p * 1)(b"f0 +* 2")
    assert P.lib.pycool_model_define(1, b"0.5*f0*f0", bad, C.byref(mid)) == P.E_INVALID
    unknown = (C.c_char_p * 1)(b"f7")                    # no such variable
    assert P.lib.pycool_model_define(1, b"0.5*f0*f0", unknown, C.byref(mid)) == P.E_INVALID
    ok = (C.c_char_p * 1)(b"p[0]*f0")
    assert P.lib.pycool_model_define(3, b"0.5*f0*f0", ok, C.byref(mid)) == P.E_INVALID
    assert P.lib.pycool_model_define(1, None, ok, C.byref(mid)) == P.E_INVALID
    assert P.lib.pycool_model_source(99, None, 0, None) == P.E_INVALID
