"""Argument checks of the allocation-free sweep, on the CPU (no GPU needed).

pycool_sweep_noalloc writes phi_out (and pi_out) while its blocks read the
neighbours of phi_in and pi_in, so an output that shares memory with an input
or with the other output would be read after it was overwritten; a short or
differently typed tensor would be read and written past its end.  Both are
refused before any device work: the C entry point checks the address ranges
(here with made-up, aligned addresses that are never dereferenced) and the
Python wrapper checks the tensors."""
import ctypes as C

import pytest

P = pytest.importorskip("paper_1201_5029_gb300")
torch = pytest.importorskip("torch")


def _cfg(n=16):
    return P.make_config(n, 10.0, "chaotic2", [1.0, 1e4], 0.005, order=2)


def _call(cfg, phi_in, pi_in, phi_out, pi_out, flush, init_pa=0):
    st = P.pycool_stage_state()
    st.a = 1.0
    st.init_pa = init_pa
    v = lambda x: None if x is None else C.c_void_p(x)  # noqa: E731
    return P.lib.pycool_sweep_noalloc(C.byref(cfg), v(phi_in), v(pi_in), v(phi_out), v(pi_out),
                                      int(flush), C.byref(st), None)


def test_overlapping_buffers_are_rejected_before_device_work():
    cfg = _cfg()
    nbytes = 2 * 16 ** 3 * 8
    a, b, c, d = (0x10000000 + i * 0x1000000 for i in range(4))
    # an output equal to an input, or overlapping one by a single element
    assert _call(cfg, a, b, a, d, False) == P.E_INVALID
    assert _call(cfg, a, b, b, d, False) == P.E_INVALID
    assert _call(cfg, a, b, c, b, False) == P.E_INVALID
    assert _call(cfg, a, b, c, a, False) == P.E_INVALID
    assert _call(cfg, a, b, c, c, False) == P.E_INVALID
    assert _call(cfg, a, b, a + nbytes - 16, d, False) == P.E_INVALID
    assert _call(cfg, a, b, b - nbytes + 16, d, True) == P.E_INVALID
    # p_a from the constraint is set by a flush only
    assert _call(cfg, a, b, c, d, False, init_pa=1) == P.E_INVALID
    # unaligned arrays
    assert _call(cfg, a + 8, b, c, d, False) == P.E_INVALID


def test_wrapper_rejects_host_short_or_mistyped_tensors():
    cfg = _cfg(8)
    st = P.pycool_stage_state()
    st.a = 1.0
    good = torch.zeros(2 * 8 ** 3, dtype=torch.float64)   # on the host: refused
    assert P.pycool_sweep_noalloc(cfg, good, good, good, good, False, st) == P.E_INVALID
    short = torch.zeros(10, dtype=torch.float64)
    assert P.pycool_sweep_noalloc(cfg, short, short, short, short, False, st) == P.E_INVALID
    f32 = torch.zeros(2 * 8 ** 3, dtype=torch.float32)
    assert P.pycool_sweep_noalloc(cfg, f32, f32, f32, f32, True, st) == P.E_INVALID
