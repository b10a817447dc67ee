"""GB300-native symplectic lattice stepper (the method of PyCOOL, arXiv:1201.5029).

Thin ctypes binding over the C ABI declared in ``include/pycool.h``: the same
function names, argument marshalling only.  Every step of the evolution runs
in the CUDA kernels of ``libpycool.so``; there is no CPU fallback.  If the
library has not been built, importing the binding raises.  The library is
mapped into the process at the first call (``load()``), so that importing the
seeded input generators (``paper_1201_5029_gb300.inputs``), which hold none of
the method's arithmetic, does not load the CUDA code.

Host arrays are numpy float64 arrays of shape (N_f, n, n, n) ([field][z][y][x]);
device arrays are CUDA torch tensors of the same shape and dtype (pass
``on_device=True``).  PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpycool.so")

MAX_FIELDS = 2
MAX_PARAMS = 8

# status codes (pycool_status)
OK, E_INVALID, E_UNSTABLE_DT, E_NOMEM, E_CUDA, E_NONFINITE, E_TIMEOUT, E_STATE, E_BUSY, \
    E_NOT_FOUND, E_CANCELLED = range(11)
# models, precisions, stencils
MODEL_FREE, MODEL_CHAOTIC2, MODEL_OSCILLON, MODEL_QBALL = range(4)
FP64, SPLIT_FP32, SPLIT_DD = 0, 1, 2
STENCIL_7PT, STENCIL_4TH, STENCIL_ISO27 = 7, 13, 27
IC_WHITE = 0

MODELS = {"free": MODEL_FREE, "chaotic2": MODEL_CHAOTIC2, "oscillon": MODEL_OSCILLON,
          "qball": MODEL_QBALL}
MODEL_NF = {MODEL_FREE: 1, MODEL_CHAOTIC2: 2, MODEL_OSCILLON: 1, MODEL_QBALL: 2}
PRECISIONS = {"fp64": FP64, "split_fp32": SPLIT_FP32, "split_dd": SPLIT_DD}
STENCILS = {"7pt": STENCIL_7PT, "4th": STENCIL_4TH, "iso27": STENCIL_ISO27}


class pycool_config(C.Structure):
    _fields_ = [("n", C.c_int32), ("model", C.c_int32), ("order", C.c_int32),
                ("precision", C.c_int32), ("stencil", C.c_int32), ("time_step", C.c_int32),
                ("L", C.c_double), ("dt", C.c_double), ("mpl", C.c_double),
                ("rho_rad0", C.c_double), ("rho_mat0", C.c_double),
                ("params", C.c_double * MAX_PARAMS)]


class pycool_energies_t(C.Structure):
    _fields_ = [("eta", C.c_double), ("a", C.c_double), ("pa", C.c_double), ("H", C.c_double),
                ("rho_kin", C.c_double * MAX_FIELDS), ("rho_grad", C.c_double * MAX_FIELDS),
                ("rho_pot", C.c_double), ("rho", C.c_double), ("P", C.c_double),
                ("residual", C.c_double),
                ("mean", C.c_double * MAX_FIELDS), ("variance", C.c_double * MAX_FIELDS),
                ("steps_done", C.c_int64), ("sweeps_done", C.c_int64)]

    def as_dict(self, nf: int = MAX_FIELDS) -> dict:
        return dict(eta=self.eta, a=self.a, pa=self.pa, H=self.H,
                    rho_kin=list(self.rho_kin)[:nf], rho_grad=list(self.rho_grad)[:nf],
                    rho_pot=self.rho_pot, rho=self.rho, P=self.P, residual=self.residual,
                    mean=list(self.mean)[:nf], variance=list(self.variance)[:nf],
                    steps_done=self.steps_done, sweeps_done=self.sweeps_done)


class pycool_stage_state(C.Structure):
    """Background record of the allocation-free sweep (pycool_sweep_noalloc)."""
    _fields_ = [("a", C.c_double), ("pa", C.c_double), ("eta", C.c_double),
                ("h_prev", C.c_double), ("sum_pi2", C.c_double), ("stage", C.c_int64),
                ("steps_done", C.c_int64), ("init_pa", C.c_int32), ("error", C.c_int32),
                ("obs", pycool_energies_t)]


class pycool_ic(C.Structure):
    _fields_ = [("background", C.c_double * MAX_FIELDS), ("momentum", C.c_double * MAX_FIELDS),
                ("noise", C.c_double), ("a0", C.c_double)]


class PycoolError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {pycool_strerror(status)} (status {status})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libpycool.so is not built ({LIB_PATH}); run "
            "`python -m paper_1201_5029_gb300.build` (or __graft_entry__.build()) first")
    lib = C.CDLL(LIB_PATH)
    P, S = C.c_void_p, C.c_int
    sig = {
        "pycool_stages_per_step": (C.c_int, [C.c_int32]),
        "pycool_stage_weights": (S, [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
        "pycool_query_bytes": (S, [C.POINTER(pycool_config), C.POINTER(C.c_size_t),
                                   C.POINTER(C.c_size_t)]),
        "pycool_create": (S, [C.POINTER(pycool_config), P, P, P, C.POINTER(P)]),
        "pycool_set_initial": (S, [P, P, P, C.c_int, C.c_double, C.c_double]),
        "pycool_evolve": (S, [P, C.c_int64]),
        "pycool_sync": (S, [P, C.c_double]),
        "pycool_energies": (S, [P, C.POINTER(pycool_energies_t)]),
        "pycool_field_stats": (S, [P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "pycool_get_fields": (S, [P, P, P, C.c_int]),
        "pycool_checkpoint_size": (S, [P, C.POINTER(C.c_size_t)]),
        "pycool_checkpoint_save": (S, [P, P, C.c_size_t]),
        "pycool_checkpoint_load": (S, [P, P, C.c_size_t]),
        "pycool_set_stream": (S, [P, P]),
        "pycool_kernel_launches": (C.c_int64, [P]),
        "pycool_linear_modes": (S, [C.c_int32, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64), P]),
        "pycool_linear_growth": (S, [C.POINTER(pycool_config), C.c_double, C.c_double, P, P, P,
                                     C.c_int64, C.c_int64, P, P, P]),
        "pycool_model_define": (S, [C.c_int32, C.c_char_p, C.POINTER(C.c_char_p),
                                    C.POINTER(C.c_int32)]),
        "pycool_model_source": (S, [C.c_int32, P, C.c_size_t, C.POINTER(C.c_size_t)]),
        "pycool_energy_fields": (S, [P, P, P, C.c_int]),
        "pycool_spectrum_bins": (C.c_int32, [C.c_int32]),
        "pycool_spectrum": (S, [P, C.c_int32, C.c_int32, P, P, C.c_int32]),
        "pycool_linear_evolve": (S, [C.POINTER(pycool_config), C.c_double, C.c_double, P, P,
                                     C.c_int64, P, P, P, P]),
        "pycool_persist_plan": (S, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                    C.c_int64, C.POINTER(C.c_int32), P, C.c_int32, P,
                                    C.c_int32]),
        "pycool_destroy": (None, [P]),
        "pycool_strerror": (C.c_char_p, [S]),
        "pycool_server_create": (S, [C.c_size_t, C.c_int32, C.POINTER(P)]),
        "pycool_server_submit": (S, [P, C.POINTER(pycool_config), C.POINTER(pycool_ic),
                                     C.c_uint64, C.c_int64, C.POINTER(C.c_uint64)]),
        "pycool_server_wait": (S, [P, C.c_uint64, C.c_double, C.POINTER(pycool_energies_t)]),
        "pycool_server_stats": (S, [P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "pycool_server_destroy": (None, [P]),
        "pycool_server_cancel": (S, [P, C.c_uint64]),
        "pycool_server_set_persistent_min_n": (S, [P, C.c_int32]),
        "pycool_debug_fail_alloc": (S, [C.c_int32]),
        "pycool_debug_barrier_stall": (S, [P, C.c_int64]),
        "pycool_noalloc_max_blocks": (C.c_size_t, []),
        "pycool_sweep_noalloc": (S, [C.POINTER(pycool_config), P, P, P, P, C.c_int32,
                                     C.POINTER(pycool_stage_state), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    return lib


if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libpycool.so is not built ({LIB_PATH}); run "
        "`python -m paper_1201_5029_gb300.build` (or __graft_entry__.build()) first")


class _Library:
    """The ctypes handle of libpycool.so, opened at the first attribute access."""
    _handle = None

    def __getattr__(self, name):
        if _Library._handle is None:
            _Library._handle = _load()
        return getattr(_Library._handle, name)


lib = _Library()


def load():
    """Map libpycool.so now (raises if it cannot be loaded); returns the handle."""
    lib.pycool_strerror  # noqa: B018  (first access opens the library)
    return _Library._handle


def _check(status: int, what: str):
    if status != OK:
        raise PycoolError(status, what)


def _ptr(arr, on_device: bool):
    if arr is None:
        return None
    if on_device:
        return C.c_void_p(int(arr.data_ptr()))
    a = np.ascontiguousarray(arr, dtype=np.float64)
    return C.c_void_p(a.ctypes.data), a


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---------------------------------------------------------------- config helpers

TIME_STEPS = {"conformal": 0, "physical": 1}


def make_config(n: int, L: float, model, params: Sequence[float], dt: float, order: int = 2,
                precision="fp64", stencil="7pt", mpl: float = 1.0, rho_rad0: float = 0.0,
                rho_mat0: float = 0.0, time_step="conformal") -> pycool_config:
    c = pycool_config()
    c.n = int(n)
    c.model = MODELS[model] if isinstance(model, str) else int(model)
    c.order = int(order)
    c.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    c.stencil = STENCILS[stencil] if isinstance(stencil, str) else int(stencil)
    c.time_step = TIME_STEPS[time_step] if isinstance(time_step, str) else int(time_step)
    c.L, c.dt, c.mpl = float(L), float(dt), float(mpl)
    c.rho_rad0, c.rho_mat0 = float(rho_rad0), float(rho_mat0)
    for i, p in enumerate(params):
        c.params[i] = float(p)
    return c


def config_from_workload(w: dict, **over) -> pycool_config:
    w = dict(w)
    w.update(over)
    return make_config(n=w["n"], L=w["L"], model=w["model"], params=w["params"], dt=w["dt"],
                       order=w["order"], precision=w.get("precision", "fp64"),
                       stencil=w.get("stencil", "7pt"), mpl=w.get("mpl", 1.0),
                       rho_rad0=w.get("rho_rad0", 0.0), rho_mat0=w.get("rho_mat0", 0.0),
                       time_step=w.get("time_step", "conformal"))


# ---------------------------------------------------------------- the C ABI, same names

def pycool_strerror(status: int) -> str:
    return lib.pycool_strerror(int(status)).decode()


def pycool_stages_per_step(order: int) -> int:
    return lib.pycool_stages_per_step(int(order))


def pycool_stage_weights(order: int) -> list:
    w = (C.c_double * 15)()
    n = C.c_int32()
    _check(lib.pycool_stage_weights(int(order), w, C.byref(n)), "pycool_stage_weights")
    return list(w)[: n.value]


def pycool_query_bytes(cfg: pycool_config) -> Tuple[int, int]:
    s, w = C.c_size_t(), C.c_size_t()
    _check(lib.pycool_query_bytes(C.byref(cfg), C.byref(s), C.byref(w)), "pycool_query_bytes")
    return s.value, w.value


def pycool_create(cfg: pycool_config, dev_state: Optional[int] = None,
                  dev_workspace: Optional[int] = None, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib.pycool_create(C.byref(cfg), dev_state, dev_workspace, _stream_ptr(stream),
                             C.byref(h)), "pycool_create")
    return h


def pycool_set_initial(sim, phi, pi, on_device: bool = False, a0: float = 1.0,
                       pa0: float = math.nan) -> None:
    if on_device:
        _check(lib.pycool_set_initial(sim, _ptr(phi, True), _ptr(pi, True), 1, a0, pa0),
               "pycool_set_initial")
        return
    p1, keep1 = _ptr(phi, False)
    p2, keep2 = _ptr(pi, False)
    _check(lib.pycool_set_initial(sim, p1, p2, 0, a0, pa0), "pycool_set_initial")


def pycool_evolve(sim, steps: int) -> None:
    _check(lib.pycool_evolve(sim, int(steps)), "pycool_evolve")


def pycool_sync(sim, timeout_s: float = -1.0) -> int:
    """Returns the status (OK, E_TIMEOUT, E_NONFINITE...) without raising."""
    return lib.pycool_sync(sim, float(timeout_s))


def pycool_energies(sim, nf: int = MAX_FIELDS) -> dict:
    e = pycool_energies_t()
    _check(lib.pycool_energies(sim, C.byref(e)), "pycool_energies")
    return e.as_dict(nf)


def pycool_field_stats(sim, field: int) -> Tuple[float, float]:
    m, v = C.c_double(), C.c_double()
    _check(lib.pycool_field_stats(sim, int(field), C.byref(m), C.byref(v)), "pycool_field_stats")
    return m.value, v.value


def pycool_get_fields(sim, phi=None, pi=None, on_device: bool = False, shape=None):
    """Copy the current fields out.  Host: pass shape=(N_f, n, n, n) to get new
    numpy arrays, or pass float64 arrays to fill.  Device: pass CUDA tensors."""
    if on_device:
        _check(lib.pycool_get_fields(sim, _ptr(phi, True) if phi is not None else None,
                                     _ptr(pi, True) if pi is not None else None, 1),
               "pycool_get_fields")
        return phi, pi
    if phi is None and shape is not None:
        phi = np.empty(shape, dtype=np.float64)
    if pi is None and shape is not None:
        pi = np.empty(shape, dtype=np.float64)
    for a in (phi, pi):
        if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous):
            raise ValueError("host arrays must be C-contiguous float64")
    _check(lib.pycool_get_fields(sim, phi.ctypes.data if phi is not None else None,
                                 pi.ctypes.data if pi is not None else None, 0),
           "pycool_get_fields")
    return phi, pi


def pycool_checkpoint_size(sim) -> int:
    s = C.c_size_t()
    _check(lib.pycool_checkpoint_size(sim, C.byref(s)), "pycool_checkpoint_size")
    return s.value


def pycool_checkpoint_save(sim) -> bytes:
    n = pycool_checkpoint_size(sim)
    buf = C.create_string_buffer(n)
    _check(lib.pycool_checkpoint_save(sim, buf, n), "pycool_checkpoint_save")
    return buf.raw


def pycool_checkpoint_load(sim, blob: bytes) -> None:
    buf = C.create_string_buffer(blob, len(blob))
    _check(lib.pycool_checkpoint_load(sim, buf, len(blob)), "pycool_checkpoint_load")


def pycool_set_stream(sim, stream) -> None:
    _check(lib.pycool_set_stream(sim, _stream_ptr(stream)), "pycool_set_stream")


def pycool_kernel_launches(sim) -> int:
    return int(lib.pycool_kernel_launches(sim))


def pycool_linear_modes(n: int, stencil="7pt"):
    """(values, index): the distinct k_eff^2 of an n^3 lattice (ascending) and
    each mode's index into them, shape (n, n, n) in numpy FFT order."""
    import numpy as np
    st = STENCILS[stencil] if isinstance(stencil, str) else int(stencil)
    cnt = C.c_int64()
    _check(lib.pycool_linear_modes(int(n), st, None, 0, C.byref(cnt), None), "pycool_linear_modes")
    vals = np.zeros(cnt.value)
    idx = np.zeros((n, n, n), dtype=np.int32)
    _check(lib.pycool_linear_modes(int(n), st, vals.ctypes.data, cnt.value, C.byref(cnt),
                                   idx.ctypes.data), "pycool_linear_modes")
    return vals, idx


def pycool_linear_growth(cfg: pycool_config, a0: float, pa0: float, phi0, pi0, k2, steps: int,
                         stream=None):
    """Growth functions of the linearised evolution: (T, background) with T of
    shape (len(k2), 2 N_f, 2 N_f) and background = (a, p_a, phi0, pi0)."""
    import numpy as np
    nf = len(phi0)
    f0 = np.ascontiguousarray(phi0, dtype=np.float64)
    p0 = np.ascontiguousarray(pi0, dtype=np.float64)
    kk = np.ascontiguousarray(k2, dtype=np.float64).ravel()
    T = np.zeros((kk.size, 2 * nf, 2 * nf))
    bg = np.zeros(2 + 2 * nf)
    _check(lib.pycool_linear_growth(C.byref(cfg), float(a0), float(pa0), f0.ctypes.data,
                                    p0.ctypes.data, kk.ctypes.data, kk.size, int(steps),
                                    T.ctypes.data, bg.ctypes.data, _stream_ptr(stream)),
           "pycool_linear_growth")
    return T, (bg[0], bg[1], bg[2:2 + nf].copy(), bg[2 + nf:].copy())


def pycool_linear_evolve(cfg: pycool_config, a0: float, pa0: float, phi, pi, steps: int,
                         phi_out, pi_out, stream=None):
    """The linearised evolution of lattice fields on the device: phi, pi,
    phi_out, pi_out are contiguous float64 CUDA tensors of shape
    (N_f, n, n, n).  Returns the final background (a, p_a, phi0, pi0)."""
    import numpy as np
    nf = MODEL_NF[int(cfg.model)]
    need = nf * int(cfg.n) ** 3
    for t in (phi, pi, phi_out, pi_out):
        if not _is_field_tensor(t, need):
            raise PycoolError(E_INVALID, "pycool_linear_evolve: arrays must be contiguous "
                                         "float64 CUDA tensors of N_f n^3 elements")
    bg = np.zeros(2 + 2 * nf)
    _check(lib.pycool_linear_evolve(C.byref(cfg), float(a0), float(pa0), phi.data_ptr(),
                                    pi.data_ptr(), int(steps), phi_out.data_ptr(),
                                    pi_out.data_ptr(), bg.ctypes.data, _stream_ptr(stream)),
           "pycool_linear_evolve")
    return (bg[0], bg[1], bg[2:2 + nf].copy(), bg[2 + nf:].copy())


def pycool_model_define(V: str, dV: Sequence[str]) -> int:
    """Compile a potential given as C expressions (fields f0, f1; parameters
    p[0..7]) and return its model id for make_config(model=...)."""
    nf = len(dV)
    arr = (C.c_char_p * nf)(*[e.encode() for e in dV])
    mid = C.c_int32()
    _check(lib.pycool_model_define(nf, V.encode(), arr, C.byref(mid)), "pycool_model_define")
    MODEL_NF[mid.value] = nf
    return mid.value


def pycool_model_source(model_id: int) -> str:
    n = C.c_size_t()
    _check(lib.pycool_model_source(int(model_id), None, 0, C.byref(n)), "pycool_model_source")
    buf = C.create_string_buffer(n.value + 1)
    _check(lib.pycool_model_source(int(model_id), buf, n.value + 1, None), "pycool_model_source")
    return buf.value.decode()


def pycool_energy_fields(sim, shape_nnn, rho=None, P=None, on_device=False):
    """rho(x), P(x) of the current synchronised state; host numpy arrays
    (allocated here when not given) or CUDA float64 tensors (on_device)."""
    import numpy as np
    if on_device:
        need = int(np.prod(shape_nnn))
        for t in (rho, P):
            if not _is_field_tensor(t, need):
                raise PycoolError(E_INVALID, "pycool_energy_fields: rho and P must be "
                                             "contiguous float64 CUDA tensors of n^3 elements")
        _check(lib.pycool_energy_fields(sim, rho.data_ptr(), P.data_ptr(), 1),
               "pycool_energy_fields")
        return rho, P
    rho = np.zeros(shape_nnn) if rho is None else rho
    P = np.zeros(shape_nnn) if P is None else P
    for a in (rho, P):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != np.prod(shape_nnn):
            raise PycoolError(E_INVALID, "pycool_energy_fields: host arrays must be contiguous "
                                         "float64 of n^3 elements")
    _check(lib.pycool_energy_fields(sim, rho.ctypes.data, P.ctypes.data, 0),
           "pycool_energy_fields")
    return rho, P


def pycool_spectrum_bins(n: int) -> int:
    return int(lib.pycool_spectrum_bins(int(n)))


def pycool_spectrum(sim, n: int, which: int, field: int):
    """(power, count) of field `field` (which = 0) or its momentum (which = 1)."""
    import numpy as np
    nb = pycool_spectrum_bins(n)
    power = np.zeros(nb)
    count = np.zeros(nb, dtype=np.int64)
    _check(lib.pycool_spectrum(sim, int(which), int(field), power.ctypes.data, count.ctypes.data,
                               nb), "pycool_spectrum")
    return power, count


def pycool_persist_plan(n: int, nf: int, precision: int, sms: int, l2_bytes: int,
                        stencil: int = STENCIL_7PT):
    """The persistent kernel's work plan (host only): (geo, units, uoff) with
    geo a dict, units an int32 array (units, 4) of (x0, y0, z0, planes + 2 H)
    and uoff the int32 block offsets into units."""
    import numpy as np
    geo = (C.c_int32 * 10)()
    _check(lib.pycool_persist_plan(n, nf, precision, stencil, sms, l2_bytes, geo, None, 0, None,
                                   0), "pycool_persist_plan")
    keys = ("n", "vx", "tx", "tiles_x", "ntiles", "rc", "rw", "nunits", "G", "halo")
    g = dict(zip(keys, list(geo)))
    units = np.zeros((g["nunits"], 4), dtype=np.int32)
    uoff = np.zeros(g["G"] + 1, dtype=np.int32)
    _check(lib.pycool_persist_plan(n, nf, precision, stencil, sms, l2_bytes, geo,
                                   units.ctypes.data, g["nunits"], uoff.ctypes.data, g["G"]),
           "pycool_persist_plan")
    return g, units, uoff


def pycool_destroy(sim) -> None:
    lib.pycool_destroy(sim)


def make_ic(background: Sequence[float], momentum: Sequence[float], noise: float,
            a0: float = 1.0) -> pycool_ic:
    ic = pycool_ic()
    for i, v in enumerate(background):
        ic.background[i] = float(v)
    for i, v in enumerate(momentum):
        ic.momentum[i] = float(v)
    ic.noise, ic.a0 = float(noise), float(a0)
    return ic


def pycool_server_create(hbm_budget: int, max_slots: int) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib.pycool_server_create(int(hbm_budget), int(max_slots), C.byref(h)),
           "pycool_server_create")
    return h


def pycool_server_submit(srv, cfg: pycool_config, ic: pycool_ic, seed: int, steps: int) -> int:
    t = C.c_uint64()
    _check(lib.pycool_server_submit(srv, C.byref(cfg), C.byref(ic), int(seed), int(steps),
                                    C.byref(t)), "pycool_server_submit")
    return t.value


def pycool_server_wait(srv, ticket: int, timeout_s: float = -1.0):
    """Returns (status, observables dict); does not raise on a run's status."""
    e = pycool_energies_t()
    st = lib.pycool_server_wait(srv, int(ticket), float(timeout_s), C.byref(e))
    return st, e


def pycool_server_stats(srv) -> dict:
    p50, p99, sus, n = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
    _check(lib.pycool_server_stats(srv, C.byref(p50), C.byref(p99), C.byref(sus), C.byref(n)),
           "pycool_server_stats")
    return dict(p50_s=p50.value, p99_s=p99.value, site_updates_per_s=sus.value,
                completed=n.value)


def pycool_server_destroy(srv) -> None:
    lib.pycool_server_destroy(srv)


def pycool_server_set_persistent_min_n(srv, min_n: int) -> None:
    """FP64 requests with side n % 32 == 0 and n >= min_n (0: none) run on the
    persistent kernel; applies to requests admitted after the call."""
    _check(lib.pycool_server_set_persistent_min_n(srv, int(min_n)),
           "pycool_server_set_persistent_min_n")


def pycool_server_cancel(srv, ticket: int) -> int:
    """Cancel a request; returns the status code (OK, E_NOT_FOUND, E_STATE)."""
    return lib.pycool_server_cancel(srv, int(ticket))


def pycool_debug_fail_alloc(count: int) -> int:
    """Fault injection: the next `count` device allocations of the library fail."""
    return lib.pycool_debug_fail_alloc(int(count))


def pycool_debug_barrier_stall(sim_handle, wait_limit_clocks: int) -> int:
    """Fault injection: the next persistent launch waits at an unreachable grid
    barrier with every wait limited to `wait_limit_clocks`; returns the status."""
    return lib.pycool_debug_barrier_stall(sim_handle, int(wait_limit_clocks))


def _is_field_tensor(t, numel: int) -> bool:
    """A contiguous float64 CUDA tensor of `numel` elements."""
    try:
        import torch
    except ImportError:  # pragma: no cover - torch is how callers pass device memory
        return False
    return (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous() and t.numel() == numel)


def pycool_noalloc_max_blocks() -> int:
    return int(lib.pycool_noalloc_max_blocks())


def pycool_sweep_noalloc(cfg: pycool_config, phi_in, pi_in, phi_out, pi_out, flush: bool,
                         state: pycool_stage_state, stream=None) -> int:
    """One stage sweep (flush=False) or synchronising flush (flush=True) with no
    device allocation; arrays are CUDA tensors.  Returns the status code.

    Each array must be a contiguous float64 CUDA tensor of N_f n^3 elements
    (pi_out may be None for a flush); anything else returns E_INVALID here,
    before the library is called, since the kernel would read or write past a
    shorter or differently typed buffer."""
    need = MODEL_NF.get(int(cfg.model), 0) * int(cfg.n) ** 3
    for t in (phi_in, pi_in, phi_out) + (() if flush and pi_out is None else (pi_out,)):
        if t is None or not _is_field_tensor(t, need):
            return E_INVALID
    ptr = lambda t: None if t is None else C.c_void_p(int(t.data_ptr()))  # noqa: E731
    return lib.pycool_sweep_noalloc(C.byref(cfg), ptr(phi_in), ptr(pi_in), ptr(phi_out),
                                    ptr(pi_out), 1 if flush else 0, C.byref(state),
                                    _stream_ptr(stream))


# ---------------------------------------------------------------- convenience wrapper

class Simulation:
    """A simulation as an object; each method is one C-ABI call."""

    def __init__(self, cfg: pycool_config, stream=None, dev_state=None, dev_workspace=None):
        self.cfg = cfg
        self.nf = MODEL_NF[cfg.model]
        self.n = cfg.n
        self.shape = (self.nf, cfg.n, cfg.n, cfg.n)
        self.handle = pycool_create(cfg, dev_state, dev_workspace, stream)

    def set_initial(self, phi, pi, on_device=False, a0=1.0, pa0=math.nan):
        pycool_set_initial(self.handle, phi, pi, on_device, a0, pa0)

    def evolve(self, steps):
        pycool_evolve(self.handle, steps)

    def sync(self, timeout_s=-1.0):
        return pycool_sync(self.handle, timeout_s)

    def energies(self):
        return pycool_energies(self.handle, self.nf)

    def field_stats(self, field):
        return pycool_field_stats(self.handle, field)

    def get_fields(self, phi=None, pi=None, on_device=False):
        return pycool_get_fields(self.handle, phi, pi, on_device, shape=self.shape)

    def checkpoint(self) -> bytes:
        return pycool_checkpoint_save(self.handle)

    def restore(self, blob: bytes):
        pycool_checkpoint_load(self.handle, blob)

    def kernel_launches(self) -> int:
        return pycool_kernel_launches(self.handle)

    def energy_fields(self, rho=None, P=None, on_device=False):
        return pycool_energy_fields(self.handle, self.shape[1:], rho, P, on_device)

    def spectrum(self, which: int, field: int):
        return pycool_spectrum(self.handle, self.n, which, field)

    def close(self):
        if self.handle:
            pycool_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
