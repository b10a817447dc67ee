"""Potentials given at run time (NVRTC) on the GPU against the oracle.

A model defined by C expressions runs the FP64 form through the library's
drift kernel, the compiled potential kernel and the library's stencil/kick
kernel.  It is held to the FP64 tolerances: the chaotic-preheating potential
written as expressions against the oracle's chaotic2, and a phi^4 potential
that is not compiled into the library against the oracle's phi4."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
import gpu_helpers as G  # noqa: E402

TOL = 1e-11

CHAOTIC = ("0.5*p[0]*f0*f0 + 0.5*p[1]*f0*f0*f1*f1",
           ("p[0]*f0 + p[1]*f0*f1*f1", "p[1]*f0*f0*f1"))
PHI4 = ("0.5*p[0]*f0*f0 + 0.25*p[1]*f0*f0*f0*f0", ("p[0]*f0 + p[1]*f0*f0*f0",))


def _check(gphi, gpi, ge, st, label):
    ef = G.field_errors(gphi, st.phi) + G.field_errors(gpi, st.pi)
    stages = int(ge["sweeps_done"]) + 1
    ff = G.fluct_errors(gphi, st.phi) + G.fluct_errors(gpi, st.pi)
    ft = G.fluct_tolerances(st.phi, stages, TOL) + G.fluct_tolerances(st.pi, stages, TOL)
    ea, epa = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa) if st.pa != 0 else 0.0
    print(f"\n{label}: fields {max(ef):.1e} a {ea:.1e} pa {epa:.1e} fluct {['%.1e' % x for x in ff]}")
    assert max(ef) < TOL and ea < TOL and epa < TOL
    assert all(e < t for e, t in zip(ff, ft)), (ff, ft)


@pytest.mark.parametrize("stencil,n,order,steps", [("7pt", 32, 4, 10), ("iso27", 20, 2, 30)])
def test_chaotic_potential_as_expressions(stencil, n, order, steps):
    mid = P.pycool_model_define(CHAOTIC[0], CHAOTIC[1])
    assert "p[1]*f0*f0*f1" in P.pycool_model_source(mid)
    w = I.workload("preheat32")
    phi, pi = I.initial_fields(w, n=n)
    cfg = P.make_config(n, w["L"], mid, w["params"], w["dt"], order=order, stencil=stencil,
                        mpl=w["mpl"])
    gphi, gpi, ge = G.run_gpu(P, cfg, phi, pi, steps, chunks=2)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=order, stencil=stencil), phi, pi, steps)
    _check(gphi, gpi, ge, st, f"runtime chaotic2 {stencil}")
    assert ge["rho"] == pytest.approx(oe["rho"], rel=1e-9)


@pytest.mark.parametrize("mpl", [1.0, math.inf])
def test_phi4_potential_not_compiled_in(mpl):
    mid = P.pycool_model_define(PHI4[0], PHI4[1])
    w = I.workload("oscillon256", model="phi4", params=(1.0, 0.5), L=20.0, dt=0.02)
    phi, pi = I.initial_fields(w, n=24)
    cfg = P.make_config(24, w["L"], mid, w["params"], w["dt"], order=6, mpl=mpl)
    gphi, gpi, ge = G.run_gpu(P, cfg, phi, pi, 8)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=24, order=6, mpl=mpl), phi, pi, 8)
    _check(gphi, gpi, ge, st, f"runtime phi4 mpl={mpl}")


def test_runtime_model_is_refused_where_unsupported():
    mid = P.pycool_model_define(PHI4[0], PHI4[1])
    w = I.workload("oscillon256")
    for kw in (dict(precision="split_fp32"), dict(precision="split_dd"), dict(stencil="4th")):
        cfg = P.make_config(32, 10.0, mid, (1.0, 0.5), 0.02, order=2, **kw)
        with pytest.raises(P.PycoolError) as ei:
            P.Simulation(cfg)
        assert ei.value.status == P.E_INVALID
    sim = P.Simulation(P.make_config(16, 10.0, mid, (1.0, 0.5), 0.02, order=2))
    sim.set_initial(*I.initial_fields(w, n=16))
    with pytest.raises(P.PycoolError):
        sim.energy_fields()
    pw, cnt = sim.spectrum(0, 0)          # spectra need no potential: available
    assert np.isfinite(pw).all() and cnt.sum() == 16 ** 3
    sim.close()
