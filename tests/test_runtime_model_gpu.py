"""Potentials given at run time (NVRTC) on the GPU against the oracle.

A model defined by C expressions runs the FP64 form through the library's
drift kernel, the compiled potential kernel and the library's stencil/kick
kernel.  It is held to the FP64 tolerances: the chaotic-preheating potential
written as expressions against the oracle's chaotic2 (with every stencil, and
its per-site energy fields), and a phi^4 potential that is not compiled into
the library against the oracle's phi4."""
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


@pytest.mark.parametrize("stencil,n,order,steps", [("7pt", 32, 4, 10), ("iso27", 20, 2, 30),
                                                   ("4th", 24, 4, 8)])
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
    for kw in (dict(precision="split_fp32"), dict(precision="split_dd")):
        cfg = P.make_config(32, 10.0, mid, (1.0, 0.5), 0.02, order=2, **kw)
        with pytest.raises(P.PycoolError) as ei:
            P.Simulation(cfg)
        assert ei.value.status == P.E_INVALID
    sim = P.Simulation(P.make_config(16, 10.0, mid, (1.0, 0.5), 0.02, order=2))
    sim.set_initial(*I.initial_fields(w, n=16))
    pw, cnt = sim.spectrum(0, 0)
    assert np.isfinite(pw).all() and cnt.sum() == 16 ** 3


@pytest.mark.parametrize("stencil", ["7pt", "4th"])
def test_energy_fields_of_a_runtime_potential(stencil):
    """rho(x), P(x) with V from the compiled kernel (run on the current state)
    against the observables oracle on its own evolved state, at the state
    parity bound of the FP64 form."""
    from oracle import pycool_observables as B
    mid = P.pycool_model_define(CHAOTIC[0], CHAOTIC[1])
    w = I.workload("preheat32")
    n, order, steps = 32, 4, 5
    phi, pi = I.initial_fields(w, n=n)
    ocfg = G.oracle_cfg(w, n=n, order=order, stencil=stencil)
    st, oe = G.run_oracle(ocfg, phi, pi, steps)
    rho_o, P_o = B.energy_fields(ocfg, st)
    with P.Simulation(P.make_config(n, w["L"], mid, w["params"], w["dt"], order=order,
                                    stencil=stencil, mpl=w["mpl"])) as sim:
        sim.set_initial(phi, pi)
        sim.evolve(steps)
        rho, Pg = sim.energy_fields()
        e = sim.energies()
    stages = int(e["sweeps_done"]) + 1
    for g, o in ((rho, rho_o), (Pg, P_o)):
        scale = np.max(np.abs(o - o.mean()))
        err = np.max(np.abs(g - o)) / scale
        bound = max(1e-10, G.fluct_tolerances(o[None], stages, 1e-10)[0])
        print(f"\nruntime chaotic2 {stencil}: field error {err:.1e} of scale {scale:.1e} "
              f"(bound {bound:.1e})")
        assert err < bound
    assert abs(rho.mean() - e["rho"]) <= 1e-12 * abs(e["rho"]) + 1e-14 * np.max(np.abs(rho))
    sim.close()
