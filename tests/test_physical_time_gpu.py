"""Physical-time steps (the adaptive conformal step of Sec. 3.1) on the GPU.

With time_step = physical each time step takes d-eta = dt / a_n (a_n at the
synchronised state that starts the step).  Here:
  - the FP64 and split-DD forms match the oracle's physical-time steps at the
    FP64 tolerances (1e-11 normwise and at the scale of the fluctuations);
  - the oscillon and Q-ball workloads at m_pl = 1, whose conformal-time runs
    overflow within their step counts (the a m stability wall of conformal
    time), run their full step counts in physical time on a 32^3 lattice with
    finite energies and a small Friedmann residual."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
import gpu_helpers as G  # noqa: E402

TOL = 1e-11


@pytest.mark.parametrize("name,order,n,steps", [
    ("preheat32", 2, 32, 60),
    ("oscillon256", 6, 32, 30),
    ("qball256", 8, 32, 8),
])
@pytest.mark.parametrize("precision", ["fp64", "split_dd"])
def test_physical_steps_match_oracle(name, order, n, steps, precision):
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=n, order=order, mpl=1.0, precision=precision,
                                           time_step="physical"), phi, pi, steps)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=order, mpl=1.0, time_step="physical"),
                          phi, pi, steps)
    ef = G.field_errors(gphi, st.phi) + G.field_errors(gpi, st.pi)
    stages = int(ge["sweeps_done"]) + 1
    ff = G.fluct_errors(gphi, st.phi) + G.fluct_errors(gpi, st.pi)
    ft = G.fluct_tolerances(st.phi, stages, TOL) + G.fluct_tolerances(st.pi, stages, TOL)
    ea, epa, eeta = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa), G.rel(ge["eta"], st.eta)
    print(f"\n{name} {precision} physical: fields {max(ef):.1e} a {ea:.1e} pa {epa:.1e} "
          f"eta {eeta:.1e} (a_end {st.a:.4f}) fluct {['%.1e' % x for x in ff]}")
    assert max(ef) < TOL and ea < TOL and epa < TOL and eeta < TOL
    assert all(e < t for e, t in zip(ff, ft)), (ff, ft)


@pytest.mark.parametrize("name", ["oscillon256", "qball256"])
def test_mpl1_workloads_run_their_length_in_physical_time(name):
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=32)
    conf = P.Simulation(G.gpu_cfg(P, w, n=32, mpl=1.0))
    conf.set_initial(phi, pi)
    conf.evolve(w["steps"])
    assert conf.sync() == P.E_NONFINITE          # the conformal-time run overflows
    conf.close()
    for precision in ("fp64", "split_dd"):
        sim = P.Simulation(G.gpu_cfg(P, w, n=32, mpl=1.0, precision=precision,
                                     time_step="physical"))
        sim.set_initial(phi, pi)
        sim.evolve(w["steps"])
        assert sim.sync() == P.OK
        e = sim.energies()
        print(f"\n{name} {precision}: {e['steps_done']} physical-time steps, a = {e['a']:.3f}, "
              f"eta = {e['eta']:.3f}, residual {e['residual']:.1e}")
        assert e["steps_done"] == w["steps"] and np.isfinite(e["rho"]) and e["a"] > 1.0
        assert e["residual"] < 1e-3
        sim.close()
