"""The fourth-order stencil on the GPU against the oracle.

The 13-point stencil (per axis (-1, 16, -30, 16, -1)/12) runs on the
persistent kernel in the FP64 and split-DD forms when n is a multiple of 32
(two halo rows, columns and planes; one launch per evolve), and on a
plain-load per-stage kernel in the FP64 form for other n and in the
split-FP32 form.  FP64 and split-DD: the tolerances of the other FP64 parity
tests (1e-11 normwise and the fluctuation-scale bound); split-FP32: its
float32 fluctuation accuracy (1e-4 of the fluctuation scale)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
import gpu_helpers as G  # noqa: E402

TOL = 1e-11


def _run(cfg, phi, pi, steps, chunks=1):
    """GPU run in `chunks` evolve calls; also the kernel launches they took."""
    sim = P.Simulation(cfg)
    sim.set_initial(phi, pi)
    before = sim.kernel_launches()
    per = [steps // chunks + (1 if i < steps % chunks else 0) for i in range(chunks)]
    for k in per:
        sim.evolve(k)
    e = sim.energies()
    launches = sim.kernel_launches() - before
    gphi, gpi = sim.get_fields()
    sim.close()
    return gphi, gpi, e, launches


@pytest.mark.parametrize("name,order,n,steps,persistent", [
    ("preheat32", 2, 32, 40, True),      # tiles at the y wrap only
    ("preheat128", 4, 64, 6, True),
    ("oscillon256", 6, 64, 4, True),     # two sites per lane
    ("qball256", 8, 96, 2, True),        # clear and wrap tiles, order 8
    ("preheat128", 4, 21, 6, False),     # ragged tiles: the per-stage kernel
    ("oscillon256", 6, 16, 5, False),
    ("qball256", 8, 12, 3, False),
    ("preheat32", 4, 4, 5, False),       # n = 4: the +-2 neighbours of a site coincide
])
def test_fourth_order_stencil_fp64(name, order, n, steps, persistent):
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    if name == "qball256":
        phi = phi + 1e-3 * np.random.default_rng(7).standard_normal(phi.shape)
    gphi, gpi, ge, launches = _run(G.gpu_cfg(P, w, n=n, order=order, stencil="4th"), phi, pi,
                                   steps, chunks=2)
    # the persistent kernel: one launch per evolve call
    assert (launches == 2) == persistent, launches
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=order, stencil="4th"), phi, pi, steps)
    ef = G.field_errors(gphi, st.phi) + G.field_errors(gpi, st.pi)
    stages = int(ge["sweeps_done"]) + 1
    ff = G.fluct_errors(gphi, st.phi) + G.fluct_errors(gpi, st.pi)
    ft = G.fluct_tolerances(st.phi, stages, TOL) + G.fluct_tolerances(st.pi, stages, TOL)
    ea, epa = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa)
    print(f"\n{name} n={n} 4th FP64: fields {max(ef):.1e} a {ea:.1e} pa {epa:.1e} "
          f"fluct {['%.1e' % x for x in ff]}")
    assert max(ef) < TOL and ea < TOL and epa < TOL
    assert all(e < t for e, t in zip(ff, ft)), (ff, ft)
    for k in ("rho", "P"):
        assert ge[k] == pytest.approx(oe[k], rel=1e-9), k


@pytest.mark.parametrize("name,order,n,steps", [("preheat128", 4, 32, 6), ("oscillon256", 6, 24, 4)])
def test_fourth_order_stencil_split(name, order, n, steps):
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=n, order=order, stencil="4th",
                                           precision="split_fp32"), phi, pi, steps)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=order, stencil="4th"), phi, pi, steps)
    fl = G.fluct_errors(gphi, st.phi)
    print(f"\n{name} n={n} 4th split: {fl}")
    assert max(fl) < 1e-4
    assert G.rel(ge["a"], st.a) < 1e-9 and G.rel(ge["rho"], oe["rho"]) < 1e-7


@pytest.mark.parametrize("name,order,n,steps", [
    ("preheat32", 2, 32, 30),
    ("preheat128", 4, 64, 5),
    ("oscillon256", 6, 64, 4),   # two sites per lane
    ("qball256", 8, 64, 2),
])
def test_fourth_order_stencil_split_dd(name, order, n, steps):
    """The split-DD form on the persistent 13-point kernel, held to the FP64
    tolerances like the form's other tests."""
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    gphi, gpi, ge, launches = _run(G.gpu_cfg(P, w, n=n, order=order, stencil="4th",
                                             precision="split_dd"), phi, pi, steps, chunks=2)
    assert launches == 2, launches
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=order, stencil="4th"), phi, pi, steps)
    ef = G.field_errors(gphi, st.phi) + G.field_errors(gpi, st.pi)
    stages = int(ge["sweeps_done"]) + 1
    ff = G.fluct_errors(gphi, st.phi) + G.fluct_errors(gpi, st.pi)
    ft = G.fluct_tolerances(st.phi, stages, TOL) + G.fluct_tolerances(st.pi, stages, TOL)
    ea, epa = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa)
    print(f"\n{name} n={n} 4th split-DD: fields {max(ef):.1e} a {ea:.1e} pa {epa:.1e} "
          f"fluct {['%.1e' % x for x in ff]} bound {['%.1e' % x for x in ft]}")
    assert max(ef) < TOL and ea < TOL and epa < TOL
    assert all(e < t for e, t in zip(ff, ft)), (ff, ft)
    for k in ("rho", "P"):
        assert ge[k] == pytest.approx(oe[k], rel=1e-9), k


def test_fourth_order_stencil_rejected_where_it_has_no_kernel():
    """split-DD runs on the persistent kernel only: n a multiple of 32."""
    w = I.workload("preheat32")
    with pytest.raises(P.PycoolError) as ei:
        P.Simulation(G.gpu_cfg(P, w, n=24, stencil="4th", precision="split_dd"))
    assert ei.value.status == P.E_INVALID
