"""Split-DD form against the CPU oracle (GPU).

The split-DD form keeps the float64 lattice mean as the background and the
fluctuations as double-float pairs (~48-bit significands), with all bulk
arithmetic on the FP32 pipe.  Its claim is float64-class accuracy, so it is
held to the FP64 form's tolerances: 1e-11 relative per field (normwise), on a
and p_a, and the fluctuation-scale bound of gpu_helpers.fluct_tolerances.
The form runs on the persistent kernel, so every lattice side here is a
multiple of 32."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
import gpu_helpers as G  # noqa: E402

TOL = 1e-11


def check(gphi, gpi, ge, st, oe, tol=TOL, label=""):
    ef = G.field_errors(gphi, st.phi)
    ep = G.field_errors(gpi, st.pi)
    ea, epa = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa)
    stages = int(ge["sweeps_done"]) + 1
    ff = G.fluct_errors(gphi, st.phi) + G.fluct_errors(gpi, st.pi)
    ft = G.fluct_tolerances(st.phi, stages, tol) + G.fluct_tolerances(st.pi, stages, tol)
    print(f"\n{label} dd: phi {['%.1e' % x for x in ef]} pi {['%.1e' % x for x in ep]} "
          f"a {ea:.1e} pa {epa:.1e} fluct {['%.1e' % x for x in ff]} "
          f"bound {['%.1e' % x for x in ft]}")
    assert max(ef) < tol and max(ep) < tol, (ef, ep)
    assert ea < tol and epa < tol, (ea, epa)
    assert all(e < t for e, t in zip(ff, ft)), (ff, ft)
    assert ge["eta"] == pytest.approx(st.eta, rel=1e-13)


def test_preheat32_leapfrog_100_steps():
    w = I.workload("preheat32")
    phi, pi = I.initial_fields(w)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, precision="split_dd"), phi, pi, w["steps"])
    st, oe = G.run_oracle(G.oracle_cfg(w), phi, pi, w["steps"])
    check(gphi, gpi, ge, st, oe, label="preheat32")
    for k in ("rho", "P", "residual"):
        assert ge[k] == pytest.approx(oe[k], rel=1e-9, abs=1e-13), k
    for f in range(2):
        assert ge["rho_kin"][f] == pytest.approx(oe["rho_kin"][f], rel=1e-10)
        assert ge["rho_grad"][f] == pytest.approx(oe["rho_grad"][f], rel=1e-9)
        assert ge["variance"][f] == pytest.approx(np.var(st.phi[f]), rel=1e-9)


@pytest.mark.parametrize("name,order,n,steps", [
    ("preheat128", 4, 64, 12),
    ("oscillon256", 6, 64, 8),
    ("qball256", 8, 64, 4),
    ("preheat128", 8, 32, 6),
    ("oscillon256", 2, 96, 10),
])
@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
def test_models_orders_stencils(name, order, n, steps, stencil):
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    if name == "qball256":
        phi = phi + 1e-3 * np.random.default_rng(7).standard_normal(phi.shape)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=n, order=order, stencil=stencil,
                                           precision="split_dd"), phi, pi, steps)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=order, stencil=stencil), phi, pi, steps)
    check(gphi, gpi, ge, st, oe, label=f"{name} n={n} {stencil}")


def test_free_field_static_background_and_evolve_chunks():
    w = I.workload("oscillon256", model="free", params=(1.0,), mpl=float("inf"))
    phi, pi = I.initial_fields(w, n=32)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=32, order=4, precision="split_dd"), phi, pi,
                              9, chunks=3)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=32, order=4), phi, pi, 9)
    check(gphi, gpi, ge, st, oe, label="free static")


def test_bitwise_reproducible_and_checkpoint_resume():
    w = I.workload("preheat32")
    phi, pi = I.initial_fields(w, n=32)
    cfg = G.gpu_cfg(P, w, n=32, order=4, precision="split_dd")
    outs = []
    for _ in range(2):
        s = P.Simulation(cfg)
        s.set_initial(phi, pi)
        s.evolve(7)
        blob = s.checkpoint()
        s.evolve(5)
        outs.append((s.get_fields(), s.energies(), blob))
        s.close()
    (f1, e1, b1), (f2, e2, b2) = outs
    assert np.array_equal(f1[0], f2[0]) and np.array_equal(f1[1], f2[1]) and b1 == b2
    r = P.Simulation(cfg)
    r.set_initial(phi, pi)
    r.restore(b1)
    r.evolve(5)
    fr = r.get_fields()
    assert np.array_equal(fr[0], f1[0]) and np.array_equal(fr[1], f1[1])
    assert r.energies()["a"] == e1["a"]
    r.close()


def test_rejected_where_it_has_no_kernel():
    w = I.workload("preheat32")
    with pytest.raises(P.PycoolError) as ei:
        P.Simulation(G.gpu_cfg(P, w, n=40, precision="split_dd"))   # not a multiple of 32
    assert ei.value.status == P.E_INVALID


@pytest.mark.parametrize("amp", [1e-6, 1e-3, 0.2])
def test_qball_log1p_tiers(amp):
    """The split-DD Q-ball takes log1p of a double-float by its Taylor series
    within 2^-12, by the atanh series within 2^-5 and in float64 beyond:
    fluctuations of 1e-6, 1e-3 and 0.2 exercise each tier."""
    w = I.workload("qball256")
    phi, pi = I.initial_fields(w, n=64)
    phi = phi + amp * np.random.default_rng(11).standard_normal(phi.shape)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=64, order=4, precision="split_dd"), phi, pi, 3)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=64, order=4), phi, pi, 3)
    check(gphi, gpi, ge, st, oe, label=f"qball amp={amp}")
