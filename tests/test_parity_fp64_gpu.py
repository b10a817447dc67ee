"""FP64 CUDA path against the CPU oracle, element by element (GPU).

Tolerance: 1e-11 relative (per field, max|gpu - oracle| / max|oracle|; and
relative on a, p_a) over the stated number of steps; and, at the scale of the
fluctuations (max|gpu - oracle| / max|oracle - mean(oracle)|), the bound of
gpu_helpers.fluct_tolerances: 40 float64 roundings at the field's magnitude
per stage, relative to the fluctuations (never below 1e-11).  The two sides differ only
in rounding order (the GPU merges the drifts of neighbouring half-stages and
sums in a fixed blocked order; the oracle applies each flow separately and
sums with correct rounding)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
from oracle import pycool_oracle as O  # noqa: E402
import gpu_helpers as G  # noqa: E402

TOL = 1e-11


def _check(gphi, gpi, ge, st, oe, tol=TOL):
    ef = G.field_errors(gphi, st.phi)
    ep = G.field_errors(gpi, st.pi)
    ea, epa = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa)
    assert max(ef) < tol, ("phi", ef)
    assert max(ep) < tol, ("pi", ep)
    assert ea < tol and epa < tol, (ea, epa)
    assert ge["eta"] == pytest.approx(st.eta, rel=1e-13)
    # the fluctuations about each field's mean, at their own scale
    stages = int(ge["sweeps_done"]) + 1
    for name, g, o in (("phi", gphi, st.phi), ("pi", gpi, st.pi)):
        fe = G.fluct_errors(g, o)
        ft = G.fluct_tolerances(o, stages, tol)
        print(f"\nfluct {name}: err {['%.2e' % x for x in fe]} bound {['%.2e' % x for x in ft]} "
              f"({stages} stages)")
        assert all(e < t for e, t in zip(fe, ft)), (name, fe, ft)
    return max(ef + ep + [ea, epa])


def test_preheat32_leapfrog_100_steps():
    """The 32^3 two-field preheating workload, full length (100 leapfrog steps)."""
    w = I.workload("preheat32")
    phi, pi = I.initial_fields(w)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w), phi, pi, w["steps"])
    st, oe = G.run_oracle(G.oracle_cfg(w), phi, pi, w["steps"])
    _check(gphi, gpi, ge, st, oe)
    for k in ("rho", "P", "residual"):
        assert ge[k] == pytest.approx(oe[k], rel=1e-9, abs=1e-13), k
    for f in range(2):
        assert ge["rho_kin"][f] == pytest.approx(oe["rho_kin"][f], rel=1e-10)
        assert ge["rho_grad"][f] == pytest.approx(oe["rho_grad"][f], rel=1e-9)
    assert ge["steps_done"] == w["steps"]


@pytest.mark.parametrize("name,order,n,steps", [
    ("preheat128", 4, 38, 12),     # ragged in x, y and z
    ("oscillon256", 6, 20, 8),
    ("qball256", 8, 17, 4),
    ("preheat128", 8, 9, 6),
])
@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
def test_models_orders_stencils_small(name, order, n, steps, stencil):
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    if name == "qball256":
        phi = phi + 1e-3 * np.random.default_rng(7).standard_normal(phi.shape)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=n, order=order, stencil=stencil), phi, pi, steps)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=order, stencil=stencil), phi, pi, steps)
    _check(gphi, gpi, ge, st, oe)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 31, 33])
def test_degenerate_and_edge_sizes(n):
    """Lattices where every stencil index wraps (n <= 3) and sizes around a tile edge."""
    w = I.workload("preheat32", L=5.0)
    phi, pi = I.initial_fields(w, n=n)
    phi = phi + 0.01 * np.random.default_rng(n).standard_normal(phi.shape)
    for stencil in ("7pt", "iso27"):
        gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=n, order=4, stencil=stencil, dt=0.002),
                                  phi, pi, 5)
        st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=4, stencil=stencil, dt=0.002), phi, pi, 5)
        _check(gphi, gpi, ge, st, oe)


def test_static_background_and_matter_radiation_terms():
    w = I.workload("oscillon256", rho_rad0=0.3, rho_mat0=0.2, mpl=2.0)
    phi, pi = I.initial_fields(w, n=12)
    for mpl in (2.0, math.inf):
        gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=12, order=4, mpl=mpl), phi, pi, 10, a0=1.3)
        st, oe = G.run_oracle(G.oracle_cfg(w, n=12, order=4, mpl=mpl), phi, pi, 10, a0=1.3)
        _check(gphi, gpi, ge, st, oe)


def test_evolve_in_chunks_matches_oracle():
    """Several evolve() calls (each ends with the synchronising flush)."""
    w = I.workload("preheat32")
    phi, pi = I.initial_fields(w, n=16)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=16, order=6), phi, pi, 9, chunks=4)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=16, order=6), phi, pi, 9)
    _check(gphi, gpi, ge, st, oe)
    assert ge["steps_done"] == 9


def test_given_pa_and_time_reversal():
    """Forward with dt, back with -dt from the checkpoint: returns to the start."""
    w = I.workload("preheat32")
    phi, pi = I.initial_fields(w, n=16)
    fwd = P.Simulation(G.gpu_cfg(P, w, n=16, order=4))
    fwd.set_initial(phi, pi)
    e0 = fwd.energies()
    fwd.evolve(40)
    blob = fwd.checkpoint()
    back = P.Simulation(G.gpu_cfg(P, w, n=16, order=4, dt=-w["dt"]))
    back.set_initial(phi, pi, pa0=e0["pa"])  # any fields; the checkpoint replaces them
    back.restore(blob)
    back.evolve(40)
    bphi, bpi = back.get_fields()
    e1 = back.energies()
    assert max(G.field_errors(bphi, phi)) < 1e-10
    assert max(G.field_errors(bpi, pi)) < 1e-10
    assert G.rel(e1["a"], 1.0) < 1e-12 and G.rel(e1["pa"], e0["pa"]) < 1e-10
    assert abs(e1["eta"]) < 1e-12


def test_device_resident_inputs_and_outputs():
    torch = pytest.importorskip("torch")
    w = I.workload("preheat32")
    phi, pi = I.initial_fields(w, n=24)
    dphi = torch.from_numpy(phi).cuda()
    dpi = torch.from_numpy(pi).cuda()
    state_b, ws_b = P.pycool_query_bytes(G.gpu_cfg(P, w, n=24))
    state = torch.empty(state_b, dtype=torch.uint8, device="cuda")
    ws = torch.empty(ws_b, dtype=torch.uint8, device="cuda")
    sim = P.Simulation(G.gpu_cfg(P, w, n=24), stream=torch.cuda.current_stream(),
                       dev_state=state.data_ptr(), dev_workspace=ws.data_ptr())
    sim.set_initial(dphi, dpi, on_device=True)
    sim.evolve(10)
    out_phi = torch.empty_like(dphi)
    out_pi = torch.empty_like(dpi)
    sim.get_fields(out_phi, out_pi, on_device=True)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=24), phi, pi, 10)
    assert max(G.field_errors(out_phi.cpu().numpy(), st.phi)) < TOL
    assert max(G.field_errors(out_pi.cpu().numpy(), st.pi)) < TOL
    sim.close()


def test_bitwise_reproducible_and_checkpoint_resume():
    w = I.workload("preheat32")
    phi, pi = I.initial_fields(w, n=20)
    cfg = G.gpu_cfg(P, w, n=20, order=4)
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
    assert np.array_equal(f1[0], f2[0]) and np.array_equal(f1[1], f2[1])
    assert e1["a"] == e2["a"] and e1["pa"] == e2["pa"] and b1 == b2
    r = P.Simulation(cfg)
    r.set_initial(phi, pi)
    r.restore(b1)
    r.evolve(5)
    fr = r.get_fields()
    er = r.energies()
    assert np.array_equal(fr[0], f1[0]) and np.array_equal(fr[1], f1[1])
    assert er["a"] == e1["a"] and er["pa"] == e1["pa"]
    r.close()


def test_nonfinite_is_detected_and_latched():
    w = I.workload("oscillon256")
    phi, pi = I.initial_fields(w, n=8)
    s = P.Simulation(G.gpu_cfg(P, w, n=8, order=2))
    s.set_initial(phi * 1e60, pi)  # V ~ phi^6 overflows
    assert s.sync() == P.E_NONFINITE
    with pytest.raises(P.PycoolError) as ei:
        s.energies()
    assert ei.value.status == P.E_NONFINITE
    s.evolve(3)  # a stopped simulation stays stopped
    assert s.sync() == P.E_NONFINITE
    s.close()


def test_invalid_configs_rejected():
    w = I.workload("preheat32")
    for bad in (dict(n=0), dict(order=3), dict(dt=0.0), dict(L=-1.0)):
        ww = dict(w)
        ww.update(bad)
        with pytest.raises(P.PycoolError) as ei:
            P.Simulation(G.gpu_cfg(P, ww))
        assert ei.value.status == P.E_INVALID
    with pytest.raises(P.PycoolError) as ei:
        P.Simulation(G.gpu_cfg(P, w, dt=1.0))
    assert ei.value.status == P.E_UNSTABLE_DT


@pytest.mark.parametrize("name,n,order,steps", [
    ("oscillon256", 64, 6, 3),    # TMA kernel, 2 sites per lane (double2)
    ("preheat128", 64, 4, 4),     # TMA kernel, 1 site per lane, 2 fields
    ("qball256", 64, 8, 2),
    ("oscillon256", 96, 2, 5),    # TMA kernel, 96 = 3 x 32
])
@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
def test_tma_kernel_sizes(name, n, order, steps, stencil):
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=n, order=order, stencil=stencil), phi, pi, steps)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=order, stencil=stencil), phi, pi, steps)
    _check(gphi, gpi, ge, st, oe)


@pytest.mark.parametrize("amp", [1e-6, 1e-3, 0.2])
def test_qball_logarithm_near_reference_all_branches(amp):
    """The FP64 Q-ball takes ln|Phi|^2 as ln(u_ref) + a log1p series when the
    site is close to the stage's reference value (5 terms within 2^-12, 11
    terms within 2^-5) and the full logarithm farther away: fluctuations of
    1e-6, 1e-3 and 0.2 exercise each branch (the TMA kernel at n = 64, the
    persistent kernel, and the plain-load kernel at n = 20)."""
    w = I.workload("qball256")
    for n in (64, 20):
        phi, pi = I.initial_fields(w, n=n)
        phi = phi + amp * np.random.default_rng(11).standard_normal(phi.shape)
        gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=n, order=4), phi, pi, 3)
        st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=4), phi, pi, 3)
        _check(gphi, gpi, ge, st, oe)
