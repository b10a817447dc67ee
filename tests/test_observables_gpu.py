"""Output-interval observables on the GPU against the observables oracle.

pycool_energy_fields (rho(x), P(x) of Eq. rho-pres with the stencil G of Eq.
G) and pycool_spectrum (shell-binned power spectrum, Sec. 2.4) at the state a
few steps into the preheating, oscillon and Q-ball workloads, for each form.
Each side evaluates the observables on its own evolved state, so the
difference carries the states' difference: for the FP64 and split-DD forms the
per-site fields agree at the scale of their fluctuations within the state
parity bound (gpu_helpers.fluct_tolerances for the stages run, never below
1e-10) and the shells (relative to the total power, which is the lattice mean
of the field squared) to 1e-10; the split-FP32 form at its float32
fluctuation accuracy, 1e-4 of the same scales."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
from oracle import pycool_observables as B  # noqa: E402
import gpu_helpers as G  # noqa: E402

CASES = [("preheat128", 4, 32, 5, "7pt"), ("oscillon256", 6, 64, 3, "iso27"),
         ("qball256", 8, 32, 2, "7pt"), ("preheat128", 4, 32, 4, "4th")]


@pytest.fixture(scope="module", params=CASES, ids=[f"{c[0]}-{c[4]}" for c in CASES])
def case(request):
    name, order, n, steps, stencil = request.param
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    ocfg = G.oracle_cfg(w, n=n, order=order, stencil=stencil)
    st, oe = G.run_oracle(ocfg, phi, pi, steps)
    rho, Pp = B.energy_fields(ocfg, st)
    spec = [[B.spectrum(arr[f]) for f in range(phi.shape[0])] for arr in (st.phi, st.pi)]
    return dict(w=w, n=n, order=order, steps=steps, stencil=stencil, phi=phi, pi=pi, st=st,
                rho=rho, P=Pp, spec=spec, oe=oe)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("split_dd", 1e-10),
                                           ("split_fp32", 1e-4)])
def test_energy_fields_and_spectra(case, precision, tol):
    w, n = case["w"], case["n"]
    sim = P.Simulation(G.gpu_cfg(P, w, n=n, order=case["order"], stencil=case["stencil"],
                                 precision=precision))
    sim.set_initial(case["phi"], case["pi"])
    sim.evolve(case["steps"])
    rho, Pg = sim.energy_fields()
    # the fluctuating parts (rho - <rho>) at their own scale, and the means
    stages = int(sim.energies()["sweeps_done"]) + 1
    for g, o in ((rho, case["rho"]), (Pg, case["P"])):
        scale = np.max(np.abs(o - o.mean()))
        err = np.max(np.abs(g - o)) / scale
        bound = max(tol, G.fluct_tolerances(o[None], stages, tol)[0]) if tol < 1e-6 else tol
        print(f"\n{w['model']} {precision}: field error {err:.1e} of fluctuation scale "
              f"{scale:.1e} (bound {bound:.1e})")
        assert err < bound
    e = sim.energies()
    assert abs(rho.mean() - e["rho"]) <= 1e-12 * abs(e["rho"]) + 1e-14 * np.max(np.abs(rho))
    for which in (0, 1):
        for f in range(case["phi"].shape[0]):
            pw, cnt = sim.spectrum(which, f)
            po, co = case["spec"][which][f]
            # a spectrum is quadratic in the field: twice the field's bound
            arr = (case["st"].phi, case["st"].pi)[which][f][None]
            sb = max(tol, 2 * G.fluct_tolerances(arr, stages, tol)[0]) if tol < 1e-6 else tol
            assert np.array_equal(cnt, co)
            # shell 0 (the mean squared) against the total power; the other
            # shells (the fluctuations) against their largest
            e0 = abs(pw[0] - po[0]) / po.sum()
            e1 = np.max(np.abs(pw[1:] - po[1:])) / np.max(po[1:])
            print(f"  spectrum which={which} f={f}: shell0 {e0:.1e} shells {e1:.1e} "
                  f"(bound {sb:.1e})")
            assert e0 < sb and e1 < sb
    sim.close()


def test_energy_fields_on_device_and_bitwise_spectrum():
    torch = pytest.importorskip("torch")
    w = I.workload("preheat32")
    phi, pi = I.initial_fields(w, n=32)
    sim = P.Simulation(G.gpu_cfg(P, w, n=32))
    sim.set_initial(phi, pi)
    sim.evolve(3)
    r = torch.empty((32, 32, 32), dtype=torch.float64, device="cuda")
    q = torch.empty_like(r)
    sim.energy_fields(r, q, on_device=True)
    hr, hq = sim.energy_fields()
    assert np.array_equal(r.cpu().numpy(), hr) and np.array_equal(q.cpu().numpy(), hq)
    a, _ = sim.spectrum(0, 1)
    b, _ = sim.spectrum(0, 1)
    assert np.array_equal(a, b)
    sim.close()
