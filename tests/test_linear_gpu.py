"""Growth functions of the linearised evolution on the GPU against the oracle.

pycool_linear_growth advances, for each distinct k_eff^2 of a lattice, the
2N_f x 2N_f transfer matrix of its Fourier modes with the background (Sec. 2.2,
Eq. Phik-1).  The oracle's ``transfer_matrices`` does the same in numpy; the
matrices and the final background must agree to 1e-11 (relative, per matrix,
and on a, p_a, phi0, pi0), as the FP64 lattice form does; and the matrices
applied to a lattice's initial modes must give the oracle's directly evolved
modes."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from oracle import pycool_linear as L  # noqa: E402
from oracle import pycool_oracle as O  # noqa: E402

TOL = 1e-11

CASES = [  # model, params, background, momentum, mpl, order, steps
    ("chaotic2", (1.0, 50.0), (1.0, 0.2), (-0.3, 0.1), 10.0, 4, 30),
    ("oscillon", (1.0, 1.0, 0.5), (0.8,), (0.0,), 10.0, 6, 20),
    ("qball", (1.0, -0.1, 1.0), (1.3, 0.4), (0.0, 0.2), 10.0, 8, 10),
    ("free", (0.7,), (0.5,), (0.1,), math.inf, 2, 200),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_growth_functions_match_oracle(case):
    model, p, bg, mom, mpl, order, steps = case
    n = 10
    cfg = O.LatticeConfig(n=n, L=8.0, model=model, params=p, dt=0.02, order=order, mpl=mpl)
    rng = np.random.default_rng(9)
    phi = np.stack([b + 1e-3 * rng.standard_normal((n, n, n)) for b in bg])
    pi = np.stack([m + 1e-3 * rng.standard_normal((n, n, n)) for m in mom])
    pa0 = 0.0 if math.isinf(mpl) else O.initial_pa(cfg, 1.0, phi, pi)
    ls = L.from_lattice(cfg, phi, pi, 1.0, pa0)
    vals, index = L.distinct_k2(L.k_eff2(n))
    T_o, bg_o = L.transfer_matrices(cfg, ls.a, ls.pa, ls.phi0, ls.pi0, vals, steps)

    gcfg = P.make_config(n=n, L=8.0, model=model, params=p, dt=0.02, order=order, mpl=mpl)
    T_g, (a, pa, f0, p0) = P.pycool_linear_growth(gcfg, ls.a, ls.pa, ls.phi0, ls.pi0, vals,
                                                  steps)
    err = np.max(np.abs(T_g - T_o), axis=(1, 2)) / np.max(np.abs(T_o), axis=(1, 2))
    print(f"\n{model}: {len(vals)} distinct k_eff^2, max rel err {err.max():.1e}, "
          f"a {abs(a - bg_o.a) / bg_o.a:.1e}")
    assert err.max() < TOL
    assert abs(a - bg_o.a) <= TOL * bg_o.a
    if pa0 != 0.0:
        assert abs(pa - bg_o.pa) <= TOL * abs(bg_o.pa)
    assert np.max(np.abs(f0 - bg_o.phi0)) <= TOL * max(1.0, np.max(np.abs(bg_o.phi0)))
    assert np.max(np.abs(p0 - bg_o.pi0)) <= TOL * max(1.0, np.max(np.abs(bg_o.pi0)))
    # the matrices reconstruct the directly evolved modes
    y0 = (ls.dphi.copy(), ls.dpi.copy())
    L.evolve(cfg, ls, steps)
    gphi, gpi = L.apply_transfer(T_g, index, *y0)
    for f in range(len(bg)):
        assert np.max(np.abs(gphi[f] - ls.dphi[f])) < TOL * np.max(np.abs(ls.dphi[f]))
        assert np.max(np.abs(gpi[f] - ls.dpi[f])) < TOL * np.max(np.abs(ls.dpi[f]))


def test_growth_rejects_bad_arguments():
    gcfg = P.make_config(n=8, L=8.0, model="chaotic2", params=(1.0, 50.0), dt=0.02, order=2)
    with pytest.raises(P.PycoolError) as ei:
        P.pycool_linear_growth(gcfg, -1.0, 0.0, (1.0, 0.0), (0.0, 0.0), [1.0], 3)
    assert ei.value.status == P.E_INVALID


LATTICE_CASES = [  # workload-like model, n, order, steps, mpl, stencil
    ("preheat128", 64, 4, 20, 1.0, "7pt"),
    ("oscillon256", 64, 6, 10, 100.0, "7pt"),
    ("qball256", 32, 8, 5, 100.0, "7pt"),
    ("preheat128", 32, 4, 10, 1.0, "4th"),
    ("oscillon256", 24, 2, 10, 100.0, "iso27"),
    ("preheat128", 32, 4, 10, 1.0, "7pt-physical"),
    ("oscillon256", 32, 6, 10, 1.0, "7pt-physical"),
]


@pytest.mark.parametrize("name,n,order,steps,mpl,stencil", LATTICE_CASES,
                         ids=[f"{c[0]}-{c[5]}" for c in LATTICE_CASES])
def test_linear_evolve_on_device_matches_oracle(name, n, order, steps, mpl, stencil):
    time_step = "physical" if stencil.endswith("-physical") else "conformal"
    stencil = stencil.split("-")[0]
    """pycool_linear_evolve (background, FFT, growth functions, per-mode
    apply, inverse FFT, all on the device) against the oracle's direct
    evolution of every mode, element by element on the lattice: the background
    to 1e-11, and the fields at the scale of their perturbations within
    gpu_helpers.fluct_tolerances for 3 log2(n) roundings (the transforms'
    levels; the output adds the perturbations to a float64 background, whose
    last bit is already 1e-16 / 1e-5 of a 1e-5 perturbation)."""
    torch = pytest.importorskip("torch")
    from paper_1201_5029_gb300 import inputs as I
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    cfg = O.LatticeConfig(n=n, L=w["L"], model=w["model"], params=w["params"], dt=w["dt"],
                          order=order, mpl=mpl, stencil=stencil, time_step=time_step)
    pa0 = O.initial_pa(cfg, 1.0, phi, pi)
    ls = L.from_lattice(cfg, phi, pi, 1.0, pa0)
    L.evolve(cfg, ls, steps)
    ophi, opi = L.to_lattice(ls)

    gcfg = P.make_config(n=n, L=w["L"], model=w["model"], params=w["params"], dt=w["dt"],
                         order=order, mpl=mpl, stencil=stencil, time_step=time_step)
    dphi, dpi = torch.from_numpy(phi).cuda(), torch.from_numpy(pi).cuda()
    outp, outq = torch.empty_like(dphi), torch.empty_like(dpi)
    a, pa, f0, p0 = P.pycool_linear_evolve(gcfg, 1.0, pa0, dphi, dpi, steps, outp, outq)
    gphi, gpi = outp.cpu().numpy(), outq.cpu().numpy()
    assert np.array_equal(dphi.cpu().numpy(), phi)          # inputs untouched
    assert abs(a - ls.a) <= TOL * ls.a and abs(pa - ls.pa) <= TOL * abs(ls.pa)
    assert np.max(np.abs(f0 - ls.phi0)) <= TOL * max(1.0, np.max(np.abs(ls.phi0)))
    import gpu_helpers as G
    levels = 3 * int(np.log2(n))
    for g, o in ((gphi, ophi), (gpi, opi)):
        fe, ft = G.fluct_errors(g, o), G.fluct_tolerances(o, levels, TOL)
        print(f"\n{name} n={n} {stencil} {time_step}: perturbation errors {['%.1e' % x for x in fe]} "
              f"bounds {['%.1e' % x for x in ft]}")
        assert all(e < t for e, t in zip(fe, ft)), (fe, ft)
