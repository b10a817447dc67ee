"""Pins of the linearised-evolution oracle (Sec. 2.2), CPU only.

What fixes it, independently of its own formulas:
  - the mass matrix against central differences of the hand-written V' of the
    full oracle;
  - k_eff^2 against the closed form 4 sum sin^2(k dx/2) (7-point) and against
    the lattice Laplacian applied to a plane wave (27-point);
  - the background against the full lattice oracle on a homogeneous lattice
    (where the linearised equations are exact);
  - the linearisation itself: on an inhomogeneous lattice the linearised and
    full evolutions differ at second order in the perturbation amplitude, so
    their relative difference in the perturbation fields must halve with the
    amplitude and vanish with it (a wrong mass-matrix entry, k_eff^2 scale or
    power of a leaves a first-order difference that does not vanish);
  - a free field on a static background against the exact per-mode matrices
    of the second-order stage;
  - the growth functions (one transfer matrix per distinct k_eff^2) against the
    direct evolution of every mode, and their symplecticity T^T J T = J."""
import math

import numpy as np
import pytest

from oracle import pycool_linear as L
from oracle import pycool_oracle as O

POINTS = {"chaotic2": ((1.0, 50.0), (0.7, -0.3)),
          "oscillon": ((1.0, 1.0, 0.5), (0.8,)),
          "qball": ((1.0, -0.1, 1.0), (1.2, 0.4))}


@pytest.mark.parametrize("model", sorted(POINTS))
def test_mass_matrix_matches_difference_quotient(model):
    p, x = POINTS[model]
    x = np.array(x)
    M = L.mass_matrix(model, p, x)
    h = 1e-6
    for j in range(len(x)):
        e = np.zeros_like(x)
        e[j] = h
        col = (O.potential_derivative(model, p, (x + e)[:, None])[:, 0]
               - O.potential_derivative(model, p, (x - e)[:, None])[:, 0]) / (2 * h)
        assert np.allclose(M[:, j], col, rtol=1e-7, atol=1e-7 * np.abs(M).max())
    assert np.allclose(M, M.T, rtol=0, atol=0)


@pytest.mark.parametrize("n", [6, 8, 16])
def test_keff2_seven_point_closed_form(n):
    k2 = L.k_eff2(n, "7pt")
    m = np.fft.fftfreq(n) * n
    s = 4.0 * np.sin(np.pi * m / n) ** 2
    closed = s[:, None, None] + s[None, :, None] + s[None, None, :]
    assert np.max(np.abs(k2 - closed)) < 1e-13


@pytest.mark.parametrize("n", [6, 8, 16])
def test_keff2_fourth_order_closed_form(n):
    """Per axis (30 - 32 cos t + 2 cos 2t)/12 = (1 - cos t)(7 - cos t)/3
    = 4 sin^2(t/2) + (4/3) sin^4(t/2), t = k dx."""
    k2 = L.k_eff2(n, "4th")
    m = np.fft.fftfreq(n) * n
    s2 = np.sin(np.pi * m / n) ** 2
    s = 4.0 * s2 + 4.0 / 3.0 * s2 ** 2
    closed = s[:, None, None] + s[None, :, None] + s[None, None, :]
    assert np.max(np.abs(k2 - closed)) < 1e-13


@pytest.mark.parametrize("mode", [(1, 2, 3), (0, 4, 1), (3, 3, 3)])
def test_keff2_matches_lattice_laplacian(mode):
    n = 8
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    th = 2 * np.pi * (mode[0] * z + mode[1] * y + mode[2] * x) / n
    for stencil in ("7pt", "iso27", "4th"):
        f = np.cos(th)[None]
        D = O.laplacian(f, stencil)[0]
        k2 = L.k_eff2(n, stencil)[mode]
        assert np.max(np.abs(D + k2 * f[0])) < 1e-12


@pytest.mark.parametrize("time_step", ["conformal", "physical"])
def test_background_equals_homogeneous_lattice(time_step):
    """The linearised evolution's background is the homogeneous lattice's
    evolution, in either time variable (physical: d-eta = dt / a per step)."""
    cfg = O.LatticeConfig(n=4, L=5.0, model="chaotic2", params=(1.0, 50.0), dt=0.02, order=4,
                          mpl=1.0, time_step=time_step)
    phi = np.stack([np.full((4, 4, 4), 0.9), np.full((4, 4, 4), 0.15)])
    pi = np.stack([np.full((4, 4, 4), -0.4), np.full((4, 4, 4), 0.05)])
    st = O.make_state(cfg, phi, pi)
    ls = L.from_lattice(cfg, phi, pi, st.a, st.pa)
    O.evolve(cfg, st, 60)
    L.evolve(cfg, ls, 60)
    assert abs(ls.a - st.a) / st.a < 1e-13
    assert abs(ls.pa - st.pa) / abs(st.pa) < 1e-13
    for f in range(2):
        assert abs(ls.phi0[f] - st.phi[f, 0, 0, 0]) < 1e-13 * max(1.0, abs(st.phi[f, 0, 0, 0]))
        assert abs(ls.pi0[f] - st.pi[f, 0, 0, 0]) < 1e-13 * max(1.0, abs(st.pi[f, 0, 0, 0]))


def _lin_vs_full(eps, steps=40, n=12, time_step="conformal"):
    cfg = O.LatticeConfig(n=n, L=6.0, model="chaotic2", params=(1.0, 50.0), dt=0.02, order=4,
                          mpl=1.0, time_step=time_step)
    rng = np.random.default_rng(5)
    phi = np.stack([1.0 + eps * rng.standard_normal((n, n, n)),
                    0.2 + eps * rng.standard_normal((n, n, n))])
    pi = np.stack([-0.3 + eps * rng.standard_normal((n, n, n)),
                   0.1 + eps * rng.standard_normal((n, n, n))])
    st = O.make_state(cfg, phi, pi)
    ls = L.from_lattice(cfg, phi, pi, st.a, st.pa)
    O.evolve(cfg, st, steps)
    L.evolve(cfg, ls, steps)
    lphi, _ = L.to_lattice(ls)
    err = 0.0
    for f in range(2):
        dfull = st.phi[f] - np.mean(st.phi[f])
        dlin = lphi[f] - ls.phi0[f]
        err = max(err, float(np.max(np.abs(dfull - dlin)) / np.max(np.abs(dfull))))
    return err, abs(st.a - ls.a) / st.a


@pytest.mark.parametrize("time_step", ["conformal", "physical"])
def test_linearisation_error_is_second_order(time_step):
    e1, a1 = _lin_vs_full(1e-4, time_step=time_step)
    e2, a2 = _lin_vs_full(2e-4, time_step=time_step)
    # perturbation fields: relative difference first order in the amplitude
    assert 1.8 < e2 / e1 < 2.2
    assert e1 < 2e-3
    # scale factor: absolute difference second order (H^(2) is neglected)
    assert 3.5 < a2 / a1 < 4.5


@pytest.mark.parametrize("order", [2, 4, 6])
def test_free_field_modes_match_exact_stage_matrices(order):
    n, dt, m2, steps = 8, 0.05, 0.7, 200
    cfg = O.LatticeConfig(n=n, L=4.0, model="free", params=(m2,), dt=dt, order=order,
                          mpl=math.inf)
    rng = np.random.default_rng(2)
    phi = rng.standard_normal((1, n, n, n))
    pi = rng.standard_normal((1, n, n, n))
    ls = L.from_lattice(cfg, phi, pi, 1.0, 0.0)
    y0 = (ls.dphi[0].copy(), ls.dpi[0].copy())
    L.evolve(cfg, ls, steps)
    w2 = L.k_eff2(n) / cfg.dx ** 2 + m2
    # one stage with a = 1: drift h/2, kick -w^2 h, drift h/2 (exact flows)
    A = np.ones_like(w2)
    B = np.zeros_like(w2)
    Cm = np.zeros_like(w2)
    Dm = np.ones_like(w2)
    for w in O.stage_weights(order):
        h = w * dt
        # M_stage = [[1, h/2],[0, 1]] [[1, 0],[-w2 h, 1]] [[1, h/2],[0, 1]]
        s11 = 1.0 - w2 * h * h / 2
        s12 = h - w2 * h ** 3 / 4
        s21 = -w2 * h
        s22 = 1.0 - w2 * h * h / 2
        A, B, Cm, Dm = s11 * A + s12 * Cm, s11 * B + s12 * Dm, s21 * A + s22 * Cm, s21 * B + s22 * Dm
    P = [[A, B], [Cm, Dm]]
    # the step matrix to the power `steps`, per mode, by repeated squaring
    R = [[np.ones_like(w2), np.zeros_like(w2)], [np.zeros_like(w2), np.ones_like(w2)]]
    e = steps
    while e:
        if e & 1:
            R = [[R[0][0] * P[0][0] + R[0][1] * P[1][0], R[0][0] * P[0][1] + R[0][1] * P[1][1]],
                 [R[1][0] * P[0][0] + R[1][1] * P[1][0], R[1][0] * P[0][1] + R[1][1] * P[1][1]]]
        P = [[P[0][0] * P[0][0] + P[0][1] * P[1][0], P[0][0] * P[0][1] + P[0][1] * P[1][1]],
             [P[1][0] * P[0][0] + P[1][1] * P[1][0], P[1][0] * P[0][1] + P[1][1] * P[1][1]]]
        e >>= 1
    exp_phi = R[0][0] * y0[0] + R[0][1] * y0[1]
    exp_pi = R[1][0] * y0[0] + R[1][1] * y0[1]
    scale = np.max(np.abs(exp_phi))
    assert np.max(np.abs(ls.dphi[0] - exp_phi)) < 1e-11 * scale
    assert np.max(np.abs(ls.dpi[0] - exp_pi)) < 1e-11 * np.max(np.abs(exp_pi))


@pytest.mark.parametrize("model,bg,mom", [("chaotic2", (1.0, 0.2), (-0.3, 0.1)),
                                          ("oscillon", (0.8,), (0.0,)),
                                          ("qball", (1.3, 0.4), (0.0, 0.2))])
def test_growth_functions_reproduce_direct_evolution(model, bg, mom):
    n = 10
    p = POINTS[model][0]
    cfg = O.LatticeConfig(n=n, L=8.0, model=model, params=p, dt=0.02, order=4, mpl=10.0)
    rng = np.random.default_rng(9)
    nf = len(bg)
    phi = np.stack([b + 1e-3 * rng.standard_normal((n, n, n)) for b in bg])
    pi = np.stack([m + 1e-3 * rng.standard_normal((n, n, n)) for m in mom])
    pa0 = O.initial_pa(cfg, 1.0, phi, pi)
    ls = L.from_lattice(cfg, phi, pi, 1.0, pa0)
    y0 = (ls.dphi.copy(), ls.dpi.copy())
    vals, index = L.distinct_k2(L.k_eff2(n))
    assert len(vals) < n ** 3 // 10          # the grouping is what saves the work
    T, bgs = L.transfer_matrices(cfg, ls.a, ls.pa, ls.phi0, ls.pi0, vals, 30)
    L.evolve(cfg, ls, 30)
    gphi, gpi = L.apply_transfer(T, index, *y0)
    assert bgs.a == ls.a and bgs.pa == ls.pa
    for f in range(nf):
        assert np.max(np.abs(gphi[f] - ls.dphi[f])) < 1e-11 * np.max(np.abs(ls.dphi[f]))
        assert np.max(np.abs(gpi[f] - ls.dpi[f])) < 1e-11 * np.max(np.abs(ls.dpi[f]))


@pytest.mark.parametrize("model,bg,mom", [("chaotic2", (1.0, 0.2), (-0.3, 0.1)),
                                          ("qball", (1.3, 0.4), (0.0, 0.2))])
def test_growth_functions_are_symplectic(model, bg, mom):
    """Each sub-flow acts on (dPhi, dPi) as [[1, h/a^2], [0, 1]] or
    [[1, 0], [-h K, 1]] with K = k_eff^2 a^2/dx^2 + a^4 M symmetric, so every
    transfer matrix satisfies T^T J T = J (J the symplectic form): a fixed
    property that a misplaced block or an asymmetric mass matrix breaks."""
    n = 8
    p = POINTS[model][0]
    cfg = O.LatticeConfig(n=n, L=8.0, model=model, params=p, dt=0.02, order=6, mpl=10.0)
    nf = len(bg)
    vals, _ = L.distinct_k2(L.k_eff2(n))
    T, _ = L.transfer_matrices(cfg, 1.0, -50.0, np.array(bg), np.array(mom), vals, 40)
    J = np.block([[np.zeros((nf, nf)), np.eye(nf)], [-np.eye(nf), np.zeros((nf, nf))]])
    for t in T:
        err = np.max(np.abs(t.T @ J @ t - J)) / max(1.0, np.max(np.abs(t)) ** 2)
        assert err < 1e-13
