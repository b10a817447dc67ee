"""Plant typical mistakes in the linearised-evolution oracle (on the CPU) and
check that its pins catch each one: a wrong mass-matrix entry, a wrong k_eff^2
scale, a wrong power of a in a flow, a wrong p_a term, an unsymmetric stage."""
import math

import numpy as np
import pytest

from oracle import pycool_linear as L
from oracle import pycool_oracle as O
import test_linear_oracle as T


def _checks():
    out = {}
    # Hessian against difference quotients of V'
    ok = True
    for model, (p, x) in T.POINTS.items():
        x = np.array(x)
        M = L.mass_matrix(model, p, x)
        for j in range(len(x)):
            e = np.zeros_like(x)
            e[j] = 1e-6
            col = (O.potential_derivative(model, p, (x + e)[:, None])[:, 0]
                   - O.potential_derivative(model, p, (x - e)[:, None])[:, 0]) / 2e-6
            ok = ok and np.allclose(M[:, j], col, rtol=1e-7, atol=1e-7 * np.abs(M).max())
    out["hessian"] = ok
    # k_eff^2 closed form
    n = 8
    m = np.fft.fftfreq(n) * n
    s = 4.0 * np.sin(np.pi * m / n) ** 2
    out["keff2"] = np.max(np.abs(L.k_eff2(n) - (s[:, None, None] + s[None, :, None]
                                                + s[None, None, :]))) < 1e-13
    # background against a homogeneous lattice
    cfg = O.LatticeConfig(n=4, L=5.0, model="chaotic2", params=(1.0, 50.0), dt=0.02, order=4,
                          mpl=1.0)
    phi = np.stack([np.full((4, 4, 4), 0.9), np.full((4, 4, 4), 0.15)])
    pi = np.stack([np.full((4, 4, 4), -0.4), np.full((4, 4, 4), 0.05)])
    st = O.make_state(cfg, phi, pi)
    ls = L.from_lattice(cfg, phi, pi, st.a, st.pa)
    O.evolve(cfg, st, 30)
    L.evolve(cfg, ls, 30)
    out["background"] = (abs(ls.a - st.a) / st.a < 1e-13
                         and abs(ls.phi0[0] - st.phi[0, 0, 0, 0]) < 1e-13)
    # linearisation error second order
    e1, a1 = T._lin_vs_full(1e-4)
    e2, a2 = T._lin_vs_full(2e-4)
    out["linearisation"] = 1.8 < e2 / e1 < 2.2 and e1 < 2e-3 and 3.5 < a2 / a1 < 4.5
    # free field against exact stage matrices (order 4)
    try:
        T.test_free_field_modes_match_exact_stage_matrices(4)
        out["free"] = True
    except AssertionError:
        out["free"] = False
    # symplectic growth functions
    try:
        T.test_growth_functions_are_symplectic("chaotic2", (1.0, 0.2), (-0.3, 0.1))
        out["symplectic"] = True
    except AssertionError:
        out["symplectic"] = False
    return out


def _hess_offdiag_half(model, p, phi0):
    M = np.array(_ORIG["mass_matrix"](model, p, phi0), dtype=np.float64)
    if M.shape[0] == 2:
        M[0, 1] *= 0.5
        M[1, 0] *= 0.5
    else:
        M = M * 1.5
    return M


def _keff2_scaled(n, stencil="7pt"):
    return 1.01 * _ORIG["k_eff2"](n, stencil)


def _h3_a2_mass(cfg, s, h, k2, modes=True):
    a, dx2 = s.a, cfg.dx ** 2
    V = float(O.potential(cfg.model, cfg.params, s.phi0[:, None])[0])
    dV = O.potential_derivative(cfg.model, cfg.params, s.phi0[:, None])[:, 0]
    if modes:
        M = L.mass_matrix(cfg.model, cfg.params, s.phi0)
        kick = np.einsum("ij,j...->i...", a ** 2 * M, s.dphi) + (a * a / dx2) * k2 * s.dphi
        s.dpi = s.dpi - kick * h
    s.pa = s.pa - 4.0 * cfg.VL * a ** 3 * V * h
    s.pi0 = s.pi0 - a ** 4 * dV * h


def _h3_pa_3V(cfg, s, h, k2, modes=True):
    a, dx2 = s.a, cfg.dx ** 2
    V = float(O.potential(cfg.model, cfg.params, s.phi0[:, None])[0])
    dV = O.potential_derivative(cfg.model, cfg.params, s.phi0[:, None])[:, 0]
    if modes:
        M = L.mass_matrix(cfg.model, cfg.params, s.phi0)
        kick = np.einsum("ij,j...->i...", a ** 4 * M, s.dphi) + (a * a / dx2) * k2 * s.dphi
        s.dpi = s.dpi - kick * h
    s.pa = s.pa - 3.0 * cfg.VL * a ** 3 * V * h
    s.pi0 = s.pi0 - a ** 4 * dV * h


def _h2_drift_1_over_a(cfg, s, h, modes=True):
    a = s.a
    s.pa = s.pa + cfg.VL * (float(np.sum(s.pi0 * s.pi0)) / a ** 3 - cfg.rho_mat0) * h
    s.phi0 = s.phi0 + s.pi0 / a * h
    if modes:
        s.dphi = s.dphi + s.dpi / (a * a) * h


def _h2_modes_1_over_a(cfg, s, h, modes=True):
    a = s.a
    s.pa = s.pa + cfg.VL * (float(np.sum(s.pi0 * s.pi0)) / a ** 3 - cfg.rho_mat0) * h
    s.phi0 = s.phi0 + s.pi0 / (a * a) * h
    if modes:
        s.dphi = s.dphi + s.dpi / a * h


def _stage_unsymmetric(cfg, s, h, k2, modes=True):
    L._flow_H1(cfg, s, h)
    L._flow_H2(cfg, s, 0.5 * h, modes)
    L._flow_H3(cfg, s, h, k2, modes)
    L._flow_H2(cfg, s, 0.5 * h, modes)
    s.eta = s.eta + h


_ORIG = {"mass_matrix": L.mass_matrix, "k_eff2": L.k_eff2}

MUTATIONS = {
    "Hessian off-diagonal halved": ("mass_matrix", _hess_offdiag_half),
    "k_eff^2 scaled by 1.01": ("k_eff2", _keff2_scaled),
    "mode kick a^2 M instead of a^4 M": ("_flow_H3", _h3_a2_mass),
    "background p_a 3V instead of 4V": ("_flow_H3", _h3_pa_3V),
    "background drift 1/a instead of 1/a^2": ("_flow_H2", _h2_drift_1_over_a),
    "mode drift 1/a instead of 1/a^2": ("_flow_H2", _h2_modes_1_over_a),
    "stage not symmetric": ("_stage", _stage_unsymmetric),
}


def test_unmutated_linear_oracle_passes_every_check():
    bad = [k for k, ok in _checks().items() if not ok]
    assert not bad, bad


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_each_planted_mistake_fails_some_linear_pin(name, monkeypatch):
    attr, repl = MUTATIONS[name]
    monkeypatch.setattr(L, attr, repl)
    with np.errstate(all="ignore"):
        try:
            res = _checks()
        except (ValueError, FloatingPointError, OverflowError, ZeroDivisionError):
            return
    failed = [k for k, ok in res.items() if not ok]
    assert failed, f"planted mistake '{name}' passed every linear pin"
