"""Plant typical mistakes in the oracle (on the CPU) and check that the pins
catch each one: a dropped term, a wrong sign, a wrong power of a, a wrong
stencil weight, a wrong coefficient order."""
import math

import numpy as np
import pytest

from oracle import pycool_oracle as O
import oracle_pins as P


def _mut_H1_sign(cfg, s, h):
    s.a = s.a + s.pa * cfg.inv_6VLm2 * h


def _mut_H2_drift_power(cfg, s, h):
    a = s.a
    sum_pi2 = O.lattice_sum(s.pi * s.pi)
    pa_new = s.pa + (a ** 3 * sum_pi2 / a ** 6 - cfg.VL * cfg.rho_mat0) * h
    s.pa, s.phi = pa_new, s.phi + s.pi / a * h


def _mut_H2_matter_sign(cfg, s, h):
    a = s.a
    sum_pi2 = O.lattice_sum(s.pi * s.pi)
    pa_new = s.pa + (a ** 3 * sum_pi2 / a ** 6 + cfg.VL * cfg.rho_mat0) * h
    s.pa, s.phi = pa_new, s.phi + s.pi / (a * a) * h


def _mut_H2_kinetic_power(cfg, s, h):
    a = s.a
    sum_pi2 = O.lattice_sum(s.pi * s.pi)
    pa_new = s.pa + (a ** 3 * sum_pi2 / a ** 5 - cfg.VL * cfg.rho_mat0) * h
    s.pa, s.phi = pa_new, s.phi + s.pi / (a * a) * h


def _make_H3(pa_grad=1.0, pa_V=4.0, kick_a4=4, kick_D=1.0):
    def flow(cfg, s, h):
        a, dx2 = s.a, cfg.dx ** 2
        D = O.laplacian(s.phi, cfg.stencil)
        V = O.potential(cfg.model, cfg.params, s.phi)
        dV = O.potential_derivative(cfg.model, cfg.params, s.phi)
        sphiD = O.lattice_sum(s.phi * D)
        sV = O.lattice_sum(V)
        pa_new = s.pa + a ** 3 * (pa_grad * sphiD / (a * a * dx2) - pa_V * sV) * h
        pi_new = s.pi + (kick_D * a * a * D / dx2 - a ** kick_a4 * dV) * h
        s.pa, s.pi = pa_new, pi_new
    return flow


def _mut_stage_unsymmetric(cfg, s, h):
    O.flow_H1(cfg, s, h)
    O.flow_H2(cfg, s, 0.5 * h)
    O.flow_H3(cfg, s, h)
    O.flow_H2(cfg, s, 0.5 * h)
    s.eta = s.eta + h


def _weights_swapped(order):
    w = list(_orig_weights(order))
    if len(w) > 2:
        w[0], w[1] = w[1], w[0]
        w[-1], w[-2] = w[-2], w[-1]
    return w


_orig_weights = O.stage_weights


def _stencil_bad_face(stencil):
    return (-6.0, 1.0, 0.0, 0.0) if stencil == "iso27" else (-6.0, 1.01, 0.0, 0.0)


def _dV_chaotic_missing_term(model, p, phi):
    if model == "chaotic2":
        return np.stack([p[0] * phi[0], p[1] * phi[0] * phi[0] * phi[1]])
    return _orig_dV(model, p, phi)


_orig_dV = O.potential_derivative


def _initial_pa_factor(cfg, a, phi, pi):
    if cfg.static:
        return 0.0
    return -math.sqrt(6.0 * cfg.VL * cfg.mpl ** 2 * O._field_energy_sum(cfg, a, phi, pi))


def _field_stats_unbiased(s, i):
    S = s.phi[i].size
    mean = O.lattice_sum(s.phi[i]) / S
    return mean, O.lattice_sum((s.phi[i] - mean) ** 2) / (S - 1)


def _field_stats_no_mean(s, i):
    S = s.phi[i].size
    return O.lattice_sum(s.phi[i]) / S, O.lattice_sum(s.phi[i] ** 2) / S


def _field_stats_wrong_field(s, i):
    return _orig_field_stats(s, 0)


_orig_field_stats = O.field_stats


def _step_size_a2(cfg, s):
    return cfg.dt / s.a ** 2 if cfg.time_step == "physical" else cfg.dt


def _step_size_ignores_a(cfg, s):
    return cfg.dt


def _checks():
    """Every pin as (name, passes?) with the same bounds as the pin tests."""
    def slope(f, *args):
        return math.log2(f(*args[0]) / f(*args[1]))
    out = {
        "transfer": all(P.free_mode_transfer_error(o) < 1e-12 for o in (2, 4, 8)),
        "continuum": 3.7 < slope(P.free_mode_continuum_error, (4, 0.2), (4, 0.1)) < 4.8,
        "homogeneous": 3.7 < slope(P.homogeneous_error, (4, 0.05), (4, 0.025)) < 4.8
                       and P.homogeneous_error(4, 0.00625) < 1e-4,
        "radiation": P.radiation_error(4) < 1e-13,
        "matter": P.matter_error(4) < 1e-13,
        "constraint": 3.7 < slope(P.constraint_error, (4, 0.04), (4, 0.02)) < 4.8,
        "constraint8": 7.7 < slope(P.constraint_error, (8, 0.1), (8, 0.05)) < 8.8,
        "friedmann2": P.second_friedmann_error() < 1e-3,
        "planewave": P.plane_wave_symbol_error("7pt", 8, (1, 2, 3)) < 1e-13
                     and P.plane_wave_symbol_error("iso27", 8, (1, 2, 3)) < 1e-13,
        "dV": P.potential_derivative_error("chaotic2", (1.0, 1e4), (1.0, 0.3)) < 1e-8,
        "composition8": 7.7 < slope(P.composition_error_harmonic, (8, 10), (8, 20)) < 8.8,
        "field_stats": P.field_stats_error() < 1e-12,
        "fourth_symbol": P.plane_wave_symbol_error("4th", 8, (1, 2, 3)) < 1e-13,
        "fourth_order": abs(P.fourth_order_accuracy_slope() - 6.0) < 0.1,
        "physical_radiation": P.radiation_physical_recurrence(4) < 1e-14,
        "physical_static": P.static_physical_equivalence() == 0.0,
    }
    return out


MUTATIONS_FOURTH = {
    "fourth-order far weight +1/12": ((1, 16.0 / 12.0), (2, 1.0 / 12.0)),
    "fourth-order near weight 15/12": ((1, 15.0 / 12.0), (2, -1.0 / 12.0)),
}

MUTATIONS = {
    "H1 sign": ("flow_H1", _mut_H1_sign),
    "H2 drift 1/a instead of 1/a^2": ("flow_H2", _mut_H2_drift_power),
    "H2 matter sign": ("flow_H2", _mut_H2_matter_sign),
    "H2 kinetic a^-2 instead of a^-3": ("flow_H2", _mut_H2_kinetic_power),
    "H3 p_a gradient term dropped": ("flow_H3", _make_H3(pa_grad=0.0)),
    "H3 p_a 3V instead of 4V": ("flow_H3", _make_H3(pa_V=3.0)),
    "H3 kick a^2 dV instead of a^4": ("flow_H3", _make_H3(kick_a4=2)),
    "H3 kick D sign": ("flow_H3", _make_H3(kick_D=-1.0)),
    "stage not symmetric": ("second_order_stage", _mut_stage_unsymmetric),
    "Table 1 weights transposed": ("stage_weights", _weights_swapped),
    "stencil weight": ("stencil_coefficients", _stencil_bad_face),
    "dV term dropped": ("potential_derivative", _dV_chaotic_missing_term),
    "constraint factor 6 instead of 12": ("initial_pa", _initial_pa_factor),
    "variance divided by S - 1": ("field_stats", _field_stats_unbiased),
    "variance without the mean": ("field_stats", _field_stats_no_mean),
    "statistics of the wrong field": ("field_stats", _field_stats_wrong_field),
    "physical step dt / a^2": ("step_size", _step_size_a2),
    "physical step without a": ("step_size", _step_size_ignores_a),
}


def test_unmutated_oracle_passes_every_check():
    bad = [k for k, ok in _checks().items() if not ok]
    assert not bad, bad


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_each_planted_mistake_fails_some_pin(name, monkeypatch):
    attr, repl = MUTATIONS[name]
    monkeypatch.setattr(O, attr, repl)
    with np.errstate(all="ignore"):
        try:
            res = _checks()
        except (ValueError, FloatingPointError, OverflowError, ZeroDivisionError):
            return  # the mistake broke the oracle outright
    failed = [k for k, ok in res.items() if not ok]
    assert failed, f"planted mistake '{name}' passed every pin"


@pytest.mark.parametrize("name", sorted(MUTATIONS_FOURTH))
def test_each_planted_fourth_order_mistake_fails_some_pin(name, monkeypatch):
    monkeypatch.setattr(O, "_FOURTH", MUTATIONS_FOURTH[name])
    with np.errstate(all="ignore"):
        res = _checks()
    failed = [k for k, ok in res.items() if not ok]
    assert failed, f"planted mistake '{name}' passed every pin"
