"""The oracle against what the paper and the mathematics fix (CPU only)."""
import math

import numpy as np
import pytest

from oracle import pycool_oracle as O
import oracle_pins as P

ORDERS = (2, 4, 6, 8)


def test_table1_matches_printed_digits():
    """Sec. 2.3, Table 1: weights as printed, centre = 1 - 2 sum, palindromic."""
    t = P.read_table1()
    for order, s in ((6, 7), (8, 15)):
        w = O.stage_weights(order)
        assert len(w) == s
        k = (s - 1) // 2
        for i in range(1, k + 1):
            assert w[i - 1] == t[order][i]
        assert w == w[::-1]
        assert w[k] == pytest.approx(1.0 - 2.0 * math.fsum(t[order].values()), abs=1e-15)
        assert math.fsum(w) == pytest.approx(1.0, abs=1e-14)


def test_triple_jump_closed_form():
    """Eq. Phi-rec with n = 1: z1 = 1/(2 - 2^(1/3)), z0 = 1 - 2 z1 (consistency)."""
    z1, z0, z1b = O.stage_weights(4)
    assert z1 == z1b
    assert z1 == pytest.approx(1.3512071919596578, abs=1e-15)
    assert z0 == pytest.approx(-1.7024143839193153, abs=1e-15)
    assert 2 * z1 + z0 == pytest.approx(1.0, abs=1e-15)
    assert O.stage_weights(2) == [1.0]


@pytest.mark.parametrize("order", ORDERS)
def test_composition_order_harmonic_and_pendulum(order):
    n1, n2 = (10, 20) if order == 8 else (20, 40)
    for f in (P.composition_error_harmonic, P.composition_error_pendulum):
        slope = math.log2(f(order, n1) / f(order, n2))
        assert order - 0.3 < slope < order + 0.8, (f.__name__, slope)


@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
@pytest.mark.parametrize("n,mode", [(8, (1, 2, 3)), (12, (5, 0, 7)), (7, (3, 3, 3)), (5, (0, 0, 1))])
def test_stencil_plane_wave_symbol(stencil, n, mode):
    assert P.plane_wave_symbol_error(stencil, n, mode) < 1e-13


@pytest.mark.parametrize("n,mode", [(10, (1, 2, 3)), (9, (4, 4, 0)), (16, (8, 1, 0))])
def test_seven_point_dispersion_closed_form(n, mode):
    """The closed form omega^2 dx^2 = sum_d 4 sin^2(k_d dx/2) of the 7-point stencil."""
    assert P.seven_point_closed_form_error(n, mode) < 1e-13


def test_iso27_is_a_laplacian_with_isotropic_k4_term():
    """Small k: symbol = -k^2 + k^4/12 + O(k^6) along every direction."""
    for direction in ((1, 0, 0), (1, 1, 0), (1, 1, 1), (0.3, 0.5, 0.81)):
        d = np.array(direction) / np.linalg.norm(direction)
        k = 1e-2
        s = P.stencil_symbol("iso27", list(k * d))
        assert s == pytest.approx(-k * k + k ** 4 / 12, rel=1e-6)


@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
def test_stokes_identity(stencil):
    assert P.stokes_error(stencil) < 1e-13


@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
def test_laplacian_symmetries(stencil):
    rng = np.random.default_rng(5)
    f = rng.standard_normal((6, 7, 5))
    D = O.laplacian(f, stencil)
    assert abs(O.lattice_sum(D)) < 1e-12
    # shift equivariance
    g = np.roll(f, (1, -2, 3), axis=(0, 1, 2))
    assert np.allclose(O.laplacian(g, stencil), np.roll(D, (1, -2, 3), axis=(0, 1, 2)), atol=1e-13)
    # axis permutation
    h = np.transpose(f, (2, 0, 1))
    assert np.allclose(O.laplacian(h, stencil), np.transpose(D, (2, 0, 1)), atol=1e-13)
    # constants are harmonic
    assert np.max(np.abs(O.laplacian(np.full((4, 4, 4), 2.5), stencil))) < 1e-14


def test_potential_values_golden():
    assert P.potential_golden_error() < 1e-15


@pytest.mark.parametrize("model,params,point", [
    ("free", (0.7,), (0.3,)),
    ("chaotic2", (1.0, 1.0e4), (1.0, 0.3)),
    ("chaotic2", (1.0, 1.0e4), (-0.4, 2e-3)),
    ("oscillon", (1.0, 1.0, 0.5), (0.8,)),
    ("oscillon", (1.0, 1.0, 0.5), (-1.7,)),
    ("qball", (1.0, -0.1, 1.0), (1.3, 0.4)),
    ("qball", (1.0, -0.1, 1.0), (0.01, -0.02)),
    ("phi4", (2.0, 3.0), (0.7,)),
])
def test_potential_derivative_matches_difference_quotient(model, params, point):
    assert P.potential_derivative_error(model, params, point) < 1e-8


def test_qball_at_origin_is_zero():
    x = np.zeros((2, 3))
    assert np.all(O.potential("qball", (1.0, -0.1, 1.0), x) == 0.0)
    assert np.all(O.potential_derivative("qball", (1.0, -0.1, 1.0), x) == 0.0)


@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
@pytest.mark.parametrize("order", ORDERS)
def test_free_mode_exact_transfer_matrix(order, stencil):
    """One Fourier mode on a static background: the scheme is a product of 2x2 matrices."""
    assert P.free_mode_transfer_error(order, stencil=stencil) < 1e-12


@pytest.mark.parametrize("order,dts", [(2, (0.1, 0.05)), (4, (0.2, 0.1)), (6, (0.4, 0.2)), (8, (0.6, 0.3))])
def test_free_mode_converges_to_discrete_dispersion(order, dts):
    e1, e2 = (P.free_mode_continuum_error(order, dt) for dt in dts)
    slope = math.log2(e1 / e2)
    assert order - 0.3 < slope < order + 0.8


@pytest.mark.parametrize("order,dts", [(2, (0.02, 0.01)), (4, (0.05, 0.025)), (6, (0.1, 0.05)), (8, (0.15, 0.075))])
def test_homogeneous_mode_against_dop853(order, dts):
    e1, e2 = (P.homogeneous_error(order, dt) for dt in dts)
    slope = math.log2(e1 / e2)
    assert order - 0.3 < slope < order + 0.8
    bound = {2: 5e-3, 4: 1e-4, 6: 1e-5, 8: 1e-6}[order]
    assert P.homogeneous_error(order, dts[1] / 4) < bound


@pytest.mark.parametrize("order", ORDERS)
def test_radiation_background_is_exactly_linear(order):
    assert P.radiation_error(order) < 1e-13


@pytest.mark.parametrize("order", ORDERS)
def test_matter_background_is_exactly_quadratic(order):
    assert P.matter_error(order) < 1e-13


@pytest.mark.parametrize("order,dts", [(2, (0.02, 0.01)), (4, (0.04, 0.02)), (6, (0.06, 0.03)), (8, (0.1, 0.05))])
def test_constraint_error_scales_as_dt_to_the_order(order, dts):
    e1, e2 = (P.constraint_error(order, dt) for dt in dts)
    slope = math.log2(e1 / e2)
    assert order - 0.3 < slope < order + 0.8


def test_constraint_error_scales_iso27():
    e1, e2 = (P.constraint_error(4, dt, stencil="iso27") for dt in (0.04, 0.02))
    assert 3.7 < math.log2(e1 / e2) < 4.8


def test_initial_state_satisfies_constraint():
    cfg = P._inhomogeneous_cfg(4, 0.01)
    phi, pi = P._inhomogeneous_ics(cfg.n)
    st = O.make_state(cfg, phi, pi)
    e = O.energies(cfg, st)
    assert abs(O.hamiltonian(cfg, st)) / (cfg.VL * e["rho"]) < 1e-14
    assert e["residual"] < 1e-13
    assert st.pa < 0


def test_time_reversibility():
    assert P.reversibility_error() < 1e-12


def test_second_friedmann_equation():
    assert P.second_friedmann_error() < 1e-3


@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
def test_plane_wave_energies(stencil):
    assert P.plane_wave_energy_error(stencil) < 1e-14


def test_field_stats_closed_forms():
    """Mean c and variance A^2/2 of c + A cos(k.x); two-valued slab field."""
    assert P.field_stats_error() < 1e-12   # inputs rounded at |c| eps, relative to A


# --- the adaptive conformal step (Sec. 3.1) ----------------------------------

@pytest.mark.parametrize("order,dts", [(2, (0.05, 0.025)), (4, (0.05, 0.025)), (6, (0.2, 0.1))])
def test_physical_steps_homogeneous_mode_against_dop853(order, dts):
    e1, e2 = (P.homogeneous_error_physical(order, dt) for dt in dts)
    assert abs(math.log2(e1 / e2) - order) < 0.5, (e1, e2)


@pytest.mark.parametrize("order,dts", [(2, (0.04, 0.02)), (4, (0.04, 0.02))])
def test_physical_steps_constraint_error_scales_as_dt_to_the_order(order, dts):
    e1, e2 = (P.constraint_error_physical(order, dt) for dt in dts)
    assert abs(math.log2(e1 / e2) - order) < 0.4, (e1, e2)


def test_physical_steps_on_static_background_are_conformal_steps_of_dt_over_a():
    assert P.static_physical_equivalence() == 0.0


@pytest.mark.parametrize("order", [2, 4, 8])
def test_physical_steps_radiation_recurrence(order):
    assert P.radiation_physical_recurrence(order) < 1e-14


# --- the fourth-order stencil (Sec. 2.1: HLATTICE's, not printed) --------------

@pytest.mark.parametrize("n,mode", [(8, (1, 2, 3)), (12, (5, 0, 2)), (9, (4, 4, 1))])
def test_fourth_order_stencil_plane_wave_symbol(n, mode):
    assert P.plane_wave_symbol_error("4th", n, mode) < 1e-13


def test_fourth_order_stencil_is_fourth_order():
    assert abs(P.fourth_order_accuracy_slope() - 6.0) < 0.1


def test_fourth_order_stencil_stokes_identity():
    assert P.stokes_error("4th") < 1e-13


def test_fourth_order_stencil_free_mode_and_constraint_slope():
    assert P.free_mode_transfer_error(4, stencil="4th") < 1e-12
    e1, e2 = (P.constraint_error(4, dt, stencil="4th") for dt in (0.04, 0.02))
    assert abs(math.log2(e1 / e2) - 4.0) < 0.4, (e1, e2)
