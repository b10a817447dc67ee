"""CPU oracle for the split-Hamiltonian symplectic lattice step of PyCOOL.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code, tables or
helpers with the CUDA path; the two meet only through seeded input arrays.

What it is
----------
A plain, slow, obviously-correct FP64 restatement of the method of
J. Sainio, "PyCOOL - a Cosmological Object-Oriented Lattice code written in
Python" (arXiv:1201.5029):

* the discrete Laplacian D[phi] and gradient stencil G[phi]   (Sec. 2.1, Eqs. D, G)
* the potentials V and dV/dphi of the three models            (Sec. 3)
* the three exact sub-flows Phi_H1, Phi_H2, Phi_H3            (Sec. 2.3, Eq. split-Phi)
* the second-order stage  Phi1(h/2) Phi2(h/2) Phi3(h) Phi2(h/2) Phi1(h/2)
                                                              (Sec. 2.3, after Eq. split-Phi)
* the stage weights: leapfrog, the triple jump (Eq. Phi-rec) and the
  symmetric compositions of Table 1
* the initial p_a from the Hamiltonian constraint H = 0       (Eqs. H2, Fried-1)
* energy density, pressure, Hubble rate and the residual curvature
                                                              (Eqs. rho-pres, res-curv)

Every flow is applied literally and separately, and every lattice sum is
recomputed from the current arrays with a correctly rounded sum (math.fsum).
There is no merging of flows, no fusion and no reordering.

Layout: fields are float64 arrays of shape (N_f, n, n, n) indexed
[field][z][y][x]; the lattice is periodic in all three directions.

Readings of the paper taken here (the paper is silent or garbled):

1. The Laplacian coefficients c_d are not printed (Sec. 2.1 cites Patra 2005).
   Two stencils are offered, both written as Eq. D with a coefficient per
   neighbour class d = number of non-zero offsets:
     '7pt'   : c = (-6, 1, 0, 0)
     'iso27' : c = (-128, 14, 3, 1) / 30   (isotropic at O(k^4))
2. V_L is the number of lattice sites n^3 (Sec. 2.1: V_L dx^3 is the box volume).
3. p_a = -6 a' V_L m_pl^2 (Eq. p-a), so an expanding universe has p_a < 0 and
   the initial p_a is the negative root of H = 0.
4. Time is conformal time eta; ``dt`` is d-eta.
5. z_0 of the triple jump has a garbled denominator in the paper; the standard
   2 - 2^{1/3} is used, which gives 2 z_1 + z_0 = 1.
6. Table 1 lists w_1 (outermost stage) first; the centre weight is
   1 - 2 * (sum of the others).
7. m_pl = inf means a static background: Phi_H1 leaves a unchanged and the
   initial p_a is 0 (the constraint cannot be imposed).
8. The complex Q-ball field is Phi = (phi_1 + i phi_2)/sqrt(2), so
   |Phi|^2 = (phi_1^2 + phi_2^2)/2 and V = dV = 0 at |Phi| = 0.
10. The fourth-order stencil (Sec. 2.1 names HLATTICE's without printing it):
   '4th' is the 13-point form that is fourth-order accurate on each axis,
   D[f](x) = sum_axes [-f(x-2e) + 16 f(x-e) - 30 f(x) + 16 f(x+e) - f(x+2e)] / 12,
   with G of Eq. G taken over the same 12 neighbours and coefficients.
9. The adaptive conformal step of Sec. 3.1 ("constant increases in physical
   time", dt_phys = a d-eta): with time_step = "physical" each time step
   takes d-eta = dt / a, a being the scale factor of the synchronised state at
   the start of the step; all stages of that step use it (h_i = w_i d-eta).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

__all__ = [
    "stage_weights", "stencil_coefficients", "laplacian", "gradient_G",
    "potential", "potential_derivative", "model_nfields",
    "LatticeConfig", "State", "flow_H1", "flow_H2", "flow_H3",
    "second_order_stage", "step", "evolve", "initial_pa", "hamiltonian",
    "energies", "field_stats", "make_state",
]

# ---------------------------------------------------------------------------
# Stage weights (Sec. 2.3: Eq. Phi-2, Eq. Phi-rec, Table 1)
# ---------------------------------------------------------------------------

# Table 1, order 6 (s = 7): w_1..w_3 as printed; w_4 = 1 - 2 (w_1 + w_2 + w_3).
_TABLE1_ORDER6 = (
    0.78451361047755726382,
    0.23557321335935813368,
    -1.17767998417887100695,
)
# Table 1, order 8 (s = 15): w_1..w_7 as printed; w_8 = 1 - 2 sum_{i<=7} w_i.
_TABLE1_ORDER8 = (
    0.74167036435061295345,
    -0.40910082580003159400,
    0.19075471029623837995,
    -0.57386247111608226666,
    0.29906418130365592384,
    0.33462491824529818378,
    0.31529309239676659663,
)


def _symmetric_from_half(half: Sequence[float]) -> List[float]:
    """w_1..w_k given, centre = 1 - 2 sum; returns w_1..w_k, centre, w_k..w_1."""
    centre = 1.0 - 2.0 * math.fsum(half)
    return list(half) + [centre] + list(reversed(half))


def stage_weights(order: int) -> List[float]:
    """Weights w_i of the Phi^(2) stages of one step, in the order applied.

    order 2: the single leapfrog stage (Eq. Phi-2).
    order 4: the triple jump of Eq. Phi-rec with n = 1:
             z_1 = 1/(2 - 2^{1/3}),  z_0 = -2^{1/3}/(2 - 2^{1/3})  -> (z_1, z_0, z_1).
    order 6, 8: the symmetric compositions of Table 1.
    """
    if order == 2:
        return [1.0]
    if order == 4:
        c = 2.0 ** (1.0 / 3.0)
        z1 = 1.0 / (2.0 - c)
        z0 = -c / (2.0 - c)
        return [z1, z0, z1]
    if order == 6:
        return _symmetric_from_half(_TABLE1_ORDER6)
    if order == 8:
        return _symmetric_from_half(_TABLE1_ORDER8)
    raise ValueError(f"unsupported integrator order {order}")


# ---------------------------------------------------------------------------
# Stencils (Sec. 2.1, Eqs. D and G)
# ---------------------------------------------------------------------------

def stencil_coefficients(stencil: str) -> tuple:
    """c_d for neighbour class d = number of non-zero offsets (0..3)."""
    if stencil == "7pt":
        return (-6.0, 1.0, 0.0, 0.0)
    if stencil == "iso27":
        return (-128.0 / 30.0, 14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0)
    raise ValueError(f"unknown stencil {stencil!r}")


def _offsets():
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                yield dz, dy, dx


def _neighbour(f: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """f(x + dx, y + dy, z + dz) on the periodic lattice; f is [..., z, y, x]."""
    return np.roll(f, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


# The fourth-order stencil: (offset along one axis, coefficient) pairs.
_FOURTH = ((1, 16.0 / 12.0), (2, -1.0 / 12.0))
_FOURTH_CENTRE = -90.0 / 12.0


def _axis_neighbour(f: np.ndarray, axis: int, k: int) -> np.ndarray:
    """f at x + k e_axis (axis 0 = z, 1 = y, 2 = x of the last three)."""
    return np.roll(f, shift=-k, axis=-3 + axis)


def laplacian(f: np.ndarray, stencil: str = "7pt") -> np.ndarray:
    """Eq. D: D[f](x) = sum over the 27 sites alpha around x of c_{d(alpha)} f(alpha)
    (for '4th': over the centre and the 12 sites up to two steps along an axis).

    Works on a single field [z][y][x] or a stack [field][z][y][x].
    D carries no 1/dx^2; the flows divide by dx^2 themselves.
    """
    if stencil == "4th":
        out = _FOURTH_CENTRE * f
        for axis in range(3):
            for k, c in _FOURTH:
                out = out + c * (_axis_neighbour(f, axis, k) + _axis_neighbour(f, axis, -k))
        return out
    c = stencil_coefficients(stencil)
    out = np.zeros_like(f)
    for dz, dy, dx in _offsets():
        d = abs(dz) + abs(dy) + abs(dx)
        if c[d] != 0.0:
            out = out + c[d] * _neighbour(f, dz, dy, dx)
    return out


def gradient_G(f: np.ndarray, stencil: str = "7pt") -> np.ndarray:
    """Eq. G: G[f](x) = 1/2 sum_alpha c_{d(alpha)} (f(alpha) - f(x))^2."""
    if stencil == "4th":
        out = np.zeros_like(f)
        for axis in range(3):
            for k, c in _FOURTH:
                for sgn in (1, -1):
                    diff = _axis_neighbour(f, axis, sgn * k) - f
                    out = out + 0.5 * c * diff * diff
        return out
    c = stencil_coefficients(stencil)
    out = np.zeros_like(f)
    for dz, dy, dx in _offsets():
        d = abs(dz) + abs(dy) + abs(dx)
        if d and c[d] != 0.0:
            diff = _neighbour(f, dz, dy, dx) - f
            out = out + 0.5 * c[d] * diff * diff
    return out


# ---------------------------------------------------------------------------
# Models (Sec. 3: chaotic preheating, oscillon, curvaton Q-ball; plus a free
# massive field used by the closed-form tests)
# ---------------------------------------------------------------------------

_MODEL_NF = {"free": 1, "free2": 2, "chaotic2": 2, "oscillon": 1, "qball": 2, "phi4": 1}


def model_nfields(model: str) -> int:
    return _MODEL_NF[model]


def potential(model: str, p: Sequence[float], phi: np.ndarray) -> np.ndarray:
    """V(phi_1..phi_N) at every site; phi has shape (N_f, ...).

    free     : V = m^2/2 sum_i phi_i^2                 p = (m2,)
    chaotic2 : V = m^2 phi^2/2 + g^2 phi^2 chi^2/2      p = (m2, g2)        (Sec. 3.1)
    oscillon : V = m^2 phi^2/2 - lam phi^4/4 + g phi^6/6 p = (m2, lam, g)   (Sec. 3.2)
    qball    : V = m^2 |Phi|^2 (1 + K ln(|Phi|^2/M^2)),
               |Phi|^2 = (phi_1^2 + phi_2^2)/2           p = (m2, K, M)     (Sec. 3.3)
    phi4     : V = m^2 phi^2/2 + lam phi^4/4               p = (m2, lam)
               (a model outside Sec. 3, for potentials given at run time)
    """
    if model == "phi4":
        m2, lam = p[0], p[1]
        ph = phi[0]
        return 0.5 * m2 * ph ** 2 + 0.25 * lam * ph ** 4
    if model in ("free", "free2"):
        m2 = p[0]
        return 0.5 * m2 * np.sum(phi * phi, axis=0)
    if model == "chaotic2":
        m2, g2 = p[0], p[1]
        ph, ch = phi[0], phi[1]
        return 0.5 * m2 * ph * ph + 0.5 * g2 * ph * ph * ch * ch
    if model == "oscillon":
        m2, lam, g = p[0], p[1], p[2]
        ph = phi[0]
        return 0.5 * m2 * ph ** 2 - 0.25 * lam * ph ** 4 + g / 6.0 * ph ** 6
    if model == "qball":
        m2, K, M = p[0], p[1], p[2]
        u = 0.5 * (phi[0] * phi[0] + phi[1] * phi[1])
        with np.errstate(divide="ignore", invalid="ignore"):
            v = m2 * u * (1.0 + K * np.log(u / (M * M)))
        return np.where(u > 0.0, v, 0.0)
    raise ValueError(f"unknown model {model!r}")


def potential_derivative(model: str, p: Sequence[float], phi: np.ndarray) -> np.ndarray:
    """dV/dphi_i at every site, shape (N_f, ...), derived by hand from V above."""
    if model == "phi4":
        return np.stack([p[0] * phi[0] + p[1] * phi[0] ** 3])
    if model in ("free", "free2"):
        return p[0] * phi
    if model == "chaotic2":
        m2, g2 = p[0], p[1]
        ph, ch = phi[0], phi[1]
        return np.stack([m2 * ph + g2 * ph * ch * ch, g2 * ph * ph * ch])
    if model == "oscillon":
        m2, lam, g = p[0], p[1], p[2]
        ph = phi[0]
        return np.stack([m2 * ph - lam * ph ** 3 + g * ph ** 5])
    if model == "qball":
        m2, K, M = p[0], p[1], p[2]
        u = 0.5 * (phi[0] * phi[0] + phi[1] * phi[1])
        with np.errstate(divide="ignore", invalid="ignore"):
            fac = m2 * (1.0 + K + K * np.log(u / (M * M)))
        fac = np.where(u > 0.0, fac, 0.0)
        return np.stack([fac * phi[0], fac * phi[1]])
    raise ValueError(f"unknown model {model!r}")


# ---------------------------------------------------------------------------
# Lattice state and the exact sub-flows (Sec. 2.3, Eq. split-Phi)
# ---------------------------------------------------------------------------

@dataclass
class LatticeConfig:
    n: int                      # lattice side; V_L = n^3 sites
    L: float                    # comoving box side; dx = L / n
    model: str
    params: Sequence[float]
    dt: float                   # conformal step d-eta (may be negative)
    order: int = 2
    stencil: str = "7pt"
    mpl: float = 1.0            # reduced Planck mass; inf = static background
    rho_rad0: float = 0.0       # homogeneous radiation, Eq. H2
    rho_mat0: float = 0.0       # homogeneous matter, Eq. H2
    time_step: str = "conformal"  # "conformal": d-eta = dt; "physical": d-eta = dt / a (Sec. 3.1)

    @property
    def VL(self) -> float:
        return float(self.n) ** 3

    @property
    def dx(self) -> float:
        return self.L / self.n

    @property
    def static(self) -> bool:
        return math.isinf(self.mpl)

    @property
    def inv_6VLm2(self) -> float:
        """1/(6 V_L m_pl^2), zero for a static background."""
        return 0.0 if self.static else 1.0 / (6.0 * self.VL * self.mpl ** 2)


@dataclass
class State:
    a: float
    pa: float
    phi: np.ndarray             # (N_f, n, n, n)
    pi: np.ndarray              # (N_f, n, n, n)
    eta: float = 0.0


def lattice_sum(x: np.ndarray) -> float:
    """Correctly rounded sum over all entries (the Sigma of the paper)."""
    return math.fsum(np.asarray(x, dtype=np.float64).ravel().tolist())


def flow_H1(cfg: LatticeConfig, s: State, h: float) -> None:
    """Phi_H1(h): a -> a - p_a h / (6 V_L m_pl^2); nothing else changes."""
    s.a = s.a - s.pa * cfg.inv_6VLm2 * h


def flow_H2(cfg: LatticeConfig, s: State, h: float) -> None:
    """Phi_H2(h): p_a -> p_a + [sum a^3 pi^2/a^6 - V_L rho_m0] h,  phi -> phi + pi h / a^2."""
    a = s.a
    sum_pi2 = lattice_sum(s.pi * s.pi)
    pa_new = s.pa + (a ** 3 * sum_pi2 / a ** 6 - cfg.VL * cfg.rho_mat0) * h
    phi_new = s.phi + s.pi / (a * a) * h
    s.pa, s.phi = pa_new, phi_new


def flow_H3(cfg: LatticeConfig, s: State, h: float) -> None:
    """Phi_H3(h): p_a -> p_a + [sum a^3 (phi D[phi]/(a^2 dx^2) - 4 V)] h,
                  pi  -> pi + [a^2 D[phi]/dx^2 - a^4 dV/dphi] h."""
    a, dx2 = s.a, cfg.dx ** 2
    D = laplacian(s.phi, cfg.stencil)
    V = potential(cfg.model, cfg.params, s.phi)
    dV = potential_derivative(cfg.model, cfg.params, s.phi)
    sum_phiD = lattice_sum(s.phi * D)
    sum_V = lattice_sum(V)
    pa_new = s.pa + a ** 3 * (sum_phiD / (a * a * dx2) - 4.0 * sum_V) * h
    pi_new = s.pi + (a * a * D / dx2 - a ** 4 * dV) * h
    s.pa, s.pi = pa_new, pi_new


def second_order_stage(cfg: LatticeConfig, s: State, h: float) -> None:
    """Phi^(2)(h) = Phi_H1(h/2) Phi_H2(h/2) Phi_H3(h) Phi_H2(h/2) Phi_H1(h/2)."""
    flow_H1(cfg, s, 0.5 * h)
    flow_H2(cfg, s, 0.5 * h)
    flow_H3(cfg, s, h)
    flow_H2(cfg, s, 0.5 * h)
    flow_H1(cfg, s, 0.5 * h)
    s.eta = s.eta + h


def step_size(cfg: LatticeConfig, s: State) -> float:
    """The conformal step d-eta of the next time step: dt (conformal time), or
    dt / a at the synchronised state that starts the step (the adaptive
    conformal step of Sec. 3.1: each step advances physical time t, dt = a
    d-eta, by about dt)."""
    if cfg.time_step == "conformal":
        return cfg.dt
    if cfg.time_step == "physical":
        return cfg.dt / s.a
    raise ValueError(f"unknown time step rule {cfg.time_step!r}")


def step(cfg: LatticeConfig, s: State) -> None:
    """One time step: the stages of the chosen order in sequence, each with
    h = w_i d-eta."""
    deta = step_size(cfg, s)
    for w in stage_weights(cfg.order):
        second_order_stage(cfg, s, w * deta)


def evolve(cfg: LatticeConfig, s: State, steps: int) -> State:
    for _ in range(int(steps)):
        step(cfg, s)
    return s


# ---------------------------------------------------------------------------
# Hamiltonian, constraint and observables (Eqs. H2, Fried-1, rho-pres, res-curv)
# ---------------------------------------------------------------------------

def _field_energy_sum(cfg: LatticeConfig, a: float, phi: np.ndarray, pi: np.ndarray) -> float:
    """sum_{i,x} a^4 (pi^2/(2 a^6) - phi D[phi]/(2 a^2 dx^2) + V) + V_L rho_r0 + a V_L rho_m0."""
    dx2 = cfg.dx ** 2
    D = laplacian(phi, cfg.stencil)
    V = potential(cfg.model, cfg.params, phi)
    fields = a ** 4 * (lattice_sum(pi * pi) / (2.0 * a ** 6)
                       - lattice_sum(phi * D) / (2.0 * a * a * dx2)
                       + lattice_sum(V))
    return fields + cfg.VL * cfg.rho_rad0 + a * cfg.VL * cfg.rho_mat0


def hamiltonian(cfg: LatticeConfig, s: State) -> float:
    """Eq. H2: -p_a^2/(12 V_L m_pl^2) + field energy + radiation + matter."""
    kin_a = 0.0 if cfg.static else s.pa ** 2 / (12.0 * cfg.VL * cfg.mpl ** 2)
    return -kin_a + _field_energy_sum(cfg, s.a, s.phi, s.pi)


def initial_pa(cfg: LatticeConfig, a: float, phi: np.ndarray, pi: np.ndarray) -> float:
    """Negative root of H = 0 (expanding branch): p_a = -sqrt(12 V_L m_pl^2 E)."""
    if cfg.static:
        return 0.0
    E = _field_energy_sum(cfg, a, phi, pi)
    return -math.sqrt(12.0 * cfg.VL * cfg.mpl ** 2 * E)


def make_state(cfg: LatticeConfig, phi: np.ndarray, pi: np.ndarray,
               a0: float = 1.0, pa0: Optional[float] = None) -> State:
    phi = np.array(phi, dtype=np.float64, copy=True)
    pi = np.array(pi, dtype=np.float64, copy=True)
    assert phi.shape == pi.shape and phi.shape[1:] == (cfg.n,) * 3
    if pa0 is None or (isinstance(pa0, float) and math.isnan(pa0)):
        pa0 = initial_pa(cfg, a0, phi, pi)
    return State(a=float(a0), pa=float(pa0), phi=phi, pi=pi, eta=0.0)


def energies(cfg: LatticeConfig, s: State) -> Dict[str, object]:
    """Lattice means of the energy components at a synchronised state.

    rho_kin[i]  = sum pi_i^2 / (2 a^6 S)
    rho_grad[i] = -sum phi_i D[phi_i] / (2 a^2 dx^2 S)   (Stokes identity, Sec. 2.1)
    rho_pot     = sum V / S
    P           = sum rho_kin - sum rho_grad / 3 - rho_pot        (Eq. rho-pres)
    H           = a'/a^2 = -p_a / (6 S m_pl^2 a^2)               (Eq. a)
    residual    = |(rho + rho_r0/a^4 + rho_m0/a^3) / (3 m_pl^2 H^2) - 1|   (Eq. res-curv)
    """
    a, S, dx2 = s.a, cfg.VL, cfg.dx ** 2
    nf = s.phi.shape[0]
    rho_kin = [lattice_sum(s.pi[i] * s.pi[i]) / (2.0 * a ** 6 * S) for i in range(nf)]
    rho_grad = [-lattice_sum(s.phi[i] * laplacian(s.phi[i], cfg.stencil)) / (2.0 * a * a * dx2 * S)
                for i in range(nf)]
    rho_pot = lattice_sum(potential(cfg.model, cfg.params, s.phi)) / S
    rho = math.fsum(rho_kin) + math.fsum(rho_grad) + rho_pot
    P = math.fsum(rho_kin) - math.fsum(rho_grad) / 3.0 - rho_pot
    if cfg.static:
        H = 0.0
        residual = float("nan")
    else:
        H = -s.pa / (6.0 * S * cfg.mpl ** 2 * a * a)
        rho_tot = rho + cfg.rho_rad0 / a ** 4 + cfg.rho_mat0 / a ** 3
        residual = abs(rho_tot / (3.0 * cfg.mpl ** 2 * H * H) - 1.0)
    return dict(eta=s.eta, a=a, pa=s.pa, H=H, rho_kin=rho_kin, rho_grad=rho_grad,
                rho_pot=rho_pot, rho=rho, P=P, residual=residual)


def field_stats(s: State, i: int) -> tuple:
    """Lattice mean and variance of field i (the field statistics of the
    post-processing, Sec. 2.4): mean = sum phi_i / S, variance = sum (phi_i - mean)^2 / S."""
    S = s.phi[i].size
    mean = lattice_sum(s.phi[i]) / S
    var = lattice_sum((s.phi[i] - mean) ** 2) / S
    return mean, var
