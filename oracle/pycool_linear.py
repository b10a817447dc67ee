"""CPU oracle for the linearised evolution of PyCOOL (Sec. 2.2).

TEST INFRASTRUCTURE ONLY, like ``pycool_oracle``: nothing in the product path
may import it.

What it is
----------
A plain FP64 restatement of the linearised method of Sec. 2.2 of J. Sainio,
"PyCOOL" (arXiv:1201.5029):

* the fields split into a homogeneous background and perturbations whose
  lattice sum vanishes                                       (Eq. phi-lin)
* the Hamiltonian H = H^(0) + H^(2), with H^(2) quadratic in the
  perturbations and neglected in the equations of a, p_a and the background
  fields                                                     (Eqs. H-lin, a-lin, phi-0)
* the perturbations evolved mode by mode in Fourier space, where the
  discrete Laplacian is the multiplier -k_eff^2 and the potential enters
  through its second derivatives at the background           (Eqs. phi-1, Phik-1, V-2)
* the same split-Hamiltonian stages and stage weights as the full lattice
  (Sec. 2.3): Phi_H1(h/2) Phi_H2(h/2) Phi_H3(h) Phi_H2(h/2) Phi_H1(h/2), with
    Phi_H1(h): a   -> a - p_a h / (6 V_L m_pl^2)
    Phi_H2(h): p_a -> p_a + V_L [sum_i pi0_i^2 / a^3 - rho_m0] h,
               phi0 -> phi0 + pi0 h / a^2,  dPhi_k -> dPhi_k + dPi_k h / a^2
    Phi_H3(h): p_a -> p_a - 4 V_L a^3 V(phi0) h,  pi0 -> pi0 - a^4 V'(phi0) h,
               dPi_k -> dPi_k - [k_eff^2 a^2 / dx^2 + a^4 M(phi0)] dPhi_k h
  (M_ij = d^2 V / dphi_i dphi_j at the background; each flow is exact: in
  Phi_H3 neither a nor the fields change);
* the paper's grouping (Sec. 2.2, after Eq. Phik-1): modes with the same
  k_eff^2 obey the same linear equations, so one 2N_f x 2N_f transfer matrix
  per distinct k_eff^2 ("growth functions") advances all of them; the state
  at a later time is that matrix applied to each mode's initial values.

Two routes are given and must agree: every mode evolved directly
(``evolve``), and the transfer matrices of the distinct k_eff^2 values
applied to the initial modes (``transfer_matrices`` + ``apply_transfer``).

Fourier convention: numpy's unnormalised forward FFT over the three lattice
axes; the zero mode of the perturbations is zero by construction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

from . import pycool_oracle as O

__all__ = ["mass_matrix", "k_eff2", "LinearState", "from_lattice", "to_lattice", "step",
           "evolve", "distinct_k2", "transfer_matrices", "apply_transfer"]


def mass_matrix(model: str, p: Sequence[float], phi0: np.ndarray) -> np.ndarray:
    """M_ij = d^2 V / dphi_i dphi_j at the homogeneous background phi0 (N_f,),
    derived by hand from the potentials of Sec. 3 (see ``pycool_oracle.potential``)."""
    phi0 = np.asarray(phi0, dtype=np.float64)
    if model in ("free", "free2"):
        return p[0] * np.eye(len(phi0))
    if model == "chaotic2":
        m2, g2 = p[0], p[1]
        ph, ch = phi0
        return np.array([[m2 + g2 * ch * ch, 2.0 * g2 * ph * ch],
                         [2.0 * g2 * ph * ch, g2 * ph * ph]])
    if model == "oscillon":
        m2, lam, g = p[0], p[1], p[2]
        x = phi0[0]
        return np.array([[m2 - 3.0 * lam * x ** 2 + 5.0 * g * x ** 4]])
    if model == "qball":
        # V = m2 u (1 + K ln(u/M^2)), u = (phi1^2 + phi2^2)/2:
        # dV/dphi_i = m2 (1 + K + K ln(u/M^2)) phi_i, so
        # M_ij = m2 (1 + K + K ln(u/M^2)) delta_ij + m2 K phi_i phi_j / u
        m2, K, M = p[0], p[1], p[2]
        u = 0.5 * float(phi0[0] ** 2 + phi0[1] ** 2)
        if u <= 0.0:
            raise ValueError("the Q-ball's second derivatives diverge at |Phi| = 0")
        fac = m2 * (1.0 + K + K * math.log(u / (M * M)))
        return fac * np.eye(2) + m2 * K * np.outer(phi0, phi0) / u
    raise ValueError(f"unknown model {model!r}")


def k_eff2(n: int, stencil: str = "7pt") -> np.ndarray:
    """k_eff^2 of every lattice mode, shape (n, n, n) in numpy FFT order: minus
    the eigenvalue of the stencil D (Eq. D) on the plane wave exp(i k.x),
    summed over the stencil's offsets (no closed form used)."""
    th = 2.0 * np.pi * np.fft.fftfreq(n)      # k dx = 2 pi m / n, m in numpy FFT order
    tz, ty, tx = np.meshgrid(th, th, th, indexing="ij")
    if stencil == "4th":
        # the 13-point stencil: the centre and, along each axis, the sites at
        # offsets +-1 and +-2 (each pair gives 2 c cos(offset k dx))
        sym = np.full((n, n, n), O._FOURTH_CENTRE)
        for t in (tz, ty, tx):
            for off, coef in O._FOURTH:
                sym = sym + 2.0 * coef * np.cos(off * t)
        return -sym
    c = O.stencil_coefficients(stencil)
    sym = np.zeros((n, n, n))
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                cls = abs(dz) + abs(dy) + abs(dx)
                if c[cls] != 0.0:
                    sym = sym + c[cls] * np.cos(dz * tz + dy * ty + dx * tx)
    return -sym


@dataclass
class LinearState:
    a: float
    pa: float
    phi0: np.ndarray        # (N_f,)
    pi0: np.ndarray         # (N_f,)
    dphi: np.ndarray        # (N_f, n, n, n) complex: Fourier modes of the perturbations
    dpi: np.ndarray         # (N_f, n, n, n) complex
    eta: float = 0.0


def from_lattice(cfg: O.LatticeConfig, phi: np.ndarray, pi: np.ndarray, a0: float,
                 pa0: float) -> LinearState:
    """Split lattice fields into the background (lattice means) and the Fourier
    modes of the perturbations (Eq. phi-lin)."""
    phi0 = np.array([O.lattice_sum(f) / f.size for f in phi])
    pi0 = np.array([O.lattice_sum(f) / f.size for f in pi])
    dphi = np.fft.fftn(phi - phi0[:, None, None, None], axes=(1, 2, 3))
    dpi = np.fft.fftn(pi - pi0[:, None, None, None], axes=(1, 2, 3))
    dphi[:, 0, 0, 0] = 0.0
    dpi[:, 0, 0, 0] = 0.0
    return LinearState(a=float(a0), pa=float(pa0), phi0=phi0, pi0=pi0, dphi=dphi, dpi=dpi)


def to_lattice(s: LinearState) -> Tuple[np.ndarray, np.ndarray]:
    """Lattice fields background + inverse FFT of the perturbation modes."""
    dphi = np.fft.ifftn(s.dphi, axes=(1, 2, 3)).real
    dpi = np.fft.ifftn(s.dpi, axes=(1, 2, 3)).real
    return s.phi0[:, None, None, None] + dphi, s.pi0[:, None, None, None] + dpi


def _flow_H1(cfg, s: LinearState, h: float) -> None:
    s.a = s.a - s.pa * cfg.inv_6VLm2 * h


def _flow_H2(cfg, s: LinearState, h: float, modes: bool = True) -> None:
    a = s.a
    s.pa = s.pa + cfg.VL * (float(np.sum(s.pi0 * s.pi0)) / a ** 3 - cfg.rho_mat0) * h
    s.phi0 = s.phi0 + s.pi0 / (a * a) * h
    if modes:
        s.dphi = s.dphi + s.dpi / (a * a) * h


def _flow_H3(cfg, s: LinearState, h: float, k2: np.ndarray, modes: bool = True) -> None:
    a, dx2 = s.a, cfg.dx ** 2
    V = float(O.potential(cfg.model, cfg.params, s.phi0[:, None])[0])
    dV = O.potential_derivative(cfg.model, cfg.params, s.phi0[:, None])[:, 0]
    if modes:
        M = mass_matrix(cfg.model, cfg.params, s.phi0)
        kick = np.einsum("ij,j...->i...", a ** 4 * M, s.dphi) + (a * a / dx2) * k2 * s.dphi
        s.dpi = s.dpi - kick * h
    s.pa = s.pa - 4.0 * cfg.VL * a ** 3 * V * h
    s.pi0 = s.pi0 - a ** 4 * dV * h


def _stage(cfg, s: LinearState, h: float, k2: np.ndarray, modes: bool = True) -> None:
    _flow_H1(cfg, s, 0.5 * h)
    _flow_H2(cfg, s, 0.5 * h, modes)
    _flow_H3(cfg, s, h, k2, modes)
    _flow_H2(cfg, s, 0.5 * h, modes)
    _flow_H1(cfg, s, 0.5 * h)
    s.eta = s.eta + h


def step(cfg: O.LatticeConfig, s: LinearState, k2: Optional[np.ndarray] = None) -> None:
    """One time step d-eta of the background and every perturbation mode;
    d-eta by the lattice's rule (O.step_size: dt, or dt / a at the step's start
    for the physical-time step of Sec. 3.1)."""
    if k2 is None:
        k2 = k_eff2(cfg.n, cfg.stencil)
    deta = O.step_size(cfg, s)
    for w in O.stage_weights(cfg.order):
        _stage(cfg, s, w * deta, k2)


def evolve(cfg: O.LatticeConfig, s: LinearState, steps: int) -> LinearState:
    k2 = k_eff2(cfg.n, cfg.stencil)
    for _ in range(int(steps)):
        step(cfg, s, k2)
    return s


def distinct_k2(k2: np.ndarray, tol: float = 1e-12) -> Tuple[np.ndarray, np.ndarray]:
    """The distinct k_eff^2 values of a lattice, ascending, and for every mode
    the index of its value.  Values closer than `tol` (relative to max(1, |v|))
    are one value: the same symbol reached through different cosines differs
    only in rounding (Sec. 2.2: equal k_eff^2 at several positions)."""
    flat = np.sort(k2.ravel())
    vals = [flat[0]]
    for v in flat[1:]:
        if v - vals[-1] > tol * max(1.0, abs(v)):
            vals.append(v)
    vals = np.array(vals)
    pos = np.searchsorted(vals, k2.ravel() + tol * np.maximum(1.0, np.abs(k2.ravel())),
                          side="right") - 1
    return vals, pos.reshape(k2.shape)


def transfer_matrices(cfg: O.LatticeConfig, a0: float, pa0: float, phi0: np.ndarray,
                      pi0: np.ndarray, k2_values: np.ndarray, steps: int) -> Tuple[np.ndarray, LinearState]:
    """The growth functions of Sec. 2.2: for each distinct k_eff^2, the
    2N_f x 2N_f matrix T with (dPhi, dPi)(eta) = T (dPhi, dPi)(0), obtained by
    evolving the 2N_f unit vectors with the background; returns T of shape
    (K, 2N_f, 2N_f) and the evolved background."""
    nf = len(phi0)
    K = len(k2_values)
    # modes laid out (N_f, K, 2N_f): column c is the c-th unit initial vector
    dphi = np.zeros((nf, K, 2 * nf))
    dpi = np.zeros((nf, K, 2 * nf))
    for i in range(nf):
        dphi[i, :, i] = 1.0
        dpi[i, :, nf + i] = 1.0
    s = LinearState(a=float(a0), pa=float(pa0), phi0=np.array(phi0, dtype=np.float64),
                    pi0=np.array(pi0, dtype=np.float64), dphi=dphi, dpi=dpi)
    k2 = np.asarray(k2_values, dtype=np.float64)[:, None]
    for _ in range(int(steps)):
        deta = O.step_size(cfg, s)
        for w in O.stage_weights(cfg.order):
            _stage(cfg, s, w * deta, k2)
    T = np.concatenate([np.transpose(s.dphi, (1, 0, 2)), np.transpose(s.dpi, (1, 0, 2))], axis=1)
    return T, s


def apply_transfer(T: np.ndarray, index: np.ndarray, dphi0: np.ndarray,
                   dpi0: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Modes at the later time from their initial values: each mode takes the
    matrix of its k_eff^2 (index: per-mode index into T)."""
    nf = dphi0.shape[0]
    y0 = np.concatenate([dphi0, dpi0], axis=0)                 # (2N_f, n, n, n)
    Tm = T[index]                                              # (n, n, n, 2N_f, 2N_f)
    y = np.einsum("...ij,j...->i...", Tm, y0)
    return y[:nf], y[nf:]
