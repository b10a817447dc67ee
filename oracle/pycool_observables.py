"""CPU oracle for the output-interval observables of PyCOOL (Sec. 2.1, 2.4).

TEST INFRASTRUCTURE ONLY, like ``pycool_oracle``: nothing in the product path
may import it.

What it is
----------
Plain FP64 numpy restatements of
* the energy density and pressure of the scalar fields at every lattice site
  (Sec. 2.1, Eq. rho-pres), with the gradient terms (nabla phi_i)^2 taken as
  G[phi_i] / dx^2 from the stencil of Eq. G and the time derivatives from the
  momenta, phi_i' = pi_i / a^2 (Eq. pi-i):
      rho(x) = sum_i [ pi_i^2 / (2 a^6) + G[phi_i](x) / (2 a^2 dx^2) ] + V(phi(x))
      P(x)   = sum_i [ pi_i^2 / (2 a^6) - G[phi_i](x) / (6 a^2 dx^2) ] - V(phi(x));
* the power spectrum of a lattice field binned in shells of the integer wave
  vector (one of the spectra of the post-processing of Sec. 2.4).

Reading (the paper only names its spectra, after LATTICEEASY and Defrost,
without definitions): with F_k = sum_x f(x) exp(-2 pi i m.x / n) (numpy's
unnormalised forward transform), m the signed integer wave vector of mode k,
the spectrum of f is
      power[b] = sum over modes with round(|m|) = b of |F_k|^2 / S^2,
      count[b] = number of those modes,
for b = 0 .. nbins - 1 with nbins = floor(sqrt(3) n / 2) + 2.  By Parseval the
bins add up to the lattice mean of f^2.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np

from . import pycool_oracle as O

__all__ = ["energy_fields", "spectrum_bins", "spectrum"]


def energy_fields(cfg: O.LatticeConfig, s: O.State) -> Tuple[np.ndarray, np.ndarray]:
    """rho(x) and P(x) of Eq. rho-pres at every site of a synchronised state."""
    a, dx2 = s.a, cfg.dx ** 2
    kin = np.zeros(s.phi.shape[1:])
    grad = np.zeros(s.phi.shape[1:])
    for i in range(s.phi.shape[0]):
        kin = kin + s.pi[i] * s.pi[i] / (2.0 * a ** 6)
        grad = grad + O.gradient_G(s.phi[i], cfg.stencil) / (a * a * dx2)
    V = O.potential(cfg.model, cfg.params, s.phi)
    rho = kin + 0.5 * grad + V
    P = kin - grad / 6.0 - V
    return rho, P


def spectrum_bins(n: int) -> int:
    """Number of shells of the binned spectrum of an n^3 lattice."""
    return int(math.floor(math.sqrt(3.0) * n / 2.0)) + 2


def spectrum(f: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(power, count) of a real field f[z][y][x] in shells round(|m|)."""
    n = f.shape[0]
    S = f.size
    F = np.fft.fftn(f)
    m = np.fft.fftfreq(n) * n                      # signed integer wave numbers
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    b = np.rint(np.sqrt(mz * mz + my * my + mx * mx)).astype(np.int64)
    nb = spectrum_bins(n)
    power = np.zeros(nb)
    count = np.zeros(nb, dtype=np.int64)
    p = (np.abs(F) ** 2 / float(S) ** 2).ravel()
    for k, bk in enumerate(b.ravel()):
        power[bk] += p[k]
        count[bk] += 1
    return power, count
