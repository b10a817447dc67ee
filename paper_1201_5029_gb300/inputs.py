"""Seeded synthetic inputs for the lattice stepper: workloads and initial fields.

This module holds no arithmetic of the method itself (no stencil, no
potential, no flow): only the workload table and random initial conditions.
It is the one place that both the CUDA path's tests/bench and the CPU oracle
draw their inputs from, so that both sides see identical arrays.

The paper's own runs (Sec. 3) need its initial-condition code (Defrost's
convolution method, only cited) and hours of GPU time; the workloads below are
synthetic stand-ins with the same models, lattice sizes and integrator orders.

Initial-condition recipes
-------------------------
white    : phi_i = background_i + N(0, noise), pi_i = momentum_i + N(0, noise),
           drawn with numpy's PCG64 (``default_rng(seed)``) in the order
           phi_1..phi_N then pi_1..pi_N, each array in [z][y][x] order.
spectral : per field, real white noise is filtered in Fourier space by
           sqrt(1/(2 w_k)) (fields) or sqrt(w_k/2) (momenta) with
           w_k^2 = k^2 + m_eff_i^2 (continuum k = 2 pi |m| / L; k = 0 removed),
           then both are scaled by the one constant that makes the field
           fluctuation rms equal to ``noise``.  The draw order is as for white.
           m_eff_i^2 is a number stated in the workload table, not computed here.
"""
from __future__ import annotations

import math
from typing import Dict, Optional, Tuple

import numpy as np

SQRT2 = math.sqrt(2.0)

# Model parameter vectors, in the order the C config's params[] takes them:
#   free / free2 : (m2,)
#   chaotic2     : (m2, g2)
#   oscillon     : (m2, lam, g)
#   qball        : (m2, K, M)
WORKLOADS: Dict[str, dict] = {
    # Two-field chaotic preheating, 32^3, leapfrog.
    "preheat32": dict(
        n=32, L=10.0, model="chaotic2", params=(1.0, 1.0e4), order=2, dt=0.005,
        steps=100, mpl=1.0, ic="white", seed=1201001,
        background=(1.0, 0.0), momentum=(-0.5, 0.0), noise=1.0e-5),
    # Same model at 128^3, 4th order, seeded spectrum |delta_k|^2 ~ 1/(2 w_k).
    "preheat128": dict(
        n=128, L=10.0, model="chaotic2", params=(1.0, 1.0e4), order=4, dt=0.01,
        steps=2000, mpl=1.0, ic="spectral", seed=1201002,
        background=(1.0, 0.0), momentum=(-0.5, 0.0), noise=1.0e-5,
        m_eff2=(1.0, 1.0e4)),
    # Single-field oscillon, 256^3, 6th order.
    "oscillon256": dict(
        n=256, L=50.0, model="oscillon", params=(1.0, 1.0, 0.5), order=6, dt=0.02,
        steps=5000, mpl=100.0, ic="white", seed=1201003,
        background=(0.8,), momentum=(0.0,), noise=1.0e-4),
    # Curvaton Q-ball, two real components, 256^3, 8th order.
    "qball256": dict(
        n=256, L=200.0, model="qball", params=(1.0, -0.1, 1.0), order=8, dt=0.05,
        steps=4000, mpl=100.0, ic="white", seed=1201004,
        background=(SQRT2 * math.cos(0.3), SQRT2 * math.sin(0.3)), momentum=(0.0, 0.0),
        noise=1.0e-6),
}

# Serving mix: lattice sides and their weights, orders, per-model step sizes.
SERVING_MIX = dict(
    sizes=(32, 64, 128, 256, 384), size_weights=(0.4, 0.3, 0.15, 0.1, 0.05),
    orders=(2, 4, 6, 8), steps=(200, 5000), models=("preheat32", "oscillon256", "qball256"),
    dt={"chaotic2": 0.005, "oscillon": 0.02, "qball": 0.05},
    L={"chaotic2": 10.0, "oscillon": 50.0, "qball": 200.0},
    requests=500, seed=1201005, arrival_seed=1201099,
)


def workload(name: str, **overrides) -> dict:
    """A copy of a named workload with fields replaced by ``overrides``."""
    w = dict(WORKLOADS[name])
    w.update(overrides)
    return w


def nfields(w: dict) -> int:
    return len(w["background"])


def white_ics(w: dict, n: Optional[int] = None, seed: Optional[int] = None
              ) -> Tuple[np.ndarray, np.ndarray]:
    """Homogeneous background plus Gaussian white noise, float64 (N_f, n, n, n)."""
    n = int(n if n is not None else w["n"])
    rng = np.random.default_rng(w["seed"] if seed is None else seed)
    nf = nfields(w)
    sig = float(w["noise"])
    phi = np.empty((nf, n, n, n), dtype=np.float64)
    pi = np.empty((nf, n, n, n), dtype=np.float64)
    for i in range(nf):
        phi[i] = w["background"][i] + sig * rng.standard_normal((n, n, n))
    for i in range(nf):
        pi[i] = w["momentum"][i] + sig * rng.standard_normal((n, n, n))
    return phi, pi


def _filter(noise: np.ndarray, L: float, m2: float, power: float) -> np.ndarray:
    n = noise.shape[0]
    kz = np.fft.fftfreq(n, d=1.0 / n)
    kx = np.fft.rfftfreq(n, d=1.0 / n)
    mz, my, mx = np.meshgrid(kz, kz, kx, indexing="ij")
    k2 = (2.0 * np.pi / L) ** 2 * (mz * mz + my * my + mx * mx)
    w = np.sqrt(k2 + m2)
    f = np.fft.rfftn(noise)
    f *= w ** power
    f[0, 0, 0] = 0.0
    return np.fft.irfftn(f, s=noise.shape, axes=(0, 1, 2))


def spectral_ics(w: dict, n: Optional[int] = None, seed: Optional[int] = None
                 ) -> Tuple[np.ndarray, np.ndarray]:
    """Background plus fluctuations with |delta_k|^2 ~ 1/(2 w_k), random phases."""
    n = int(n if n is not None else w["n"])
    rng = np.random.default_rng(w["seed"] if seed is None else seed)
    nf = nfields(w)
    raw_phi = [rng.standard_normal((n, n, n)) for _ in range(nf)]
    raw_pi = [rng.standard_normal((n, n, n)) for _ in range(nf)]
    phi = np.empty((nf, n, n, n), dtype=np.float64)
    pi = np.empty((nf, n, n, n), dtype=np.float64)
    for i in range(nf):
        m2 = float(w["m_eff2"][i])
        dphi = _filter(raw_phi[i], w["L"], m2, -0.5) / math.sqrt(2.0)
        dpi = _filter(raw_pi[i], w["L"], m2, 0.5) / math.sqrt(2.0)
        scale = float(w["noise"]) / float(np.sqrt(np.mean(dphi * dphi)))
        phi[i] = w["background"][i] + scale * dphi
        pi[i] = w["momentum"][i] + scale * dpi
    return phi, pi


def initial_fields(w: dict, n: Optional[int] = None, seed: Optional[int] = None
                   ) -> Tuple[np.ndarray, np.ndarray]:
    """The workload's initial (phi, pi), optionally at another lattice side/seed."""
    if w.get("ic", "white") == "spectral":
        return spectral_ics(w, n, seed)
    return white_ics(w, n, seed)


def plane_wave(n: int, mode: Tuple[int, int, int], amplitude: float = 1.0,
               phase: float = 0.0) -> np.ndarray:
    """cos(2 pi (m_x x + m_y y + m_z z)/n + phase) on an n^3 lattice, [z][y][x]."""
    idx = np.arange(n)
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    mx, my, mz = mode
    arg = 2.0 * np.pi * (mx * x + my * y + mz * z) / n + phase
    return amplitude * np.cos(arg)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) on numpy arrays of
    32-bit counters held in uint64: ten rounds of
      (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
    with the key advanced by (W0, W1) before every round but the first."""
    M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
    mask = np.uint64(0xFFFFFFFF)
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & mask for c in (c0, c1, c2, c3))
    ka, kb = np.uint64(k0 & 0xFFFFFFFF), np.uint64(k1 & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            ka = np.uint64((int(ka) + W0) & 0xFFFFFFFF)
            kb = np.uint64((int(kb) + W1) & 0xFFFFFFFF)
        p0 = np.uint64(M0) * c0
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ ka, lo1, hi0 ^ c3 ^ kb, lo0
    return c0, c1, c2, c3


def philox_normals(seed: int, arr: int, count: int) -> np.ndarray:
    """Standard normals z_e, e = 0..count-1, of array `arr`: element e is
    component e mod 4 of counter block e // 4 = (e//4, arr, 0, 0), key = seed;
    uniforms u = (x + 1/2) 2^-32, Box-Muller on (u0, u1) and (u2, u3)."""
    e = np.arange(count, dtype=np.uint64)
    blk = e >> np.uint64(2)
    comp = (e & np.uint64(3)).astype(np.int64)
    r0, r1, r2, r3 = philox4x32_10(blk, np.full_like(blk, arr), np.zeros_like(blk),
                                   np.zeros_like(blk), seed & 0xFFFFFFFF, seed >> 32)
    a = np.where(comp < 2, r0, r2).astype(np.float64)
    b = np.where(comp < 2, r1, r3).astype(np.float64)
    s = 2.0 ** -32
    u1, u2 = (a + 0.5) * s, (b + 0.5) * s
    rad = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * np.pi * u2
    return np.where(comp & 1, rad * np.sin(th), rad * np.cos(th))


def philox_white_ics(n: int, background, momentum, noise: float, seed: int
                     ) -> Tuple[np.ndarray, np.ndarray]:
    """The white-noise initial conditions a serving request generates on the
    device: phi_i = bg_i + noise z (array i), pi_i = mom_i + noise z (array N+i)."""
    nf = len(background)
    S = n ** 3
    phi = np.empty((nf, n, n, n), dtype=np.float64)
    pi = np.empty((nf, n, n, n), dtype=np.float64)
    for i in range(nf):
        phi[i] = (background[i] + noise * philox_normals(seed, i, S)).reshape(n, n, n)
        pi[i] = (momentum[i] + noise * philox_normals(seed, nf + i, S)).reshape(n, n, n)
    return phi, pi


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def serving_requests(count: Optional[int] = None, seed: Optional[int] = None,
                     steps_scale: float = 1.0) -> list:
    """The serving mix's request list: (workload name, n, order, steps, ic seed)."""
    mix = SERVING_MIX
    count = int(mix["requests"] if count is None else count)
    rng = np.random.default_rng(mix["seed"] if seed is None else seed)
    out = []
    for r in range(count):
        n = int(rng.choice(mix["sizes"], p=mix["size_weights"]))
        name = mix["models"][int(rng.integers(0, len(mix["models"])))]
        order = int(rng.choice(mix["orders"]))
        lo, hi = mix["steps"]
        steps = max(1, int(round(int(rng.integers(lo, hi + 1)) * steps_scale)))
        out.append(dict(workload=name, n=n, order=order, steps=steps,
                        seed=int(mix["seed"]) * 1000 + r))
    return out
