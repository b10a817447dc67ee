"""Pins of the observables oracle (CPU only): energy density and pressure at
every site (Sec. 2.1, Eq. rho-pres with the gradient stencil of Eq. G) and
the binned power spectrum (Sec. 2.4), against closed forms, the Stokes
identity, Parseval's theorem and a direct (non-FFT) Fourier sum; and planted
mistakes that each pin must catch."""
import math

import numpy as np
import pytest

from oracle import pycool_oracle as O
from oracle import pycool_observables as B


def _plane_wave_free(n=16, k_index=3, A=0.2, a=1.3, m2=0.7, L=5.0):
    """phi = A cos(theta), theta = 2 pi k x / n, pi = 0, free field, 7-point:
    G = 1/2 sum_faces (phi(x+e) - phi(x))^2; only the two x-neighbours differ,
    and cos(t +- k) - cos t = -+2 sin(t +- k/2) sin(k/2) gives
    G = 2 A^2 sin^2(k/2) (1 - cos(2 t) cos k)  (k = 2 pi k_index / n)."""
    cfg = O.LatticeConfig(n=n, L=L, model="free", params=(m2,), dt=0.01, mpl=math.inf)
    x = np.arange(n)
    t = 2.0 * math.pi * k_index * x / n
    phi = np.broadcast_to(A * np.cos(t)[None, None, :], (n, n, n))[None].copy()
    s = O.State(a=a, pa=0.0, phi=phi, pi=np.zeros_like(phi))
    kk = 2.0 * math.pi * k_index / n
    G = 2.0 * A * A * math.sin(kk / 2) ** 2 * (1.0 - np.cos(2 * t) * math.cos(kk))
    G = np.broadcast_to(G[None, None, :], (n, n, n))
    dx2 = cfg.dx ** 2
    V = 0.5 * m2 * phi[0] ** 2
    rho_want = G / (2 * a * a * dx2) + V
    P_want = -G / (6 * a * a * dx2) - V
    return cfg, s, rho_want, P_want


def plane_wave_error():
    cfg, s, rw, pw = _plane_wave_free()
    rho, P = B.energy_fields(cfg, s)
    return float(max(np.max(np.abs(rho - rw)) / np.max(np.abs(rw)),
                     np.max(np.abs(P - pw)) / np.max(np.abs(pw))))


def kinetic_error(a=1.7, B0=0.3, C0=-0.2):
    """phi = 0 (V = 0, G = 0), two constant momenta: rho = P = (B0^2 + C0^2)/(2 a^6)."""
    n = 6
    cfg = O.LatticeConfig(n=n, L=3.0, model="chaotic2", params=(1.0, 10.0), dt=0.01)
    z = np.zeros((2, n, n, n))
    pi = np.stack([np.full((n, n, n), B0), np.full((n, n, n), C0)])
    s = O.State(a=a, pa=-1.0, phi=z, pi=pi)
    rho, P = B.energy_fields(cfg, s)
    want = (B0 ** 2 + C0 ** 2) / (2 * a ** 6)
    return float(max(np.max(np.abs(rho - want)), np.max(np.abs(P - want))) / want)


def stokes_mean_error(stencil):
    """Lattice mean of rho(x) (G stencil) against energies() (sum phi D via the
    Stokes identity of Sec. 2.1), for a random two-field state."""
    n = 8
    cfg = O.LatticeConfig(n=n, L=4.0, model="chaotic2", params=(1.0, 30.0), dt=0.01,
                          stencil=stencil)
    rng = np.random.default_rng(3)
    phi = np.stack([1.0 + 0.1 * rng.standard_normal((n, n, n)), 0.1 * rng.standard_normal((n, n, n))])
    pi = np.stack([-0.5 + 0.1 * rng.standard_normal((n, n, n)), 0.1 * rng.standard_normal((n, n, n))])
    s = O.make_state(cfg, phi, pi, a0=1.2)
    rho, P = B.energy_fields(cfg, s)
    e = O.energies(cfg, s)
    return float(max(abs(rho.mean() - e["rho"]) / abs(e["rho"]), abs(P.mean() - e["P"]) / abs(e["P"])))


def direct_dft_spectrum(f):
    """The binned spectrum with every coefficient summed directly (no FFT) and
    the shells found by enumerating integer vectors (small n only)."""
    n = f.shape[0]
    S = f.size
    nb = int(math.floor(math.sqrt(3.0) * n / 2.0)) + 2
    power = np.zeros(nb)
    count = np.zeros(nb, dtype=np.int64)
    idx = np.arange(n)
    zz, yy, xx = np.meshgrid(idx, idx, idx, indexing="ij")
    for kz in range(n):
        for ky in range(n):
            for kx in range(n):
                ph = np.exp(-2j * math.pi * (kz * zz + ky * yy + kx * xx) / n)
                Fk = np.sum(f * ph)
                m = [(v if v <= n // 2 else v - n) for v in (kz, ky, kx)]
                bb = int(round(math.sqrt(sum(v * v for v in m))))
                power[bb] += abs(Fk) ** 2 / S ** 2
                count[bb] += 1
    return power, count


def spectrum_errors():
    rng = np.random.default_rng(5)
    f = rng.standard_normal((5, 5, 5)) + 0.3
    p, c = B.spectrum(f)
    pd, cd = direct_dft_spectrum(f)
    parseval = abs(p.sum() - np.mean(f * f)) / np.mean(f * f)
    direct = float(np.max(np.abs(p - pd)) / np.max(pd))
    counts_ok = np.array_equal(c, cd) and c.sum() == f.size
    # a plane wave of |m| = 3 puts A^2/2 into shell 3 and nothing elsewhere
    n = 12
    x = np.arange(n)
    A = 0.7
    w = np.broadcast_to(A * np.cos(2 * math.pi * 3 * x / n)[None, None, :], (n, n, n))
    pw, cw = B.spectrum(w)
    wave = abs(pw[3] - A * A / 2) / (A * A / 2) + float(np.sum(np.abs(np.delete(pw, 3))))
    shells = cw[0] == 1 and cw[1] == 18     # |m|^2 = 1 (6 vectors) and 2 (12 vectors)
    return parseval, direct, wave, bool(counts_ok and shells)


def _checks():
    par, direct, wave, counts = spectrum_errors()
    return {"plane_wave": plane_wave_error() < 1e-12, "kinetic": kinetic_error() < 1e-14,
            "stokes7": stokes_mean_error("7pt") < 1e-12,
            "stokes27": stokes_mean_error("iso27") < 1e-12,
            "parseval": par < 1e-12, "direct": direct < 1e-12, "wave": wave < 1e-12,
            "counts": counts}


def test_energy_fields_plane_wave_closed_form():
    assert plane_wave_error() < 1e-12


def test_energy_fields_kinetic_closed_form():
    assert kinetic_error() < 1e-14


@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
def test_energy_field_means_match_the_stokes_form(stencil):
    assert stokes_mean_error(stencil) < 1e-12


def test_spectrum_parseval_direct_sum_plane_wave_and_shells():
    par, direct, wave, counts = spectrum_errors()
    assert par < 1e-12 and direct < 1e-12 and wave < 1e-12 and counts


def _ef_grad_factor(cfg, s):     # (nabla phi)^2 / a^2 instead of / (2 a^2)
    rho, P = _orig_ef(cfg, s)
    a, dx2 = s.a, cfg.dx ** 2
    g = sum(O.gradient_G(s.phi[i], cfg.stencil) for i in range(s.phi.shape[0])) / (a * a * dx2)
    return rho + 0.5 * g, P


def _ef_pressure_third(cfg, s):  # -G/(3 a^2 dx^2) in P
    rho, P = _orig_ef(cfg, s)
    a, dx2 = s.a, cfg.dx ** 2
    g = sum(O.gradient_G(s.phi[i], cfg.stencil) for i in range(s.phi.shape[0])) / (a * a * dx2)
    return rho, P - g / 6.0


def _ef_kinetic_a4(cfg, s):      # pi^2 / (2 a^4)
    rho, P = _orig_ef(cfg, s)
    a = s.a
    k = sum(s.pi[i] ** 2 for i in range(s.pi.shape[0]))
    return rho + k * (1 / (2 * a ** 4) - 1 / (2 * a ** 6)), P + k * (1 / (2 * a ** 4) - 1 / (2 * a ** 6))


def _spec_S_norm(f):             # |F|^2 / S instead of / S^2
    p, c = _orig_spec(f)
    return p * f.size, c


def _spec_floor(f):              # shells floor(|m|) instead of round(|m|)
    n = f.shape[0]
    F = np.fft.fftn(f)
    m = np.fft.fftfreq(n) * n
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    b = np.floor(np.sqrt(mz * mz + my * my + mx * mx)).astype(np.int64)
    nb = B.spectrum_bins(n)
    p = np.zeros(nb)
    c = np.zeros(nb, dtype=np.int64)
    np.add.at(p, b.ravel(), (np.abs(F) ** 2 / float(f.size) ** 2).ravel())
    np.add.at(c, b.ravel(), 1)
    return p, c


_orig_ef = B.energy_fields
_orig_spec = B.spectrum

MUTATIONS = {
    "gradient term 1/a^2": ("energy_fields", _ef_grad_factor),
    "pressure gradient 1/3": ("energy_fields", _ef_pressure_third),
    "kinetic 1/a^4": ("energy_fields", _ef_kinetic_a4),
    "spectrum over S": ("spectrum", _spec_S_norm),
    "shells by floor": ("spectrum", _spec_floor),
}


def test_unmutated_observables_pass_every_check():
    bad = [k for k, ok in _checks().items() if not ok]
    assert not bad, bad


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_each_planted_observable_mistake_fails_some_pin(name, monkeypatch):
    attr, repl = MUTATIONS[name]
    monkeypatch.setattr(B, attr, repl)
    failed = [k for k, ok in _checks().items() if not ok]
    assert failed, f"planted mistake '{name}' passed every pin"
