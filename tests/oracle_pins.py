"""Pins for the CPU oracle: each function returns an error measure that the
mathematics (or the paper's printed numbers) fixes, independently of how the
oracle computes it.  ``test_oracle_pins.py`` asserts the bounds;
``test_oracle_mutations.py`` plants typical mistakes in the oracle and checks
that at least one pin sees each of them.
"""
from __future__ import annotations

import math
import os

import numpy as np

from oracle import pycool_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Table 1 and the triple jump -------------------------------------------

def read_table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_weights.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            order, idx, val = line.split()
            rows.setdefault(int(order), {})[int(idx)] = float(val)
    return rows


def composition_error_harmonic(order: int, nsteps: int, T: float = 2.0) -> float:
    """Kick-drift-kick leapfrog for q'' = -q (written here, not the oracle's flows)
    composed with the oracle's stage weights; error against cos(T)."""
    q, p = 1.0, 0.0
    h0 = T / nsteps
    w = O.stage_weights(order)
    for _ in range(nsteps):
        for wi in w:
            h = wi * h0
            p -= 0.5 * h * q
            q += h * p
            p -= 0.5 * h * q
    return math.hypot(q - math.cos(T), p + math.sin(T))


def composition_error_pendulum(order: int, nsteps: int, T: float = 2.0) -> float:
    """Same for the nonlinear pendulum q'' = -sin q, against a fine reference."""
    def run(n):
        q, p = 1.2, 0.0
        h0 = T / n
        w = O.stage_weights(order)
        for _ in range(n):
            for wi in w:
                h = wi * h0
                p -= 0.5 * h * math.sin(q)
                q += h * p
                p -= 0.5 * h * math.sin(q)
        return q, p
    from scipy.integrate import solve_ivp
    sol = solve_ivp(lambda t, y: [y[1], -math.sin(y[0])], (0.0, T), [1.2, 0.0],
                    method="DOP853", rtol=1e-14, atol=1e-14)
    qr, pr = sol.y[0, -1], sol.y[1, -1]
    q, p = run(nsteps)
    return math.hypot(q - qr, p - pr)


# --- Stencils ---------------------------------------------------------------

def stencil_symbol(stencil: str, theta) -> float:
    """Fourier symbol of Eq. D for the coefficient classes c_0..c_3:
    c0 + 2 c1 sum cos + 4 c2 sum_{d<e} cos cos + 8 c3 prod cos;
    for the fourth-order stencil, per axis (4 sin^2 t - 64 sin^2(t/2)) / 12
    (from 1 - cos t = 2 sin^2(t/2) applied to (-2 cos 2t + 32 cos t - 30)/12)."""
    if stencil == "4th":
        return sum((4 * math.sin(t) ** 2 - 64 * math.sin(t / 2) ** 2) / 12.0 for t in theta)
    c = O.stencil_coefficients(stencil)
    cs = [math.cos(t) for t in theta]
    pair = cs[0] * cs[1] + cs[0] * cs[2] + cs[1] * cs[2]
    return c[0] + 2 * c[1] * sum(cs) + 4 * c[2] * pair + 8 * c[3] * cs[0] * cs[1] * cs[2]


def plane_wave(n, mode, phase=0.3):
    idx = np.arange(n)
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    mx, my, mz = mode
    return np.cos(2 * np.pi * (mx * x + my * y + mz * z) / n + phase)


def plane_wave_symbol_error(stencil: str, n: int, mode) -> float:
    f = plane_wave(n, mode)
    theta = [2 * np.pi * m / n for m in mode]
    D = O.laplacian(f, stencil)
    return float(np.max(np.abs(D - stencil_symbol(stencil, theta) * f)))


def seven_point_closed_form_error(n: int, mode) -> float:
    """The 7-point symbol must be -sum_d 4 sin^2(k_d dx / 2) (dx = 1 here)."""
    f = plane_wave(n, mode)
    lam = -sum(4 * math.sin(math.pi * m / n) ** 2 for m in mode)
    return float(np.max(np.abs(O.laplacian(f, "7pt") - lam * f)))


def stokes_error(stencil: str, n: int = 9, seed: int = 3) -> float:
    """Sec. 2.1: sum phi D[phi] = -sum G[phi] on a periodic lattice."""
    f = np.random.default_rng(seed).standard_normal((n, n, n))
    lhs = O.lattice_sum(f * O.laplacian(f, stencil))
    rhs = -O.lattice_sum(O.gradient_G(f, stencil))
    return abs(lhs - rhs) / abs(rhs)


# --- Single Fourier mode of a free field on a static background --------------

def free_mode_cfg(n, order, dt, a0=1.3, m2=0.7, stencil="7pt"):
    cfg = O.LatticeConfig(n=n, L=n * 0.5, model="free", params=(m2,), dt=dt,
                          order=order, stencil=stencil, mpl=math.inf)
    return cfg


def free_mode_transfer_error(order: int, n: int = 10, mode=(1, 2, 3), steps: int = 60,
                             dt: float = 0.05, stencil: str = "7pt", a0: float = 1.3) -> float:
    """On a plane wave every flow acts as a 2x2 matrix on (phi_k, pi_k):
    Phi_H2(h): [[1, h/a^2], [0, 1]],  Phi_H3(h): [[1, 0], [(a^2 Dk/dx^2 - a^4 m^2) h, 1]],
    Phi_H1 is the identity (static a).  The oracle must equal the matrix product."""
    cfg = free_mode_cfg(n, order, dt, a0=a0, stencil=stencil)
    m2 = cfg.params[0]
    f = plane_wave(n, mode)
    A, B = 0.8, -0.35
    st = O.make_state(cfg, (A * f)[None], (B * f)[None], a0=a0)
    O.evolve(cfg, st, steps)
    theta = [2 * np.pi * m / n for m in mode]
    Dk = stencil_symbol(stencil, theta)
    K = a0 ** 2 * Dk / cfg.dx ** 2 - a0 ** 4 * m2
    M = np.eye(2)
    for _ in range(steps):
        for w in O.stage_weights(order):
            h = w * dt
            drift = np.array([[1.0, 0.5 * h / a0 ** 2], [0.0, 1.0]])
            kick = np.array([[1.0, 0.0], [K * h, 1.0]])
            M = drift @ kick @ drift @ M
    phik, pik = M @ np.array([A, B])
    e1 = np.max(np.abs(st.phi[0] - phik * f)) / max(abs(A), abs(phik))
    e2 = np.max(np.abs(st.pi[0] - pik * f)) / max(abs(B), abs(pik))
    return float(max(e1, e2))


def free_mode_continuum_error(order: int, dt: float, T: float = 3.0, n: int = 8,
                              mode=(1, 1, 0), a0: float = 1.3) -> float:
    """Against the exact time evolution of the spatially discrete system:
    phi'' = (Dk/dx^2 - a^2 m^2) phi, i.e. omega^2 = sum_d 4 sin^2(k_d dx/2)/dx^2 + a^2 m^2."""
    steps = int(round(T / dt))
    cfg = free_mode_cfg(n, order, dt, a0=a0)
    m2 = cfg.params[0]
    f = plane_wave(n, mode)
    A, B = 1.0, 0.0
    st = O.make_state(cfg, (A * f)[None], (B * f)[None], a0=a0)
    O.evolve(cfg, st, steps)
    omega2 = sum(4 * math.sin(math.pi * m / n) ** 2 for m in mode) / cfg.dx ** 2 + a0 ** 2 * m2
    w = math.sqrt(omega2)
    t = steps * dt
    phik = A * math.cos(w * t)
    pik = -A * a0 ** 2 * w * math.sin(w * t)
    return float(max(np.max(np.abs(st.phi[0] - phik * f)),
                     np.max(np.abs(st.pi[0] - pik * f)) / (a0 ** 2 * w)))


# --- Homogeneous mode against a high-accuracy ODE solve ----------------------

def homogeneous_error(order: int, dt: float, T: float = 1.5, model="chaotic2",
                      params=(1.0, 50.0), bg=(1.0, 0.3), mom=(-0.5, 0.2), mpl=1.0,
                      rho_m0=0.02, rho_r0=0.01) -> float:
    """Zero fluctuations: the lattice is homogeneous and the system is the
    background ODEs of Sec. 2.2 (Eqs. a-lin, phi-0) plus the matter term of
    Eq. H2, integrated here by scipy's DOP853 at rtol 1e-13."""
    from scipy.integrate import solve_ivp
    n = 2
    cfg = O.LatticeConfig(n=n, L=1.0, model=model, params=params, dt=dt, order=order,
                          mpl=mpl, rho_mat0=rho_m0, rho_rad0=rho_r0)
    nf = len(bg)
    phi = np.array([np.full((n, n, n), b) for b in bg])
    pi = np.array([np.full((n, n, n), p) for p in mom])
    st = O.make_state(cfg, phi, pi)
    y0 = [st.a, st.pa] + list(bg) + list(mom)
    VL = cfg.VL
    g2 = params[1] if model == "chaotic2" else 0.0
    m2 = params[0]

    def V_and_dV(f):
        # chaotic2 only: V = m^2 phi^2/2 + g^2 phi^2 chi^2/2
        ph, ch = f
        V = 0.5 * m2 * ph ** 2 + 0.5 * g2 * ph ** 2 * ch ** 2
        return V, [m2 * ph + g2 * ph * ch ** 2, g2 * ph ** 2 * ch]

    def rhs(t, y):
        a, pa = y[0], y[1]
        f, p = y[2:2 + nf], y[2 + nf:]
        V, dV = V_and_dV(f)
        da = -pa / (6 * VL * mpl ** 2)
        dpa = VL * a ** 3 * (sum(pi_ ** 2 for pi_ in p) / a ** 6 - 4 * V) - VL * rho_m0
        dphi = [pi_ / a ** 2 for pi_ in p]
        dpi = [-a ** 4 * d for d in dV]
        return [da, dpa] + dphi + dpi

    steps = int(round(T / dt))
    O.evolve(cfg, st, steps)
    sol = solve_ivp(rhs, (0.0, steps * dt), y0, method="DOP853", rtol=1e-13, atol=1e-13)
    yT = sol.y[:, -1]
    got = [st.a, st.pa] + [st.phi[i, 0, 0, 0] for i in range(nf)] + [st.pi[i, 0, 0, 0] for i in range(nf)]
    scale = [abs(v) + 1e-300 for v in yT]
    scale[1] = abs(yT[1])
    return float(max(abs(g - r) / max(s, 1e-3) for g, r, s in zip(got, yT, scale)))


# --- Exact background solutions (radiation, matter) -------------------------

def radiation_error(order: int, rho_r0: float = 3.0, a0: float = 1.1, dt: float = 0.07,
                    steps: int = 40) -> float:
    """Fields zero, radiation only: H = 0 fixes a' = sqrt(rho_r0/(3 m^2)) and p_a is
    constant (Eq. H2), so a(eta) = a0 + eta sqrt(rho_r0/3) exactly."""
    n = 2
    cfg = O.LatticeConfig(n=n, L=1.0, model="free", params=(1.0,), dt=dt, order=order,
                          mpl=1.0, rho_rad0=rho_r0)
    z = np.zeros((1, n, n, n))
    st = O.make_state(cfg, z, z, a0=a0)
    O.evolve(cfg, st, steps)
    exact = a0 + st.eta * math.sqrt(rho_r0 / 3.0)
    return abs(st.a - exact) / exact


def matter_error(order: int, rho_m0: float = 2.0, a0: float = 0.9, dt: float = 0.05,
                 steps: int = 40) -> float:
    """Fields zero, matter only: p_a' = -V_L rho_m0 is constant, so
    a(eta) = a0 + a0' eta + rho_m0 eta^2/(12 m^2) with a0' = sqrt(a0 rho_m0/(3 m^2)),
    which a symmetric composition of the exact flows reproduces to round-off."""
    n = 2
    cfg = O.LatticeConfig(n=n, L=1.0, model="free", params=(1.0,), dt=dt, order=order,
                          mpl=1.0, rho_mat0=rho_m0)
    z = np.zeros((1, n, n, n))
    st = O.make_state(cfg, z, z, a0=a0)
    O.evolve(cfg, st, steps)
    eta = st.eta
    exact = a0 + math.sqrt(a0 * rho_m0 / 3.0) * eta + rho_m0 * eta ** 2 / 12.0
    return abs(st.a - exact) / exact


# --- Constraint conservation, reversibility, second Friedmann equation -------

def _inhomogeneous_cfg(order, dt, n=12, g2=50.0, stencil="7pt"):
    return O.LatticeConfig(n=n, L=6.0, model="chaotic2", params=(1.0, g2), dt=dt,
                           order=order, stencil=stencil, mpl=1.0)


def _inhomogeneous_ics(n, seed=11, amp=0.05):
    rng = np.random.default_rng(seed)
    phi = np.stack([1.0 + amp * rng.standard_normal((n, n, n)),
                    0.2 + amp * rng.standard_normal((n, n, n))])
    pi = np.stack([-0.5 + amp * rng.standard_normal((n, n, n)),
                   amp * rng.standard_normal((n, n, n))])
    return phi, pi


def constraint_error(order: int, dt: float, T: float = 0.6, stencil="7pt") -> float:
    """max over the run of |H| / (a^4 V_L rho), sampled every step (Eq. H2 = 0)."""
    cfg = _inhomogeneous_cfg(order, dt, stencil=stencil)
    phi, pi = _inhomogeneous_ics(cfg.n)
    st = O.make_state(cfg, phi, pi)
    worst = 0.0
    for _ in range(int(round(T / dt))):
        O.step(cfg, st)
        e = O.energies(cfg, st)
        worst = max(worst, abs(O.hamiltonian(cfg, st)) / (st.a ** 4 * cfg.VL * e["rho"]))
    return worst


def reversibility_error(order: int = 4, steps: int = 30, dt: float = 0.02) -> float:
    cfg = _inhomogeneous_cfg(order, dt, n=8)
    phi, pi = _inhomogeneous_ics(cfg.n)
    st = O.make_state(cfg, phi, pi)
    a0, pa0 = st.a, st.pa
    O.evolve(cfg, st, steps)
    cfg.dt = -dt
    O.evolve(cfg, st, steps)
    return float(max(np.max(np.abs(st.phi - phi)) / np.max(np.abs(phi)),
                     np.max(np.abs(st.pi - pi)) / np.max(np.abs(pi)),
                     abs(st.a - a0) / a0, abs(st.pa - pa0) / abs(pa0)))


def second_friedmann_error(order: int = 4, dt: float = 0.002) -> float:
    """Central difference of a(eta) against a'' = a^3 <rho - 3P>/(6 m^2) + rho_m0/(6 m^2).

    Eq. Fried-2 prints a'' = -a^3<rho - 3P>/(6 m^2); the Hamiltonian flows (and the
    standard conformal-time result, a ~ eta^2 for matter) give the + sign used here."""
    cfg = _inhomogeneous_cfg(order, dt, n=8)
    cfg.rho_mat0 = 0.05
    phi, pi = _inhomogeneous_ics(cfg.n)
    st = O.make_state(cfg, phi, pi)
    O.evolve(cfg, st, 20)
    a_m = st.a
    O.step(cfg, st)
    e = O.energies(cfg, st)
    a_c = st.a
    O.step(cfg, st)
    a_p = st.a
    fd = (a_p - 2 * a_c + a_m) / dt ** 2
    rho3p = e["rho"] - 3 * e["P"]
    pred = a_c ** 3 * rho3p / 6.0 + cfg.rho_mat0 / 6.0
    return abs(fd - pred) / abs(pred)


def plane_wave_energy_error(stencil="7pt") -> float:
    """phi = A cos(k.x), pi = B cos(k.x), static a: rho_grad = -A^2 Dk/(4 a^2 dx^2),
    rho_kin = B^2/(4 a^6), rho_pot = m^2 A^2/4 (free model)."""
    n, mode, a0, A, B = 8, (1, 2, 0), 1.4, 0.3, -0.7
    cfg = free_mode_cfg(n, 2, 0.01, a0=a0, stencil=stencil)
    f = plane_wave(n, mode, phase=0.0)
    st = O.make_state(cfg, (A * f)[None], (B * f)[None], a0=a0)
    e = O.energies(cfg, st)
    Dk = stencil_symbol(stencil, [2 * np.pi * m / n for m in mode])
    want = [-A * A * Dk / (4 * a0 ** 2 * cfg.dx ** 2), B * B / (4 * a0 ** 6), cfg.params[0] * A * A / 4]
    got = [e["rho_grad"][0], e["rho_kin"][0], e["rho_pot"]]
    return max(abs(g - w) / abs(w) for g, w in zip(got, want))


def potential_golden_error() -> float:
    worst = 0.0
    with open(os.path.join(GOLDEN, "potential_values.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            model, params, fields, val = [s.strip() for s in line.split("|")]
            p = [float(v) for v in params.split()]
            x = np.array([[float(v)] for v in fields.split()])
            got = float(O.potential(model, p, x)[0])
            worst = max(worst, abs(got - float(val)) / abs(float(val)))
    return worst


def potential_derivative_error(model: str, params, point, h=1e-5) -> float:
    x = np.array([[v] for v in point], dtype=np.float64)
    dV = O.potential_derivative(model, params, x)[:, 0]
    worst = 0.0
    for i in range(len(point)):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (O.potential(model, params, xp)[0] - O.potential(model, params, xm)[0]) / (2 * h)
        worst = max(worst, abs(fd - dV[i]) / max(1.0, abs(dV[i])))
    return worst


# --- field statistics --------------------------------------------------------

def field_stats_error(n: int = 8) -> float:
    """Mean and variance of fields whose statistics are known in closed form:
      c + A cos(2 pi m.x / n) with a lattice mode m whose doubled mode is not
        zero mod n: the cosine sums to zero over the periods, its square to
        S/2, so mean = c and variance = A^2/2 exactly;
      a field equal to u on half the sites and v on the other half (the z < n/2
        slab): mean (u + v)/2, variance ((u - v)/2)^2.
    Returns the largest relative error of the oracle's (mean, variance)."""
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    worst = 0.0
    for c, A, m in ((1.0, 1e-3, (1, 2, 3)), (-0.5, 2.0, (0, 1, 0)), (3.0, 0.25, (2, 0, 1))):
        wave = np.cos(2.0 * math.pi * (m[0] * z + m[1] * y + m[2] * x) / n)
        s = O.State(a=1.0, pa=0.0, phi=(c + A * wave)[None].copy(), pi=np.zeros((1, n, n, n)))
        mean, var = O.field_stats(s, 0)
        worst = max(worst, abs(mean - c) / abs(c), abs(var - A * A / 2) / (A * A / 2))
    u, v = 1.25, -0.75
    f = np.where(z < n // 2, u, v).astype(np.float64)
    s = O.State(a=1.0, pa=0.0, phi=np.stack([np.zeros_like(f), f]), pi=np.zeros((2, n, n, n)))
    mean, var = O.field_stats(s, 1)
    worst = max(worst, abs(mean - (u + v) / 2) / abs((u + v) / 2),
                abs(var - ((u - v) / 2) ** 2) / ((u - v) / 2) ** 2)
    return worst


# --- the adaptive conformal step (physical-time steps, Sec. 3.1) -------------

def homogeneous_error_physical(order: int, dt: float, steps: int = 24) -> float:
    """Physical-time steps (d-eta = dt / a per step) on a homogeneous lattice
    against DOP853 on the background ODEs (Sec. 2.2, Eqs. a-lin, phi-0), both
    at the conformal time the steps reached; the oscillon potential at
    m_pl = 1, where a grows several-fold.  Error ~ dt^order."""
    from scipy.integrate import solve_ivp
    n = 2
    m2, lam, g = 1.0, 1.0, 0.5
    cfg = O.LatticeConfig(n=n, L=1.0, model="oscillon", params=(m2, lam, g), dt=dt, order=order,
                          mpl=1.0, time_step="physical")
    phi = np.full((1, n, n, n), 0.8)
    pi = np.full((1, n, n, n), 0.1)
    st = O.make_state(cfg, phi, pi)
    y0 = [st.a, st.pa, 0.8, 0.1]
    VL = cfg.VL

    def rhs(t, y):
        a, pa, f, p = y
        V = 0.5 * m2 * f ** 2 - 0.25 * lam * f ** 4 + g * f ** 6 / 6.0
        dV = m2 * f - lam * f ** 3 + g * f ** 5
        return [-pa / (6 * VL), VL * a ** 3 * (p * p / a ** 6 - 4 * V), p / a ** 2, -a ** 4 * dV]

    O.evolve(cfg, st, steps * int(round(0.2 / dt)))
    sol = solve_ivp(rhs, (0.0, st.eta), y0, method="DOP853", rtol=1e-13, atol=1e-14)
    yT = sol.y[:, -1]
    got = [st.a, st.pa, st.phi[0, 0, 0, 0], st.pi[0, 0, 0, 0]]
    return float(max(abs(u - r) / max(abs(r), 1e-3) for u, r in zip(got, yT)))


def constraint_error_physical(order: int, dt: float, T: float = 0.6) -> float:
    """max |H| / (a^4 V_L rho) over a run of physical-time steps (Eq. H2 = 0)."""
    cfg = _inhomogeneous_cfg(order, dt)
    cfg.time_step = "physical"
    phi, pi = _inhomogeneous_ics(cfg.n)
    st = O.make_state(cfg, phi, pi)
    worst = 0.0
    for _ in range(int(round(T / dt))):
        O.step(cfg, st)
        e = O.energies(cfg, st)
        worst = max(worst, abs(O.hamiltonian(cfg, st)) / (st.a ** 4 * cfg.VL * e["rho"]))
    return worst


def static_physical_equivalence() -> float:
    """On a static background (m_pl = inf) a stays a0, so physical-time steps
    of dt are conformal steps of dt / a0: with a0 = 2 (dt / a0 exact) the two
    runs must agree bit for bit.  Returns the largest difference."""
    cfg_p = _inhomogeneous_cfg(4, 0.03, n=8)
    cfg_p.mpl = math.inf
    cfg_p.time_step = "physical"
    cfg_c = _inhomogeneous_cfg(4, 0.015, n=8)
    cfg_c.mpl = math.inf
    phi, pi = _inhomogeneous_ics(8)
    sp = O.make_state(cfg_p, phi, pi, a0=2.0)
    sc = O.make_state(cfg_c, phi, pi, a0=2.0)
    O.evolve(cfg_p, sp, 12)
    O.evolve(cfg_c, sc, 12)
    return float(max(np.max(np.abs(sp.phi - sc.phi)), np.max(np.abs(sp.pi - sc.pi)),
                     abs(sp.eta - sc.eta)))


def radiation_physical_recurrence(order: int, rho_r0: float = 3.0, a0: float = 1.1,
                                  dt: float = 0.07, steps: int = 40) -> float:
    """Fields zero, radiation only: p_a is constant and every Phi_H1 moves a by
    -p_a h / (6 V_L m^2), so a step of d-eta = dt / a_n (the stage weights sum
    to one) gives a_{n+1} = a_n + C dt / a_n, C = -p_a / (6 V_L m^2), with a_n
    the scale factor at the start of the step.  Largest relative deviation
    from that recurrence."""
    n = 2
    cfg = O.LatticeConfig(n=n, L=1.0, model="free", params=(1.0,), dt=dt, order=order,
                          mpl=1.0, rho_rad0=rho_r0, time_step="physical")
    z = np.zeros((1, n, n, n))
    st = O.make_state(cfg, z, z, a0=a0)
    C = -st.pa / (6.0 * cfg.VL)
    worst = 0.0
    for _ in range(steps):
        a_n = st.a
        O.step(cfg, st)
        want = a_n + C * dt / a_n
        worst = max(worst, abs(st.a - want) / want)
    return worst


# --- the fourth-order stencil -------------------------------------------------

def fourth_order_accuracy_slope(mode=(1, 0, 0)) -> float:
    """The symbol of the fourth-order stencil on a plane wave, lambda(theta),
    against -|theta|^2: the difference must fall as theta^6 (fourth order in
    dx relative to theta^2).  Log2 ratio of |lambda + theta^2| at n = 32 and
    n = 64 (theta halves)."""
    errs = []
    for n in (32, 64):
        f = plane_wave(n, mode)
        D = O.laplacian(f, "4th")
        lam = float(np.sum(D * f) / np.sum(f * f))     # the eigenvalue on this wave
        th2 = sum((2 * math.pi * m / n) ** 2 for m in mode)
        errs.append(abs(lam + th2))
    return math.log2(errs[0] / errs[1])
