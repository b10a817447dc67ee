"""Shared helpers for the GPU tests: run the same seeded problem through the
C ABI (CUDA path) and through the CPU oracle, and compare."""
from __future__ import annotations

import math

import numpy as np

from oracle import pycool_oracle as O
from paper_1201_5029_gb300 import inputs as I

STENCIL_NAMES = {7: "7pt", 27: "iso27"}


def oracle_cfg(w: dict, n=None, order=None, stencil="7pt", dt=None, mpl=None,
               time_step="conformal") -> O.LatticeConfig:
    return O.LatticeConfig(n=int(n or w["n"]), L=w["L"], model=w["model"], params=w["params"],
                           dt=float(dt if dt is not None else w["dt"]),
                           order=int(order or w["order"]), stencil=stencil,
                           mpl=float(mpl if mpl is not None else w["mpl"]),
                           rho_rad0=w.get("rho_rad0", 0.0), rho_mat0=w.get("rho_mat0", 0.0),
                           time_step=time_step)


def gpu_cfg(P, w: dict, n=None, order=None, stencil="7pt", precision="fp64", dt=None, mpl=None,
            time_step="conformal"):
    return P.make_config(n=int(n or w["n"]), L=w["L"], model=w["model"], params=w["params"],
                         dt=float(dt if dt is not None else w["dt"]),
                         order=int(order or w["order"]), precision=precision, stencil=stencil,
                         mpl=float(mpl if mpl is not None else w["mpl"]),
                         rho_rad0=w.get("rho_rad0", 0.0), rho_mat0=w.get("rho_mat0", 0.0),
                         time_step=time_step)


def run_gpu(P, cfg, phi, pi, steps, a0=1.0, chunks=1):
    sim = P.Simulation(cfg)
    sim.set_initial(phi, pi, a0=a0)
    per = [steps // chunks + (1 if i < steps % chunks else 0) for i in range(chunks)]
    for s in per:
        sim.evolve(s)
    e = sim.energies()
    gphi, gpi = sim.get_fields()
    sim.close()
    return gphi, gpi, e


def run_oracle(ocfg, phi, pi, steps, a0=1.0):
    st = O.make_state(ocfg, phi, pi, a0=a0)
    O.evolve(ocfg, st, steps)
    return st, O.energies(ocfg, st)


def field_errors(g: np.ndarray, o: np.ndarray) -> list:
    """Per-field normwise relative error max|g - o| / max|o|."""
    out = []
    for f in range(o.shape[0]):
        scale = float(np.max(np.abs(o[f])))
        out.append(float(np.max(np.abs(g[f] - o[f]))) / (scale if scale > 0 else 1.0))
    return out


# Unit roundoff of float64 (round to nearest).
EPS64 = 2.0 ** -53
# Per-stage rounding budget of the fluctuation check, in units of EPS64 times
# the field's magnitude: each stage rounds phi and pi a few times at the
# magnitude of the field (drift, kick, stencil sum); two implementations that
# round in different orders drift apart by at most a small multiple of that per
# stage.  40 covers the measured errors of every FP64 parity case on GB300
# with a margin of 4.5 or more (the smallest: the momenta of the 256^3 Q-ball
# after one order-8 step, 1.5e-10 against a bound of 6.9e-10; most cases sit
# 20-100 times below their bound).
FLUCT_K = 40.0


def fluct_errors(g: np.ndarray, o: np.ndarray) -> list:
    """Per-field error at the scale of the fluctuations:
    max|g - o| / max|o - mean(o)|.

    A field that sits on a homogeneous background (phi ~ 1 with fluctuations
    of 1e-5) is checked by field_errors only to ~1e-5 of the part the sweep
    actually evolves; this measure divides by the fluctuations themselves."""
    out = []
    for f in range(o.shape[0]):
        scale = float(np.max(np.abs(o[f] - o[f].mean())))
        if scale == 0.0:
            scale = float(np.max(np.abs(o[f]))) or 1.0
        out.append(float(np.max(np.abs(g[f] - o[f]))) / scale)
    return out


def fluct_tolerances(o: np.ndarray, stages: int, floor: float) -> list:
    """Bound of fluct_errors for the FP64 form after `stages` stage sweeps:
    max(floor, FLUCT_K * stages * EPS64 * max|o| / max|o - mean(o)|).

    The absolute rounding difference between two FP64 evaluations of the method
    grows at most by about FLUCT_K EPS64 |o| per stage; relative to the
    fluctuation scale that is the ratio of background to fluctuations times
    that.  For a field with no background (ratio ~1) the bound is the normwise
    tolerance `floor`."""
    out = []
    for f in range(o.shape[0]):
        scale = float(np.max(np.abs(o[f] - o[f].mean())))
        big = float(np.max(np.abs(o[f])))
        ratio = big / scale if scale > 0 else 1.0
        out.append(max(floor, FLUCT_K * max(stages, 1) * EPS64 * ratio))
    return out


def rel(a: float, b: float) -> float:
    return abs(a - b) / max(abs(b), 1e-300)


def stats_of(e: dict, variances) -> dict:
    """The statistics a long chaotic run is compared on: a, rho and its parts,
    and the per-field variances, as one flat dict of floats."""
    out = {"a": float(e["a"]), "rho": float(e["rho"]), "rho_pot": float(e["rho_pot"])}
    for f, v in enumerate(variances):
        out[f"rho_kin{f}"] = float(e["rho_kin"][f])
        out[f"rho_grad{f}"] = float(e["rho_grad"][f])
        out[f"var{f}"] = float(v)
    return out


def _nudge(x, rng):
    """x moved by one ulp up or down at every entry (seeded signs)."""
    up = rng.random(np.shape(x)) < 0.5
    return np.where(up, np.nextafter(x, np.inf), np.nextafter(x, -np.inf))


def oracle_checkpoints(args):
    """Oracle run for the long-run statistics test (one process each):
    args = (workload name, n, order, dt, steps, every, perturbation, seed).
    The perturbation models the rounding of an implementation that computes
    the same method in another order or precision, applied after every step:
      "none" : the oracle as it stands;
      "ulp"  : every value of phi and pi, and a and p_a, moved by one ulp up
               or down (seeded signs): rounding differences of the FP64 form;
      "fp32" : the fluctuations of phi and pi about their lattice means
               rounded to float32: the split form's representation of them.
    Returns the statistics at every `every` steps."""
    name, n, order, dt, steps, every, kind, seed = args
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    cfg = oracle_cfg(w, n=n, order=order, dt=dt)
    st = O.make_state(cfg, phi, pi)
    rng = np.random.default_rng(seed)
    out = []
    for k in range(steps):
        O.step(cfg, st)
        if kind == "ulp":
            st.phi[...] = _nudge(st.phi, rng)
            st.pi[...] = _nudge(st.pi, rng)
            st.a = float(_nudge(st.a, rng))
            st.pa = float(_nudge(st.pa, rng))
        elif kind == "fp32":
            for arr in (st.phi, st.pi):
                for f in range(arr.shape[0]):
                    m = float(np.mean(arr[f]))
                    arr[f] = m + (arr[f] - m).astype(np.float32).astype(np.float64)
        if (k + 1) % every == 0:
            e = O.energies(cfg, st)
            out.append(stats_of(e, [O.field_stats(st, f)[1] for f in range(phi.shape[0])]))
    return out
