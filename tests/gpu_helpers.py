"""Shared helpers for the GPU tests: run the same seeded problem through the
C ABI (CUDA path) and through the CPU oracle, and compare."""
from __future__ import annotations

import math

import numpy as np

from oracle import pycool_oracle as O
from paper_1201_5029_gb300 import inputs as I

STENCIL_NAMES = {7: "7pt", 27: "iso27"}


def oracle_cfg(w: dict, n=None, order=None, stencil="7pt", dt=None, mpl=None) -> O.LatticeConfig:
    return O.LatticeConfig(n=int(n or w["n"]), L=w["L"], model=w["model"], params=w["params"],
                           dt=float(dt if dt is not None else w["dt"]),
                           order=int(order or w["order"]), stencil=stencil,
                           mpl=float(mpl if mpl is not None else w["mpl"]),
                           rho_rad0=w.get("rho_rad0", 0.0), rho_mat0=w.get("rho_mat0", 0.0))


def gpu_cfg(P, w: dict, n=None, order=None, stencil="7pt", precision="fp64", dt=None, mpl=None):
    return P.make_config(n=int(n or w["n"]), L=w["L"], model=w["model"], params=w["params"],
                         dt=float(dt if dt is not None else w["dt"]),
                         order=int(order or w["order"]), precision=precision, stencil=stencil,
                         mpl=float(mpl if mpl is not None else w["mpl"]),
                         rho_rad0=w.get("rho_rad0", 0.0), rho_mat0=w.get("rho_mat0", 0.0))


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


def rel(a: float, b: float) -> float:
    return abs(a - b) / max(abs(b), 1e-300)
