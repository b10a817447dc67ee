"""Throughput of the symplectic lattice step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload qball256]
                    [--extra preheat128,oscillon256] [--impl ours|reference]

Headline workload (default): the curvaton Q-ball problem on a 256^3 lattice,
two real field components, L = 200/m, 8th-order composition (15 stages per
step), d-eta = 0.05, seeded white-noise initial fluctuations -- the largest
configuration that is timed; its state (1.07 GB in FP64) is larger than L2.
The two other timed configurations (two-field preheating at 128^3, order 4;
the one-field oscillon at 256^3, order 6) are measured in the same run and
reported under "extra".  Every workload is timed in each form (FP64 and
split-FP32).  A "step" is one time step through the C ABI: evolve(1) = s
fused stage sweeps + the synchronising flush sweep (every row of the hot
path: background update, fused sweep, reductions, flush/energies), one launch
of the persistent kernel.

Metric: site-updates/s per stage = n^3 x stages / time, whole job (all ranks).
L2 is flushed (256 MiB write) between timed steps; each step is timed with CUDA
events on the simulation's stream.

--impl reference times the CPU oracle (oracle/pycool_oracle.py, the method as
written in the paper) on the host cores on the same workload: each timed step
is one second-order stage of the workload (a bounded sample of a time step).

Multi-GPU: the simulations are independent (replicas only, no collective on
the data path); under torchrun each rank runs its own replica and rank 0
reports the whole-job rate over the slowest rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "site-updates/s per stage vs HBM roofline (FP64, split-FP32); serving p50/p99"
UNIT = "site-updates/s"
FORMS = ("fp64", "split_fp32", "split_dd")
WORD = {"fp64": 8, "split_fp32": 4, "split_dd": 8}
KERNEL_FORM = {"fp64": "FP64", "split_fp32": "split", "split_dd": "splitDD"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# Algorithmic float64 operations per site (FMA = 2) of the method with the
# 7-point stencil, counted from the arithmetic each site needs (not from the
# instructions the kernel issues):
#   stage sweep: drift 2/field, Laplacian 7/field (6 adds + the centre FMA),
#     kick 4/field, sums pi^2 and phi D 4/field, sum V 1, plus the potential and
#     its gradient (chaotic2 9, oscillon 11, qball 12 + one log, free 3);
#   flush: drift 2/field, Laplacian 7/field, sums pi^2, phi D 4/field,
#     sum (phi - K) 1/field, sum (phi - K)^2 2/field, sum V 1, plus V alone
#     (chaotic2 5, oscillon 6, qball 6 + one log, free 2).
FP64_FLOPS_PER_SITE = {"chaotic2": 44.0, "oscillon": 29.0, "qball": 47.0, "free": 21.0}
FP64_FLUSH_FLOPS_PER_SITE = {"chaotic2": 38.0, "oscillon": 23.0, "qball": 39.0, "free": 19.0}
# GB300 float64 peak: 2 DFMA lanes per SM per clock (ncu: 304 predicated-on
# DFMA thread instructions per cycle for the 152 SMs) x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 304 * 2 * 2.07e9 / 1e12
# DRAM traffic per launch measured by ncu, one line per (workload, form):
#   <workload> <form> <kernel source hash> <dram read bytes> <dram write bytes>
# A figure counts only while the kernel sources still hash to the value it was
# taken with; otherwise the line's traffic is reported as null.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
NOMINAL_HBM_GBS = 8000.0   # GB300's nominal HBM3e bandwidth (the fractions also quote it)


# the sources evolve_persist is compiled from (its translation units and headers)
KERNEL_SOURCES = ("persist.cuh", "persist_fp64.cu", "persist_split.cu", "persist_dd.cu",
                  "persist_fp64_wide.cu", "persist_dd_wide.cu", "sweep.cuh", "internal.cuh",
                  "models.cuh", "models_dd.cuh", "dd.cuh")


def kernel_source_hash() -> str:
    """SHA-256 (first 16 hex digits) of the sources of the persistent evolve
    kernel: a traffic figure measured on other sources is not used."""
    h = hashlib.sha256()
    for name in sorted(KERNEL_SOURCES):
        with open(os.path.join(ROOT, "paper_1201_5029_gb300", "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, form: str):
    """DRAM bytes per launch from the ncu capture of the current kernels, or None."""
    try:
        cur = kernel_source_hash()
        with open(TRAFFIC_FILE) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 5 and not line.startswith("#") and parts[0] == workload \
                        and parts[1] == form and parts[2] == cur:
                    return float(parts[3]) + float(parts[4])
    except OSError:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 100 ms during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, tag: str = "main"):
        self.index = index
        self.proc = None
        self.used = False   # a second `with` appends: summary() covers every region
        self.path = os.path.join("/tmp", f"pycool_clocks_{os.getpid()}_{tag}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "a" if self.used else "w")
            self.used = True
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest_rank_ms(tot, forms, device):
    """Max over ranks of each form's timed total (ms).

    The replicas run independently; the job ends when the slowest rank ends,
    so the whole-job time of a form is the maximum of the ranks' totals.
    Identity when no process group is initialised (one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return {f: float(tot[f]) for f in forms}
    t = torch.tensor([tot[f] for f in forms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return {f: float(t[i]) for i, f in enumerate(forms)}


def whole_job_rate(ws, sites, stages, steps, total_ms):
    """Site-updates per second of the whole job: every rank updated `sites`
    sites `stages` times per step for `steps` steps within `total_ms`."""
    return ws * sites * stages * steps / (total_ms / 1e3)


def run_form(P, torch, w, precision, steps, warmup, flush_buf, phi, pi, stream):
    """Time `steps` evolve(1) calls of one form; returns a dict of measurements."""
    cfg = P.config_from_workload(w, precision=precision)
    sim = P.Simulation(cfg, stream=stream)
    sim.set_initial(phi, pi)
    for _ in range(warmup):
        sim.evolve(1)
    assert sim.sync() == P.OK
    s = P.pycool_stages_per_step(w["order"])
    launches0 = sim.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush_buf.add_(1)           # 256 MiB read+write: evicts the lattice from L2
        ev[i][0].record(stream)
        sim.evolve(1)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    st = sim.sync()
    launches = sim.kernel_launches() - launches0
    ms = [a.elapsed_time(b) for a, b in ev]
    e = sim.energies()
    sim.close()
    return dict(ms=ms, total_ms=sum(ms), launches=launches, stages=s, status=st, energies=e)


def e2e_form(P, torch, w, precision, steps, phi_pin, pi_pin, out_phi, out_pi, stream):
    """Through the public API with host buffers: H2D of the inputs, one time step,
    D2H of the result, every step."""
    cfg = P.config_from_workload(w, precision=precision)
    sim = P.Simulation(cfg, stream=stream)
    sim.set_initial(phi_pin, pi_pin)
    sim.evolve(1)
    sim.get_fields(out_phi, out_pi)
    torch.cuda.synchronize()
    phases = [0.0, 0.0, 0.0]
    t0 = time.perf_counter()
    for _ in range(steps):
        ta = time.perf_counter()
        sim.set_initial(phi_pin, pi_pin)     # H2D from pinned host memory
        tb = time.perf_counter()
        sim.evolve(1)
        sim.sync()
        tc = time.perf_counter()
        sim.get_fields(out_phi, out_pi)      # D2H of the step's result
        td = time.perf_counter()
        phases[0] += tb - ta
        phases[1] += tc - tb
        phases[2] += td - tc
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    sim.close()
    return dt, {"set_initial": 1e3 * phases[0] / steps, "evolve": 1e3 * phases[1] / steps,
                "get_fields": 1e3 * phases[2] / steps}


def roofline(w, form, s, ms_per_step, hbm, peak_kind):
    """Roofline object of the persistent kernel (one launch per time step of s
    stages) of a workload and form, from the CUDA-event time per launch."""
    S = w["n"] ** 3
    nf = len(w["background"])
    # algorithmic bytes per launch: s sweeps read and write phi and pi, the
    # flush reads both and writes phi
    launch_bytes = (s * 4 + 3) * nf * WORD[form] * S
    gbs = launch_bytes / (ms_per_step / 1e3) / 1e9
    kname = f"evolve_persist<{w['model']},7pt,{KERNEL_FORM[form]}>"
    traffic = measured_traffic(w["name"], form)
    common = {"traffic": traffic, "kernel": kname + " (one launch per time step)",
              "algorithmic_bytes_per_launch": launch_bytes,
              "traffic_over_algorithmic": (traffic / launch_bytes) if traffic else None}
    if form == "fp64":
        flops = S * (s * FP64_FLOPS_PER_SITE.get(w["model"], 40.0)
                     + FP64_FLUSH_FLOPS_PER_SITE.get(w["model"], 35.0))
        tf = flops / (ms_per_step / 1e3) / 1e12
        out = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": tf / FP64_PEAK_TFLOPS,
               "peak_kind": "float64 pipe: 2 DFMA/SM/clk x 152 SMs x 2.07 GHz (GB300 FP64 is "
                            "1/64 of FP32; float64 arithmetic binds this form, not HBM)",
               "flops_per_launch": flops, "achieved_gbs": gbs, "hbm_frac": gbs / hbm,
               "hbm_peak_gbs": hbm, "hbm_frac_of_nominal": gbs / NOMINAL_HBM_GBS}
    else:
        out = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
               "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
               "frac_of_nominal": gbs / NOMINAL_HBM_GBS}
        if form == "split_dd":
            out["note"] = ("double-float fluctuations: 8 bytes per value like FP64, arithmetic "
                           "on the FP32 pipe (error-free transformations); the form is held to "
                           "the FP64 parity tolerances")
    out.update(common)
    return out


def _serving_configs(P, I, reqs, prec):
    mix = I.SERVING_MIX
    out = []
    for r in reqs:
        w = I.workload(r["workload"])
        cfg = P.make_config(r["n"], mix["L"][w["model"]], w["model"], w["params"],
                            mix["dt"][w["model"]], order=r["order"], precision=prec, mpl=w["mpl"])
        out.append((cfg, P.make_ic(w["background"], w["momentum"], w["noise"]), r))
    return out


def _serve(P, items, arrivals, slots=64, budget=96 << 30, persist_min_n=None):
    """Submit each request at its arrival time (None: all at once), wait for all.
    Returns the server's latency percentiles and the aggregate rate.
    persist_min_n: side from which FP64 members run on the persistent kernel
    (None: the server's default)."""
    srv = P.pycool_server_create(budget, slots)
    if persist_min_n is not None:
        P.pycool_server_set_persistent_min_n(srv, persist_min_n)
    t0 = time.perf_counter()
    tickets, work = [], 0
    for i, (cfg, ic, r) in enumerate(items):
        if arrivals is not None:
            dt = arrivals[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
        tickets.append(P.pycool_server_submit(srv, cfg, ic, r["seed"], r["steps"]))
        work += r["n"] ** 3 * r["steps"] * P.pycool_stages_per_step(r["order"])
    bad = sum(P.pycool_server_wait(srv, t, 1800.0)[0] != P.OK for t in tickets)
    wall = time.perf_counter() - t0
    s = P.pycool_server_stats(srv)
    P.pycool_server_destroy(srv)
    return dict(p50_s=s["p50_s"], p99_s=s["p99_s"], site_updates_per_s=work / wall,
                completed=s["completed"], failed=int(bad), wall_s=wall)


def serving_leg(P, I, count, steps_scale, load, other_loads=(), calib_count=100,
                persist_min_n=256, compare_per_stage=False):
    """Serving mix (sizes 32..384^3, three models, orders 2..8): a closed-loop
    calibration of the FP64 form's capacity on the first `calib_count`
    requests, then the Poisson arrival stream of all `count` requests at
    `load` x that capacity for each form (the headline), and both forms at
    each of `other_loads` x that capacity (reported under "by_load").
    FP64 members of side >= persist_min_n (a multiple of 32; 0: none) run on
    the persistent kernel; compare_per_stage adds the FP64 replay of the same
    arrival stream with every member on the per-stage kernels."""
    reqs = I.serving_requests(count=count, steps_scale=steps_scale)
    work_of = lambda r: r["n"] ** 3 * r["steps"] * P.pycool_stages_per_step(r["order"])  # noqa
    mean_work = sum(work_of(r) for r in reqs) / len(reqs)
    items64 = _serving_configs(P, I, reqs, "fp64")
    calib = _serve(P, items64[:calib_count], None, persist_min_n=persist_min_n)
    capacity = calib["site_updates_per_s"] / mean_work          # requests/s
    rate = load * capacity
    arr = I.poisson_arrivals(rate, len(reqs), I.SERVING_MIX["arrival_seed"])
    out = {"requests": len(reqs), "steps_scale": steps_scale, "offered_load": load,
           "arrival_rate_per_s": rate, "capacity_fp64_req_per_s": capacity,
           "capacity_calibration": f"closed loop, first {min(calib_count, len(reqs))} requests, "
                                   "FP64",
           "mean_site_stages_per_request": mean_work,
           "persistent_min_n": persist_min_n,
           "latency": "submit (Poisson arrival) -> observables read back on the host"}
    items32 = _serving_configs(P, I, reqs, "split_fp32")
    for prec, items in (("fp64", items64), ("split_fp32", items32)):
        out[prec] = _serve(P, items, arr, persist_min_n=persist_min_n)
    if compare_per_stage:
        out["fp64_all_per_stage"] = _serve(P, items64, arr, persist_min_n=0)
    by_load = {}
    keep = ("p50_s", "p99_s", "site_updates_per_s", "completed", "failed")
    for lo in other_loads:
        arr_lo = I.poisson_arrivals(lo * capacity, len(reqs), I.SERVING_MIX["arrival_seed"])
        by_load[str(lo)] = {prec: {k: v for k, v in
                                   _serve(P, items, arr_lo, persist_min_n=persist_min_n).items()
                                   if k in keep}
                            for prec, items in (("fp64", items64), ("split_fp32", items32))}
    if by_load:
        out["by_load"] = by_load
    return out


def _oracle_stage_rate(args):
    """Oracle stages on one host core for about `budget` seconds (one process)."""
    name, n, budget = args
    from oracle import pycool_oracle as O
    from paper_1201_5029_gb300 import inputs as I
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    cfg = O.LatticeConfig(n=n, L=w["L"], model=w["model"], params=w["params"], dt=w["dt"],
                          order=w["order"], mpl=w["mpl"])
    st = O.make_state(cfg, phi, pi)
    ws = O.stage_weights(w["order"])
    done, t0 = 0, time.perf_counter()
    while True:
        O.second_order_stage(cfg, st, ws[done % len(ws)] * cfg.dt)
        done += 1
        el = time.perf_counter() - t0
        if el > budget:
            break
    return n ** 3 * done, el


def cpu_baseline(w, budget_s=15.0, all_core_n=64):
    """The oracle as it stands, on the host cores.  One thread on the
    workload's own lattice (second-order stages of its time step), and every
    host core running its own replica of the same model on an all_core_n^3
    lattice (independent processes, as the GPU's replicas are independent)."""
    import multiprocessing as mp
    sites, el = _oracle_stage_rate((w["name"], w["n"], budget_s))
    single = sites / el
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")        # no fork after the process has used the GPU
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_stage_rate, [(w["name"], all_core_n, budget_s)] * cores)
        wall = time.perf_counter() - t0
    agg = sum(s for s, _ in res) / max(e for _, e in res)
    return {"value": agg, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, one per host core, each running second-order stages "
                      f"of the {w['name']} model on its own {all_core_n}^3 lattice for "
                      f"~{budget_s:.0f} s (numpy FP64; {wall:.1f} s wall)",
            "single_thread": {"value": single, "unit": UNIT, "cores": 1,
                              "sample": f"second-order stages of the {w['n']}^3 workload itself, "
                                        f"{el:.1f} s, numpy FP64, one thread"}}


def reference_arm(args, w):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    from paper_1201_5029_gb300 import inputs as I
    from oracle import pycool_oracle as O
    phi, pi = I.initial_fields(w)
    cfg = O.LatticeConfig(n=w["n"], L=w["L"], model=w["model"], params=w["params"], dt=w["dt"],
                          order=w["order"], mpl=w["mpl"])
    st = O.make_state(cfg, phi, pi)
    wts = O.stage_weights(w["order"])
    # warm-up: at most one stage (the oracle has no caches to warm)
    for i in range(min(args.warmup, 1)):
        O.second_order_stage(cfg, st, wts[i % len(wts)] * cfg.dt)
    # each timed step is one second-order stage of the workload (a bounded
    # sample of its time step); stop once ~2 minutes are used
    done, t0 = 0, time.perf_counter()
    while done < args.steps:
        O.second_order_stage(cfg, st, wts[(done + 1) % len(wts)] * cfg.dt)
        done += 1
        if time.perf_counter() - t0 > 120.0:
            break
    el = time.perf_counter() - t0
    value = w["n"] ** 3 * done / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": done, "warmup": args.warmup,
        "ms_per_step": el / done * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{done} second-order stage(s) of the {w['n']}^3 workload "
                                   f"({el:.1f} s; numpy FP64, single thread)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def linear_leg(P, w, steps):
    """Growth functions of the linearised evolution (Sec. 2.2) for the
    workload's lattice: one transfer matrix per distinct k_eff^2 of its
    stencil (the library's grouping), advanced `steps` time steps with the
    homogeneous background.  Times the growth-function call (device buffers,
    copies and the kernel) after one warm-up call."""
    import numpy as np
    n = w["n"]
    vals, _ = P.pycool_linear_modes(n, w.get("stencil", "7pt"))
    cfg = P.config_from_workload(w)
    nf = len(w["background"])
    phi0 = np.array(w["background"], dtype=np.float64)
    pi0 = np.array(w["momentum"], dtype=np.float64)
    # p_a of the homogeneous background from the library's own constraint
    with P.Simulation(P.config_from_workload(w, n=32)) as sim:
        sim.set_initial(np.broadcast_to(phi0[:, None, None, None], (nf, 32, 32, 32)).copy(),
                        np.broadcast_to(pi0[:, None, None, None], (nf, 32, 32, 32)).copy())
        pa32 = sim.energies()["pa"]
    pa0 = pa32 * (n / 32.0) ** 3          # p_a scales with V_L for a homogeneous state
    stages = P.pycool_stages_per_step(w["order"])
    P.pycool_linear_growth(cfg, 1.0, pa0, phi0, pi0, vals, 1)
    t0 = time.perf_counter()
    T, bg = P.pycool_linear_growth(cfg, 1.0, pa0, phi0, pi0, vals, steps)
    el = time.perf_counter() - t0
    ok = bool(np.all(np.isfinite(T)))
    return {"metric": "linearised evolution: growth-function stage updates/s (one per distinct "
                      "k_eff^2 and stage)",
            "value": len(vals) * steps * stages / el, "unit": "k-value stage updates/s",
            "distinct_k2": int(len(vals)), "lattice_modes": n ** 3, "steps": steps,
            "seconds": el, "lattice_equivalent_site_updates_per_s": n ** 3 * steps * stages / el,
            "finite": ok, "a_end": bg[0], "config": _config(w)}


# C expressions of the compiled-in potentials, for the runtime-compiled leg
RUNTIME_EXPRESSIONS = {
    "chaotic2": ("0.5*p[0]*f0*f0 + 0.5*p[1]*f0*f0*f1*f1",
                 ("p[0]*f0 + p[1]*f0*f1*f1", "p[1]*f0*f0*f1")),
    "oscillon": ("0.5*p[0]*f0*f0 - 0.25*p[1]*f0*f0*f0*f0 + p[2]/6.0*f0*f0*f0*f0*f0*f0",
                 ("p[0]*f0 - p[1]*f0*f0*f0 + p[2]*f0*f0*f0*f0*f0",)),
}


def _event_ms(torch, stream, fn, reps):
    """Mean CUDA-event time (ms) of fn() over reps calls on `stream`, after one warm-up."""
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def next_rows_leg(P, torch, I, w, stream, steps=3):
    """The paths beyond the fused step, each timed on the workload's lattice:
      linear_evolve : the linearised evolution end to end on the device
                      (means, FFTs, growth functions of every distinct
                      k_eff^2 for `steps` steps, per-mode apply, inverse FFTs);
      observables   : per-site energy density and pressure, and the spectra of
                      every field (FP64 state of the workload);
      fourth_order  : `steps` time steps with the 13-point stencil, FP64 (the
                      persistent kernel when n is a multiple of 32);
      fourth_order_split_dd : the same in the split-DD form (persistent kernel);
      runtime_model : `steps` time steps of a potential compiled at run time
                      (the workload's own potential as C expressions), FP64.
    Each figure is site-updates/s (n^3 x stages x steps / time) or, for the
    observables, sites/s and GB/s of their algorithmic bytes."""
    import numpy as np
    out = {}
    n = w["n"]
    S = n ** 3
    nf = len(w["background"])
    stages = P.pycool_stages_per_step(w["order"])
    phi, pi = I.initial_fields(w)
    dphi = torch.from_numpy(phi).cuda()
    dpi = torch.from_numpy(pi).cuda()
    try:
        cfg = P.config_from_workload(w)
        with P.Simulation(P.config_from_workload(w)) as sim:
            sim.set_initial(phi, pi)
            pa0 = sim.energies()["pa"]
            # observables of the initial FP64 state
            r = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
            q = torch.empty_like(r)
            ms_e = _event_ms(torch, stream, lambda: sim.energy_fields(r, q, on_device=True), 3)
            sim.spectrum(0, 0)                     # the first call makes the plan and tables
            t0 = time.perf_counter()
            for f in range(nf):
                sim.spectrum(0, f)
            ms_s = (time.perf_counter() - t0) * 1e3 / nf
        e_bytes = S * (2 * nf * 8 + 2 * 8)      # read phi, pi of every field; write rho, P
        out["observables"] = {"energy_fields_ms": ms_e, "energy_fields_gbs": e_bytes / ms_e / 1e6,
                              "spectrum_ms_per_field": ms_s,
                              "note": "energy fields: CUDA events; spectrum: wall time of one "
                                      "pycool_spectrum call (FFT, shell sums, copy back)"}
        outp, outq = torch.empty_like(dphi), torch.empty_like(dpi)
        ms_l = _event_ms(torch, stream,
                         lambda: P.pycool_linear_evolve(cfg, 1.0, pa0, dphi, dpi, steps, outp,
                                                        outq, stream), 2)
        out["linear_evolve"] = {"value": S * stages * steps / (ms_l / 1e3), "unit": UNIT,
                                "ms_per_call": ms_l, "steps": steps,
                                "note": "whole call incl. its device allocations, after one "
                                        "call that made the lattice's tables and FFT plans"}
    except Exception as e:  # noqa: BLE001
        out["error"] = f"{type(e).__name__}: {e}"
    for name, make in (("fourth_order", lambda: P.config_from_workload(w, stencil="4th")),
                       ("fourth_order_split_dd", lambda: P.config_from_workload(
                           w, stencil="4th", precision="split_dd")),
                       ("runtime_model", lambda: P.make_config(
                           n, w["L"], P.pycool_model_define(*RUNTIME_EXPRESSIONS[w["model"]]),
                           w["params"], w["dt"], order=w["order"], mpl=w["mpl"]))):
        if name == "runtime_model" and w["model"] not in RUNTIME_EXPRESSIONS:
            continue
        try:
            with P.Simulation(make(), stream=stream) as sim:
                sim.set_initial(phi, pi)
                ms = _event_ms(torch, stream, lambda: sim.evolve(1), steps)
                st = sim.sync()
            out[name] = {"value": S * stages / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                         "status": st, "form": "split_dd" if name.endswith("split_dd") else "fp64"}
        except Exception as e:  # noqa: BLE001
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    return out


def _config(w):
    state = 2 * len(w["background"]) * w["n"] ** 3 * 8
    return {"workload": f"{w['name']}: {w['model']} {len(w['background'])}-field, "
                        f"{w['n']}^3 periodic lattice, L={w['L']}, order {w['order']} "
                        f"(Yoshida), dt={w['dt']}, m_pl={w['mpl']}",
            "n": w["n"], "fields": len(w["background"]), "order": w["order"],
            "stencil": "7pt", "ic": w.get("ic", "white"), "seed": w["seed"],
            "step": "evolve(1): one fused sweep per stage + synchronising flush",
            "l2": "flushed between timed steps (256 MiB write); FP64 state "
                  + (f"{state / 1e6:.0f} MB < L2" if state < 120e6 else
                     f"{state / 1e6:.0f} MB > L2"),
            "parallelism": "replicas (independent lattice per GPU)"}


def time_workload(P, torch, I, name, forms, steps, warmup, flush_buf, stream, ws, hbm, peak_kind):
    """Every form of one workload: CUDA-event timing of `steps` evolve(1) calls
    after `warmup` untimed ones; the per-form results with their rooflines."""
    w = I.workload(name)
    w["name"] = name
    phi, pi = I.initial_fields(w)
    S = w["n"] ** 3
    res = {prec: run_form(P, torch, w, prec, steps, warmup, flush_buf, phi, pi, stream)
           for prec in forms}
    tot = slowest_rank_ms({k: v["total_ms"] for k, v in res.items()}, forms, "cuda")
    out = {"config": _config(w), "forms": {}}
    for prec in forms:
        r = res[prec]
        rate = whole_job_rate(ws, S, r["stages"], steps, tot[prec])
        msps = tot[prec] / steps
        out["forms"][prec] = {"value": rate, "unit": UNIT, "ms_per_step": msps,
                              "steps_per_s": ws * 1e3 / msps,
                              "launches": r["launches"], "status": r["status"],
                              "roofline": roofline(w, prec, r["stages"], msps, hbm, peak_kind)}
    for f, dt in (("split_fp32", "f32 fluctuations + f64 background/sums"),
                  ("split_dd", "f32 pairs (double-float fluctuations) + f64 background/sums")):
        if f in forms:
            out["forms"][f]["dtype"] = dt
            if "fp64" in forms:
                out["forms"][f]["speedup_vs_fp64"] = (out["forms"][f]["value"]
                                                      / out["forms"]["fp64"]["value"])
    return w, phi, pi, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="qball256")
    ap.add_argument("--extra", default="preheat128,oscillon256",
                    help="further workloads timed in the same run (comma list)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--linear", action="store_true",
                    help="time the linearised evolution's growth functions instead")
    ap.add_argument("--no-linear", action="store_true",
                    help="leave the growth-function measurement out of the main line")
    ap.add_argument("--next-rows", default="preheat128",
                    help="workload of the linearised / observables / fourth-order / runtime-model "
                         "timings (empty: leave them out)")
    ap.add_argument("--only-next-rows", action="store_true",
                    help="time only those paths (profiling them)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=500)
    ap.add_argument("--serving-steps-scale", type=float, default=0.02)
    ap.add_argument("--serving-load", type=float, default=0.7)
    ap.add_argument("--serving-other-loads", default="",
                    help="further offered loads (comma list), both forms, under by_load")
    ap.add_argument("--serving-persist-min-n", type=int, default=256,
                    help="FP64 serving members of this side and above (a multiple of 32) run "
                         "on the persistent kernel; 0: none")
    ap.add_argument("--serving-compare-per-stage", action="store_true",
                    help="also replay the FP64 stream with every member on the per-stage kernels")
    ap.add_argument("--forms", default="fp64,split_fp32,split_dd",
                    help="comma list of forms to time (profiling a single kernel)")
    args = ap.parse_args()
    forms = [f for f in args.forms.split(",") if f]
    extras = [x for x in args.extra.split(",") if x and x != args.workload]
    args.warmup = max(args.warmup, 3)

    from paper_1201_5029_gb300 import inputs as I
    w = I.workload(args.workload)
    w["name"] = args.workload
    if args.impl == "reference":
        return reference_arm(args, w)
    if args.linear:
        import paper_1201_5029_gb300 as P
        print(json.dumps(linear_leg(P, w, args.steps)), flush=True)
        return 0
    if args.only_next_rows:
        import torch
        import paper_1201_5029_gb300 as P
        wn = I.workload(args.next_rows)
        wn["name"] = args.next_rows
        print(json.dumps(next_rows_leg(P, torch, I, wn, torch.cuda.current_stream())), flush=True)
        return 0

    import torch
    import paper_1201_5029_gb300 as P

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    stream = torch.cuda.current_stream()
    flush_buf = torch.zeros(256 << 20, dtype=torch.uint8, device="cuda")
    peaks, peak_kind = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    clk = ClockSampler(local)
    with clk:
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        w, phi, pi, head = time_workload(P, torch, I, args.workload, forms, args.steps,
                                         args.warmup, flush_buf, stream, ws, hbm, peak_kind)
        torch.cuda.synchronize()
    nf = phi.shape[0]
    S = w["n"] ** 3
    s = P.pycool_stages_per_step(w["order"])
    full = forms == list(FORMS)

    # e2e through the public API with host buffers (FP64 form, headline workload),
    # right after the headline's device timing
    e2e = None
    if full and rank == 0 and not args.no_e2e:
        phi_pin = torch.from_numpy(phi).pin_memory().numpy()
        pi_pin = torch.from_numpy(pi).pin_memory().numpy()
        out_phi = torch.empty(phi.shape, dtype=torch.float64).pin_memory().numpy()
        out_pi = torch.empty(pi.shape, dtype=torch.float64).pin_memory().numpy()
        k = args.e2e_steps
        eclk = ClockSampler(local, "e2e")
        with eclk:
            dt, phases = e2e_form(P, torch, w, "fp64", k, phi_pin, pi_pin, out_phi, out_pi,
                                  stream)
        e2e = {"value": ws * S * s * k / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(phi.nbytes + pi.nbytes),
               "d2h_bytes_per_step": int(out_phi.nbytes + out_pi.nbytes),
               "form": "fp64", "steps": k, "ms_per_step_phases": phases,
               "clocks": eclk.summary(),
               "note": "set_initial(host) + evolve(1) + get_fields(host) per step"}

    extra = {}
    with clk:
        if ws > 1:
            torch.distributed.barrier()
        for name in extras:
            extra[name] = time_workload(P, torch, I, name, forms, args.steps, args.warmup,
                                        flush_buf, stream, ws, hbm, peak_kind)[3]
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
    clocks = clk.summary()

    if not full:
        if rank == 0:  # profiling run: a short line per workload and form, no baselines
            for name, leg in [(args.workload, head)] + list(extra.items()):
                for f in forms:
                    r = leg["forms"][f]
                    print(json.dumps({"workload": name, "form": f, "value": r["value"],
                                      "unit": UNIT, "ms_per_step": r["ms_per_step"],
                                      "launches": r["launches"], "status": r["status"],
                                      "roofline_frac": r["roofline"]["frac"]}), flush=True)
        return 0

    serving = None
    if rank == 0 and not args.no_serving:
        serving = serving_leg(P, I, args.serving_requests, args.serving_steps_scale,
                              args.serving_load,
                              [float(x) for x in args.serving_other_loads.split(",") if x],
                              persist_min_n=args.serving_persist_min_n,
                              compare_per_stage=args.serving_compare_per_stage)

    # the linearised evolution's growth functions on the same lattice (Sec. 2.2):
    # a side measurement, never allowed to take the main line down
    linear = None
    if rank == 0 and not args.no_linear:
        try:
            lin = linear_leg(P, w, 20)
            linear = {k: lin[k] for k in ("metric", "value", "unit", "distinct_k2", "lattice_modes",
                                          "steps", "seconds",
                                          "lattice_equivalent_site_updates_per_s", "finite")}
        except Exception as e:  # noqa: BLE001
            linear = {"error": f"{type(e).__name__}: {e}"}

    next_rows = None
    if rank == 0 and args.next_rows:
        wn = I.workload(args.next_rows)
        wn["name"] = args.next_rows
        next_rows = next_rows_leg(P, torch, I, wn, stream)
        next_rows["workload"] = _config(wn)["workload"]

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(w)
        f64 = head["forms"]["fp64"]
        launches = sum(leg["forms"][f]["launches"] for leg in [head] + list(extra.values())
                       for f in forms)
        line = {
            "metric": METRIC, "value": f64["value"], "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": f64["ms_per_step"],
            "steps_per_s": f64["steps_per_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded white-noise / spectral initial fluctuations, no dataset)",
            "config": head["config"],
            "roofline": f64["roofline"],
            "forms": head["forms"],
            "extra": extra,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "serving": serving,
            "linear": linear,
            "next_rows": next_rows,
            "gpu_launches": int(launches),
            "kernel_source_hash": kernel_source_hash(),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
