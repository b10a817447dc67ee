"""Serving (continuous batching) on the GPU: a served request equals the
oracle run on the same device-generated initial fields; a request's result is
bit-identical alone and in a mix of other sizes, models, orders and precisions;
admission by HBM budget; a failing request does not disturb the others."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
from oracle import pycool_oracle as O  # noqa: E402

GB = 1 << 30


def _req(name, n, order, precision="fp64", stencil="7pt", mpl=None):
    w = I.workload(name)
    cfg = P.make_config(n, w["L"], w["model"], w["params"], w["dt"], order=order,
                        precision=precision, stencil=stencil,
                        mpl=w["mpl"] if mpl is None else mpl)
    ic = P.make_ic(w["background"], w["momentum"], w["noise"])
    return w, cfg, ic


def _obs_tuple(e):
    nf = 2
    return (e.eta, e.a, e.pa, e.H, tuple(e.rho_kin)[:nf], tuple(e.rho_grad)[:nf], e.rho_pot,
            e.rho, e.P, e.residual, tuple(e.mean)[:nf], tuple(e.variance)[:nf], e.steps_done,
            e.sweeps_done)


def _run(requests, budget=8 * GB, slots=32, persist_min_n=None):
    srv = P.pycool_server_create(budget, slots)
    try:
        if persist_min_n is not None:
            P.pycool_server_set_persistent_min_n(srv, persist_min_n)
        tickets = [P.pycool_server_submit(srv, cfg, ic, seed, steps)
                   for (cfg, ic, seed, steps) in requests]
        out = [P.pycool_server_wait(srv, t, 120.0) for t in tickets]
        stats = P.pycool_server_stats(srv)
    finally:
        P.pycool_server_destroy(srv)
    return out, stats


@pytest.mark.parametrize("name,n,order", [("preheat32", 32, 2), ("oscillon256", 24, 6),
                                          ("qball256", 32, 4),
                                          ("preheat128", 128, 4),    # TMA-staged member
                                          ("oscillon256", 128, 2)])
def test_served_request_matches_oracle(name, n, order):
    w, cfg, ic = _req(name, n, order)
    seed, steps = 77 + n, 6
    [(st, e)], stats = _run([(cfg, ic, seed, steps)])
    assert st == P.OK
    phi, pi = I.philox_white_ics(n, w["background"], w["momentum"], w["noise"], seed)
    ocfg = O.LatticeConfig(n=n, L=w["L"], model=w["model"], params=w["params"], dt=w["dt"],
                           order=order, mpl=w["mpl"])
    s = O.make_state(ocfg, phi, pi)
    O.evolve(ocfg, s, steps)
    oe = O.energies(ocfg, s)
    assert e.steps_done == steps
    for key in ("a", "pa", "rho", "P"):
        assert math.isclose(getattr(e, key), oe[key], rel_tol=1e-10), key
    for f in range(len(w["background"])):
        m, v = O.field_stats(s, f)
        assert math.isclose(e.mean[f], m, rel_tol=1e-10, abs_tol=1e-14)
        assert math.isclose(e.variance[f], v, rel_tol=1e-6)
    assert stats["completed"] == 1 and stats["p50_s"] > 0


@pytest.mark.parametrize("name,n,order,stencil,steps", [("preheat128", 64, 8, "7pt", 3),
                                                        ("qball256", 64, 6, "iso27", 4),
                                                        ("oscillon256", 96, 4, "7pt", 5)])
def test_persistent_member_matches_oracle(name, n, order, stencil, steps):
    """An FP64 member on the persistent kernel (the threshold lowered to its
    side): launches of 8 stage sweeps that end mid-step with the stage boundary
    pending (45, 28 and 15 sweeps here), the last one with the flush.  The
    result equals the oracle's on the same device-generated initial fields."""
    w, cfg, ic = _req(name, n, order, stencil=stencil)
    seed = 91 + n
    [(st, e)], stats = _run([(cfg, ic, seed, steps)], persist_min_n=64)
    assert st == P.OK
    phi, pi = I.philox_white_ics(n, w["background"], w["momentum"], w["noise"], seed)
    ocfg = O.LatticeConfig(n=n, L=w["L"], model=w["model"], params=w["params"], dt=w["dt"],
                           order=order, stencil=stencil, mpl=w["mpl"])
    s = O.make_state(ocfg, phi, pi)
    O.evolve(ocfg, s, steps)
    oe = O.energies(ocfg, s)
    assert e.steps_done == steps
    assert e.sweeps_done == steps * P.pycool_stages_per_step(order)   # stage sweeps only
    for key in ("a", "pa", "rho", "P"):
        assert math.isclose(getattr(e, key), oe[key], rel_tol=1e-10), key
    for f in range(len(w["background"])):
        m, v = O.field_stats(s, f)
        assert math.isclose(e.mean[f], m, rel_tol=1e-10, abs_tol=1e-14)
        assert math.isclose(e.variance[f], v, rel_tol=1e-6)
    assert stats["completed"] == 1


def test_persistent_members_bitwise_alone_and_in_mix():
    """Threshold 64: FP64 members of 64^3, 96^3 and 128^3 run on the persistent
    kernel, one after another between the per-stage groups' graphs, beside
    per-stage members of every kind; each persistent member's result alone
    equals its result in the mix bit for bit."""
    extra = []
    for i, (name, n, order) in enumerate([("qball256", 128, 8), ("preheat32", 64, 4),
                                          ("oscillon256", 64, 6)]):
        w, cfg, ic = _req(name, n, order)
        extra.append((cfg, ic, 500 + i, 2 + i))
    mix = _mix() + extra
    out, stats = _run(mix, persist_min_n=64)
    assert all(st == P.OK for st, _ in out) and stats["completed"] == len(mix)
    persistent = [i for i, (cfg, _, _, _) in enumerate(mix)
                  if cfg.precision == P.FP64 and cfg.n % 32 == 0 and cfg.n >= 64]
    assert len(persistent) == 4
    for i in persistent:
        [(st, e)], _ = _run([mix[i]], persist_min_n=64)
        assert st == P.OK
        assert _obs_tuple(e) == _obs_tuple(out[i][1]), i


def test_persistent_member_zero_steps_cancel_and_threshold():
    """A persistent member with zero steps returns its initial state's
    observables (the same admission flush as a per-stage member's, so the same
    bits); a long one is cancelled at a boundary; invalid thresholds are
    refused."""
    w, cfg, ic = _req("preheat32", 64, 8)
    [(st0, e0)], _ = _run([(cfg, ic, 5, 0)], persist_min_n=0)
    [(st1, e1)], _ = _run([(cfg, ic, 5, 0)], persist_min_n=64)
    assert st0 == st1 == P.OK and _obs_tuple(e0) == _obs_tuple(e1)
    srv = P.pycool_server_create(4 * GB, 4)
    try:
        for bad in (-32, 16, 48, 100):
            with pytest.raises(Exception):
                P.pycool_server_set_persistent_min_n(srv, bad)
        P.pycool_server_set_persistent_min_n(srv, 64)
        t = P.pycool_server_submit(srv, cfg, ic, 6, 10 ** 6)
        import time
        time.sleep(0.5)
        assert P.pycool_server_cancel(srv, t) == P.OK
        st, e = P.pycool_server_wait(srv, t, 60.0)
        assert st == P.E_CANCELLED
        assert 0 < e.sweeps_done < 15 * 10 ** 6
        # the server carries on: a short request after it completes
        t2 = P.pycool_server_submit(srv, cfg, ic, 7, 2)
        st2, e2 = P.pycool_server_wait(srv, t2, 60.0)
        assert st2 == P.OK and e2.steps_done == 2
    finally:
        P.pycool_server_destroy(srv)


def test_device_initial_conditions_match_numpy_generator():
    """Zero steps: the result is the initial state's observables, so the device
    generator and the numpy restatement must agree on the fields' statistics."""
    w, cfg, ic = _req("preheat32", 32, 2)
    [(st, e)], _ = _run([(cfg, ic, 1234, 0)])
    assert st == P.OK
    phi, pi = I.philox_white_ics(32, w["background"], w["momentum"], w["noise"], 1234)
    for f in range(2):
        assert math.isclose(e.mean[f], float(np.mean(phi[f])), rel_tol=1e-12, abs_tol=1e-16)
        assert math.isclose(e.variance[f], float(np.var(phi[f])), rel_tol=1e-9)


def _mix(seed0=1000):
    """A mix of sizes, models, orders, precisions and stencils."""
    mix = []
    spec = [("preheat32", 32, 2, "fp64", "7pt"), ("oscillon256", 64, 6, "split_fp32", "7pt"),
            ("qball256", 32, 8, "fp64", "iso27"), ("preheat32", 64, 4, "split_fp32", "7pt"),
            ("oscillon256", 40, 4, "fp64", "7pt"), ("qball256", 64, 2, "split_fp32", "iso27"),
            ("preheat32", 96, 2, "fp64", "7pt"), ("oscillon256", 32, 8, "split_fp32", "iso27")]
    for i, (name, n, order, prec, st) in enumerate(spec):
        w, cfg, ic = _req(name, n, order, prec, st)
        mix.append((cfg, ic, seed0 + i, 3 + (i % 4)))
    return mix


@pytest.mark.parametrize("prec", ["fp64", "split_fp32"])
def test_result_bitwise_identical_alone_and_in_mix(prec):
    w, cfg, ic = _req("preheat32", 64, 4, prec)
    x = (cfg, ic, 4242, 5)
    [(st1, e1)], _ = _run([x])
    mix = _mix()
    out, stats = _run(mix[:4] + [x] + mix[4:])
    st2, e2 = out[4]
    assert st1 == st2 == P.OK
    assert _obs_tuple(e1) == _obs_tuple(e2)
    assert all(s == P.OK for s, _ in out)
    assert stats["completed"] == len(mix) + 1


def test_twenty_sampled_requests_bitwise_alone_and_in_mix():
    """20 requests of the serving mix's own stream (its first 16 and its first
    two of 256^3 and of 384^3: the three models, orders 2..8, both forms
    alternately, a few steps each): each result, run alone, equals its result
    in the mix of all 20 bit for bit."""
    mixd = I.SERVING_MIX
    pool = I.serving_requests(steps_scale=0.002)          # the 500-request stream
    reqs = (pool[:16] + [r for r in pool if r["n"] == 256][:2] +
            [r for r in pool if r["n"] == 384][:2])
    items = []
    for i, r in enumerate(reqs):
        w = I.workload(r["workload"])
        cfg = P.make_config(r["n"], mixd["L"][w["model"]], w["model"], w["params"],
                            mixd["dt"][w["model"]], order=r["order"],
                            precision="fp64" if i % 2 == 0 else "split_fp32", mpl=w["mpl"])
        ic = P.make_ic(w["background"], w["momentum"], w["noise"])
        items.append((cfg, ic, r["seed"], r["steps"]))
    assert len(reqs) == 20 and {r["n"] for r in reqs} >= {32, 64, 128, 256, 384}
    out, stats = _run(items, budget=40 * GB, slots=32)
    assert all(s == P.OK for s, _ in out) and stats["completed"] == 20
    for i, x in enumerate(items):
        [(st, e)], _ = _run([x], budget=40 * GB)
        assert st == P.OK
        assert _obs_tuple(e) == _obs_tuple(out[i][1]), i


@pytest.mark.parametrize("name,n,prec", [("preheat32", 256, "split_fp32"),
                                         ("preheat32", 320, "split_fp32"),
                                         ("qball256", 256, "fp64")])
def test_long_z_chunks_are_reproducible_run_to_run(name, n, prec):
    """Members whose blocks stream 64-plane z-chunks through the 8-slot TMA
    ring (each slot refilled seven times per sweep): the same request, served
    three times in turn by one server (each run on the arena the previous one
    left) and once after a different request, gives the same result bit for
    bit.  A refill that overtook a read of its slot (a missing proxy fence
    between the generic reads and the TMA write) changed the last digits of
    the observables from run to run here."""
    w, cfg, ic = _req(name, n, 8 if prec == "split_fp32" else 4, prec)
    x = (cfg, ic, 4321, 2)
    other = _req("oscillon256", 128, 2)
    srv = P.pycool_server_create(8 * GB, 4)
    try:
        res = []
        for item in (x, x, x, (other[1], other[2], 7, 1), x):
            t = P.pycool_server_submit(srv, *item)
            st, e = P.pycool_server_wait(srv, t, 120.0)
            assert st == P.OK
            res.append(_obs_tuple(e))
    finally:
        P.pycool_server_destroy(srv)
    assert res[0] == res[1] == res[2] == res[4]


def test_admission_under_a_tight_budget_gives_the_same_results():
    mix = _mix(2000)
    free, _ = _run(mix)
    tight, stats = _run(mix, budget=64 << 20, slots=3)   # a few lattices at a time
    for (s1, e1), (s2, e2) in zip(free, tight):
        assert s1 == s2 == P.OK
        assert _obs_tuple(e1) == _obs_tuple(e2)
    assert stats["completed"] == len(mix)


def test_failing_request_is_isolated():
    good = _mix(3000)[:3]
    w, bad_cfg, bad_ic = _req("oscillon256", 16, 2)
    bad_ic.background[0] = 1e60           # V ~ phi^6 overflows at once
    out, _ = _run(good[:1] + [(bad_cfg, bad_ic, 1, 4)] + good[1:])
    ref, _ = _run(good)
    assert out[1][0] == P.E_NONFINITE
    for (s1, e1), (s2, e2) in zip([out[0]] + out[2:], ref):
        assert s1 == s2 == P.OK and _obs_tuple(e1) == _obs_tuple(e2)


def test_submit_validation_and_unknown_ticket():
    srv = P.pycool_server_create(64 << 20, 2)
    try:
        w, cfg, ic = _req("preheat32", 32, 2)
        big = P.make_config(512, 10.0, "chaotic2", (1.0, 1e4), 0.001, order=2)
        with pytest.raises(P.PycoolError) as ei:
            P.pycool_server_submit(srv, big, ic, 1, 1)       # could never fit 64 MiB
        assert ei.value.status == P.E_NOMEM
        bad = P.make_config(32, 10.0, "chaotic2", (1.0, 1e4), 5.0, order=2)
        with pytest.raises(P.PycoolError) as ei:
            P.pycool_server_submit(srv, bad, ic, 1, 1)
        assert ei.value.status == P.E_UNSTABLE_DT
        assert P.pycool_server_wait(srv, 999999, 0.1)[0] == P.E_NOT_FOUND
        t = P.pycool_server_submit(srv, cfg, ic, 5, 3)
        st, e = P.pycool_server_wait(srv, t, 60.0)
        assert st == P.OK and e.steps_done == 3
        assert P.pycool_server_wait(srv, t, 0.1)[0] == P.E_NOT_FOUND   # collected once
    finally:
        P.pycool_server_destroy(srv)
