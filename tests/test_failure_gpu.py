"""Failure detection without a GPU fault (GPU).

Every failure here is made on the host or through a bounded device-side wait,
and each test checks that the error comes back as a status while the CUDA
context stays usable:
  - pycool_sync's host deadline returns E_TIMEOUT for work still running and
    OK once it has finished (nothing is poisoned by a host timeout);
  - a grid barrier that waits for an arrival that never comes (fault test of
    the persistent kernel, with a short wait limit) makes every block give up
    and return: pycool_sync returns E_TIMEOUT, the simulation is poisoned,
    and a new simulation on the same context computes the same result as
    before;
  - the allocation-failure hook makes pycool_create and pycool_server_create
    return E_NOMEM;
  - a request cancelled while queued or while resident returns E_CANCELLED,
    and the requests around it finish normally."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
import gpu_helpers as G  # noqa: E402


def test_sync_deadline_returns_timeout_then_ok():
    w = I.workload("qball256")
    phi, pi = I.initial_fields(w)
    sim = P.Simulation(G.gpu_cfg(P, w))
    sim.set_initial(phi, pi)
    sim.evolve(4)                      # ~0.1 s of FP64 work on the device
    assert sim.sync(1e-4) == P.E_TIMEOUT
    assert sim.sync() == P.OK          # a host deadline poisons nothing
    assert sim.energies()["steps_done"] == 4
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "split_fp32"])
def test_device_wait_runs_out_and_returns_a_status(precision):
    w = I.workload("preheat128")
    phi, pi = I.initial_fields(w, n=64)
    cfg = G.gpu_cfg(P, w, n=64, precision=precision)

    def run():
        s = P.Simulation(cfg)
        s.set_initial(phi, pi)
        s.evolve(2)
        out = s.get_fields()
        s.close()
        return out

    before = run()
    sim = P.Simulation(cfg)
    sim.set_initial(phi, pi)
    assert P.pycool_debug_barrier_stall(sim.handle, 1 << 20) == P.OK   # ~0.5 ms limit
    sim.evolve(2)
    t0 = time.perf_counter()
    assert sim.sync(30.0) == P.E_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    with pytest.raises(P.PycoolError) as ei:
        sim.evolve(1)
    assert ei.value.status == P.E_STATE
    sim.close()
    after = run()                      # the context is still usable: same result as before
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])


def test_allocation_failure_hook():
    w = I.workload("preheat32")
    cfg = G.gpu_cfg(P, w, n=16)
    assert P.pycool_debug_fail_alloc(1) == P.OK
    with pytest.raises(P.PycoolError) as ei:
        P.Simulation(cfg)
    assert ei.value.status == P.E_NOMEM
    s = P.Simulation(cfg)              # the hook fired once
    s.close()
    assert P.pycool_debug_fail_alloc(1) == P.OK
    with pytest.raises(P.PycoolError) as ei:
        P.pycool_server_create(64 << 20, 4)
    assert ei.value.status == P.E_NOMEM
    srv = P.pycool_server_create(64 << 20, 4)
    P.pycool_server_destroy(srv)
    assert P.pycool_debug_fail_alloc(0) == P.OK


def test_server_cancel_queued_and_resident():
    mix = I.SERVING_MIX
    wq = I.workload("qball256")
    wp = I.workload("preheat32")
    long_cfg = P.make_config(128, mix["L"]["qball"], "qball", wq["params"], mix["dt"]["qball"],
                             order=8, mpl=wq["mpl"])
    short_cfg = P.make_config(32, mix["L"]["chaotic2"], "chaotic2", wp["params"],
                              mix["dt"]["chaotic2"], order=2, mpl=wp["mpl"])
    icq = P.make_ic(wq["background"], wq["momentum"], wq["noise"])
    icp = P.make_ic(wp["background"], wp["momentum"], wp["noise"])
    srv = P.pycool_server_create(4 << 30, 1)            # one slot: the second request queues
    t_long = P.pycool_server_submit(srv, long_cfg, icq, 11, 100000)
    t_queued = P.pycool_server_submit(srv, short_cfg, icp, 12, 10)
    assert P.pycool_server_cancel(srv, t_queued) == P.OK
    st, _ = P.pycool_server_wait(srv, t_queued, 5.0)
    assert st == P.E_CANCELLED
    time.sleep(0.5)                                     # the long request is resident by now
    assert P.pycool_server_cancel(srv, t_long) == P.OK
    st, obs = P.pycool_server_wait(srv, t_long, 60.0)
    assert st == P.E_CANCELLED
    assert obs.sweeps_done > 0 and obs.steps_done < 100000
    assert P.pycool_server_cancel(srv, t_long) == P.E_NOT_FOUND       # collected already
    t_ok = P.pycool_server_submit(srv, short_cfg, icp, 13, 10)
    st, obs = P.pycool_server_wait(srv, t_ok, 60.0)
    assert st == P.OK and obs.steps_done == 10
    assert P.pycool_server_stats(srv)["completed"] == 1                # cancelled ones not counted
    P.pycool_server_destroy(srv)
