"""The bench's serving leg (host only, no GPU): a fake binding records what the
leg asks of the server.  Every replay sets the persistent threshold the bench
was given (the calibration included), the optional comparison replays the FP64
stream with the threshold at 0 on the same arrival times, and each replay
submits the whole stream in order."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_1201_5029_gb300 import inputs as I  # noqa: E402


class FakeServing:
    OK = 0
    STAGES = {2: 1, 4: 3, 6: 7, 8: 15}

    def __init__(self):
        self.servers = []

    def make_config(self, n, L, model, params, dt, order, precision, mpl):
        return dict(n=n, model=model, order=order, precision=precision)

    def make_ic(self, background, momentum, noise):
        return (tuple(background), tuple(momentum), noise)

    def pycool_stages_per_step(self, order):
        return self.STAGES[order]

    def pycool_server_create(self, budget, slots):
        srv = dict(min_n=None, submitted=[])
        self.servers.append(srv)
        return srv

    def pycool_server_set_persistent_min_n(self, srv, n):
        assert n == 0 or (n >= 32 and n % 32 == 0)
        srv["min_n"] = n

    def pycool_server_submit(self, srv, cfg, ic, seed, steps):
        srv["submitted"].append((cfg["n"], cfg["order"], cfg["precision"], seed, steps))
        return len(srv["submitted"])

    def pycool_server_wait(self, srv, ticket, timeout):
        return self.OK, None

    def pycool_server_stats(self, srv):
        return dict(p50_s=0.01, p99_s=0.02, site_updates_per_s=1e9,
                    completed=len(srv["submitted"]))

    def pycool_server_destroy(self, srv):
        srv["destroyed"] = True


def _leg(**kw):
    P = FakeServing()
    out = bench.serving_leg(P, I, count=6, steps_scale=0.002, load=0.7, calib_count=3, **kw)
    return P, out


def test_threshold_reaches_every_replay():
    P, out = _leg(persist_min_n=128)
    assert out["persistent_min_n"] == 128
    # calibration, FP64 and split-FP32 replays
    assert len(P.servers) == 3
    assert all(s["min_n"] == 128 and s["destroyed"] for s in P.servers)
    assert "fp64_all_per_stage" not in out
    reqs = I.serving_requests(count=6, steps_scale=0.002)
    calib, fp64, split = P.servers
    assert [x[0] for x in calib["submitted"]] == [r["n"] for r in reqs[:3]]
    assert [(x[0], x[1], x[3], x[4]) for x in fp64["submitted"]] == \
        [(r["n"], r["order"], r["seed"], r["steps"]) for r in reqs]
    assert {x[2] for x in fp64["submitted"]} == {"fp64"}
    assert {x[2] for x in split["submitted"]} == {"split_fp32"}


def test_comparison_replays_the_fp64_stream_per_stage():
    P, out = _leg(persist_min_n=256, compare_per_stage=True)
    assert len(P.servers) == 4
    calib, fp64, split, per_stage = P.servers
    assert per_stage["min_n"] == 0 and fp64["min_n"] == 256
    assert per_stage["submitted"] == fp64["submitted"]
    assert set(out["fp64_all_per_stage"]) >= {"p50_s", "p99_s", "completed", "failed"}
