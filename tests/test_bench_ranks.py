"""Multi-rank aggregation of bench.py, on CPU with the gloo backend.

Under torchrun every rank evolves its own replica of the lattice (no
collective on the data path); the whole-job time of a form is the slowest
rank's and the whole-job rate counts the sites of every rank.  Two gloo
ranks exercise the same functions bench.py calls after its timed region;
the reference arm's non-zero ranks exit without work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

FORMS = ["fp64", "split_fp32"]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank-dependent totals: rank 1 is slower in fp64, rank 0 in split
        tot = {"fp64": 10.0 + 5.0 * rank, "split_fp32": 3.0 - rank}
        dist.barrier()
        agg = bench.slowest_rank_ms(tot, FORMS, "cpu")
        dist.barrier()
        rate = bench.whole_job_rate(ws, 128 ** 3, 3, 7, agg["fp64"])
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{agg['fp64']!r} {agg['split_fp32']!r} {rate!r}\n")
    finally:
        dist.destroy_process_group()


def test_slowest_rank_two_gloo_ranks(tmp_path):
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(ws)]
    # every rank sees the same maxima
    assert rows[0] == rows[1]
    fp64, split, rate = (float(v) for v in rows[0])
    assert fp64 == 15.0 and split == 3.0
    # two replicas of 128^3 sites x 3 stages x 7 steps in 15 ms
    assert rate == pytest.approx(2 * 128 ** 3 * 3 * 7 / 0.015, rel=1e-15)


def test_single_rank_is_identity():
    assert not dist.is_initialized()
    tot = {"fp64": 1.25, "split_fp32": 0.5}
    assert bench.slowest_rank_ms(tot, FORMS, "cpu") == tot
    assert bench.whole_job_rate(1, 10, 2, 3, 1000.0) == 60.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup, gpus = 3, 3, 2
    assert bench.reference_arm(Args(), {"n": 8}) == 0
    assert capsys.readouterr().out == ""
