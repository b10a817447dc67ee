"""The bench's roofline plumbing (host only, no GPU).

roofline.traffic is the DRAM traffic per launch from an ncu capture of the
persistent kernel, stored in profiles/traffic_per_launch.txt under the hash of
the sources that kernel is built from; the bench uses a line only while that
hash matches, so a changed kernel reports null rather than a stale figure.
The algorithmic bytes and flops of a launch are checked against their
definitions."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_1201_5029_gb300 import inputs as I  # noqa: E402

CSRC = os.path.join(ROOT, "paper_1201_5029_gb300", "csrc")


def test_hash_covers_the_persistent_kernel_sources():
    for name in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(CSRC, name)), name
    # every translation unit that instantiates evolve_persist is covered
    for name in os.listdir(CSRC):
        if name.startswith("persist") and name.endswith(".cu"):
            assert name in bench.KERNEL_SOURCES, name
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()


def test_traffic_lines_parse_and_match_only_their_hash(tmp_path, monkeypatch):
    with open(bench.TRAFFIC_FILE) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows, "no traffic lines"
    for r in rows:
        assert len(r) == 6 and r[1] in bench.FORMS and len(r[2]) == 16
        assert int(r[3]) > 0 and int(r[4]) > 0 and int(r[5]) > 0
    cur = bench.kernel_source_hash()
    fake = tmp_path / "traffic.txt"
    fake.write_text("# comment\n"
                    f"qball256 fp64 {cur} 100 23 5\n"
                    "qball256 split_dd 0123456789abcdef 7 7 7\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(fake))
    assert bench.measured_traffic("qball256", "fp64") == 123.0
    assert bench.measured_traffic("qball256", "split_dd") is None   # another kernel's figure
    assert bench.measured_traffic("oscillon256", "fp64") is None


@pytest.mark.parametrize("name,form", [("qball256", "fp64"), ("qball256", "split_fp32"),
                                       ("oscillon256", "split_dd")])
def test_roofline_algorithmic_bytes(name, form):
    w = I.workload(name)
    w["name"] = name
    s = {2: 1, 4: 3, 6: 7, 8: 15}[w["order"]]
    r = bench.roofline(w, form, s, 1.0, 6674.5, "measured")
    nf, n = len(w["background"]), w["n"]
    word = 4 if form == "split_fp32" else 8
    # s sweeps read and write phi and pi, the flush reads both and writes phi
    alg = (4 * s + 3) * nf * word * n ** 3
    assert r["algorithmic_bytes_per_launch"] == alg
    if r["bound"] == "hbm":
        assert r["achieved"] == pytest.approx(alg / 1e-3 / 1e9)
        assert r["frac"] == pytest.approx(r["achieved"] / 6674.5)
    else:   # FP64: algorithmic flops (FMA = 2) of s sweeps and the flush over the float64 peak
        assert r["achieved"] == pytest.approx(r["flops_per_launch"] / 1e-3 / 1e12)
        assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS)
        assert r["hbm_frac"] == pytest.approx(alg / 1e-3 / 1e9 / 6674.5)
