"""Parity at the full lattice sizes of the timed workloads (GPU).

The workloads `bench.py` times run on 128^3 (two-field preheating, order 4)
and 256^3 (oscillon, order 6; Q-ball, order 8) lattices, in the launch
configuration of the persistent kernel (one cooperative launch per evolve,
one block per SM, the geometry chosen for that size).  Here the same
configurations run a few stages and are compared with the CPU oracle on the
whole lattice:
  - FP64 form: every field value, a and p_a within 1e-11 relative (the
    tolerance of the other FP64 parity tests);
  - split-FP32 form: the bounds of test_split_fp32_gpu.py.
One oracle run per workload serves both forms (module-scoped fixture)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
import gpu_helpers as G  # noqa: E402

TOL64 = 1e-11

# (workload, order, time steps), each in the order the bench times it:
# 128^3 preheating (order 4, 2 steps = 6 stages), 256^3 oscillon (order 6,
# 1 step = 7 stages), 256^3 Q-ball (order 8, 1 step = 15 stages; the oracle
# takes a few minutes for it)
CASES = [("preheat128", 4, 2), ("oscillon256", 6, 1), ("qball256", 8, 1)]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    name, order, steps = request.param
    w = I.workload(name)
    phi, pi = I.initial_fields(w)
    st, oe = G.run_oracle(G.oracle_cfg(w, order=order), phi, pi, steps)
    return dict(name=name, order=order, steps=steps, w=w, phi=phi, pi=pi, st=st, oe=oe)


def test_fp64_full_size(case):
    w, st = case["w"], case["st"]
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, order=case["order"]), case["phi"], case["pi"],
                              case["steps"])
    ef = G.field_errors(gphi, st.phi)
    ep = G.field_errors(gpi, st.pi)
    ea, epa = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa)
    stages = int(ge["sweeps_done"]) + 1
    ff = G.fluct_errors(gphi, st.phi) + G.fluct_errors(gpi, st.pi)
    ft = G.fluct_tolerances(st.phi, stages, TOL64) + G.fluct_tolerances(st.pi, stages, TOL64)
    print(f"\n{case['name']} n={w['n']} FP64: phi {ef} pi {ep} a {ea:.1e} pa {epa:.1e} "
          f"fluct {['%.2e' % x for x in ff]} bound {['%.2e' % x for x in ft]}")
    assert max(ef) < TOL64 and max(ep) < TOL64
    assert ea < TOL64 and epa < TOL64
    assert all(e < t for e, t in zip(ff, ft)), (ff, ft)
    assert ge["steps_done"] == case["steps"]


def test_split_full_size(case):
    w, st, oe = case["w"], case["st"], case["oe"]
    phi = case["phi"]
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, order=case["order"], precision="split_fp32"),
                              phi, case["pi"], case["steps"])
    fl = []
    for f in range(phi.shape[0]):
        scale = float(np.max(np.abs(st.phi[f] - st.phi[f].mean())))
        fl.append(float(np.max(np.abs(gphi[f] - st.phi[f]))) / scale)
    ea, epa = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa)
    erho = G.rel(ge["rho"], oe["rho"])
    evar = [G.rel(ge["variance"][f], np.var(st.phi[f])) for f in range(phi.shape[0])]
    print(f"\n{case['name']} n={w['n']} split: dphi/scale={fl} a={ea:.1e} pa={epa:.1e} "
          f"rho={erho:.1e} var={evar}")
    assert max(fl) < 1e-4
    assert ea < 1e-9 and epa < 1e-7
    assert erho < 1e-7
    assert max(evar) < 1e-4


def test_split_dd_full_size(case):
    """The split-DD form in the bench's launch configuration, at the FP64 tolerances."""
    w, st = case["w"], case["st"]
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, order=case["order"], precision="split_dd"),
                              case["phi"], case["pi"], case["steps"])
    ef = G.field_errors(gphi, st.phi)
    ep = G.field_errors(gpi, st.pi)
    ea, epa = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa)
    stages = int(ge["sweeps_done"]) + 1
    ff = G.fluct_errors(gphi, st.phi) + G.fluct_errors(gpi, st.pi)
    ft = G.fluct_tolerances(st.phi, stages, TOL64) + G.fluct_tolerances(st.pi, stages, TOL64)
    print(f"\n{case['name']} n={w['n']} split-DD: phi {ef} pi {ep} a {ea:.1e} pa {epa:.1e} "
          f"fluct {['%.2e' % x for x in ff]} bound {['%.2e' % x for x in ft]}")
    assert max(ef) < TOL64 and max(ep) < TOL64
    assert ea < TOL64 and epa < TOL64
    assert all(e < t for e, t in zip(ff, ft)), (ff, ft)
