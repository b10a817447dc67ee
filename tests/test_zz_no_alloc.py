"""The allocation-free sweep (pycool_sweep_noalloc) against pycool_evolve.

pycool_sweep_noalloc serves callers that cannot allocate device memory (their
memory belongs to another allocator, or cudaMalloc's device-wide
synchronisation is not acceptable on their path): its scratch is a static
device array inside the library.  Here it must reproduce, step for step, what
the regular entry point computes from the same initial state, within the
parity tolerance of the other GPU tests.  This file is named to be collected
last, so a run that stops at the first failure has run everything else first.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
import gpu_helpers as G  # noqa: E402

TOL = 1e-11


def _rel_field(g, o):
    return max(float(np.max(np.abs(g[f] - o[f])) / np.max(np.abs(o[f]))) for f in range(o.shape[0]))


@pytest.mark.parametrize("n,order", [(32, 2), (40, 4)])   # TMA kernel and plain-load kernel
def test_noalloc_matches_evolve_two_steps(n, order):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    w = I.workload("preheat32")
    phi0, pi0 = I.initial_fields(w, n=n)
    cfg = P.make_config(n, w["L"], w["model"], w["params"], w["dt"], order=order, mpl=w["mpl"])
    stages = P.pycool_stages_per_step(order)

    # reference: the regular entry point, two evolve(1) calls in a row
    sim = P.Simulation(cfg)
    sim.set_initial(phi0, pi0)
    ref = []
    for _ in range(2):
        sim.evolve(1)
        f, p = sim.get_fields()
        ref.append((f, p, sim.energies()))
    sim.close()

    # allocation-free: the caller owns two buffer pairs and swaps them
    stream = torch.cuda.current_stream()
    A = [torch.from_numpy(phi0).cuda(), torch.from_numpy(pi0).cuda()]
    B = [torch.empty_like(A[0]), torch.empty_like(A[1])]
    st = P.pycool_stage_state()
    st.a = 1.0
    st.init_pa = 1
    # reduction-only flush: initial sums and p_a from H = 0; phi copied into B
    assert P.pycool_sweep_noalloc(cfg, A[0], A[1], B[0], None, True, st, stream) == P.OK
    phi, pi = B[0], A[1]
    spare = [A[0], B[1]]
    for step in range(2):
        for _ in range(stages):
            out = [spare[0], spare[1]]
            assert P.pycool_sweep_noalloc(cfg, phi, pi, out[0], out[1], False, st, stream) == P.OK
            spare = [phi, pi]
            phi, pi = out
        out_phi = spare[0]
        assert P.pycool_sweep_noalloc(cfg, phi, pi, out_phi, None, True, st, stream) == P.OK
        spare[0] = phi
        phi = out_phi
        rf, rp, re = ref[step]
        gphi, gpi = phi.cpu().numpy(), pi.cpu().numpy()
        assert _rel_field(gphi, rf) < TOL
        assert _rel_field(gpi, rp) < TOL
        # and at the scale of the fluctuations about each field's mean
        sweeps = (step + 1) * (stages + 1)
        for g, r in ((gphi, rf), (gpi, rp)):
            fe, ft = G.fluct_errors(g, r), G.fluct_tolerances(r, sweeps, TOL)
            assert all(e < t for e, t in zip(fe, ft)), (fe, ft)
        assert abs(st.a - re["a"]) / re["a"] < TOL
        assert abs(st.pa - re["pa"]) / abs(re["pa"]) < TOL
        assert st.steps_done == step + 1 and st.h_prev == 0.0
        assert math.isclose(st.obs.rho, re["rho"], rel_tol=TOL)
        assert math.isclose(st.obs.residual, re["residual"], rel_tol=1e-6, abs_tol=1e-12)


def test_noalloc_rejects_oversized_lattice_and_bad_precision():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    w = I.workload("preheat32")
    t = torch.zeros(64, dtype=torch.float64, device="cuda")
    st = P.pycool_stage_state()
    st.a = 1.0
    big = P.make_config(1024, 100.0, w["model"], w["params"], 0.001, order=2)
    assert P.pycool_sweep_noalloc(big, t, t, t, t, False, st) == P.E_INVALID
    split = P.make_config(32, w["L"], w["model"], w["params"], w["dt"], precision="split_fp32")
    assert P.pycool_sweep_noalloc(split, t, t, t, t, False, st) == P.E_INVALID
    assert P.pycool_noalloc_max_blocks() > 1000
