"""Split-FP32 form against the FP64 oracle (GPU).

The split form stores the fluctuations around the float64 lattice mean in
float32, so it does not reproduce the oracle to round-off; its error on every
reported quantity is measured here and bounded (the bounds are stated in the
asserts and are the form's accuracy claim at these workloads)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
import gpu_helpers as G  # noqa: E402


@pytest.mark.parametrize("name,order,n,steps", [
    ("preheat32", 2, 32, 100),
    ("preheat128", 4, 24, 20),
    ("oscillon256", 6, 20, 10),
    ("qball256", 8, 16, 6),
    ("oscillon256", 6, 128, 2),   # TMA kernel, 4 sites per lane (float4)
    ("preheat128", 4, 64, 5),     # TMA kernel, 2 sites per lane, 2 fields
    ("qball256", 8, 96, 1),       # TMA kernel, 1 site per lane
])
@pytest.mark.parametrize("stencil", ["7pt", "iso27"])
def test_split_errors_against_oracle(name, order, n, steps, stencil):
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=n, order=order, stencil=stencil,
                                           precision="split_fp32"), phi, pi, steps)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=order, stencil=stencil), phi, pi, steps)
    # fluctuation error relative to the fluctuation scale of each field
    fl = []
    for f in range(phi.shape[0]):
        scale = float(np.max(np.abs(st.phi[f] - st.phi[f].mean())))
        fl.append(float(np.max(np.abs(gphi[f] - st.phi[f]))) / scale)
    ea, epa = G.rel(ge["a"], st.a), G.rel(ge["pa"], st.pa)
    erho = G.rel(ge["rho"], oe["rho"])
    evar = [G.rel(ge["variance"][f], np.var(st.phi[f])) for f in range(phi.shape[0])]
    print(f"\n{name} n={n} order={order} {stencil}: dphi/scale={fl} a={ea:.2e} pa={epa:.2e} "
          f"rho={erho:.2e} var={evar}")
    assert max(fl) < 1e-4
    assert ea < 1e-9 and epa < 1e-7
    assert erho < 1e-7
    assert max(evar) < 1e-4
    assert max(G.field_errors(gphi, st.phi)) < 1e-5


@pytest.mark.parametrize("amp", [1e-6, 0.05])
@pytest.mark.parametrize("n", [64, 24])
def test_qball_log1p_branches(amp, n):
    """The split Q-ball takes log1p(du/u0) by its Taylor series for |du/u0| <
    2^-7 and by log1pf beyond: fluctuations of 1e-6 keep every site on the
    series, 0.05 puts many on log1pf (persistent kernel at 64, per-stage
    kernel at 24).  Errors at 1e-4 of the fluctuation scale, as above."""
    w = I.workload("qball256")
    phi, pi = I.initial_fields(w, n=n)
    phi = phi + amp * np.random.default_rng(12).standard_normal(phi.shape)
    gphi, gpi, ge = G.run_gpu(P, G.gpu_cfg(P, w, n=n, order=4, precision="split_fp32"),
                              phi, pi, 3)
    st, oe = G.run_oracle(G.oracle_cfg(w, n=n, order=4), phi, pi, 3)
    for g, o in ((gphi, st.phi), (gpi, st.pi)):
        for f in range(2):
            scale = float(np.max(np.abs(o[f] - o[f].mean())))
            err = float(np.max(np.abs(g[f] - o[f]))) / scale
            print(f"\nqball split amp={amp} n={n}: error {err:.1e} of scale {scale:.1e}")
            assert err < 1e-4, (amp, n, f, err)
    # p_a sums V and phi D over fluctuations up to 0.05 in float32 parts
    assert G.rel(ge["a"], st.a) < 1e-9 and G.rel(ge["pa"], st.pa) < 1e-6
