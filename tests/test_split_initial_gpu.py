"""The split forms' initial state and read-out on the device (GPU).

set_initial splits each field into its lattice mean (the float64 background)
and the rest (float32, or a double-float pair), and get_fields adds them back,
both in kernels.  Checked here:
- host and device inputs give the same state bit for bit, and host and device
  read-outs the same values bit for bit;
- the background is the lattice mean (against math.fsum, to a few ulps);
- the round trip x -> (mean, fluctuation) -> x is within the form's rounding
  of the fluctuation: 2^-24 of it for float32, 2^-48 for a double-float pair,
  plus float64 roundings of x itself;
- the first time steps from either input are identical.
Lattice sides cover the persistent kernel (32) and the per-stage kernels of
other sides (24, split-FP32 only), one field and two; the split-FP32 read-out of one field
runs in two chunks, the others in one."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1201_5029_gb300")
from paper_1201_5029_gb300 import inputs as I  # noqa: E402
import gpu_helpers as G  # noqa: E402

FRAC = {"split_fp32": 2.0 ** -23, "split_dd": 2.0 ** -47}

CASES = [("split_fp32", "oscillon256", 24), ("split_fp32", "preheat128", 32),
         ("split_fp32", "oscillon256", 32), ("split_dd", "oscillon256", 32),
         ("split_dd", "qball256", 32), ("split_dd", "preheat128", 32)]


@pytest.mark.parametrize("precision,name,n", CASES)
def test_host_and_device_initial_state(precision, name, n):
    w = I.workload(name)
    phi, pi = I.initial_fields(w, n=n)
    cfg = G.gpu_cfg(P, w, n=n, order=2, precision=precision)
    dphi = torch.from_numpy(phi).cuda()
    dpi = torch.from_numpy(pi).cuda()
    with P.Simulation(cfg) as sh, P.Simulation(cfg) as sd:
        sh.set_initial(phi, pi)
        sd.set_initial(dphi, dpi, on_device=True)
        torch.cuda.synchronize()
        eh, ed = sh.energies(), sd.energies()
        hphi, hpi = sh.get_fields()
        gphi, gpi = sd.get_fields()
        assert np.array_equal(hphi, gphi) and np.array_equal(hpi, gpi)
        assert sh.checkpoint() == sd.checkpoint()
        # device read-out equals the host read-out bit for bit
        ophi, opi = torch.empty_like(dphi), torch.empty_like(dpi)
        sd.get_fields(ophi, opi, on_device=True)
        torch.cuda.synchronize()
        assert np.array_equal(ophi.cpu().numpy(), hphi)
        assert np.array_equal(opi.cpu().numpy(), hpi)
        # the lattice mean of phi (background + mean fluctuation) is the
        # input's, within the rounding of the fluctuations
        for f in range(phi.shape[0]):
            x = phi[f]
            m = math.fsum(x.ravel()) / x.size
            bound = FRAC[precision] * np.max(np.abs(x - m)) + 4 * 2.0 ** -53 * np.max(np.abs(x))
            assert abs(eh["mean"][f] - m) <= bound, (f, eh["mean"][f], m)
        # the round trip is within the rounding of the fluctuation
        for x, y in ((phi, hphi), (pi, hpi)):
            for f in range(x.shape[0]):
                scale = np.max(np.abs(x[f] - x[f].mean()))
                err = np.max(np.abs(y[f] - x[f]))
                bound = FRAC[precision] * scale + 4 * 2.0 ** -53 * np.max(np.abs(x[f]))
                assert err <= bound, (f, err, bound)
        for k in ("rho", "P", "a", "pa"):
            assert eh[k] == ed[k], k
        sh.evolve(2)
        sd.evolve(2)
        a1, b1 = sh.get_fields()
        a2, b2 = sd.get_fields()
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
