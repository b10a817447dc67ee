"""The library's grouping of lattice modes by k_eff^2 (host only, no GPU).

pycool_linear_modes lists the distinct k_eff^2 of an n^3 lattice and each
mode's index into them: the grouping by which the linearised evolution
advances one transfer matrix per distinct value (Sec. 2.2).  It must agree
with the oracle's grouping of the symbols it computes from the stencil's
offsets, and with the 7-point closed form."""
import numpy as np
import pytest

P = pytest.importorskip("paper_1201_5029_gb300")
from oracle import pycool_linear as L  # noqa: E402


@pytest.mark.parametrize("n,stencil", [(8, "7pt"), (10, "7pt"), (12, "iso27"), (64, "7pt"),
                                       (96, "iso27"), (8, "4th"), (12, "4th"), (64, "4th")])
def test_modes_match_oracle_grouping(n, stencil):
    vals, idx = P.pycool_linear_modes(n, stencil)
    ov, oi = L.distinct_k2(L.k_eff2(n, stencil))
    assert len(vals) == len(ov)
    assert np.max(np.abs(vals - ov)) < 1e-12
    assert np.array_equal(idx, oi)
    assert np.all(np.diff(vals) > 0)


@pytest.mark.parametrize("n", [16, 32])
def test_seven_point_values_closed_form(n):
    vals, idx = P.pycool_linear_modes(n, "7pt")
    m = np.fft.fftfreq(n) * n
    s = 4.0 * np.sin(np.pi * m / n) ** 2
    closed = s[:, None, None] + s[None, :, None] + s[None, None, :]
    assert np.max(np.abs(vals[idx] - closed)) < 1e-12
    assert vals[0] == pytest.approx(0.0, abs=1e-15) and vals[-1] == pytest.approx(12.0)
    # far fewer equations than modes: the point of the grouping
    assert len(vals) < n ** 3 / 20


def test_modes_reject_bad_arguments():
    with pytest.raises(P.PycoolError):
        P.pycool_linear_modes(0)
    with pytest.raises(P.PycoolError):
        P.pycool_linear_modes(8, 5)
