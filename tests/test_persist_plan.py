"""The persistent kernel's work plan (host logic, no GPU).

pycool_evolve on an n = 32k lattice runs one cooperative launch whose blocks
walk a host-made table of units (a tile of (32 vx) x 16 sites and a z-range,
loaded with one z-halo plane per side, two for the 13-point stencil).
The kernel trusts the table, so here every plan the library can make for the
timed and tested shapes is checked on the CPU:
  - every (tile, z) pair of the lattice is in exactly one unit and every unit
    lies inside the lattice (tile-aligned x0, y0; 1 <= planes; z0 + planes <= n);
  - at most 64 units per block, at most min(sms, 208) blocks;
  - the blocks' work is even: with the plan's cost model (a plane costs 1,
    or 1.24 at the periodic y boundary in the split form; a unit adds 2h for
    its z-halo planes and switch) the busiest block is within a few percent of
    the mean for the full-size lattices;
  - the plan is a pure function of its arguments."""
import numpy as np
import pytest

P = pytest.importorskip("paper_1201_5029_gb300")

L2 = 126 << 20   # bytes of L2 (a GB300's order of magnitude)

SHAPES = [(n, nf, prec, st) for n in (32, 64, 96, 128, 256, 512) for nf in (1, 2)
          for prec, st in ((P.FP64, P.STENCIL_7PT), (P.SPLIT_FP32, P.STENCIL_7PT),
                           (P.SPLIT_DD, P.STENCIL_7PT), (P.FP64, P.STENCIL_4TH),
                           (P.SPLIT_DD, P.STENCIL_4TH))]


def _vx(n, nf, prec):
    word = 4 if prec == P.SPLIT_FP32 else 8
    for v in (4, 2, 1):
        if v * nf * word <= 16 and n % (32 * v) == 0:
            return v
    return 1


def _model(n, nf, prec, l2):
    word = 4 if prec == P.SPLIT_FP32 else 8
    resident = l2 > 0 and 4 * nf * n ** 3 * word <= 0.75 * l2
    return (0.25, 1.0) if prec != P.SPLIT_FP32 else ((1.5 if resident else 0.3), 1.24)


def _cost(units, n, h, pen, halo=1):
    tiles_y = n // 16
    ty = units[:, 1] // 16
    wrap = (ty == 0) | (ty == tiles_y - 1)
    return (units[:, 3] - 2 * halo + 2 * halo * h) * np.where(wrap, pen, 1.0)


@pytest.mark.parametrize("n,nf,prec,stencil", SHAPES)
@pytest.mark.parametrize("sms,l2", [(152, L2), (148, L2), (152, 0)])
def test_plan_covers_lattice_once(n, nf, prec, stencil, sms, l2):
    g, units, uoff = P.pycool_persist_plan(n, nf, prec, sms, l2, stencil)
    vx = _vx(n, nf, prec)
    halo = 2 if stencil == P.STENCIL_4TH else 1
    assert g["halo"] == halo
    assert g["n"] == n and g["vx"] == vx and g["tx"] == 32 * vx
    assert g["tiles_x"] == n // (32 * vx) and g["ntiles"] == g["tiles_x"] * (n // 16)
    assert 1 <= g["G"] <= min(sms, 208)
    assert uoff[0] == 0 and uoff[-1] == len(units) == g["nunits"]
    counts = np.diff(uoff)
    assert (counts >= 1).all() and (counts <= 64).all()
    x0, y0, z0, w = units.T
    planes = w - 2 * halo
    assert (x0 % g["tx"] == 0).all() and (x0 >= 0).all() and (x0 + g["tx"] <= n).all()
    assert (y0 % 16 == 0).all() and (y0 >= 0).all() and (y0 + 16 <= n).all()
    assert (planes >= 1).all() and (z0 >= 0).all() and (z0 + planes <= n).all()
    seen = np.zeros((g["ntiles"], n), dtype=np.int32)
    tile = (y0 // 16) * g["tiles_x"] + x0 // g["tx"]
    for t, z, p in zip(tile, z0, planes):
        seen[t, z:z + p] += 1
    assert (seen == 1).all()


@pytest.mark.parametrize("n,nf,prec,bound", [
    (128, 2, P.SPLIT_FP32, 1.08), (256, 1, P.SPLIT_FP32, 1.02), (256, 2, P.SPLIT_FP32, 1.02),
    (128, 2, P.FP64, 1.03), (256, 1, P.FP64, 1.02), (256, 2, P.FP64, 1.02)])
def test_plan_balances_blocks(n, nf, prec, bound):
    g, units, uoff = P.pycool_persist_plan(n, nf, prec, 152, L2)
    h, pen = _model(n, nf, prec, L2)
    load = np.add.reduceat(_cost(units, n, h, pen), uoff[:-1])
    assert g["G"] == 152
    assert load.max() <= bound * load.mean(), (load.max(), load.mean())
    # and no block does more than an even share of the planes plus one unit's worth
    tiles_y = n // 16
    share = n * g["tiles_x"] * ((tiles_y - 2) + 2 * pen) / 152
    assert load.max() <= share + 2 * h * pen * (np.diff(uoff).max()) + 1.0


def test_plan_is_deterministic():
    a = P.pycool_persist_plan(256, 2, P.SPLIT_FP32, 152, L2)
    b = P.pycool_persist_plan(256, 2, P.SPLIT_FP32, 152, L2)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("n,nf,prec,bound", [(128, 2, P.FP64, 1.04), (256, 2, P.FP64, 1.02),
                                             (256, 1, P.SPLIT_DD, 1.02)])
def test_plan_balances_blocks_13_point(n, nf, prec, bound):
    """Four z-halo planes per unit (13-point stencil): still an even split (at
    128^3 a block holds ~28 planes, so one plane is 3.6 % of it)."""
    g, units, uoff = P.pycool_persist_plan(n, nf, prec, 152, L2, P.STENCIL_4TH)
    h, pen = _model(n, nf, prec, L2)
    load = np.add.reduceat(_cost(units, n, h, pen, halo=2), uoff[:-1])
    assert g["G"] == 152 and g["halo"] == 2
    assert load.max() <= bound * load.mean(), (load.max(), load.mean())


@pytest.mark.parametrize("args", [(48, 1, P.FP64, 152, L2), (0, 1, P.FP64, 152, L2),
                                  (64, 3, P.FP64, 152, L2), (64, 1, 7, 152, L2),
                                  (64, 1, P.FP64, 0, L2), (64, 1, P.FP64, 152, -1),
                                  (64, 1, P.FP64, 152, L2, 9),
                                  (64, 1, P.SPLIT_FP32, 152, L2, P.STENCIL_4TH)])
def test_plan_rejects_bad_arguments(args):
    with pytest.raises(P.PycoolError) as ei:
        P.pycool_persist_plan(*args)
    assert ei.value.status == P.E_INVALID
