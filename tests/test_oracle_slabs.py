"""The z-slab harness (oracle/slabs.py) that the full-size GPU parity test uses to run the oracle
over millions of nodes: on a small channel its slab-parallel steps and read-outs equal the
whole-grid oracle bit for bit (no GPU)."""
import numpy as np
import pytest

import oracle as O
from oracle import slabs
from paper_1704_07559_gb300 import inputs as I

TAU0 = 0.51
RATES = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / TAU0, 1.4, 1 / TAU0, 1.4, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1.98,
         1.98, 1.98]
CHANNEL = [O.PERIODIC, O.PERIODIC, O.WALL, O.WALL, O.PERIODIC, O.PERIODIC]


@pytest.mark.parametrize("formula,steps,workers", [(O.YU, 2, 3), (O.CHAI, 1, 4), (O.YU, 3, 5)])
def test_slabs_equal_the_whole_grid(formula, steps, workers):
    nx, ny, nz = 12, 10, 11
    kw = dict(q=19, rates=RATES, closure=O.SMAG, smag_cs=0.17, formula=formula, bc=CHANNEL)
    G = O.Grid(O.make_params(**kw), nx, ny, nz)
    drho, u = I.channel_profile(nx, ny, nz, u_centre=0.1, noise=0.01, seed=2)
    F = np.array([1e-5, 0.0, 0.0])
    f0 = G.run(G.init(drho, u, force=F), 2, force=F)
    want = G.run(f0, steps, force=F)
    got, reads = slabs.run(kw, f0, steps=steps, force=F, readouts=("yu", "chai"), workers=workers)
    assert np.array_equal(got, want)
    for fm, code in (("yu", O.YU), ("chai", O.CHAI)):
        r = O.Grid(O.make_params(**dict(kw, formula=code)), nx, ny, nz).readout(f0, force=F)
        assert np.array_equal(reads[fm][0], r["S"])
        assert np.array_equal(reads[fm][1], r["tau"])


@pytest.mark.parametrize("steps,workers", [(1, 3), (2, 4)])
def test_slabs_cut_along_walled_y_equal_the_whole_grid(steps, workers):
    """Cuts along y, the channel's walled axis: slabs at the walls keep them, interior cuts get a
    dummy wall whose effect stays in the dropped halo rows."""
    nx, ny, nz = 9, 13, 5
    kw = dict(q=19, rates=RATES, closure=O.SMAG, smag_cs=0.17, formula=O.YU, bc=CHANNEL)
    G = O.Grid(O.make_params(**kw), nx, ny, nz)
    drho, u = I.channel_profile(nx, ny, nz, u_centre=0.1, noise=0.01, seed=2)
    F = np.array([1e-5, 0.0, 2e-6])
    f0 = G.run(G.init(drho, u, force=F), 2, force=F)
    got, reads = slabs.run(kw, f0, steps=steps, force=F, readouts=("yu", "chai"), workers=workers, axis="y")
    assert np.array_equal(got, G.run(f0, steps, force=F))
    for fm, code in (("yu", O.YU), ("chai", O.CHAI)):
        r = O.Grid(O.make_params(**dict(kw, formula=code)), nx, ny, nz).readout(f0, force=F)
        assert np.array_equal(reads[fm][0], r["S"])
        assert np.array_equal(reads[fm][1], r["tau"])


def test_d2q9_power_law_cavity_cut_along_y():
    n, U = 24, 0.05
    lid = [[0.0, 0.0, 0.0] for _ in range(6)]
    lid[3] = [U, 0.0, 0.0]
    rates9 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 1 / 0.7, 1 / 0.7]
    kw = dict(q=9, rates=rates9, closure=O.POWERLAW, formula=O.CHAI, pl_n=0.5, pl_k=0.01,
              bc=[O.WALL, O.WALL, O.WALL, O.LID, O.PERIODIC, O.PERIODIC], lid_u=lid, pl_tol=1e-14)
    G = O.Grid(O.make_params(**kw), n, n, 1)
    f0 = G.run(G.init(np.zeros((1, n, n)), np.zeros((2, 1, n, n))), 5)
    got, reads = slabs.run(kw, f0, steps=2, readouts=("yu", "chai"), workers=5, axis="y")
    assert np.array_equal(got, G.run(f0, 2))
    r = G.readout(f0)
    assert np.array_equal(reads["chai"][0], r["S"])
    assert np.array_equal(reads["chai"][1], r["tau"])
