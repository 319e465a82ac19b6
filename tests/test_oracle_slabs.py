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
