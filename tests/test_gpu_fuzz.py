"""Seeded random configurations against the FP64 oracle, element by element (same checks and bars
as test_gpu_parity): lattice, storage, closure, route, boundary kind per axis (periodic, walls,
a moving wall), force (none, uniform, per-node field) and grid extents from 1 to 40 (odd and even,
so both the one-node and the two-node 16-bit kernels and every pull path are exercised)."""
import numpy as np
import pytest

from test_gpu_parity import Case

pytestmark = pytest.mark.gpu

N_CASES = 96
N_16BIT = 48  # further draws on D3Q19 / D3Q15 with 16-bit storage (one- and two-node kernels)


def draw(k, sixteen=False):
    rng = np.random.default_rng(1000 + k + (50_000 if sixteen else 0))
    q = int(rng.choice([19, 15])) if sixteen else int(rng.choice([19, 19, 15, 9]))
    d = 2 if q == 9 else 3
    if sixteen:
        precision = str(rng.choice(["fp16s", "bf16s"]))
    else:
        precision = str(rng.choice(["fp64", "fp32", "fp16s", "bf16s"] if q != 9 else ["fp64", "fp32"]))
    closures = ["newton", "smag"]
    if precision in ("fp64", "fp32"):
        closures += ["powerlaw", "smag_lagged", "smag_dev"]
    closure = str(rng.choice(closures))
    formula = str(rng.choice(["yu", "chai"]))
    dims = [int(rng.integers(1, 41)), int(rng.integers(1, 21)), int(rng.integers(1, 9)) if d == 3 else 1]
    bc, lid = [], {}
    for a in range(d):
        kind = rng.choice(["periodic", "wall", "lid"], p=[0.5, 0.3, 0.2])
        if kind == "periodic":
            bc += ["periodic", "periodic"]
        else:
            dims[a] = max(dims[a], 2)
            face = 2 * a + int(rng.integers(2))
            bc += ["wall", "wall"]
            if kind == "lid":
                bc[face] = "lid"
                v = [0.0, 0.0, 0.0]
                v[(a + 1) % d] = float(rng.uniform(-0.05, 0.05))
                lid[face] = tuple(v)
    bc += ["periodic"] * (6 - len(bc))
    extra = dict(bc=bc, lid=lid, tau=float(rng.uniform(0.51, 0.9)))
    fk = rng.integers(3)
    if fk == 1:
        extra["force"] = list(rng.normal(scale=1e-5, size=d))
    elif fk == 2:
        extra["force_field"] = True
    if closure == "powerlaw":
        extra["pl"] = (float(rng.choice([0.6, 1.0, 1.4])), float(rng.uniform(0.005, 0.05)))
    return q, tuple(dims), precision, closure, formula, extra


@pytest.mark.parametrize("k,sixteen", [(k, False) for k in range(N_CASES)] + [(k, True) for k in range(N_16BIT)])
def test_random_configuration(k, sixteen):
    q, dims, precision, closure, formula, extra = draw(k, sixteen)
    c = Case(q, dims, precision, closure, formula, seed=k, **extra)
    c.check_init()
    for _ in range(2):
        c.check_step()
    c.check_sums()
