"""The library's adjoint (lbm_adjoint) against the FP64 CPU reference gradient and against
finite differences of the FP64 oracle.

Bars: FP64 populations, 1e-10 relative (normwise) to the autograd reference; FP32 populations
with FP64 accumulation, 1e-4 relative to finite differences and to the reference (the stated
bar for the gradient)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from oracle import autograd_ref as AR
from paper_1704_07559_gb300 import inputs as I
from paper_1704_07559_gb300 import lbm

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "adjoint_fd_24.json")
TAU0, CS = 0.51, 0.17
RATES = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / TAU0, 1.4, 1 / TAU0, 1.4, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1.98, 1.98,
         1.98]


def setup(dims, precision, closure="smag", formula="yu", rms=0.02, kmax=2, develop=2):
    """Lattice with the force field bound and the state set to f0: the seeded Fourier field at
    equilibrium, advanced `develop` oracle steps so that it carries a strain rate."""
    nx, ny, nz = dims
    drho, u = I.random_fourier(nx, ny, nz, kmax=kmax, rms=rms, seed=6)
    g = I.gaussian_force(3, (nz, ny, nx), std=1e-5, seed=5)
    G = O.Grid(O.make_params(19, RATES, closure=O.SMAG if closure == "smag" else O.NEWTON, smag_cs=CS), nx, ny, nz)
    f0 = G.run(G.init(drho, u, force=g), develop, force=g)
    lat = lbm.Lattice(19, nx, ny, nz, rates=RATES, precision=precision, closure=closure, smag_cs=CS, formula=formula,
                      force_field=torch.from_numpy(g))
    lat.set_state(torch.from_numpy(f0))
    return lat, f0, g


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("seg", [1, 3, 7, 10])
def test_fp64_adjoint_matches_reference(seg):
    """Every checkpoint segmentation gives the reference gradient (ragged last segment included)."""
    dims, T = (10, 8, 6), 7
    lat, f0, g = setup(dims, "fp64")
    L, grad = lat.adjoint(T, seg)
    Lr, gr, fT = AR.loss_and_grad(f0, g, RATES, CS, T)
    assert abs(L - Lr) <= 1e-12 * abs(Lr)
    assert rel(grad.cpu().numpy(), gr) <= 1e-10
    # the context holds the state after T steps
    assert np.abs(lat.get_state().cpu().numpy() - fT).max() <= 1e-12 * np.abs(fT).max()


def test_fp64_newtonian_and_chai_forward():
    """The derivative is that of the common function of both routes (Sec. 5.1): a context whose
    step uses Chai's formula, and the Newtonian closure, both match the reference."""
    dims, T = (8, 6, 6), 5
    lat, f0, g = setup(dims, "fp64", formula="chai")
    L, grad = lat.adjoint(T, 2)
    Lr, gr, _ = AR.loss_and_grad(f0, g, RATES, CS, T)
    assert rel(grad.cpu().numpy(), gr) <= 1e-10
    lat2, f0, g = setup(dims, "fp64", closure="newton")
    L2, grad2 = lat2.adjoint(T, 2)
    Lr2, gr2, _ = AR.loss_and_grad(f0, g, RATES, 0.0, T)
    assert abs(L2 - Lr2) <= 1e-12 * abs(Lr2)
    assert rel(grad2.cpu().numpy(), gr2) <= 1e-10


def test_zero_steps_is_the_direct_term():
    lat, f0, g = setup((8, 6, 4), "fp64")
    L, grad = lat.adjoint(0, 1)
    Lr, gr, _ = AR.loss_and_grad(f0, g, RATES, CS, 0)
    assert abs(L - Lr) <= 1e-12 * abs(Lr)
    assert rel(grad.cpu().numpy(), gr) <= 1e-10


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-7), ("fp32", 1e-4)])
def test_adjoint_matches_finite_differences_24(precision, tol):
    """24^3, T = 16: the 32 seeded components of the golden finite differences of the FP64 oracle."""
    doc = json.load(open(GOLD))
    n, T = doc["n"], doc["T"]
    lat, f0, g = setup((n, n, n), precision, rms=0.01, kmax=4, develop=0)
    L, grad = lat.adjoint(T, 4)
    grad = grad.cpu().numpy()
    fd = np.array([e["dLdg"] for e in doc["entries"]])
    ad = np.array([grad[tuple(e["component"])] for e in doc["entries"]])
    assert np.abs(ad - fd).max() <= tol * np.abs(fd).max()
    assert abs(L - doc["loss"]) <= (1e-12 if precision == "fp64" else 1e-5) * abs(doc["loss"])


def test_fp32_adjoint_matches_reference_gradient_24():
    """All 3 x 24^3 components of the FP32 gradient against the FP64 reference: 1e-4 relative."""
    n, T = 24, 16
    lat, f0, g = setup((n, n, n), "fp32", rms=0.01, kmax=4, develop=0)
    L, grad = lat.adjoint(T, 4)
    Lr, gr, _ = AR.loss_and_grad(f0, g, RATES, CS, T, segment=4)
    assert rel(grad.cpu().numpy(), gr) <= 1e-4


def test_autograd_function():
    """DissipationLoss wires the adjoint into torch.autograd."""
    dims, T = (8, 6, 6), 4
    lat, f0, g = setup(dims, "fp64")
    gt = torch.tensor(g, device="cuda", requires_grad=True)
    L = lbm.DissipationLoss.apply(gt, lat, torch.from_numpy(f0).cuda(), T, 2)
    (3.0 * L).backward()
    Lr, gr, _ = AR.loss_and_grad(f0, g, RATES, CS, T)
    assert abs(float(L.detach()) - Lr) <= 1e-12 * abs(Lr)
    assert rel(gt.grad.cpu().numpy(), 3.0 * gr) <= 1e-10


def test_adjoint_rejects_unsupported_setups():
    lat = lbm.Lattice(19, 8, 8, 8, rates=RATES, closure="smag", smag_cs=CS)  # no force field
    with pytest.raises(lbm.LBMError) as e:
        lat.adjoint(4)
    assert e.value.code == -1
    g = torch.zeros(3, 8, 8, 8, dtype=torch.float32)
    lat2 = lbm.Lattice(19, 8, 8, 8, rates=RATES, closure="smag", smag_cs=CS, force_field=g,
                       bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2)
    with pytest.raises(lbm.LBMError):
        lat2.adjoint(4)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_at_rest_is_exactly_zero(precision):
    """|S| is not differentiable at S = 0 (its derivative is taken as 0 there).  A fluid at rest
    under a zero force field has S = 0 at every node and step, L = 0, and L is quadratic in g
    there, so dL/dg = 0: the adjoint must return exact zeros, not NaN."""
    n = 8
    g = torch.zeros(3, n, n, n, dtype=torch.float64)
    lat = lbm.Lattice(19, n, n, n, rates=RATES, precision=precision, closure="smag", smag_cs=CS,
                      force_field=g)
    lat.init(np.zeros((n, n, n)), np.zeros((3, n, n, n)))
    L, grad = lat.adjoint(6, 2)
    assert L == 0.0
    assert torch.isfinite(grad).all() and float(grad.abs().max()) == 0.0
