"""Pins of the FP64 CPU reference gradient (oracle/autograd_ref.py): its forward map is the C
oracle's, and its gradient equals finite differences of the C oracle (no GPU)."""
import json
import os

import numpy as np
import torch

import oracle as O
from oracle import autograd_ref as AR
from paper_1704_07559_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden", "adjoint_fd_24.json")


def test_forward_equals_c_oracle():
    tau0, cs = 0.51, 0.17
    r = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / tau0, 1.4, 1 / tau0, 1.4, 1 / tau0, 1 / tau0, 1 / tau0, 1.98, 1.98,
         1.98]
    n = 6
    drho, u = I.random_fourier(n, n, n, kmax=2, rms=0.02, seed=6)
    g = I.gaussian_force(3, (n, n, n), std=1e-5, seed=5)
    G = O.Grid(O.make_params(19, r, closure=O.SMAG, smag_cs=cs), n, n, n)
    f = G.init(drho, u, force=g)
    M = AR.Model(r, cs)
    ft = torch.tensor(f)
    for _ in range(3):
        f, _ = G.step(f, force=g)
        ft = M.step(ft, torch.tensor(g))
    assert np.abs(ft.numpy() - f).max() <= 1e-14 * np.abs(f).max()


def test_gradient_equals_oracle_finite_differences():
    """autograd through the restatement = central differences (Richardson) of the C oracle on the
    32 seeded components of the golden file, to the differences' own accuracy."""
    doc = json.load(open(GOLD))
    n, T = doc["n"], doc["T"]
    G = O.Grid(O.make_params(19, doc["rates"], closure=O.SMAG, smag_cs=doc["smag_cs"]), n, n, n)
    drho, u = I.random_fourier(n, n, n, kmax=4, rms=0.01, seed=6)
    g = I.gaussian_force(3, (n, n, n), std=1e-5, seed=5)
    f0 = G.init(drho, u, force=g)
    L, grad, _ = AR.loss_and_grad(f0, g, doc["rates"], doc["smag_cs"], T, segment=4)
    assert abs(L - doc["loss"]) <= 1e-13 * abs(doc["loss"])
    fd = np.array([e["dLdg"] for e in doc["entries"]])
    ad = np.array([grad[tuple(e["component"])] for e in doc["entries"]])
    assert np.abs(ad - fd).max() <= 1e-7 * np.abs(fd).max()
