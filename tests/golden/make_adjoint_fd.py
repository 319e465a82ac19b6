"""Write adjoint_fd_24.json: central finite differences of the dissipation functional with
respect to seeded components of the body-force field, computed with the FP64 oracle only.

Setup (the adjoint check of the 128^3 adjoint workload, at 24^3): D3Q19 MRT, rates
s1 = 1.19, s2 = s10 = s12 = 1.4, s4 = s6 = s8 = 1.2, s16..18 = 1.98, viscous 1/tau0 with
tau0 = 0.51; Smagorinsky Cs = 0.17; periodic 24^3; initial velocity: divergence-free random
Fourier field (|k| <= 4, rms 0.01, seed 6) at equilibrium; force field N(0, (1e-5)^2), seed 5;
T = 16 steps; L = sum nu_eff S:S of the state step 17 would see.  Each derivative is the
Richardson combination (4 D(h/2) - D(h))/3 of central differences D with h = 2e-7.

    python tests/golden/make_adjoint_fd.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1704_07559_gb300 import inputs as I  # noqa: E402

N, T, TAU0, CS = 24, 16, 0.51, 0.17
RATES = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / TAU0, 1.4, 1 / TAU0, 1.4, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1.98, 1.98, 1.98]


def setup():
    p = O.make_params(19, RATES, closure=O.SMAG, smag_cs=CS)
    G = O.Grid(p, N, N, N)
    drho, u = I.random_fourier(N, N, N, kmax=4, rms=0.01, seed=6)
    g = I.gaussian_force(3, (N, N, N), std=1e-5, seed=5)
    f0 = G.init(drho, u, force=g)
    return G, f0, g


def functional(G, f0, g):
    f = f0.copy()
    for _ in range(T):
        f, _ = G.step(f, force=g)
    r = G.readout(f, force=g)
    S = r["S"]
    SS = S[0] ** 2 + S[1] ** 2 + S[2] ** 2 + 2 * (S[3] ** 2 + S[4] ** 2 + S[5] ** 2)
    return float((((r["tau"] - 0.5) / 3) * SS).sum())


def main():
    G, f0, g = setup()
    rng = np.random.default_rng(24)
    comps = [tuple(int(v) for v in (rng.integers(0, 3), rng.integers(0, N), rng.integers(0, N), rng.integers(0, N)))
             for _ in range(32)]
    h = 2e-7
    out = []
    for c in comps:
        def D(hh):
            gp = g.copy()
            gp[c] += hh
            gm = g.copy()
            gm[c] -= hh
            return (functional(G, f0, gp) - functional(G, f0, gm)) / (2 * hh)
        d1, d2 = D(h), D(h / 2)
        out.append({"component": list(c), "dLdg": (4 * d2 - d1) / 3, "central_h": d1, "central_h2": d2})
        print(c, out[-1]["dLdg"])
    doc = {"description": __doc__.strip().splitlines()[0], "n": N, "T": T, "tau0": TAU0, "smag_cs": CS,
           "rates": RATES, "loss": functional(G, f0, g), "entries": out}
    with open(os.path.join(HERE, "adjoint_fd_24.json"), "w") as fh:
        json.dump(doc, fh, indent=1)


if __name__ == "__main__":
    main()
