"""Exact-arithmetic brute force of whole time steps, against the FP64 oracle.

A second, independent statement of the step in rational arithmetic (fractions.Fraction): the
moment matrix is built from the basis polynomials of the moment vector evaluated on the velocity
set (not the oracle's table typed from the paper), the equilibrium moments are T f_eq of the
He-Luo equilibrium (not the closed form), the inverse is an exact Gauss-Jordan, the strain rate is
Chai's definition -sum_i c_i c_i (T^-1 L T f_neq)_i / (2 rho0 cs2) with f_neq = f - f_eq + Fbar/2.
Rates and force are dyadic, so the oracle's float inputs equal the rational ones exactly; two
periodic steps with a uniform force on a 2x2x2 D3Q19 and a 3x3 D2Q9 grid, Newtonian closure (the
Smagorinsky closure is pinned by its fixed-point residual elsewhere).  Bar: a few units of FP64
roundoff: 4 ulp of max |f*| and 8 ulp of max |S| (measured: at most 2.9 and 2.8).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O

EPS = 2.0 ** -52


def poly_rows(q, c):
    """Rows of the moment matrix: the basis polynomials evaluated on the velocities."""
    rows = []
    for cx, cy, cz in c:
        c2 = cx * cx + cy * cy + cz * cz
        if q == 19:  # d'Humieres et al. (2002) D3Q19 basis, moment order of eq. (moment)
            rows.append([1, 19 * c2 - 30, Fr(21 * c2 * c2 - 53 * c2 + 24, 2), cx, (5 * c2 - 9) * cx, cy,
                         (5 * c2 - 9) * cy, cz, (5 * c2 - 9) * cz, 3 * cx * cx - c2, (3 * c2 - 5) * (3 * cx * cx - c2),
                         cy * cy - cz * cz, (3 * c2 - 5) * (cy * cy - cz * cz), cx * cy, cy * cz, cx * cz,
                         (cy * cy - cz * cz) * cx, (cz * cz - cx * cx) * cy, (cx * cx - cy * cy) * cz])
        else:  # Lallemand-Luo D2Q9 basis
            rows.append([1, -4 + 3 * c2, 4 - Fr(21, 2) * c2 + Fr(9, 2) * c2 * c2, cx, (-5 + 3 * c2) * cx, cy,
                         (-5 + 3 * c2) * cy, cx * cx - cy * cy, cx * cy])
    return [[Fr(rows[i][k]) for i in range(q)] for k in range(q)]  # T[k][i]


def inverse(T):
    n = len(T)
    M = [list(T[r]) + [Fr(int(r == k)) for k in range(n)] for r in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        inv = 1 / M[col][col]
        M[col] = [v * inv for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                fct = M[r][col]
                M[r] = [a - fct * b for a, b in zip(M[r], M[col])]
    return [row[n:] for row in M]


def weights(q, c):
    table = {19: {0: Fr(1, 3), 1: Fr(1, 18), 2: Fr(1, 36)}, 9: {0: Fr(4, 9), 1: Fr(1, 9), 2: Fr(1, 36)}}[q]
    return [table[cx * cx + cy * cy + cz * cz] for cx, cy, cz in c]


def matvec(M, v):
    return [sum((a * b for a, b in zip(row, v)), Fr(0)) for row in M]


def exact_step(q, c, T, Ti, w, s, F, f, dims):
    """One pull + collide step in rational arithmetic; returns (f*, S of the pre-collision state)."""
    nx, ny, nz = dims
    d = 2 if q == 9 else 3
    out = {}
    Sout = {}
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)] if d == 3 else [(0, 0), (1, 1), (0, 1)]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                fin = [f[i][((z - c[i][2]) % nz, (y - c[i][1]) % ny, (x - c[i][0]) % nx)] for i in range(q)]
                drho = sum(fin, Fr(0))
                j = [sum((c[i][a] * fin[i] for i in range(q)), Fr(0)) + F[a] / 2 for a in range(3)]
                u = j  # rho0 = 1
                uu = sum(v * v for v in u)
                feq, Fb = [], []
                for i in range(q):
                    cu = sum(c[i][a] * u[a] for a in range(3))
                    cF = sum(c[i][a] * F[a] for a in range(3))
                    uF = sum(u[a] * F[a] for a in range(3))
                    feq.append(w[i] * (drho + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * uu))
                    Fb.append(w[i] * (3 * (cF - uF) + 9 * cu * cF))
                m, meq, TF = matvec(T, fin), matvec(T, feq), matvec(T, Fb)
                ms = [m[k] - s[k] * (m[k] - meq[k]) + (1 - s[k] / 2) * TF[k] for k in range(q)]
                out[(z, y, x)] = matvec(Ti, ms)
                fneq = [fin[i] - feq[i] + Fb[i] / 2 for i in range(q)]
                Om = matvec(Ti, [s[k] * v for k, v in enumerate(matvec(T, fneq))])
                Sout[(z, y, x)] = [-sum((c[i][a] * c[i][b] * Om[i] for i in range(q)), Fr(0)) * Fr(3, 2)
                                   for a, b in comps]
    fnew = [{key: out[key][i] for key in out} for i in range(q)]
    return fnew, Sout


@pytest.mark.parametrize("q,dims", [(19, (2, 2, 2)), (9, (3, 3, 1))])
def test_two_steps_match_exact_rational_arithmetic(q, dims):
    c, _, _, _, _ = O.tables(q)
    c = [tuple(int(v) for v in row) for row in c]
    T = poly_rows(q, c)
    Ti = inverse(T)
    w = weights(q, c)
    # dyadic rates (exact in binary) with s_nu = 3/2 on the viscous moments
    if q == 19:
        s = [0, 1.1875, 1.375, 0, 1.25, 0, 1.25, 0, 1.25, 1.5, 1.375, 1.5, 1.375, 1.5, 1.5, 1.5, 1.9375, 1.9375, 1.9375]
    else:
        s = [0, 1.1875, 1.375, 0, 1.25, 0, 1.25, 1.5, 1.5]
    F = [2.0 ** -16, -(2.0 ** -17), 2.0 ** -18 if q == 19 else 0.0]
    nx, ny, nz = dims
    rng = np.random.default_rng(q)
    f0 = rng.normal(scale=1e-2, size=(q, nz, ny, nx))
    G = O.Grid(O.make_params(q, s, formula=O.CHAI), nx, ny, nz)
    Fd = np.array(F[:2 if q == 9 else 3])
    fex = [{(z, y, x): Fr(float(f0[i, z, y, x])) for z in range(nz) for y in range(ny) for x in range(nx)}
           for i in range(q)]
    sfr, Ffr = [Fr(v) for v in s], [Fr(v) for v in F]
    fo = f0
    for _ in range(2):
        fex, Sex = exact_step(q, c, T, Ti, w, sfr, Ffr, fex, dims)
        fo, out = G.step(fo, force=Fd, want=("S",))
        exact = np.array([[[[float(fex[i][(z, y, x)]) for x in range(nx)] for y in range(ny)] for z in range(nz)]
                          for i in range(q)])
        assert np.abs(fo - exact).max() <= 4 * EPS * np.abs(exact).max()
        Se = np.array([[[[float(Sex[(z, y, x)][k]) for x in range(nx)] for y in range(ny)] for z in range(nz)]
                       for k in range(len(Sex[(0, 0, 0)]))])
        assert np.abs(out["S"] - Se).max() <= 8 * EPS * np.abs(Se).max()
    # the Yu route gives the same S (Sec. 5.1 / 5.4)
    G.p.formula = O.YU
    r = G.readout(fo, force=Fd)
    Sex_next = exact_step(q, c, T, Ti, w, sfr, Ffr, fex, dims)[1]
    Se = np.array([[[[float(Sex_next[(z, y, x)][k]) for x in range(nx)] for y in range(ny)] for z in range(nz)]
                   for k in range(len(Sex_next[(0, 0, 0)]))])
    assert np.abs(r["S"] - Se).max() <= 8 * EPS * np.abs(Se).max()
