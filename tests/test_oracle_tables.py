"""Pins of the oracle's lattice tables, equilibria and strain-rate formulas against what the
paper prints and what the lattice mathematics fixes (no GPU)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def read_matrix(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([Fraction(t) for t in line.split()])
    return rows


def exact_inverse(T):
    """Exact rational inverse by Gauss-Jordan elimination on Fractions."""
    n = len(T)
    M = [[Fraction(int(T[r][k])) for k in range(n)] + [Fraction(int(r == k)) for k in range(n)] for r in range(n)]
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


def test_d3q19_velocity_set_and_weights():
    c, w, T, Ti, opp = O.tables(19)
    # eq. (HeLuoD3Q19): rest + 6 axis + 12 edge velocities, each +-pair present
    c2 = (c * c).sum(1)
    assert list(c2) == [0] + [1] * 6 + [2] * 12
    assert all((c[opp[i]] == -c[i]).all() for i in range(19))
    # eq. (omega) with the textbook isotropy of the D3Q19 quadrature
    assert abs(w.sum() - 1) < 1e-15
    d = np.eye(3)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), d / 3, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-15)
    # rows 3, 5, 7 of T are the velocity components (moment vector eq. (moment): j = rho0 u)
    assert (T[3] == c[:, 0]).all() and (T[5] == c[:, 1]).all() and (T[7] == c[:, 2]).all()


def test_d3q15_velocity_set_and_weights():
    """D3Q15 (named, not printed, by the paper): rest + 6 axis + 8 corner velocities with weights
    2/9, 1/9, 1/72; the quadrature is isotropic to fourth order like D3Q19's."""
    c, w, T, Ti, opp = O.tables(15)
    c2 = (c * c).sum(1)
    assert list(c2) == [0] + [1] * 6 + [3] * 8
    assert all((c[opp[i]] == -c[i]).all() for i in range(15))
    assert abs(w.sum() - 1) < 1e-15
    d = np.eye(3)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), d / 3, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-15)
    assert (T[3] == c[:, 0]).all() and (T[5] == c[:, 1]).all() and (T[7] == c[:, 2]).all()


def test_d3q15_rows_are_the_basis_polynomials():
    """Each row of the D3Q15 matrix is its defining polynomial of the velocity (d'Humieres et al.
    2002 basis) evaluated on the velocity set."""
    c, w, T, Ti, opp = O.tables(15)
    x, y, z = (c[:, a].astype(float) for a in range(3))
    c2 = x * x + y * y + z * z
    rows = [np.ones(15), c2 - 2, (15 * c2 ** 2 - 55 * c2 + 32) / 2, x, (5 * c2 - 13) * x / 2, y,
            (5 * c2 - 13) * y / 2, z, (5 * c2 - 13) * z / 2, 3 * x * x - c2, y * y - z * z, x * y, y * z, x * z,
            x * y * z]
    assert np.array_equal(T, np.array(rows))


def test_d2q9_velocity_set_and_weights():
    c, w, T, Ti, opp = O.tables(9)
    assert abs(w.sum() - 1) < 1e-15
    d = np.eye(2)
    c2 = c[:, :2]
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c2, c2), d / 3, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c2, c2, c2, c2)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-15)
    assert (T[3] == c[:, 0]).all() and (T[5] == c[:, 1]).all()


@pytest.mark.parametrize("q", [19, 15, 9])
def test_moment_matrix_orthogonal_and_inverse(q):
    c, w, T, Ti, opp = O.tables(q)
    G = T @ T.T
    assert np.allclose(G, np.diag(np.diag(G)), atol=0)  # integer rows, exactly orthogonal
    # the elimination inverse equals the orthogonality form T^T D^-1 and inverts T
    assert np.abs(Ti - T.T / np.diag(G)).max() < 1e-15
    assert np.abs(T @ Ti - np.eye(q)).max() < 1e-14
    if q == 19:
        assert list(np.diag(G)) == [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
    elif q == 15:
        assert list(np.diag(G)) == [15, 18, 360, 10, 40, 10, 40, 10, 40, 12, 4, 8, 8, 8, 8]
    else:
        assert list(np.diag(G)) == [9, 36, 36, 6, 12, 6, 12, 4, 4]


@pytest.mark.parametrize("k,name", [(0, "x"), (1, "y"), (2, "z")])
def test_advection_matrices_match_printed(k, name):
    """T C_k T^-1 from the oracle's T and velocity set reproduces the printed C^_k of Sec. 4.1
    exactly (rational arithmetic).  This pins every entry of T and the velocity order."""
    c, w, T, Ti, opp = O.tables(19)
    Tinv = exact_inverse(T)
    C = [[Fraction(0)] * 19 for _ in range(19)]
    for r in range(19):
        for s in range(19):
            C[r][s] = sum(Fraction(int(T[r][i])) * int(c[i][k]) * Tinv[i][s] for i in range(19))
    P = read_matrix("chat_%s.txt" % name)
    diffs = [(r, s, P[r][s], C[r][s]) for r in range(19) for s in range(19) if P[r][s] != C[r][s]]
    if name == "z":
        # the single misprint documented in the fixture header
        assert diffs == [(16, 13, Fraction(1), Fraction(0))]
    else:
        assert diffs == []


def rng_states(n, seed=0):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield rng.normal(scale=1e-2), rng.normal(scale=3e-2, size=3)


@pytest.mark.parametrize("q", [19, 15, 9])
def test_equilibrium_moments_closed_form(q):
    """eq. (meq) (closed-form m_eq) equals T f_eq of eq. (edf), at random states and rho0 != 1."""
    c, w, T, Ti, opp = O.tables(q)
    for drho, j in rng_states(50, seed=q):
        for rho0 in (1.0, 1.3):
            if q == 9:
                j = j.copy()
                j[2] = 0
            fe = O.feq(q, drho, j, rho0)
            me = O.meq(q, drho, j, rho0)
            assert np.abs(T @ fe - me).max() < 1e-15


@pytest.mark.parametrize("q", [19, 15, 9])
def test_equilibrium_velocity_moments(q):
    """The He-Luo equilibrium satisfies eq. (cfeqmoment_) of Sec. 4.2:
    sum f = drho, sum c f = j, sum cc f = cs2 drho I + rho0 u u, sum ccc f = cs2 rho0 (delta u)."""
    c, w, T, Ti, opp = O.tables(q)
    d = 2 if q == 9 else 3
    cc = c[:, :d].astype(float)
    I = np.eye(d)
    for drho, j in rng_states(20, seed=7):
        rho0 = 1.2
        j = j[:d]
        u = j / rho0
        fe = O.feq(q, drho, j, rho0)
        assert abs(fe.sum() - drho) < 1e-15
        assert np.abs(cc.T @ fe - j).max() < 1e-15
        P = np.einsum("i,ia,ib->ab", fe, cc, cc)
        assert np.abs(P - (drho / 3 * I + rho0 * np.outer(u, u))).max() < 1e-15
        Q = np.einsum("i,ia,ib,ic->abc", fe, cc, cc, cc)
        ref = rho0 / 3 * (np.einsum("ab,c->abc", I, u) + np.einsum("ac,b->abc", I, u) + np.einsum("bc,a->abc", I, u))
        assert np.abs(Q - ref).max() < 1e-15


def test_chai_second_moments_match_printed_N():
    """Chai's contraction applied to a single non-equilibrium moment e_k reproduces the printed
    N_ab coefficients of Sec. 5.1 (golden/n_alpha_beta.txt); S = -N / (2 rho0 cs2)."""
    c, w, T, Ti, opp = O.tables(19)
    comps = ["xx", "yy", "zz", "xy", "yz", "xz"]
    gold = {}
    with open(os.path.join(GOLD, "n_alpha_beta.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            comp, k, coef = line.split()
            gold[(comp, int(k))] = float(Fraction(coef))
    rng = np.random.default_rng(3)
    s = rng.uniform(0.5, 1.9, size=19)
    s[[0, 3, 5, 7]] = 0.0
    for k in range(1, 19):
        e = np.zeros(19)
        e[k] = 1.0
        fneq = Ti @ e
        S = O.strain_chai(19, fneq, s)
        N = -S * 2.0 / 3.0
        for p, comp in enumerate(comps):
            want = gold.get((comp, k), 0.0) * s[k]
            assert abs(N[p] - want) < 1e-15, (comp, k, N[p], want)


def yu_chai_pair(q, s, seed, scale=1e-3, n=30, rho0=1.0):
    c, w, T, Ti, opp = O.tables(q)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(n):
        f = rng.normal(scale=scale, size=q)
        drho = f.sum()
        j = c.T @ f
        fneq = f - O.feq(q, drho, j, rho0)
        mneq = T @ f - O.meq(q, drho, j, rho0)
        Sy = O.strain_yu(q, mneq, s, rho0)
        Sc = O.strain_chai(q, fneq, s, rho0)
        worst = max(worst, np.abs(Sy - Sc).max() / np.abs(Sc).max())
    return worst


def test_yu_equals_chai_d3q19():
    """Sec. 5.1: Yu's formula and Chai's formula give the same S on D3Q19 (to rounding), for
    arbitrary states and any rates with s9 = s11 = s13 = s14 = s15."""
    tau = 0.6
    s = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / tau, 1.4, 1 / tau, 1.4, 1 / tau, 1 / tau, 1 / tau, 1.98, 1.98,
         1.98]
    assert yu_chai_pair(19, s, 1) < 1e-13
    rng = np.random.default_rng(2)
    for _ in range(5):
        s = list(rng.uniform(0.3, 1.95, size=19))
        for k in (0, 3, 5, 7):
            s[k] = 0.0
        for k in (11, 13, 14, 15):
            s[k] = s[9]
        assert yu_chai_pair(19, s, 5, rho0=1.1) < 1e-13


def test_yu_chai_differ_when_rates_split():
    """Yu's formula assumes one viscous rate; with s13 != s9 the two routes differ (Chai uses the
    individual rate), which is why the library rejects the Yu route for split rates."""
    s = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1.6, 1.4, 1.6, 1.4, 1.2, 1.6, 1.6, 1.98, 1.98, 1.98]
    assert yu_chai_pair(19, s, 1) > 1e-3


def test_yu_type_equals_chai_d3q15():
    """Sec. 5.4 procedure on D3Q15: the Yu-type formula derived from Chai's equals Chai's, for the
    workload rates and for random rates with one viscous rate on moments 9..13."""
    s = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2] + [1 / 0.6] * 5 + [1.98]
    assert yu_chai_pair(15, s, 6) < 1e-13
    rng = np.random.default_rng(8)
    for _ in range(5):
        s = list(rng.uniform(0.3, 1.95, size=15))
        for k in (0, 3, 5, 7):
            s[k] = 0.0
        for k in (10, 11, 12, 13):
            s[k] = s[9]
        assert yu_chai_pair(15, s, 9, rho0=0.9) < 1e-13


def test_yu_type_equals_chai_d2q9():
    """Sec. 5.4 procedure on D2Q9: the Yu-type formula derived from Chai's equals Chai's."""
    s = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 1 / 0.7, 1 / 0.7]
    assert yu_chai_pair(9, s, 4) < 1e-13


@pytest.mark.parametrize("q", [19, 15, 9])
def test_force_moments(q):
    """Guo-type discrete force: sum Fbar = 0, sum c Fbar = F, sum cc Fbar = uF + Fu, and T Fbar is
    the derivative of the closed-form m_eq along F (central difference of a quadratic)."""
    c, w, T, Ti, opp = O.tables(q)
    d = 2 if q == 9 else 3
    rng = np.random.default_rng(11)
    for _ in range(10):
        rho0 = 1.0 + 0.2 * rng.random()
        j = np.zeros(3)
        j[:d] = rng.normal(scale=0.03, size=d)
        F = np.zeros(3)
        F[:d] = rng.normal(scale=1e-3, size=d)
        Fb = O.force_bar(q, j, F, rho0)
        u = j[:d] / rho0
        cc = c[:, :d].astype(float)
        assert abs(Fb.sum()) < 1e-17
        assert np.abs(cc.T @ Fb - F[:d]).max() < 1e-17
        P = np.einsum("i,ia,ib->ab", Fb, cc, cc)
        assert np.abs(P - (np.outer(u, F[:d]) + np.outer(F[:d], u))).max() < 1e-17
        # m_eq is quadratic in j, so the central difference is exact for any step h
        h = 1.0
        dm = (O.meq(q, 0.3, j + h * F, rho0) - O.meq(q, 0.3, j - h * F, rho0)) / (2 * h)
        assert np.abs(T @ Fb - dm).max() < 1e-15


VISCOUS_SET = {19: [1, 9, 11, 13, 14, 15], 15: [1, 9, 10, 11, 12, 13], 9: [1, 7, 8]}


@pytest.mark.parametrize("q", [19, 15, 9])
def test_first_order_moments_by_advection_matrices(q):
    """Sec. 4.1 / 5.4: the first-order non-equilibrium moments that initialise a velocity
    gradient are m1 = -L^-1 [sum_a C^_a d_a m_eq + d_t m_eq] with C^_a = T C_a T^-1, worked out here
    numerically from the tables (d_t drho = -div j, j linear in x, drho uniform).  The oracle's
    initialisation, typed in by hand per lattice (D3Q19: eq. (YuLuobasis)), must hold exactly these
    values in the moments that carry the strain rate."""
    c, w, T, Ti, opp = O.tables(q)
    d = 2 if q == 9 else 3
    rng = np.random.default_rng(20 + q)
    s = rng.uniform(0.6, 1.9, size=q)
    nu = VISCOUS_SET[q][1:]
    s[nu] = s[nu[0]]
    for _ in range(4):
        Gm = np.zeros((3, 3))
        Gm[:d, :d] = rng.normal(scale=1e-2, size=(d, d))  # G[a, b] = d u_a / d x_b, rho0 = 1
        # d m_eq / d j . v at j = 0 (m_eq is quadratic in j: the central difference is exact)
        def dmeq(v):
            return (O.meq(q, 0.0, v) - O.meq(q, 0.0, -v)) / 2
        dmeq_drho = O.meq(q, 1.0, np.zeros(3)) - O.meq(q, 0.0, np.zeros(3))
        src = -np.trace(Gm) * dmeq_drho
        for a in range(d):
            Ca = T @ np.diag(c[:, a].astype(float)) @ Ti
            src += Ca @ dmeq(Gm[:, a])
        m1 = -src / s
        # the oracle's initial state on a single periodic node (pointwise, so no streaming mixes it)
        shape = (1, 1, 1)
        p = O.make_params(q, list(s))
        G = O.Grid(p, 1, 1, 1)
        grad = np.zeros((d * d,) + shape)
        for a in range(d):
            for b in range(d):
                grad[a * d + b] = Gm[a, b]
        f = G.init(np.zeros(shape), np.zeros((d,) + shape), grad_u=grad).reshape(q)
        mneq = T @ f - O.meq(q, f.sum(), c.T @ f)
        for k in VISCOUS_SET[q]:
            assert abs(mneq[k] - m1[k]) < 1e-15, (k, mneq[k], m1[k])
