"""FP64 CPU oracle of the MRT lattice Boltzmann step with Yu and Chai strain rates.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the CPU-baseline /
reference legs of the benchmark.  The product library never imports it.  The arithmetic lives
in ``lbm_oracle.c`` (plain C, FP64, dense matrices, one node at a time); this module only
marshals numpy arrays into it.

Array conventions (all float64, C order):
  populations  f[i, z, y, x]   shape (q, nz, ny, nx)   (D2Q9: nz = 1)
  strain rate  S[c, z, y, x]   c = xx, yy, zz, xy, yz, xz (3D) or xx, yy, xy (2D)
  velocity     u[a, z, y, x]   a < d;   grad_u[a*d + b] = d u_a / d x_b
  force        F               None, a length-d vector (uniform), or an array (d, nz, ny, nx)
Faces are ordered -x, +x, -y, +y, -z, +z.
"""
import ctypes
import os

import numpy as np

from . import build as _build

PERIODIC, WALL, LID = 0, 1, 2
NEWTON, SMAG, POWERLAW, SMAG_LAGGED, SMAG_DEV = 0, 1, 2, 3, 4
YU, CHAI = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.or_tables.argtypes = [ctypes.c_int, ip, dp, dp, dp, ip]
        _lib.or_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp]
        _lib.or_meq.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp]
        _lib.or_force_bar.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp]
        _lib.or_strain_yu.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
        _lib.or_strain_chai.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
        pp = ctypes.POINTER(Params)
        _lib.or_collide.argtypes = [pp, dp, dp, ctypes.c_double, dp, dp, dp, ip, dp]
        _lib.or_node.argtypes = [pp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, dp,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, ip, dp, dp]
        _lib.or_step.argtypes = [pp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, dp,
                                 dp, dp, dp, dp, dp, dp]
        _lib.or_init.argtypes = [pp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
                                 ctypes.c_int, dp, dp]
        _lib.or_readout.argtypes = [pp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                    dp, dp, dp, dp, dp]
        _lib.or_sums.argtypes = [pp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, dp]
    return _lib


class Params(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int),
        ("closure", ctypes.c_int),
        ("formula", ctypes.c_int),
        ("smag_iters", ctypes.c_int),
        ("pl_max_iter", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("rho0", ctypes.c_double),
        ("s", ctypes.c_double * 19),
        ("smag_cs", ctypes.c_double),
        ("pl_n", ctypes.c_double),
        ("pl_k", ctypes.c_double),
        ("pl_tau_min", ctypes.c_double),
        ("pl_tau_max", ctypes.c_double),
        ("pl_tol", ctypes.c_double),
        ("lid_u", (ctypes.c_double * 3) * 6),
    ]


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    if a is None:
        return None
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def tables(q):
    """(c [q,3] int, w [q], T [q,q], Tinv [q,q] by elimination, opp [q])."""
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q)
    T = np.zeros((q, q))
    Ti = np.zeros((q, q))
    opp = np.zeros(q, np.int32)
    rc = lib().or_tables(q, _ip(c), _dp(w), _dp(T), _dp(Ti), _ip(opp))
    if rc != 0:
        raise ValueError("bad lattice %r" % q)
    return c, w, T, Ti, opp


def _vec3(j):
    v = np.zeros(3)
    j = np.asarray(j, dtype=np.float64).ravel()
    v[: len(j)] = j
    return v


def feq(q, drho, j, rho0=1.0):
    out = np.zeros(q)
    lib().or_feq(q, float(drho), _dp(_vec3(j)), float(rho0), _dp(out))
    return out


def meq(q, drho, j, rho0=1.0):
    out = np.zeros(q)
    lib().or_meq(q, float(drho), _dp(_vec3(j)), float(rho0), _dp(out))
    return out


def force_bar(q, j, F, rho0=1.0):
    out = np.zeros(q)
    lib().or_force_bar(q, _dp(_vec3(j)), float(rho0), _dp(_vec3(F)), _dp(out))
    return out


def n_strain(q):
    return 3 if q == 9 else 6


def strain_yu(q, mneq, s, rho0=1.0):
    out = np.zeros(n_strain(q))
    lib().or_strain_yu(q, _dp(_f64(mneq)), _dp(_f64(s)), float(rho0), _dp(out))
    return out


def strain_chai(q, fneq, s, rho0=1.0):
    out = np.zeros(n_strain(q))
    lib().or_strain_chai(q, _dp(_f64(fneq)), _dp(_f64(s)), float(rho0), _dp(out))
    return out


def make_params(q, rates, closure=NEWTON, formula=YU, rho0=1.0, bc=None, lid_u=None, smag_cs=0.0,
                smag_iters=6, pl_n=1.0, pl_k=0.0, pl_tau_min=0.505, pl_tau_max=5.0, pl_tol=1e-14,
                pl_max_iter=200):
    p = Params()
    p.q = q
    p.closure = closure
    p.formula = formula
    p.smag_iters = smag_iters
    p.pl_max_iter = pl_max_iter
    bc = bc if bc is not None else [PERIODIC] * 6
    for k in range(6):
        p.bc[k] = bc[k]
    p.rho0 = rho0
    rates = list(rates)
    assert len(rates) == q
    for k in range(q):
        p.s[k] = rates[k]
    p.smag_cs = smag_cs
    p.pl_n, p.pl_k, p.pl_tau_min, p.pl_tau_max, p.pl_tol = pl_n, pl_k, pl_tau_min, pl_tau_max, pl_tol
    if lid_u is not None:
        for f in range(6):
            for a in range(3):
                p.lid_u[f][a] = lid_u[f][a]
    return p


def collide(p, fin, F=None, tau_prev=0.0, with_next=False):
    """Collision of one node: returns (fout, S, tau, iters) and, with with_next, the tau to store
    for the next step.  tau_prev: the node's stored tau (lagged closure)."""
    q = p.q
    fout = np.zeros(q)
    S = np.zeros(n_strain(q))
    tau = ctypes.c_double()
    it = ctypes.c_int()
    tn = ctypes.c_double()
    Fv = None if F is None else _vec3(F)
    lib().or_collide(ctypes.byref(p), _dp(_f64(fin)), _dp(Fv), float(tau_prev), _dp(fout), _dp(S),
                     ctypes.byref(tau), ctypes.byref(it), ctypes.byref(tn))
    if with_next:
        return fout, S, tau.value, it.value, tn.value
    return fout, S, tau.value, it.value


class Grid:
    """A lattice of nx x ny x nz nodes with the oracle's parameters."""

    def __init__(self, params, nx, ny, nz=1):
        self.p = params
        self.q = params.q
        self.d = 2 if self.q == 9 else 3
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz
        self.shape = (nz, ny, nx)

    def _force(self, force):
        if force is None:
            return None, 0
        F = _f64(force)
        if F.ndim == 1:
            return F, 0
        assert F.shape == (self.d,) + self.shape
        return F, 1

    def init(self, drho, u, grad_u=None, force=None, with_tau=False):
        """Post-collision buffer of step -1 whose pull gives the requested pre-collision state;
        with_tau: also each node's closure tau at the prescribed gradient (the lagged closure's
        first stored tau), returned as (fpost, tau)."""
        fpost = np.zeros((self.q,) + self.shape)
        tau = np.zeros(self.shape)
        F, ff = self._force(force)
        rc = lib().or_init(ctypes.byref(self.p), self.nx, self.ny, self.nz, _dp(_f64(drho)), _dp(_f64(u)),
                           _dp(_f64(grad_u)), _dp(F), ff, _dp(fpost), _dp(tau))
        if rc != 0:
            raise ValueError("or_init rejected the arguments")
        return (fpost, tau) if with_tau else fpost

    def step(self, fpost, force=None, want=(), tau=None):
        """One time step.  want: any of 'S', 'tau', 'drho', 'u' (pre-collision state of this step)
        and 'tau_next' (the taus the next step reads).  tau: the stored tau per node (lagged
        closure)."""
        fnew = np.zeros_like(fpost)
        F, ff = self._force(force)
        out = {}
        S = np.zeros((n_strain(self.q),) + self.shape) if "S" in want else None
        tau_o = np.zeros(self.shape) if "tau" in want else None
        drho = np.zeros(self.shape) if "drho" in want else None
        u = np.zeros((self.d,) + self.shape) if "u" in want else None
        tn = np.zeros(self.shape) if "tau_next" in want else None
        rc = lib().or_step(ctypes.byref(self.p), self.nx, self.ny, self.nz, _dp(_f64(fpost)), _dp(F), ff,
                           _dp(_f64(tau)), _dp(fnew), _dp(S), _dp(tau_o), _dp(drho), _dp(u), _dp(tn))
        if rc != 0:
            raise ValueError("or_step rejected the arguments")
        for k, v in (("S", S), ("tau", tau_o), ("drho", drho), ("u", u), ("tau_next", tn)):
            if v is not None:
                out[k] = v
        return fnew, out

    def run(self, fpost, n, force=None, tau=None):
        """n steps; with a stored tau field (lagged closure) returns (fpost, tau)."""
        for _ in range(n):
            if tau is None:
                fpost, _ = self.step(fpost, force)
            else:
                fpost, out = self.step(fpost, force, want=("tau_next",), tau=tau)
                tau = out["tau_next"]
        return fpost if tau is None else (fpost, tau)

    def readout(self, fpost, force=None, tau=None):
        """S, tau, drho, u of the pre-collision state that the next step would see."""
        _, out = self.step(fpost, force, want=("S", "tau", "drho", "u"), tau=tau)
        return out

    def node(self, fpost, x, y, z=0, force=None, tau=None, with_next=False):
        """(fout, S, tau, iters, fin) of one node of the next step, without touching the grid
        (with_next: also the node's tau for the next step).  tau: stored taus (lagged closure)."""
        F, ff = self._force(force)
        fout = np.zeros(self.q)
        S = np.zeros(n_strain(self.q))
        fin = np.zeros(self.q)
        tau_o = ctypes.c_double()
        it = ctypes.c_int()
        tn = ctypes.c_double()
        rc = lib().or_node(ctypes.byref(self.p), self.nx, self.ny, self.nz, _dp(_f64(fpost)), _dp(F), ff,
                           _dp(_f64(tau)), x, y, z, _dp(fout), _dp(S), ctypes.byref(tau_o), ctypes.byref(it),
                           _dp(fin), ctypes.byref(tn))
        if rc != 0:
            raise ValueError("or_node rejected the arguments")
        if with_next:
            return fout, S, tau_o.value, it.value, fin, tn.value
        return fout, S, tau_o.value, it.value, fin

    def sums(self, fpost, force=None):
        out = np.zeros(1 + self.d)
        F, ff = self._force(force)
        rc = lib().or_sums(ctypes.byref(self.p), self.nx, self.ny, self.nz, _dp(_f64(fpost)), _dp(F), ff,
                           _dp(out))
        if rc != 0:
            raise ValueError("or_sums rejected the arguments")
        return out


__all__ = ["tables", "feq", "meq", "force_bar", "strain_yu", "strain_chai", "make_params", "collide",
           "Grid", "PERIODIC", "WALL", "LID", "NEWTON", "SMAG", "POWERLAW", "SMAG_LAGGED", "SMAG_DEV", "YU", "CHAI",
           "n_strain"]
