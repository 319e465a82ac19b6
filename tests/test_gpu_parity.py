"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element, on the
same seeded inputs.  Every step is checked from the same input state: the oracle takes the GPU's
populations (converted exactly to float64), advances one step, and the GPU's output must match.

Tolerances (normwise: max |gpu - oracle| / max |oracle| per array):
  FP64 path     1e-12 on S, tau, drho, u and the populations;
  FP32 path     1e-5 on S and tau (the stated FP32 bar), 2e-6 on populations, drho and u;
  FP16S / BF16S populations within one unit roundoff of the 16-bit format of |f*| (FP16 also its
                subnormal spacing 2^-24) plus the FP32 bound;
                S and tau of a 16-bit state 1e-5 (the read-out is FP32 arithmetic on exactly
                converted values).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1704_07559_gb300 import inputs as I
from paper_1704_07559_gb300 import lbm

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(S=1e-12, f=1e-12, m=1e-12), "fp32": dict(S=1e-5, f=2e-6, m=2e-6),
       "fp16s": dict(S=1e-5, f=2e-6, m=2e-6, eps=2.0 ** -11, abs=2.0 ** -24),
       "bf16s": dict(S=1e-5, f=2e-6, m=2e-6, eps=2.0 ** -8)}
BCN = {"periodic": O.PERIODIC, "wall": O.WALL, "lid": O.LID}


def rates(q, tau):
    if q == 19:
        return [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / tau, 1.4, 1 / tau, 1.4, 1 / tau, 1 / tau, 1 / tau, 1.98,
                1.98, 1.98]
    if q == 15:
        return [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / tau, 1 / tau, 1 / tau, 1 / tau, 1 / tau, 1.98]
    return [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 1 / tau, 1 / tau]


def relerr(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def f64(t):
    return t.detach().to(torch.float64).cpu().numpy()


class Case:
    def __init__(self, q, dims, precision="fp32", closure="newton", formula="yu", tau=0.6, bc=None, lid=None,
                 force=None, force_field=False, smag_cs=0.17, pl=(1.0, 0.0), seed=0):
        self.q, self.dims, self.precision = q, dims, precision
        self.d = 2 if q == 9 else 3
        self.shape = (dims[2], dims[1], dims[0])
        self.bc = list(bc or ["periodic"] * 6)
        self.bc += ["periodic"] * (6 - len(self.bc))
        self.lid = lid or {}
        rng = np.random.default_rng(seed)
        self.force = force
        self.ffield = I.gaussian_force(self.d, self.shape, std=2e-5, seed=seed + 7) if force_field else None
        kw = dict(rates=rates(q, tau), precision=precision, closure=closure, formula=formula, bc=self.bc,
                  lid_u=self.lid, smag_cs=smag_cs, pl_n=pl[0], pl_k=pl[1])
        if force is not None:
            kw["force"] = force
        if force_field:
            kw["force_field"] = torch.from_numpy(self.ffield)
        self.lat = lbm.Lattice(q, *dims, **kw)
        lid_u = [[0.0, 0.0, 0.0] for _ in range(6)]
        for f, v in self.lid.items():
            lid_u[f] = list(v)
        self.p = O.make_params(q, rates(q, tau), closure={"newton": O.NEWTON, "smag": O.SMAG, "powerlaw": O.POWERLAW,
                                                          "smag_lagged": O.SMAG_LAGGED,
                                                          "smag_dev": O.SMAG_DEV}[closure],
                               formula=O.YU if formula == "yu" else O.CHAI, bc=[BCN[b] for b in self.bc],
                               lid_u=lid_u, smag_cs=smag_cs, pl_n=pl[0], pl_k=pl[1],
                               pl_tol=1e-14 if precision == "fp64" else 1e-7)
        self.G = O.Grid(self.p, *dims)
        # random smooth-ish macroscopic fields (any state is a valid parity input)
        self.drho = rng.normal(scale=1e-3, size=self.shape)
        self.u = rng.normal(scale=0.02, size=(self.d,) + self.shape)
        self.g = rng.normal(scale=2e-3, size=(self.d * self.d,) + self.shape)

    @property
    def oforce(self):
        if self.ffield is not None:
            return self.ffield
        return None if self.force is None else np.array(self.force, dtype=np.float64)

    def check_init(self):
        self.lat.init(self.drho, self.u, self.g)
        fg = f64(self.lat.get_state())
        fo, to = self.G.init(self.drho, self.u, self.g, force=self.oforce, with_tau=True)
        t = TOL[self.precision]
        bound = t.get("eps", 0.0) * np.abs(fo) + t["f"] * np.abs(fo).max() + t.get("abs", 0.0)
        assert np.all(np.abs(fg - fo) <= bound), relerr(fg, fo)
        if self.lat.tau is not None:  # the lagged closure's first stored tau
            assert relerr(f64(self.lat.tau), to) <= t["m"]
        return fg

    @property
    def tau_in(self):
        return None if self.lat.tau is None else f64(self.lat.tau)

    def check_step(self, formulas=("yu", "chai")):
        """Read-outs of the current state, then one step, each against the oracle."""
        t = TOL[self.precision]
        fin = f64(self.lat.get_state())
        tin = self.tau_in
        fo, out = self.G.step(fin, force=self.oforce, want=("S", "tau", "drho", "u", "tau_next"), tau=tin)
        for fm in formulas:
            S, tau = self.lat.strain_rate(fm, with_tau=True)
            p_saved = self.p.formula
            self.p.formula = O.YU if fm == "yu" else O.CHAI
            ro = self.G.readout(fin, force=self.oforce, tau=tin)
            self.p.formula = p_saved
            assert relerr(f64(S), ro["S"]) <= t["S"], (fm, relerr(f64(S), ro["S"]))
            assert relerr(f64(tau), ro["tau"]) <= t["S"], (fm, relerr(f64(tau), ro["tau"]))
        drho, u = self.lat.macroscopic()
        assert relerr(f64(drho), out["drho"]) <= t["m"]
        assert relerr(f64(u), out["u"]) <= t["m"]
        self.lat.step(1)
        fg = f64(self.lat.get_state())
        bound = t.get("eps", 0.0) * np.abs(fo) + t["f"] * np.abs(fo).max() + t.get("abs", 0.0)
        assert np.all(np.abs(fg - fo) <= bound), relerr(fg, fo)
        if self.lat.tau is not None:  # the tau stored for the next step
            assert relerr(f64(self.lat.tau), out["tau_next"]) <= t["S"]
        return fg

    def check_sums(self):
        fin = f64(self.lat.get_state())
        so = self.G.sums(fin, force=self.oforce)
        sg = self.lat.sums()
        scale = self.G.N * np.abs(fin).max()
        tol = 1e-13 if self.precision == "fp64" else 1e-6
        assert np.abs(sg - so).max() <= tol * scale, (sg, so)


CASES = [
    # lattice, dims, precision, closure, formula, extra
    (19, (150, 7, 5), "fp64", "newton", "yu", {}),
    (19, (150, 7, 5), "fp64", "smag", "chai", dict(force=[1e-5, -2e-5, 3e-6])),
    (19, (37, 6, 9), "fp64", "smag", "yu", dict(bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
                                                 force=[1e-5, 0, 0])),
    (19, (9, 8, 7), "fp64", "newton", "chai", dict(bc=["wall"] * 5 + ["lid"], lid={5: (0.05, 0.02, 0.0)})),
    (19, (150, 7, 5), "fp32", "newton", "yu", {}),
    (19, (150, 7, 5), "fp32", "newton", "chai", {}),
    (19, (130, 9, 6), "fp32", "smag", "yu", dict(bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
                                                  force=[1e-5, 0, 0], tau=0.51)),
    (19, (130, 9, 6), "fp32", "smag", "chai", dict(bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
                                                    force=[1e-5, 0, 0], tau=0.51)),
    (19, (33, 17, 5), "fp32", "smag", "chai", dict(force_field=True)),
    (19, (33, 17, 5), "fp32", "powerlaw", "yu", dict(pl=(0.7, 0.01), tau=0.7)),
    (19, (11, 10, 9), "fp32", "newton", "yu", dict(bc=["wall"] * 5 + ["lid"], lid={5: (0.05, 0.0, 0.01)})),
    (19, (150, 7, 5), "fp16s", "smag", "yu", dict(tau=0.51)),
    (19, (150, 7, 5), "bf16s", "smag", "chai", dict(tau=0.51)),
    (19, (64, 6, 6), "fp16s", "newton", "chai", dict(bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
                                                      force=[1e-5, 0, 0])),
    # odd nx: 16-bit storage on the one-node kernel (even nx takes two nodes per thread)
    (19, (33, 17, 5), "bf16s", "smag", "yu", dict(tau=0.51, force_field=True)),
    (19, (33, 8, 6), "fp16s", "smag", "chai", dict(tau=0.51, bc=["wall"] * 2 + ["periodic"] * 4)),
    # even nx with walls at x: the two-node kernel's general pull at the x faces
    (19, (40, 8, 6), "fp16s", "smag", "yu", dict(tau=0.51, bc=["wall"] * 2 + ["periodic"] * 2 + ["wall", "lid"],
                                                  lid={5: (0.04, 0.0, 0.0)})),
    # even nx, the two-node kernel's packed pair arithmetic with the per-node force field (read as
    # one pair per component), on both routes, and with fixed rates
    (19, (34, 17, 5), "fp16s", "smag", "chai", dict(tau=0.51, force_field=True)),
    (19, (34, 17, 5), "bf16s", "smag", "yu", dict(tau=0.51, force_field=True)),
    (19, (66, 7, 5), "bf16s", "newton", "yu", dict(force=[1e-5, -2e-5, 3e-6])),
    (15, (34, 9, 6), "fp16s", "smag", "chai", dict(tau=0.51, force_field=True)),
    (9, (150, 37, 1), "fp64", "powerlaw", "chai", dict(bc=["wall"] * 3 + ["lid"], lid={3: (0.05, 0.0, 0.0)},
                                                       pl=(0.5, 7e-4), tau=1.0)),
    (9, (150, 37, 1), "fp32", "powerlaw", "chai", dict(bc=["wall"] * 3 + ["lid"], lid={3: (0.05, 0.0, 0.0)},
                                                       pl=(1.5, 2.0), tau=1.0)),
    (9, (150, 37, 1), "fp32", "powerlaw", "yu", dict(pl=(0.5, 7e-4), tau=1.0)),
    (9, (97, 40, 1), "fp32", "smag", "yu", dict(force=[1e-5, 2e-6])),
    (9, (97, 40, 1), "fp64", "newton", "chai", dict(force_field=True)),
    (15, (150, 7, 5), "fp64", "smag", "yu", dict(force=[1e-5, -2e-5, 3e-6], tau=0.55)),
    (15, (37, 6, 9), "fp64", "newton", "chai", dict(bc=["wall"] * 5 + ["lid"], lid={5: (0.05, 0.02, 0.0)})),
    (15, (130, 9, 6), "fp32", "smag", "yu", dict(bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
                                                  force=[1e-5, 0, 0], tau=0.51)),
    (15, (130, 9, 6), "fp32", "smag", "chai", dict(bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
                                                    force=[1e-5, 0, 0], tau=0.51)),
    (15, (33, 17, 5), "fp32", "powerlaw", "chai", dict(force_field=True, pl=(0.7, 0.01), tau=0.7)),
    (15, (11, 10, 9), "fp32", "newton", "yu", dict(bc=["wall"] * 4 + ["periodic"] * 2)),
    (15, (64, 9, 6), "fp16s", "smag", "yu", dict(tau=0.51, bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
                                                  force=[1e-5, 0, 0])),
    (15, (33, 9, 6), "bf16s", "smag", "chai", dict(tau=0.51, force_field=True)),
    (19, (130, 9, 6), "fp64", "smag_lagged", "yu", dict(bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
                                                         force=[1e-5, 0, 0], tau=0.51)),
    (19, (130, 9, 6), "fp32", "smag_lagged", "chai", dict(force_field=True, tau=0.51)),
    (19, (150, 7, 5), "fp64", "smag_dev", "chai", dict(force=[1e-5, -2e-5, 3e-6], tau=0.51)),
    (19, (130, 9, 6), "fp32", "smag_dev", "yu", dict(bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
                                                      force=[1e-5, 0, 0], tau=0.51)),
    (15, (33, 17, 5), "fp32", "smag_lagged", "yu", dict(tau=0.51)),
    (9, (97, 40, 1), "fp32", "smag_dev", "chai", dict(bc=["wall"] * 3 + ["lid"], lid={3: (0.05, 0.0, 0.0)}, tau=0.51)),
]


@pytest.mark.parametrize("q,dims,precision,closure,formula,extra", CASES,
                         ids=["%d-%s-%s-%s-%s-%d" % (c[0], "x".join(map(str, c[1])), c[2], c[3], c[4], k)
                              for k, c in enumerate(CASES)])
def test_step_parity(q, dims, precision, closure, formula, extra):
    c = Case(q, dims, precision, closure, formula, seed=len(dims) + dims[0], **extra)
    c.check_init()
    for _ in range(3):
        c.check_step()
    c.check_sums()


@pytest.mark.parametrize("q", [19, 15])
def test_fp64_trajectory_matches_oracle(q):
    """Twenty FP64 steps run independently on both sides stay within 1e-12 (TGV, Smagorinsky)."""
    n = 12
    drho, u, g = I.taylor_green_3d(n, u0=0.04, pressure=True)
    r = rates(q, 0.51)
    for formula in ("yu", "chai"):
        lat = lbm.Lattice(q, n, n, n, rates=r, precision="fp64", closure="smag", smag_cs=0.17, formula=formula)
        lat.init(drho, u, g).step(20)
        G = O.Grid(O.make_params(q, r, closure=O.SMAG, smag_cs=0.17, formula=O.YU if formula == "yu" else O.CHAI),
                   n, n, n)
        fo = G.run(G.init(drho, u, g), 20)
        assert relerr(f64(lat.get_state()), fo) <= 1e-12
        assert relerr(f64(lat.strain_rate("yu")), G.readout(fo)["S"]) <= 1e-12


@pytest.mark.parametrize("q", [19, 15])
@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 5, 3), (4, 1, 1), (2, 2, 2)])
def test_degenerate_periodic_grids(dims, q):
    """Grids of extent 1 or 2 on an axis (every neighbour wraps onto the node itself or its twin)."""
    c = Case(q, dims, "fp64", "smag", "chai", tau=0.55, seed=3)
    c.check_init()
    c.check_step()
    c.check_sums()


@pytest.mark.parametrize("q", [19, 15])
def test_zero_steps_and_yu_equals_chai_on_gpu(q):
    """lbm_step(0) leaves the state untouched; both routes give the same S (Sec. 5.1 on D3Q19,
    the Sec. 5.4 Yu-type formula on D3Q15) on the GPU too, to FP32 rounding."""
    c = Case(q, (40, 12, 10), "fp32", "smag", "yu", tau=0.51, seed=9)
    c.lat.init(c.drho, c.u, c.g)
    f0 = f64(c.lat.get_state())
    c.lat.step(0)
    assert np.array_equal(f64(c.lat.get_state()), f0)
    c.lat.step(2)
    Sy = f64(c.lat.strain_rate("yu"))
    Sc = f64(c.lat.strain_rate("chai"))
    assert relerr(Sy, Sc) <= 1e-5


def test_errors_are_reported_not_raised_as_faults():
    lat = lbm.Lattice(19, 8, 8, 8, rates=rates(19, 0.6))
    with pytest.raises(lbm.LBMError) as e:
        lat.step(-1)
    assert e.value.code == -1
    assert lbm.lib().lbm_strain_rate(lat.ctx, 7, None, None) == -1  # unknown formula
    # split viscous rates: Chai accepted, Yu read-out refused
    r = rates(19, 0.6)
    r[13] = 1.2
    lat2 = lbm.Lattice(19, 8, 8, 8, rates=r, formula="chai")
    with pytest.raises(lbm.LBMError):
        lat2.strain_rate("yu")
    lat2.strain_rate("chai")


def test_lagged_closure_needs_its_tau_field():
    """Through the raw C ABI: with the lagged closure and no tau field bound, init, step and
    read-outs report LBM_ERR_STATE (no kernel runs); after lbm_bind_tau they succeed."""
    import ctypes

    L = lbm.lib()
    p = lbm.default_params()
    p.closure = 3
    p.smag_cs = 0.17
    r = rates(19, 0.6)
    ctx = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(ctx), 19, 8, 8, 8, (ctypes.c_double * 19)(*r), None, ctypes.byref(p)) == 0
    stride = ctypes.c_int64()
    L.lbm_layout(ctx, None, ctypes.byref(stride), None)
    fa = torch.zeros((19, stride.value), dtype=torch.float32, device="cuda")
    fb = torch.zeros_like(fa)
    s = torch.cuda.current_stream()
    assert L.lbm_bind(ctx, ctypes.c_void_p(fa.data_ptr()), ctypes.c_void_p(fb.data_ptr()), None,
                      ctypes.c_void_p(s.cuda_stream)) == 0
    drho = torch.zeros(512, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * 512, dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    assert L.lbm_init(ctx, vp(drho.data_ptr()), vp(u.data_ptr()), None) == -5
    assert L.lbm_step(ctx, 1) == -5
    S = torch.empty(6 * 512, dtype=torch.float32, device="cuda")
    assert L.lbm_strain_rate(ctx, 0, vp(S.data_ptr()), None) == -5
    assert L.lbm_bind_tau(ctx, None) == -1
    tau = torch.empty(512, dtype=torch.float32, device="cuda")
    assert L.lbm_bind_tau(ctx, vp(tau.data_ptr())) == 0
    assert L.lbm_init(ctx, vp(drho.data_ptr()), vp(u.data_ptr()), None) == 0
    assert L.lbm_step(ctx, 2) == 0
    torch.cuda.synchronize()
    assert torch.all(tau == torch.tensor(1 / r[9], dtype=torch.float32, device="cuda"))  # fluid at rest
    L.lbm_destroy(ctx)
