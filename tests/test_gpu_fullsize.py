"""Parity at the full workload sizes, through the same library calls and launches that bench.py
times (its own workload constructors build every lattice here).

The headline channel (256 x 128 x 128) is compared whole: every node's read-outs and populations
against the oracle run over z-slabs in parallel host processes; so is the 4096^2 D2Q9 cavity (the
oracle over y-slabs).  The 512^3 box and the channel's variants are compared at sampled nodes:
after a few GPU steps, the strain-rate read-outs and the next step are compared with the FP64
oracle at corners, face and edge centres, and seeded random nodes.  For each
sampled node the oracle gets the node's neighbourhood, a patch of up to 3 x 3 x 3 nodes cut from
the GPU's populations (converted exactly to float64) with the workload's boundary kind on every
face the node touches, and computes that node's collision on its own (or_node).  Bars are those
of the element-by-element parity tests, normwise over the sample: FP64 1e-12; FP32 1e-5 on S
and tau, 2e-6 on populations; 16-bit storage one unit roundoff of the format on top.

The 32^3 FP64 Taylor-Green workload is small enough for whole-array parity over its 500 steps.
The adjoint workload (128^3, T = 256) is checked by a property that holds at any size: the
gradient's directional derivative dL/dg . v equals the central difference of the loss along v
(losses from the FP64 path), to 1e-4 relative for the FP32 adjoint.
"""
import numpy as np
import pytest
import torch

import bench
import oracle as O
from paper_1704_07559_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(S=1e-12, f=1e-12), "fp32": dict(S=1e-5, f=2e-6),
       "fp16s": dict(S=1e-5, f=2e-6, eps=2.0 ** -11, abs=2.0 ** -24),
       "bf16s": dict(S=1e-5, f=2e-6, eps=2.0 ** -8)}
BCN = {"periodic": O.PERIODIC, "wall": O.WALL, "lid": O.LID}
CL = {"newton": O.NEWTON, "smag": O.SMAG, "powerlaw": O.POWERLAW, "smag_lagged": O.SMAG_LAGGED,
      "smag_dev": O.SMAG_DEV}


def sample_nodes(dims, n_random, seed, d):
    nx, ny, nz = dims
    pts = set()
    for x in (0, nx // 2, nx - 1):
        for y in (0, ny // 2, ny - 1):
            for z in ((0, nz // 2, nz - 1) if d == 3 else (0,)):
                pts.add((x, y, z))
    rng = np.random.default_rng(seed)
    while len(pts) < 27 + n_random:
        pts.add((int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))))
    return sorted(pts)


def patch(f, node, dims, bc, d):
    """The neighbourhood of `node` cut from f (q, nz, ny, nx), as float64, with the centre's
    index in the patch and the patch's face kinds (the workload's kinds: on a walled axis the
    patch stops at the wall, so the centre sees the same boundary as in the full grid)."""
    idx, centre, kinds = [], [], []
    for a in range(3):
        n, p = dims[a], node[a]
        if d == 2 and a == 2:
            ii, c = [p], 0
        elif bc[2 * a] == "periodic":
            ii, c = [(p - 1) % n, p, (p + 1) % n], 1
        else:
            lo, hi = max(0, p - 1), min(n - 1, p + 1)
            ii, c = list(range(lo, hi + 1)), p - lo
        idx.append(torch.tensor(ii, device=f.device))
        centre.append(c)
        kinds += [BCN[bc[2 * a]], BCN[bc[2 * a + 1]]]
    ix, iy, iz = idx
    sub = f[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]
    return np.ascontiguousarray(sub.to(torch.float64).cpu().numpy()), centre, kinds


def at_nodes(t, nodes):
    xs = torch.tensor([p[0] for p in nodes], device=t.device)
    ys = torch.tensor([p[1] for p in nodes], device=t.device)
    zs = torch.tensor([p[2] for p in nodes], device=t.device)
    if t.dim() == 3:
        return t[zs, ys, xs].to(torch.float64).cpu().numpy()
    return t[:, zs, ys, xs].to(torch.float64).cpu().numpy()


def relerr(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)


def check_sampled(lat, rates, precision, closure, formula, bc, nodes, force=None, lid=None, smag_cs=0.0,
                  pl=(1.0, 0.0), formulas=("yu", "chai")):
    """Read-outs by each formula and one step of `lat`, against the oracle at `nodes`."""
    t = TOL[precision]
    q, d, dims = lat.q, lat.d, (lat.nx, lat.ny, lat.nz)
    fin = lat.get_state()
    patches = [patch(fin, p, dims, bc, d) for p in nodes]
    del fin
    lagged = lat.tau is not None  # the lagged closure reads each node's stored tau
    tau_in = at_nodes(lat.tau, nodes) if lagged else None
    reads = {}
    for fm in formulas:
        S, tau = lat.strain_rate(fm, with_tau=True)
        reads[fm] = (at_nodes(S, nodes), at_nodes(tau, nodes))
        del S, tau
    lat.step(1)
    fout = at_nodes(lat.get_state(), nodes)
    tau_next = at_nodes(lat.tau, nodes) if lagged else None
    lid_u = [[0.0, 0.0, 0.0] for _ in range(6)]
    for fc, v in (lid or {}).items():
        lid_u[fc] = list(v)
    ffield = lat.force_field

    def params(kinds, fm):
        return O.make_params(q, rates, closure=CL[closure], formula=O.YU if fm == "yu" else O.CHAI, bc=kinds,
                             lid_u=lid_u, smag_cs=smag_cs, pl_n=pl[0], pl_k=pl[1],
                             pl_tol=1e-14 if precision == "fp64" else 1e-7)

    fo = np.zeros((q, len(nodes)))
    tn_o = np.zeros(len(nodes))
    So = {fm: np.zeros((lat.ns, len(nodes))) for fm in formulas}
    to = {fm: np.zeros(len(nodes)) for fm in formulas}
    for k, (node, (sub, c, kinds)) in enumerate(zip(nodes, patches)):
        if ffield is not None:
            F = ffield[:, node[2], node[1], node[0]].to(torch.float64).cpu().numpy()
        else:
            F = None if force is None else np.array(force, dtype=np.float64)
        pdims = (sub.shape[3], sub.shape[2], sub.shape[1])
        tp = np.full(sub.shape[1:], tau_in[k]) if lagged else None
        for fm in formulas:
            G = O.Grid(params(kinds, fm), *pdims)
            f1, S1, t1, _, _, tn1 = G.node(sub, c[0], c[1], c[2], force=F, tau=tp, with_next=True)
            So[fm][:, k], to[fm][k] = S1, t1
            if fm == formula:
                fo[:, k], tn_o[k] = f1, tn1
    for fm in formulas:
        assert relerr(reads[fm][0], So[fm]) <= t["S"], (fm, relerr(reads[fm][0], So[fm]))
        assert relerr(reads[fm][1], to[fm]) <= t["S"], (fm, relerr(reads[fm][1], to[fm]))
    bound = t.get("eps", 0.0) * np.abs(fo) + t["f"] * np.abs(fo).max() + t.get("abs", 0.0)
    assert np.all(np.abs(fout - fo) <= bound), relerr(fout, fo)
    if lagged:
        assert relerr(tau_next, tn_o) <= t["S"]
    return So[formula]


@pytest.mark.parametrize("lattice,precision,formula,closure", [
    (19, "fp32", "yu", "smag"), (19, "fp32", "chai", "smag"), (19, "fp16s", "yu", "smag"),
    (19, "bf16s", "chai", "smag"), (19, "fp64", "yu", "smag"), (15, "fp32", "yu", "smag"), (15, "fp32", "chai", "smag"),
    (19, "fp32", "yu", "smag_lagged"), (19, "fp32", "chai", "smag_dev")])
def test_channel_256x128x128_sampled(lattice, precision, formula, closure):
    """The headline channel (walls at y, g_x = 1e-6, Smagorinsky or a variant) after 10 steps."""
    lat = bench.make_lattice(precision, formula, lattice=lattice, closure=closure)
    lat.step(10)
    nodes = sample_nodes((lat.nx, lat.ny, lat.nz), 120, seed=lattice + len(precision), d=3)
    nodes += [(x, y, 64) for x in (3, 200) for y in (0, 1, 126, 127)]  # wall rows
    rates = bench.RATES if lattice == 19 else bench.RATES15
    S = check_sampled(lat, rates, precision, closure, formula, bench.BC, sorted(set(nodes)), force=[bench.G, 0, 0],
                      smag_cs=bench.CS)
    assert np.abs(S).max() > 1e-4  # the sample carries a real strain rate
    lat.close()


@pytest.mark.parametrize("precision,formula", [("fp32", "yu"), ("fp32", "chai"), ("fp16s", "yu")])
def test_channel_256x128x128_whole_array(precision, formula):
    """The headline channel compared with the oracle at every one of its 4.2M nodes, through the
    headline's own launch.  After 20 steps (the automatic schedule: one multi-step launch), the
    read-outs of that state by both formulas (eqs. (LuoS), (ChaiS)) and tau are compared whole;
    then two more steps run as one multi-step launch and the populations after them are compared
    whole with two oracle steps from the same state.  The oracle runs over z-slabs in one spawned
    process per host core (oracle/slabs.py, bit-identical to the whole-grid oracle).  Bars: S and
    tau 1e-5 (normwise); populations after two steps 2 x the one-step FP32 bound (2e-6 max|f|) per
    element, and for 16-bit storage 2 x one unit roundoff of the format of max|f| on top (two
    roundings, each carried by one step)."""
    from oracle import slabs

    t = TOL[precision]
    lat = bench.make_lattice(precision, formula)
    lat.step(20)
    steps0, launches0 = lat.stats()
    f20 = lat.get_state().to(torch.float64).cpu().numpy()
    reads = {fm: [x.to(torch.float64).cpu().numpy() for x in lat.strain_rate(fm, with_tau=True)]
             for fm in ("yu", "chai")}
    lat.step(2)
    steps1, launches1 = lat.stats()
    assert (steps1 - steps0, launches1 - launches0) == (2, 1)  # one multi-step launch
    f22 = lat.get_state().to(torch.float64).cpu().numpy()
    lat.close()
    kw = dict(q=19, rates=bench.RATES, closure=O.SMAG, smag_cs=bench.CS, formula=O.YU if formula == "yu" else O.CHAI,
              bc=[BCN[b] for b in bench.BC], pl_tol=1e-7)
    fo, ro = slabs.run(kw, f20, steps=2, force=np.array([bench.G, 0.0, 0.0]), readouts=("yu", "chai"))
    for fm in ("yu", "chai"):
        S, tau = reads[fm]
        assert relerr(S, ro[fm][0]) <= t["S"], (fm, relerr(S, ro[fm][0]))
        assert relerr(tau, ro[fm][1]) <= t["S"], (fm, relerr(tau, ro[fm][1]))
    assert np.abs(reads["yu"][0]).max() > 1e-4  # the state carries a real strain rate
    fmax = np.abs(fo).max()
    bound = 2 * t["f"] * fmax + 2 * t.get("eps", 0.0) * fmax
    err = np.abs(f22 - fo)
    assert np.all(err <= bound), (err.max() / fmax, bound / fmax)


@pytest.mark.parametrize("precision,formula", [("fp32", "yu"), ("fp16s", "chai"), ("bf16s", "yu")])
def test_box_512_sampled(precision, formula):
    """The reduced-precision workload: 512^3 periodic Smagorinsky box, random Fourier start."""
    lat = bench.box_lattice(512, precision, formula, 8, 0.03, 4)
    lat.step(3)
    nodes = sample_nodes((512, 512, 512), 100, seed=len(precision), d=3)
    check_sampled(lat, bench.RATES, precision, "smag", formula, ["periodic"] * 6, nodes, smag_cs=bench.CS)
    lat.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("nidx,formula", [(0.5, "chai"), (1.5, "chai"), (1.0, "yu")])
def test_cavity_4096_sampled(nidx, formula):
    """The D2Q9 power-law lid-driven cavity, 4096^2, after 300 steps (the lid layer moves)."""
    lat = bench.cavity_lattice(4096, nidx, formula)
    lat.step(300)
    nodes = sample_nodes((4096, 4096, 1), 100, seed=int(10 * nidx), d=2)
    nodes += [(x, y, 0) for x in (0, 1, 7, 2048, 4094, 4095) for y in (4093, 4094, 4095)]  # lid layer
    U = bench.CAVITY_U
    K = U ** (2 - nidx) * 4096 ** nidx / bench.CAVITY_RE
    tau_ref = 0.5 + 3 * U * 4096 / bench.CAVITY_RE
    rates = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 1 / tau_ref, 1 / tau_ref]
    S = check_sampled(lat, rates, "fp32", "powerlaw", formula, ["wall", "wall", "wall", "lid", "periodic", "periodic"],
                      sorted(set(nodes)), lid={3: (U, 0.0, 0.0)}, pl=(nidx, K))
    assert np.abs(S).max() > 1e-4  # the lid layer shears
    lat.close()


@pytest.mark.parametrize("nidx,formula", [(0.5, "chai"), (1.5, "yu")])
def test_cavity_4096_whole_array(nidx, formula):
    """The D2Q9 power-law lid-driven cavity at its full 4096^2 size, every node: after 300 steps
    (one launch per step, as the bench runs it), the read-outs of that state by both formulas
    (Chai's and the Yu-type formula of the Sec. 5.4 procedure) and tau, and the populations after
    one more step, against the oracle run over y-slabs in one spawned process per host core (the
    cavity's walls and lid kept where a slab reaches them).  Same bars as the channel's
    whole-array test."""
    from oracle import slabs

    t = TOL["fp32"]
    lat = bench.cavity_lattice(4096, nidx, formula)
    lat.step(300)
    f300 = lat.get_state().to(torch.float64).cpu().numpy()
    reads = {fm: [x.to(torch.float64).cpu().numpy() for x in lat.strain_rate(fm, with_tau=True)]
             for fm in ("yu", "chai")}
    lat.step(1)
    f301 = lat.get_state().to(torch.float64).cpu().numpy()
    lat.close()
    U = bench.CAVITY_U
    K = U ** (2 - nidx) * 4096 ** nidx / bench.CAVITY_RE
    tau_ref = 0.5 + 3 * U * 4096 / bench.CAVITY_RE
    lid = [[0.0, 0.0, 0.0] for _ in range(6)]
    lid[3] = [U, 0.0, 0.0]
    kw = dict(q=9, rates=[0, 1.19, 1.4, 0, 1.2, 0, 1.2, 1 / tau_ref, 1 / tau_ref], closure=O.POWERLAW,
              formula=O.YU if formula == "yu" else O.CHAI, bc=[O.WALL, O.WALL, O.WALL, O.LID, O.PERIODIC, O.PERIODIC],
              lid_u=lid, pl_n=nidx, pl_k=K, pl_tol=1e-7)
    fo, ro = slabs.run(kw, f300, steps=1, readouts=("yu", "chai"), axis="y")
    for fm in ("yu", "chai"):
        S, tau = reads[fm]
        assert relerr(S, ro[fm][0]) <= t["S"], (fm, relerr(S, ro[fm][0]))
        assert relerr(tau, ro[fm][1]) <= t["S"], (fm, relerr(tau, ro[fm][1]))
    assert np.abs(reads["chai"][0]).max() > 1e-4  # the lid layer shears
    err = np.abs(f301 - fo)
    bound = t["f"] * np.abs(fo).max()
    assert np.all(err <= bound), (err.max() / np.abs(fo).max())


def test_tgv_32_fp64_whole_trajectory():
    """The 32^3 FP64 Taylor-Green workload: 500 steps run independently on the GPU and in the
    oracle agree to 1e-12 (populations) and so do both formulas' S at the end; the two formulas
    agree with each other to 1e-13, and the S amplitude follows the linear (Stokes) decay
    exp(-3 nu k^2 t) within 5% (the 3D vortex is not an exact solution; Re is about 3)."""
    lat = bench.tgv_lattice("yu")
    S0 = float(lat.strain_rate("yu").abs().max())
    lat.step(bench.TGV_STEPS)
    n = bench.TGV_N
    drho, u, g = I.taylor_green_3d(n, u0=bench.TGV_U0)
    G = O.Grid(O.make_params(19, bench.tgv_rates()), n, n, n)
    fo = G.run(G.init(drho, u, g), bench.TGV_STEPS)
    fg = lat.get_state().cpu().numpy()
    assert relerr(fg, fo) <= 1e-12
    for fm, code in (("yu", O.YU), ("chai", O.CHAI)):
        G.p.formula = code
        assert relerr(lat.strain_rate(fm).cpu().numpy(), G.readout(fo)["S"]) <= 1e-12
    Sy, Sc = lat.strain_rate("yu").cpu().numpy(), lat.strain_rate("chai").cpu().numpy()
    assert relerr(Sy, Sc) <= 1e-13
    nu, k = (bench.TGV_TAU - 0.5) / 3, 2 * np.pi / n
    ratio = np.abs(Sy).max() / S0 / np.exp(-3 * nu * k * k * bench.TGV_STEPS)
    assert abs(ratio - 1) <= 0.05, ratio
    lat.close()


def test_adjoint_128_directional_derivative():
    """dL/dg . v of the FP32 adjoint at the bench's 128^3, T = 256, 16-step checkpoints, against
    (L(g + h v) - L(g - h v)) / 2h from the FP64 path, for a seeded random direction v."""
    n = bench.ADJ_N
    g = torch.from_numpy(I.gaussian_force(3, (n, n, n), std=1e-5, seed=5))
    v = torch.from_numpy(I.gaussian_force(3, (n, n, n), std=1e-5, seed=17))
    lat = bench.adjoint_lattice("fp32", g)
    L32, grad = lat.adjoint(bench.ADJ_T, bench.ADJ_SEG)
    dirder = float((grad * v.cuda()).sum())
    lat.close()
    lat64 = bench.adjoint_lattice("fp64", g)
    f0 = lat64.get_state().clone()
    h = 1e-2
    losses = []
    for sgn in (1.0, -1.0):
        lat64.force_field.copy_((g + sgn * h * v).cuda())
        lat64.set_state(f0)
        losses.append(lat64.adjoint(bench.ADJ_T, bench.ADJ_SEG)[0])
    fd = (losses[0] - losses[1]) / (2 * h)
    lat64.force_field.copy_(g.cuda())
    lat64.set_state(f0)
    L64, grad64 = lat64.adjoint(bench.ADJ_T, bench.ADJ_SEG)
    dir64 = float((grad64 * v.cuda()).sum())
    lat64.close()
    assert abs(L32 - L64) <= 1e-5 * abs(L64)
    assert abs(dir64 - fd) <= 1e-5 * abs(fd), (dir64, fd)
    assert abs(dirder - fd) <= 1e-4 * abs(fd), (dirder, fd)
