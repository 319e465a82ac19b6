"""Several steps per launch (the streamed schedule) against one launch per step and the oracle.

A streamed launch runs each node's step with the arithmetic of the one-step kernel, scheduled
unit by unit (one z plane by a band of y rows), so after any number of steps its state must equal
the per-step state bit for bit; a wrong dependency (a unit that ran before a neighbour finished
the previous step, or overwrote a buffer a neighbour was still reading) shows up as a difference.
The FP32 cases are also compared with the FP64 oracle over the same steps.  Sizes are chosen so
that the units have ragged last bands, planes wrap and walls/lids sit on band edges."""
import numpy as np
import pytest
import torch

from paper_1704_07559_gb300 import lbm
from test_gpu_parity import Case, f64, relerr

pytestmark = pytest.mark.gpu

WALL_Y = ["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2
LID_Y = ["periodic"] * 2 + ["wall", "lid"] + ["periodic"] * 2

STREAM_CASES = [
    # lattice, dims (nx, ny, nz), precision, closure, formula, extra
    (19, (300, 20, 6), "fp32", "smag", "yu", dict(force=[1e-5, -2e-5, 3e-6])),
    (19, (300, 20, 6), "fp32", "smag", "chai", dict(bc=WALL_Y, force=[2e-5, 0, 0])),
    (19, (301, 9, 5), "fp32", "newton", "yu", dict(bc=["wall"] * 6)),
    (19, (256, 13, 4), "fp32", "powerlaw", "chai", dict(pl=(0.7, 0.01), bc=LID_Y, lid={3: (0.05, 0, 0.01)})),
    (19, (200, 11, 7), "fp32", "smag_dev", "yu", dict(force_field=True)),
    (19, (300, 20, 6), "fp16s", "smag", "yu", dict(bc=WALL_Y, force=[1e-5, 0, 0])),
    (19, (301, 20, 6), "fp16s", "smag", "chai", {}),
    (19, (300, 17, 5), "bf16s", "newton", "chai", dict(bc=LID_Y, lid={3: (0.05, 0, 0)})),
    (15, (300, 20, 6), "fp32", "smag", "yu", dict(force=[1e-5, 0, 2e-6])),
    (15, (300, 20, 6), "fp16s", "smag", "chai", dict(bc=WALL_Y)),
    (15, (302, 14, 3), "bf16s", "smag", "yu", {}),
    (9, (513, 40, 1), "fp32", "powerlaw", "yu", dict(pl=(0.5, 0.02), bc=["wall"] * 3 + ["lid"], lid={3: (0.1, 0, 0)})),
    (9, (1030, 12, 1), "fp32", "smag", "chai", dict(force=[1e-5, 2e-6])),
]


def make(q, dims, precision, closure, formula, extra):
    return Case(q, dims, precision=precision, closure=closure, formula=formula,
                tau=0.55 if closure != "powerlaw" else 0.6, **extra)


@pytest.mark.parametrize("nsteps", [7, 8])
@pytest.mark.parametrize("q,dims,precision,closure,formula,extra", STREAM_CASES)
def test_streamed_steps_equal_per_step(q, dims, precision, closure, formula, extra, nsteps):
    c = make(q, dims, precision, closure, formula, extra)
    c.lat.init(c.drho, c.u, c.g)
    f0 = c.lat.get_state().clone()
    c.lat.set_schedule("per_step").step(nsteps)
    ref = c.lat.get_state().clone()
    c.lat.set_state(f0)
    c.lat.set_schedule("stream").step(nsteps).status()
    got = c.lat.get_state()
    assert torch.equal(got.view(torch.int16 if got.element_size() == 2 else torch.int32),
                       ref.view(torch.int16 if ref.element_size() == 2 else torch.int32)), \
        (f64(got) != f64(ref)).sum()
    # the read-outs after an odd or even number of streamed steps see the same current buffer
    S1 = c.lat.strain_rate(formula)
    c.lat.set_state(ref)
    assert torch.equal(S1, c.lat.strain_rate(formula))


@pytest.mark.parametrize("q,dims,precision,closure,formula,extra",
                         [cs for cs in STREAM_CASES if cs[2] == "fp32"])
def test_streamed_steps_match_the_oracle(q, dims, precision, closure, formula, extra):
    """Five streamed steps against five oracle steps from the same (exactly converted) state:
    populations within 1e-5 of max|f| (five times the one-step FP32 bound)."""
    c = make(q, dims, precision, closure, formula, extra)
    c.lat.init(c.drho, c.u, c.g)
    fo = f64(c.lat.get_state())
    for _ in range(5):
        fo, _ = c.G.step(fo, force=c.oforce)
    c.lat.set_schedule("stream").step(5).status()
    fg = f64(c.lat.get_state())
    assert relerr(fg, fo) <= 1e-5, relerr(fg, fo)


def test_auto_schedule_on_the_channel_equals_per_step():
    """The channel the benchmark times (256x128x128, walls at y, force, Smagorinsky): the automatic
    schedule takes the streamed launch there; 20 steps equal 20 one-step launches bit for bit, for
    FP32 and FP16 storage (two nodes per thread)."""
    import bench
    for precision in ("fp32", "fp16s"):
        lat = bench.make_lattice(precision, "yu")
        f0 = lat.get_state().clone()
        lat.set_schedule("per_step").step(20)
        ref = lat.get_state().clone()
        lat.set_state(f0)
        steps0, launches0 = lat.stats()
        lat.set_schedule("auto").step(20).status()
        steps1, launches1 = lat.stats()
        assert (steps1 - steps0, launches1 - launches0) == (20, 1), precision
        got = lat.get_state()
        w = torch.int16 if got.element_size() == 2 else torch.int32
        assert torch.equal(got.view(w), ref.view(w)), precision
        lat.close()


def test_fp64_keeps_one_launch_per_step():
    """FP64 (arithmetic-bound) steps one launch per step even under a forced streamed schedule."""
    c = make(19, (300, 20, 6), "fp64", "smag", "yu", {})
    c.lat.init(c.drho, c.u, c.g)
    f0 = c.lat.get_state().clone()
    c.lat.set_schedule("per_step").step(4)
    ref = c.lat.get_state().clone()
    c.lat.set_state(f0)
    steps0, launches0 = c.lat.stats()
    c.lat.set_schedule("stream").step(4).status()
    steps1, launches1 = c.lat.stats()
    assert (steps1 - steps0, launches1 - launches0) == (4, 4)
    assert torch.equal(c.lat.get_state(), ref)


@pytest.mark.parametrize("formula", ["yu", "chai"])
def test_lagged_closure_streamed_equals_per_step(formula):
    """The lagged closure's stored tau is read and rewritten by the node's own unit, one step after
    another (possibly on different SMs): populations and the tau field after 7 streamed steps equal
    7 one-step launches bit for bit."""
    c = make(19, (300, 20, 6), "fp32", "smag_lagged", formula, dict(bc=WALL_Y, force=[1e-5, 0, 0]))
    c.lat.init(c.drho, c.u, c.g)
    f0, t0 = c.lat.get_state().clone(), c.lat.tau.clone()
    c.lat.set_schedule("per_step").step(7)
    ref, tref = c.lat.get_state().clone(), c.lat.tau.clone()
    c.lat.set_state(f0)
    c.lat.tau.copy_(t0)
    c.lat.set_schedule("stream").step(7).status()
    assert torch.equal(c.lat.get_state().view(torch.int32), ref.view(torch.int32))
    assert torch.equal(c.lat.tau.view(torch.int32), tref.view(torch.int32))


def test_a_dependency_wait_that_runs_out_is_reported():
    """The one-shot stall check starts a streamed launch one step ahead: no unit can ever see its
    neighbours finish the step before, every wait runs out (bounded at about two seconds), the
    launch ends, lbm_status reports LBM_ERR_STATE once, and the context works afterwards."""
    c = make(19, (300, 20, 6), "fp32", "smag", "yu", {})
    c.lat.init(c.drho, c.u, c.g)
    c.lat.set_schedule("stall_check").step(3)
    with pytest.raises(lbm.LBMError) as e:
        c.lat.status()
    assert e.value.code == -5 and "ran out" in str(e.value)
    c.lat.status()  # reported once
    c.lat.init(c.drho, c.u, c.g)
    f0 = c.lat.get_state().clone()
    c.lat.set_schedule("per_step").step(3)
    ref = c.lat.get_state().clone()
    c.lat.set_state(f0)
    c.lat.set_schedule("stream").step(3)
    assert np.all(np.isfinite(c.lat.sums()))
    assert torch.equal(c.lat.get_state(), ref)


@pytest.mark.parametrize("seg", [1, 4, 5])
def test_adjoint_under_the_streamed_schedule_equals_per_step(seg):
    """lbm_adjoint's forward sweep runs the middle steps of each checkpoint segment through the
    multi-step launch when the schedule allows; the functional, the gradient and the final state
    equal those of one launch per step bit for bit (the adjoint has no atomics, so it is
    deterministic)."""
    from paper_1704_07559_gb300 import inputs as I
    from test_gpu_parity import rates

    nx, ny, nz = 300, 20, 6
    drho, u = I.random_fourier(nx, ny, nz, kmax=2, rms=0.02, seed=6)
    g = I.gaussian_force(3, (nz, ny, nx), std=1e-5, seed=5)
    lat = lbm.Lattice(19, nx, ny, nz, rates=rates(19, 0.55), precision="fp32", closure="smag", smag_cs=0.17,
                      formula="yu", force_field=torch.from_numpy(g))
    lat.init(drho, u)
    f0 = lat.get_state().clone()
    out = {}
    for sched in ("per_step", "stream"):
        lat.set_state(f0)
        L, grad = lat.set_schedule(sched).adjoint(13, seg)
        lat.status()
        out[sched] = (L, grad.clone(), lat.get_state().clone())
    assert out["per_step"][0] == out["stream"][0]
    assert torch.equal(out["per_step"][1], out["stream"][1])
    assert torch.equal(out["per_step"][2].view(torch.int32), out["stream"][2].view(torch.int32))


def test_long_runs_are_split_into_launches_of_at_most_4096_steps():
    """lbm_step(5000) under the streamed schedule makes two multi-step launches (4096 + 904) and
    equals 5000 one-step launches bit for bit."""
    c = make(19, (300, 20, 6), "fp32", "smag", "yu", dict(force=[1e-6, 0, 0]))
    c.lat.init(c.drho, c.u, c.g)
    f0 = c.lat.get_state().clone()
    ref = c.lat.set_schedule("per_step").step(5000).get_state().clone()
    c.lat.set_state(f0)
    steps0, launches0 = c.lat.stats()
    got = c.lat.set_schedule("stream").step(5000).status().get_state()
    steps1, launches1 = c.lat.stats()
    assert (steps1 - steps0, launches1 - launches0) == (5000, 2)
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32))


def test_two_multi_step_launches_running_concurrently():
    """Two contexts on two streams, each running 200 steps as one multi-step launch at the same
    time (their blocks share the SMs; neither launch is cooperative): both end bit-identical to
    one launch per step, with no wait running out."""
    from paper_1704_07559_gb300 import inputs as I
    from test_gpu_parity import rates

    dims = [(256, 64, 64), (192, 48, 80)]
    lats, refs = [], []
    for k, (nx, ny, nz) in enumerate(dims):
        st = torch.cuda.Stream()
        lat = lbm.Lattice(19, nx, ny, nz, rates=rates(19, 0.55), precision="fp32", closure="smag", smag_cs=0.17,
                          formula="yu" if k == 0 else "chai", force=[1e-6, 0, 0], stream=st)
        drho, u = I.random_fourier(nx, ny, nz, kmax=3, rms=0.02, seed=10 + k)
        lat.init(drho, u)
        g = lat.get_state()  # copied on the lattice's stream
        torch.cuda.synchronize()
        f0 = g.clone()
        lat.set_schedule("per_step").step(200)
        g = lat.get_state()
        torch.cuda.synchronize()
        refs.append(g.clone())
        lat.set_state(f0)
        torch.cuda.synchronize()
        lats.append(lat)
    for lat in lats:  # both launches queued before either is waited for
        lat.set_schedule("stream").step(200)
    for lat, ref in zip(lats, refs):
        lat.status()
        got = lat.get_state()
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
