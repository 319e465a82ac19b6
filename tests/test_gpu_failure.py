"""Failure detection on the GPU, with every fault made on the host: a NaN written into a state that
is uploaded (lbm_set_state) or written into the bound buffer between steps, and conserved totals
knocked off balance by editing the bound buffer between steps.  Nothing here faults the GPU: the
library's sums kernels read the corrupted values like any others and the host reads the result.

- lbm_sums and lbm_sums_noalloc return LBM_ERR_NONFINITE with the sums filled in;
- the watchdog (lbm_set_watchdog) stays quiet on healthy runs, including the exact momentum
  growth N F per step under a uniform force on a periodic lattice (the balance of the collision,
  eq. (mrteqvT) with s_0 = s_3 = s_5 = s_7 = 0), and reports LBM_ERR_DRIFT / LBM_ERR_NONFINITE at
  the first check after the fault, with the state and the step count of that check.
"""
import ctypes

import numpy as np
import pytest

from paper_1704_07559_gb300 import lbm

pytestmark = pytest.mark.gpu

TAU0 = 0.6
RATES19 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / TAU0, 1.4, 1 / TAU0, 1.4, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1.98,
           1.98, 1.98]
CHANNEL = ["periodic", "periodic", "wall", "wall", "periodic", "periodic"]


def lattice(precision="fp32", bc=None, force=None, dims=(40, 12, 9), closure="smag", formula="yu", seed=3):
    lat = lbm.Lattice(lbm.D3Q19, *dims, rates=RATES19, precision=precision, closure=closure, smag_cs=0.17,
                      formula=formula, bc=bc, force=force)
    rng = np.random.default_rng(seed)
    lat.init(rng.normal(scale=1e-3, size=lat.shape), rng.normal(scale=0.02, size=(3,) + lat.shape),
             rng.normal(scale=2e-3, size=(9,) + lat.shape))
    return lat


def raw_sums(lat):
    out = (ctypes.c_double * 4)()
    rc = lbm.lib().lbm_sums(lat.ctx, out)
    return rc, np.array(out[:])


def noalloc_sums(lat, buf, force=None):
    fn = lbm.lib().lbm_sums_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(lbm.Params),
                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    out = (ctypes.c_double * 4)()
    fv = None if force is None else (ctypes.c_double * 3)(*force)
    rc = fn(lat.q, lat.nx, lat.ny, lat.nz, ctypes.byref(lat.params), fv, ctypes.c_void_p(buf.data_ptr()), lat.stride,
            None, out, ctypes.c_void_p(lat.stream.cuda_stream))
    return rc, np.array(out[:])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_nan_in_an_uploaded_state_is_reported_by_the_sums(precision):
    """A NaN in the rest population of one node, uploaded from host memory: the mass sum is NaN,
    lbm_sums and lbm_sums_noalloc return LBM_ERR_NONFINITE and still fill every sum (the momentum
    sums, which the rest population does not enter, stay finite and equal)."""
    lat = lattice(precision, bc=CHANNEL, force=[1e-5, 0.0, 0.0])
    lat.step(3)
    f = lat.get_state().cpu()
    f[0, 4, 5, 6] = float("nan")
    lat.set_state(f)
    rc, s = raw_sums(lat)
    assert rc == -4
    assert np.isnan(s[0]) and np.all(np.isfinite(s[1:]))
    with pytest.raises(lbm.LBMError) as ei:
        lat.sums()
    assert ei.value.code == -4
    cur = lat.f_b if lat.stats()[0] % 2 else lat.f_a  # the buffer the last step wrote
    rc2, s2 = noalloc_sums(lat, cur, force=[1e-5, 0.0, 0.0])
    assert rc2 == -4
    assert np.isnan(s2[0]) and np.all(np.isfinite(s2[1:]))
    assert np.abs(s2[1:] - s[1:]).max() <= 1e-6 * lat.N * 0.1


@pytest.mark.parametrize("precision,bc,force,tol", [
    ("fp64", None, [1e-5, -3e-6, 2e-6], 1e-12),   # periodic: mass and momentum balance checked
    ("fp32", None, [1e-5, 0.0, 0.0], 1e-6),
    ("fp32", CHANNEL, [1e-5, 0.0, 0.0], 1e-6),    # walls: mass only
    ("fp16s", CHANNEL, [1e-5, 0.0, 0.0], 1e-5),   # 16-bit rounding: a random walk of ~1e-3 in 60 steps
])
def test_watchdog_is_quiet_on_a_healthy_run(precision, bc, force, tol):
    """60 steps checked every 7 (the last chunk ragged): no report, every step counted, and the
    state equals the same 60 steps run without the watchdog (it does not change the results)."""
    a = lattice(precision, bc=bc, force=force)
    b = lattice(precision, bc=bc, force=force)
    a.set_watchdog(7, tol).step(60)
    b.step(60)
    assert a.stats()[0] == 60
    assert bool((a.get_state() == b.get_state()).all())
    # the drift actually seen is far inside the bound
    s0 = lattice(precision, bc=bc, force=force).sums()
    s1 = a.sums()
    assert abs(s1[0] - s0[0]) <= tol * a.N


def test_watchdog_reports_an_injected_mass_drift():
    """Between two lbm_step calls 1e-6 of mass is added to one node of the bound buffer (not
    through lbm_set_state, which would reset the reference): the next check, 4 steps later,
    reports LBM_ERR_DRIFT naming the mass; the steps of that chunk are counted."""
    lat = lattice("fp64", force=[1e-5, 0.0, 0.0])
    lat.set_watchdog(4, 1e-12)
    lat.step(8)  # two checks, both quiet; 8 steps: the current buffer is A again
    with torch_no_grad():
        lat.f_a[0, 100] += 1e-6
    with pytest.raises(lbm.LBMError) as ei:
        lat.step(12)
    assert ei.value.code == -6
    assert "mass" in str(ei.value)
    assert lat.stats()[0] == 12
    # re-arming takes the new state as the reference
    lat.set_watchdog(4, 1e-12).step(8)


def test_watchdog_reports_an_injected_momentum_drift():
    """A momentum kick that conserves mass (+d on f_1 and -d on f_2, c_x = +1 and -1, at one node)
    on an all-periodic lattice: LBM_ERR_DRIFT naming momentum component 0.  With walls the
    momentum is not checked (the walls exchange momentum with the fluid) and the same kick passes."""
    for bc, reported in ((None, True), (CHANNEL, False)):
        lat = lattice("fp64", bc=bc, force=[1e-5, 0.0, 0.0])
        lat.set_watchdog(5, 1e-12)
        lat.step(10)
        with torch_no_grad():
            lat.f_a[1, 77] += 5e-7
            lat.f_a[2, 77] -= 5e-7
        if reported:
            with pytest.raises(lbm.LBMError) as ei:
                lat.step(10)
            assert ei.value.code == -6
            assert "momentum 0" in str(ei.value)
        else:
            lat.step(10)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16s"])
def test_watchdog_reports_a_nan_written_between_steps(precision):
    """A NaN written into the bound buffer between steps spreads through the next steps; the next
    check returns LBM_ERR_NONFINITE and stepping stops there (3 of the 9 requested steps)."""
    lat = lattice(precision, bc=CHANNEL, force=[1e-5, 0.0, 0.0])
    lat.set_watchdog(3, 1e-6)
    lat.step(6)
    with torch_no_grad():
        lat.f_a[5, 321] = float("nan")
    with pytest.raises(lbm.LBMError) as ei:
        lat.step(9)
    assert ei.value.code == -4
    assert lat.stats()[0] == 9


def test_watchdog_arguments():
    lat = lattice("fp32")
    for every, tol in ((-1, 1e-6), (3, -1.0), (3, float("nan")), (3, float("inf"))):
        with pytest.raises(lbm.LBMError) as ei:
            lat.set_watchdog(every, tol)
        assert ei.value.code == -1
    lat.set_watchdog(0, float("nan"))  # off: tol is not read
    lat.step(2)


def torch_no_grad():
    import torch

    return torch.no_grad()
