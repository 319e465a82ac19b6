"""The allocation-free sums entry point (lbm_sums_noalloc) against the regular lbm_sums.

lbm_sums_noalloc serves callers that cannot allocate device memory when they need the global
mass and momentum sums (their memory belongs to another allocator, or they run a time-stepping
loop where cudaMalloc may synchronise the device).  It keeps its scratch in a static device
array instead of the context's cudaMalloc'ed buffer.  This file is collected last so that a run
stopping at the first failure has already run every other test; it passes both alone in a fresh
process and after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_1704_07559_gb300 import build, lbm

RATES19 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / 0.51, 1.4, 1 / 0.51, 1.4, 1 / 0.51, 1 / 0.51, 1 / 0.51, 1.98,
           1.98, 1.98]
RATES9 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 1 / 0.7, 1 / 0.7]
RATES15 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2] + [1 / 0.51] * 5 + [1.98]


def entry():
    build.build()
    L = lbm.lib()
    fn = L.lbm_sums_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(lbm.Params),
                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def call(fn, lat, buf, force=None):
    out = (ctypes.c_double * (1 + lat.d))()
    fv = None if force is None else (ctypes.c_double * 3)(*(list(force) + [0.0] * (3 - len(force))))
    ff = None if lat.force_field is None else ctypes.c_void_p(lat.force_field.data_ptr())
    rc = fn(lat.q, lat.nx, lat.ny, lat.nz, ctypes.byref(lat.params), fv, ctypes.c_void_p(buf.data_ptr()), lat.stride,
            ff, out, ctypes.c_void_p(lat.stream.cuda_stream))
    return rc, np.array(out[:])


def test_rejects_too_many_rows_without_touching_the_gpu():
    """More than LBM_NOALLOC_MAX_ROWS rows (ny * nz) exceed the static scratch: LBM_ERR_ARG."""
    fn = entry()
    p = lbm.default_params()
    out = (ctypes.c_double * 4)()
    rc = fn(19, 4, 1024, 257, ctypes.byref(p), None, ctypes.c_void_p(16), 4 * 1024 * 257, None, out, None)
    assert rc == -1
    rc = fn(19, 4, 4, 4, None, None, ctypes.c_void_p(16), 64, None, out, None)
    assert rc == -1


CASES = [
    dict(q=19, dims=(70, 12, 9), precision="fp32", bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
         force=[1e-5, 0.0, 2e-6], tol=1e-6),
    dict(q=19, dims=(40, 10, 8), precision="fp64", bc=None, force=None, tol=1e-13),
    dict(q=9, dims=(90, 33, 1), precision="fp32", bc=["wall"] * 3 + ["lid"], lid={3: (0.05, 0.0, 0.0)}, force=None,
         tol=1e-6),
    dict(q=15, dims=(50, 12, 7), precision="fp32", bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
         force=[1e-5, 0.0, 2e-6], tol=1e-6),
    dict(q=15, dims=(40, 10, 6), precision="bf16s", bc=None, force=[2e-6, 0.0, 0.0], tol=1e-6),
    dict(q=19, dims=(48, 10, 7), precision="fp16s", bc=["periodic"] * 2 + ["wall"] * 2 + ["periodic"] * 2,
         force=[1e-5, 0.0, 0.0], tol=1e-6),
    dict(q=19, dims=(33, 9, 6), precision="fp32", bc=None, force=None, force_field=True, tol=1e-6),
]


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=["d3q19-fp32-channel", "d3q19-fp64-periodic", "d2q9-fp32-lid",
                                           "d3q15-fp32-channel", "d3q15-bf16-periodic", "d3q19-fp16-channel",
                                           "d3q19-fp32-force-field"])
def test_matches_lbm_sums_on_two_calls_in_a_row(case):
    """Two calls in a row (before and after a step, so the scratch holds the first call's
    contents when the second runs) agree with lbm_sums within the sums tolerance of the parity
    tests (1e-13 x N max|f| in FP64, 1e-6 x N max|f| otherwise)."""
    import torch

    fn = entry()
    q = case["q"]
    rng = np.random.default_rng(11)
    ff = None
    if case.get("force_field"):
        d = 2 if q == 9 else 3
        ff = torch.tensor(rng.normal(scale=1e-5, size=(d,) + tuple(reversed(case["dims"]))), dtype=torch.float32)
    lat = lbm.Lattice(q, *case["dims"], rates={19: RATES19, 15: RATES15, 9: RATES9}[q], precision=case["precision"],
                      closure="smag", smag_cs=0.17, bc=case["bc"], lid_u=case.get("lid"), force=case["force"],
                      force_field=ff)
    d = lat.d
    lat.init(rng.normal(scale=1e-3, size=lat.shape), rng.normal(scale=0.02, size=(d,) + lat.shape),
             rng.normal(scale=2e-3, size=(d * d,) + lat.shape))
    bufs = [lat.f_a, lat.f_b]
    for call_no in range(2):
        cur = bufs[call_no % 2]  # A after init, B after one step
        ref = lat.sums()
        rc, got = call(fn, lat, cur, case["force"])
        assert rc == 0
        fmax = float(cur[:, :lat.N].abs().max().to(torch.float64))
        assert np.abs(got - ref).max() <= case["tol"] * lat.N * fmax, (call_no, got, ref)
        lat.step(1)


@pytest.mark.gpu
def test_allocates_nothing():
    """The property the entry point exists for: after one warm-up call (which loads the module
    and with it the static array), repeated calls leave the device's free memory unchanged; and
    torch's caching allocator sees no allocation either."""
    import torch

    fn = entry()
    lat = lbm.Lattice(19, 64, 24, 16, rates=RATES19, precision="fp32", closure="smag", smag_cs=0.17,
                      force=[1e-5, 0.0, 0.0])
    rng = np.random.default_rng(5)
    lat.init(rng.normal(scale=1e-3, size=lat.shape), rng.normal(scale=0.02, size=(3,) + lat.shape))
    rc, first = call(fn, lat, lat.f_a, [1e-5, 0.0, 0.0])
    assert rc == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(20):
        rc, got = call(fn, lat, lat.f_a, [1e-5, 0.0, 0.0])
        assert rc == 0
        assert np.array_equal(got, first)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
