"""The C-ABI library builds, loads and exports every call declared in include/lbm.h, and its
host-side argument checks reject bad input without touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1704_07559_gb300 import build, lbm

    build.build()
    return lbm.lib()


def header_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(lbm_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_call(L):
    names = header_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(L, name), name
    from paper_1704_07559_gb300 import lbm

    assert sorted(lbm.API) == names


def test_default_params(L):
    from paper_1704_07559_gb300 import lbm

    p = lbm.default_params()
    assert p.precision == 1 and p.closure == 0 and p.formula == 0
    assert p.smag_iters == 6 and p.rho0 == 1.0 and list(p.bc) == [0] * 6


D3 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1.6, 1.4, 1.6, 1.4, 1.6, 1.6, 1.6, 1.98, 1.98, 1.98]
D15 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1.6, 1.6, 1.6, 1.6, 1.6, 1.98]


def create(L, lattice=19, dims=(8, 8, 8), rates=None, mutate=None):
    from paper_1704_07559_gb300 import lbm

    p = lbm.default_params()
    if mutate:
        mutate(p)
    r = rates if rates is not None else {19: D3, 15: D15}.get(lattice, [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 1.6, 1.6])
    arr = (ctypes.c_double * len(r))(*r)
    ctx = ctypes.c_void_p()
    rc = L.lbm_create(ctypes.byref(ctx), lattice, dims[0], dims[1], dims[2], arr, None, ctypes.byref(p))
    return rc, ctx


@pytest.mark.parametrize("case", [
    dict(lattice=7),
    dict(dims=(0, 8, 8)),
    dict(lattice=9, dims=(8, 8, 2)),
    dict(dims=(8, 70000, 1)),
    dict(dims=(2048, 2048, 1024)),
    dict(rates=D3[:3] + [0.1] + D3[4:]),                       # nonzero conserved rate
    dict(rates=D3[:1] + [2.5] + D3[2:]),                       # rate outside (0, 2)
    dict(rates=D3[:13] + [1.2] + D3[14:]),                     # split viscous rates with Yu
    dict(mutate=lambda p: setattr(p, "precision", 9)),
    dict(mutate=lambda p: setattr(p, "closure", 5)),
    dict(mutate=lambda p: setattr(p, "formula", 2)),
    dict(mutate=lambda p: p.bc.__setitem__(0, 1)),             # -x wall with +x periodic
    dict(mutate=lambda p: setattr(p, "rho0", 0.0)),
    dict(mutate=lambda p: setattr(p, "smag_iters", 0)),
    dict(mutate=lambda p: (setattr(p, "precision", 2), setattr(p, "closure", 2))),
    dict(lattice=9, mutate=lambda p: setattr(p, "precision", 2)),
    dict(mutate=lambda p: (setattr(p, "closure", 2), setattr(p, "pl_tau_min", 0.5))),
    dict(lattice=15, mutate=lambda p: (setattr(p, "precision", 3), setattr(p, "closure", 2))),  # 16-bit power law
    dict(lattice=15, rates=D15[:7] + [0.3] + D15[8:]),                  # D3Q15 conserved j_z rate
    dict(lattice=15, rates=D15[:12] + [1.5] + D15[13:]),                # D3Q15 split viscous rates, Yu
    dict(lattice=15, dims=(8, 8, 0)),
    dict(mutate=lambda p: setattr(p, "closure", 5)),
    dict(mutate=lambda p: (setattr(p, "precision", 2), setattr(p, "closure", 3))),  # 16-bit: lagged
    dict(mutate=lambda p: (setattr(p, "precision", 3), setattr(p, "closure", 4))),  # 16-bit: deviatoric
    dict(rates=D3[:13] + [1.2] + D3[14:], mutate=lambda p: (setattr(p, "formula", 1), setattr(p, "closure", 3))),
    dict(mutate=lambda p: p.bc.__setitem__(4, 3)),                         # one halo z face
    dict(mutate=lambda p: (p.bc.__setitem__(0, 3), p.bc.__setitem__(1, 3))),  # halo faces on x
    dict(mutate=lambda p: (p.bc.__setitem__(4, 3), p.bc.__setitem__(5, 1))),  # halo with a wall
    dict(dims=(8, 8, 65534), mutate=lambda p: (p.bc.__setitem__(4, 3), p.bc.__setitem__(5, 3))),  # nz + 2 planes
])
def test_create_rejects_bad_arguments(L, case):
    rc, ctx = create(L, **case)
    assert rc == -1
    assert ctx.value is None
    assert L.lbm_last_error(None).startswith(b"lbm_create: invalid")


def test_chai_accepts_split_viscous_rates_host_checks(L):
    """Chai's formula uses each viscous rate on its own, so split rates pass the host checks
    (the call then needs a GPU for its scratch; without one it reports a CUDA error)."""
    rc, ctx = create(L, rates=D3[:13] + [1.2] + D3[14:], mutate=lambda p: setattr(p, "formula", 1))
    assert rc in (0, -2, -3)
    if rc == 0:
        L.lbm_destroy(ctx)


def test_d3q15_host_checks_pass(L):
    """A valid D3Q15 context passes every host check (then needs a GPU for its scratch)."""
    rc, ctx = create(L, lattice=15)
    assert rc in (0, -2, -3)
    if rc == 0:
        L.lbm_destroy(ctx)


def test_null_context_calls_fail_cleanly(L):
    assert L.lbm_step(None, 1) == -1
    assert L.lbm_bind_tau(None, None) == -1
    assert L.lbm_destroy(None) == 0
    assert L.lbm_layout(None, None, None, None) == -1
    assert L.lbm_set_schedule(None, 0) == -1
    assert L.lbm_status(None) == -1
    assert L.lbm_stats(None, None, None) == -1
    assert L.lbm_set_watchdog(None, 1, 1e-6) == -1
    assert L.lbm_halo_layout(None, None, None) == -1
    assert L.lbm_halo_pack(None, None, None) == -1
    assert L.lbm_halo_unpack(None, None, None) == -1


def test_halo_faces_pass_the_host_checks(L):
    """Both z faces LBM_HALO on D3Q19 and D3Q15 pass the host checks (then need a GPU for the
    context's scratch); on D2Q9 the z faces are ignored."""
    for lattice in (19, 15):
        rc, ctx = create(L, lattice=lattice, mutate=lambda p: (p.bc.__setitem__(4, 3), p.bc.__setitem__(5, 3)))
        assert rc in (0, -2, -3)
        if rc == 0:
            L.lbm_destroy(ctx)


def test_noalloc_rejects_bad_arguments_before_any_cuda_call(L):
    """lbm_sums_noalloc checks its arguments on the host first (a rejected call touches no CUDA
    state, so these run without a GPU): a non-finite or non-positive rho0, a non-finite force or
    wall velocity, an unpaired boundary, a row count beyond its static scratch."""
    from paper_1704_07559_gb300 import lbm

    fn = L.lbm_sums_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(lbm.Params),
                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    out = (ctypes.c_double * 4)()

    def call(mutate=None, force=None, dims=(4, 4, 4)):
        p = lbm.default_params()
        if mutate:
            mutate(p)
        fv = None if force is None else (ctypes.c_double * 3)(*force)
        n = dims[0] * dims[1] * dims[2]
        return fn(19, dims[0], dims[1], dims[2], ctypes.byref(p), fv, ctypes.c_void_p(256), n, None, out, None)

    inf, nan = float("inf"), float("nan")
    assert call(lambda p: setattr(p, "rho0", inf)) == -1
    assert call(lambda p: setattr(p, "rho0", 0.0)) == -1
    assert call(lambda p: setattr(p, "rho0", nan)) == -1
    assert call(force=(1e-6, nan, 0.0)) == -1
    assert call(force=(inf, 0.0, 0.0)) == -1

    def lid_nan(p):
        p.bc[2], p.bc[3] = 1, 2
        p.lid_u[3][0] = nan
    assert call(lid_nan) == -1

    def unpaired(p):
        p.bc[2] = 1
    assert call(unpaired) == -1
    assert call(dims=(4, 1024, 257)) == -1
    assert call(lambda p: setattr(p, "precision", 7)) == -1


def header_constants(prefix):
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (%s\w+) (-?\d+)" % prefix, text, re.M)}


def test_binding_constants_match_the_header():
    """The binding's name tables carry the header's values (schedules, closures, precisions,
    boundary kinds, formulas, error codes)."""
    from paper_1704_07559_gb300 import lbm

    sched = header_constants("LBM_SCHEDULE_")
    assert {k: sched["LBM_SCHEDULE_" + k.upper()] for k in lbm.SCHEDULE} == lbm.SCHEDULE
    cl = header_constants("LBM_")
    assert lbm.CLOSURE == {"newton": cl["LBM_NEWTON"], "smag": cl["LBM_SMAG"], "powerlaw": cl["LBM_POWERLAW"],
                           "smag_lagged": cl["LBM_SMAG_LAGGED"], "smag_dev": cl["LBM_SMAG_DEV"]}
    assert lbm.PRECISION == {"fp64": cl["LBM_FP64"], "fp32": cl["LBM_FP32"], "fp16s": cl["LBM_FP16S"],
                             "bf16s": cl["LBM_BF16S"]}
    assert lbm.FORMULA == {"yu": cl["LBM_YU"], "chai": cl["LBM_CHAI"]}
    assert lbm.BC == {"periodic": cl["LBM_PERIODIC"], "wall": cl["LBM_WALL"], "lid": cl["LBM_LID"],
                      "halo": cl["LBM_HALO"]}
    errs = header_constants("LBM_ERR_")
    assert {v: k for k, v in errs.items()} == {k: v for k, v in lbm.ERRORS.items()}
