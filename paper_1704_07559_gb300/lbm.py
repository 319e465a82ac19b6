"""Python binding of the C ABI in include/lbm.h (liblbm.so), argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module allocates the
population buffers and output fields as torch tensors on the GPU, passes their raw pointers and
the current torch stream to the library, and turns status codes into exceptions.  There is no
CPU fallback: if the library is missing or no GPU is present, calls raise.

Array conventions match the header: populations (q, stride) in the storage dtype, fields
(components, nz, ny, nx) in the compute dtype (float64 for 'fp64', float32 otherwise).
"""
import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

D2Q9, D3Q15, D3Q19 = 9, 15, 19
PRECISION = {"fp64": 0, "fp32": 1, "fp16s": 2, "bf16s": 3}
CLOSURE = {"newton": 0, "smag": 1, "powerlaw": 2, "smag_lagged": 3, "smag_dev": 4}
FORMULA = {"yu": 0, "chai": 1}
BC = {"periodic": 0, "wall": 1, "lid": 2, "halo": 3}
SCHEDULE = {"auto": 0, "per_step": 1, "stream": 2, "stall_check": 3}
STORAGE_DTYPE = {0: torch.float64, 1: torch.float32, 2: torch.float16, 3: torch.bfloat16}
ERRORS = {-1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_NOMEM", -4: "LBM_ERR_NONFINITE", -5: "LBM_ERR_STATE",
          -6: "LBM_ERR_DRIFT"}
API = ["lbm_default_params", "lbm_create", "lbm_destroy", "lbm_layout", "lbm_bind", "lbm_bind_tau", "lbm_init",
       "lbm_step", "lbm_strain_rate", "lbm_macroscopic", "lbm_sums", "lbm_get_state", "lbm_set_state", "lbm_last_error",
       "lbm_sums_noalloc", "lbm_adjoint_workspace", "lbm_adjoint", "lbm_set_schedule", "lbm_status",
       "lbm_stats", "lbm_set_watchdog", "lbm_halo_layout", "lbm_halo_pack", "lbm_halo_unpack"]


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class Params(ctypes.Structure):
    """Mirror of struct lbm_params."""
    _fields_ = [
        ("precision", ctypes.c_int),
        ("closure", ctypes.c_int),
        ("formula", ctypes.c_int),
        ("smag_iters", ctypes.c_int),
        ("pl_max_iter", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("force_field", ctypes.c_int),
        ("rho0", ctypes.c_double),
        ("smag_cs", ctypes.c_double),
        ("pl_n", ctypes.c_double),
        ("pl_k", ctypes.c_double),
        ("pl_tau_min", ctypes.c_double),
        ("pl_tau_max", ctypes.c_double),
        ("pl_tol", ctypes.c_double),
        ("lid_u", (ctypes.c_double * 3) * 6),
    ]


_lib = None


def lib():
    """Load liblbm.so (built by paper_1704_07559_gb300.build); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblbm.so is not built (run paper_1704_07559_gb300.build.build()); "
                           "there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    L.lbm_default_params.argtypes = [ctypes.POINTER(Params)]
    L.lbm_default_params.restype = None
    L.lbm_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                             ctypes.POINTER(Params)]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_layout.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int64), ip]
    L.lbm_bind.argtypes = [vp, vp, vp, vp, vp]
    L.lbm_bind_tau.argtypes = [vp, vp]
    L.lbm_init.argtypes = [vp, vp, vp, vp]
    L.lbm_step.argtypes = [vp, ctypes.c_int]
    L.lbm_set_schedule.argtypes = [vp, ctypes.c_int]
    L.lbm_status.argtypes = [vp]
    L.lbm_set_watchdog.argtypes = [vp, ctypes.c_int, ctypes.c_double]
    L.lbm_halo_layout.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int64)]
    L.lbm_halo_pack.argtypes = [vp, vp, vp]
    L.lbm_halo_unpack.argtypes = [vp, vp, vp]
    L.lbm_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.lbm_strain_rate.argtypes = [vp, ctypes.c_int, vp, vp]
    L.lbm_macroscopic.argtypes = [vp, vp, vp]
    L.lbm_sums.argtypes = [vp, dp]
    L.lbm_get_state.argtypes = [vp, vp]
    L.lbm_set_state.argtypes = [vp, vp]
    L.lbm_adjoint_workspace.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    L.lbm_adjoint.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int64, vp, dp]
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = ctypes.c_char_p
    for name in API:
        if name not in ("lbm_default_params", "lbm_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def default_params():
    p = Params()
    lib().lbm_default_params(ctypes.byref(p))
    return p


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Lattice:
    """One lattice and its two population buffers on a CUDA device.

    rates: q relaxation rates (conserved entries 0, viscous entries 1/tau0).  force: uniform
    body-force density (d values) or None.  force_field: a (d, nz, ny, nx) tensor of the compute
    dtype (kept referenced) or None.  bc: 6 face kinds ('periodic' | 'wall' | 'lid' | 'halo'),
    faces -x, +x, -y, +y, -z, +z; lid_u: {face index: (ux, uy, uz)}.  With 'halo' z faces (a slab
    of a lattice cut along z, see slab.py) nz counts the slab's own planes and every array of the
    lattice spans nz + 2 planes, the first and last being ghost planes.
    """

    def __init__(self, lattice, nx, ny, nz=1, rates=None, force=None, precision="fp32", closure="newton",
                 formula="yu", bc=None, lid_u=None, smag_cs=0.0, smag_iters=6, pl_n=1.0, pl_k=0.0,
                 pl_tau_min=0.505, pl_tau_max=5.0, pl_tol=None, pl_max_iter=64, rho0=1.0, force_field=None,
                 device="cuda", stream=None):
        L = lib()
        self.q = int(lattice)
        self.d = 2 if self.q == D2Q9 else 3
        self.ns = 3 if self.q == D2Q9 else 6
        bc = list(bc) if bc is not None else ["periodic"] * 6
        bc += ["periodic"] * (6 - len(bc))  # 2D lattices may give only the four x / y faces
        self.halo = bc[4] == "halo" and bc[5] == "halo"
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz) + (2 if self.halo else 0)
        self.N = self.nx * self.ny * self.nz
        self.shape = (self.nz, self.ny, self.nx)
        self.device = torch.device(device)
        p = default_params()
        p.precision = PRECISION[precision]
        p.closure = CLOSURE[closure]
        p.formula = FORMULA[formula]
        p.smag_iters = smag_iters
        p.pl_max_iter = pl_max_iter
        for f in range(6):
            p.bc[f] = BC[bc[f]] if isinstance(bc[f], str) else int(bc[f])
        p.force_field = 1 if force_field is not None else 0
        p.rho0 = rho0
        p.smag_cs = smag_cs
        p.pl_n, p.pl_k, p.pl_tau_min, p.pl_tau_max = pl_n, pl_k, pl_tau_min, pl_tau_max
        if pl_tol is not None:
            p.pl_tol = pl_tol
        for f, v in (lid_u or {}).items():
            for a in range(3):
                p.lid_u[f][a] = v[a]
        self.params = p
        self.precision = p.precision
        self.storage_dtype = STORAGE_DTYPE[p.precision]
        self.compute_dtype = torch.float64 if p.precision == 0 else torch.float32
        r = (ctypes.c_double * self.q)(*[float(v) for v in rates])
        fv = None
        if force is not None:
            fv = (ctypes.c_double * 3)(*([float(v) for v in force] + [0.0] * (3 - len(force))))
        ctx = ctypes.c_void_p()
        rc = L.lbm_create(ctypes.byref(ctx), self.q, self.nx, self.ny, self.nz - (2 if self.halo else 0), r, fv,
                          ctypes.byref(p))
        if rc != 0:
            raise LBMError(rc, L.lbm_last_error(None).decode())
        self.ctx = ctx
        q = ctypes.c_int()
        stride = ctypes.c_int64()
        eb = ctypes.c_int()
        L.lbm_layout(ctx, ctypes.byref(q), ctypes.byref(stride), ctypes.byref(eb))
        self.stride = stride.value
        self.f_a = torch.empty((self.q, self.stride), dtype=self.storage_dtype, device=self.device)
        self.f_b = torch.empty((self.q, self.stride), dtype=self.storage_dtype, device=self.device)
        self.force_field = None
        if force_field is not None:
            self.force_field = force_field.to(device=self.device, dtype=self.compute_dtype).contiguous()
            assert self.force_field.shape == (self.d,) + self.shape
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._check(L.lbm_bind(ctx, _ptr(self.f_a), _ptr(self.f_b), _ptr(self.force_field),
                               ctypes.c_void_p(self.stream.cuda_stream)))
        # the lagged closure's per-node tau (state carried from step to step)
        self.tau = None
        if p.closure == CLOSURE["smag_lagged"]:
            self.tau = torch.empty(self.shape, dtype=self.compute_dtype, device=self.device)
            self._check(L.lbm_bind_tau(ctx, _ptr(self.tau)))

    # -- plumbing --------------------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise LBMError(rc, lib().lbm_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            lib().lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _field(self, t, comps, dtype):
        t = torch.as_tensor(t, dtype=dtype, device=self.device).contiguous()
        shape = (comps,) + self.shape if comps else self.shape
        return t.reshape(shape)

    # -- API -------------------------------------------------------------------------------
    def init(self, drho, u, grad_u=None):
        """Initial state from delta rho (nz,ny,nx), u (d,...) and optionally grad u (d*d,...)."""
        dr = self._field(drho, 0, torch.float64)
        uu = self._field(u, self.d, torch.float64)
        gu = None if grad_u is None else self._field(grad_u, self.d * self.d, torch.float64)
        self._check(lib().lbm_init(self.ctx, _ptr(dr), _ptr(uu), _ptr(gu)))
        self._keep = (dr, uu, gu)  # alive until the stream has consumed them
        return self

    def step(self, n=1):
        self._check(lib().lbm_step(self.ctx, int(n)))
        return self

    def set_schedule(self, schedule):
        """How step(n >= 2) launches: "auto", "per_step" or "stream" (several steps per launch)."""
        self._check(lib().lbm_set_schedule(self.ctx, SCHEDULE[schedule]))
        return self

    def set_watchdog(self, every, tol=1e-6):
        """Check the conserved totals every `every` steps inside step() (0 turns it off); step()
        then raises LBMError LBM_ERR_DRIFT or LBM_ERR_NONFINITE when they go off balance."""
        self._check(lib().lbm_set_watchdog(self.ctx, int(every), float(tol)))
        return self

    def stats(self):
        """(steps advanced, step kernels launched) since the context was created."""
        steps, launches = ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(lib().lbm_stats(self.ctx, ctypes.byref(steps), ctypes.byref(launches)))
        return steps.value, launches.value

    def status(self):
        """Synchronise the bound stream; raises LBMError on an asynchronous failure."""
        self._check(lib().lbm_status(self.ctx))
        return self

    def strain_rate(self, formula=None, with_tau=False):
        fm = self.params.formula if formula is None else FORMULA[formula]
        S = torch.empty((self.ns,) + self.shape, dtype=self.compute_dtype, device=self.device)
        tau = torch.empty(self.shape, dtype=self.compute_dtype, device=self.device) if with_tau else None
        self._check(lib().lbm_strain_rate(self.ctx, fm, _ptr(S), _ptr(tau)))
        return (S, tau) if with_tau else S

    def macroscopic(self):
        drho = torch.empty(self.shape, dtype=self.compute_dtype, device=self.device)
        u = torch.empty((self.d,) + self.shape, dtype=self.compute_dtype, device=self.device)
        self._check(lib().lbm_macroscopic(self.ctx, _ptr(drho), _ptr(u)))
        return drho, u

    def sums(self):
        out = (ctypes.c_double * (1 + self.d))()
        self._check(lib().lbm_sums(self.ctx, out))
        return np.array(out[:], dtype=np.float64)

    def get_state(self, out=None):
        """Post-collision populations of the current buffer as a dense (q, nz, ny, nx) tensor."""
        if out is None:
            out = torch.empty((self.q,) + self.shape, dtype=self.storage_dtype, device=self.device)
        assert out.dtype == self.storage_dtype and out.is_contiguous() and out.numel() == self.q * self.N
        self._check(lib().lbm_get_state(self.ctx, _ptr(out)))
        return out

    def adjoint(self, T, seg=None):
        """(L, dL/dg) after T steps from the current state: L as a float, dL/dg as a float64
        tensor (d, nz, ny, nx).  seg defaults to round(sqrt(T)).  The current state afterwards is
        the state after T steps."""
        seg = int(seg or max(1, round(T ** 0.5)))
        L = lib()
        nbytes = ctypes.c_int64()
        self._check(L.lbm_adjoint_workspace(self.ctx, int(T), seg, ctypes.byref(nbytes)))
        work = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        off = (-work.data_ptr()) % 256
        grad = torch.empty((self.d,) + self.shape, dtype=torch.float64, device=self.device)
        loss = ctypes.c_double()
        self._check(L.lbm_adjoint(self.ctx, int(T), seg, ctypes.c_void_p(work.data_ptr() + off), nbytes.value,
                                  _ptr(grad), ctypes.byref(loss)))
        return loss.value, grad

    def halo_layout(self):
        """(crossing populations per z face, elements per halo buffer) of a lattice with halo faces."""
        pops, elems = ctypes.c_int(), ctypes.c_int64()
        self._check(lib().lbm_halo_layout(self.ctx, ctypes.byref(pops), ctypes.byref(elems)))
        return pops.value, elems.value

    def halo_pack(self, send_lo, send_hi):
        """Copy the populations leaving through the lower / upper z face into two device tensors."""
        self._check(lib().lbm_halo_pack(self.ctx, _ptr(send_lo), _ptr(send_hi)))
        return self

    def halo_unpack(self, recv_lo, recv_hi):
        """Write the lower / upper neighbours' outgoing populations into the ghost planes."""
        self._check(lib().lbm_halo_unpack(self.ctx, _ptr(recv_lo), _ptr(recv_hi)))
        return self

    def set_state(self, f):
        f = f.to(dtype=self.storage_dtype).contiguous()
        assert f.numel() == self.q * self.N
        self._check(lib().lbm_set_state(self.ctx, _ptr(f)))
        self._keep = f
        return self


class DissipationLoss(torch.autograd.Function):
    """L(g): the dissipation functional after T steps from the state f0 under the force field g
    (bound to `lat`, which must have been created with a force field).  Forward runs the steps and
    the library's adjoint together; backward returns grad_output * dL/dg."""

    @staticmethod
    def forward(ctx, g, lat, f0, T, seg=None):
        lat.force_field.copy_(g.detach().to(lat.force_field.dtype).reshape(lat.force_field.shape))
        lat.set_state(f0)
        loss, grad = lat.adjoint(T, seg)
        ctx.save_for_backward(grad.to(g.dtype).reshape(g.shape))
        return torch.tensor(loss, dtype=torch.float64, device=g.device)

    @staticmethod
    def backward(ctx, grad_output):
        (grad,) = ctx.saved_tensors
        return grad_output.to(grad.dtype) * grad, None, None, None, None
