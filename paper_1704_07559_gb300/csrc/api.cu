// api.cu -- the C ABI declared in include/lbm.h: argument checks, the context, and dispatch to
// the kernel instantiations.  No call aborts; every failure returns a status and a message.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/lbm.h"
#include "adjoint.cuh"
#include "adjoint_launch.h"
#include "launch.h"
#include "step.cuh"

struct lbm_ctx {
    int q, d, ns;
    int nx, ny, nz;   // nz counts every plane held, ghost planes included
    int halo;         // 1: both z faces are LBM_HALO (planes 0 and nz - 1 are ghost planes)
    int z0, nzc;      // planes computed: [z0, z0 + nzc)
    int hpop_up[5], hpop_dn[5], hpops;  // populations crossing the z faces (c_z = +1 / -1)
    long long N, stride;
    int elem_bytes;
    double rates[19];
    double force[3];
    lbm_params p;
    // bound resources
    void* buf[2];
    const void* force_field;
    void* tau_field;  // lagged closure: the stored tau per node (caller-owned)
    cudaStream_t stream;
    int bound;
    int cur;  // index of the current buffer
    // library-owned scratch: per-block partial sums and the final row
    double* partial;
    double* result;
    // several steps per launch: synchronisation words (error flag, ticket, per-unit step counts)
    // and the unit geometry; schedule is one of LBM_SCHEDULE_*
    int* sync;
    int stream_rows, stream_tiles;
    int schedule;
    long long n_steps, n_step_launches;  // steps advanced and step kernels launched by lbm_step
    // watchdog (lbm_set_watchdog): check the global sums every watch_every steps against the
    // reference sums watch_ref taken at step watch_ref_step (watch_ref_ok 0: take it first)
    int watch_every;
    double watch_tol;
    int watch_ref_ok;
    double watch_ref[4];
    long long watch_ref_step;
    char err[512];
};

namespace {

// message of the last failed lbm_create on this thread (lbm_last_error(NULL) returns it)
thread_local char create_err[256] = "";

int fail(lbm_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_finite(double v) { return std::isfinite(v); }

bool is_viscous(int q, int k) {
    switch (q) {
        case 19: return lbm::D3Q19::viscous(k);
        case 15: return lbm::D3Q15::viscous(k);
        default: return lbm::D2Q9::viscous(k);
    }
}
bool is_conserved(int q, int k) {
    switch (q) {
        case 19: return lbm::D3Q19::conserved(k);
        case 15: return lbm::D3Q15::conserved(k);
        default: return lbm::D2Q9::conserved(k);
    }
}
int first_viscous(int q) { return q == 9 ? lbm::D2Q9::NU0 : lbm::D3Q19::NU0; }
int row_norm2(int q, int k) {
    switch (q) {
        case 19: return lbm::norm2<lbm::D3Q19>(k);
        case 15: return lbm::norm2<lbm::D3Q15>(k);
        default: return lbm::norm2<lbm::D2Q9>(k);
    }
}

bool viscous_rates_equal(const lbm_ctx* c) {
    const double s = c->rates[first_viscous(c->q)];
    for (int k = 0; k < c->q; ++k)
        if (is_viscous(c->q, k) && c->rates[k] != s) return false;
    return true;
}

template <class R>
void fill_args(const lbm_ctx* c, lbm::StepArgs<R>* a) {
    std::memset(a, 0, sizeof(*a));
    a->nx = c->nx;
    a->ny = c->ny;
    a->nz = c->nz;
    a->z0 = c->z0;
    a->nzc = c->nzc;
    a->stride = c->stride;
    for (int k = 0; k < 19; ++k) {
        a->s[k] = R(k < c->q ? c->rates[k] : 0.0);
        const int n2 = k >= c->q ? 1 : row_norm2(c->q, k);
        a->skn[k] = R(k < c->q ? c->rates[k] / n2 : 0.0);
    }
    for (int d = 0; d < 3; ++d) a->F[d] = R(c->force[d]);
    a->rho0 = R(c->p.rho0);
    a->inv_rho0 = R(1.0 / c->p.rho0);
    a->tau0 = R(1.0 / c->rates[first_viscous(c->q)]);
    a->smag_c3 = R(3.0 * c->p.smag_cs * c->p.smag_cs);
    a->pl_k3 = R(3.0 * c->p.pl_k);
    a->pl_nm1 = R(c->p.pl_n - 1.0);
    a->pl_tau_min = R(c->p.pl_tau_min);
    a->pl_tau_max = R(c->p.pl_tau_max);
    a->pl_tol = R(c->p.pl_tol);
    a->smag_iters = c->p.smag_iters;
    a->pl_max_iter = c->p.pl_max_iter;
    int wall = 0, lid = 0;
    for (int f = 0; f < 6; ++f) {
        if (c->d == 2 && f >= 4) continue;
        if (c->p.bc[f] == LBM_WALL || c->p.bc[f] == LBM_LID) wall |= 1 << f;  // a halo face reads its ghost plane
        if (c->p.bc[f] == LBM_LID) lid |= 1 << f;
        for (int k = 0; k < 3; ++k) a->lid[f][k] = R(c->p.lid_u[f][k]);
    }
    a->wall_mask = wall;
    a->lid_mask = lid;
    a->force_field = c->p.force_field ? static_cast<const R*>(c->force_field) : nullptr;
    a->tau_field = static_cast<R*>(c->tau_field);
}

// source / destination buffers and their per-population base pointers
template <class R>
void set_buffers(const lbm_ctx* c, lbm::StepArgs<R>* a, const void* src, void* dst) {
    a->src = src;
    a->dst = dst;
    const size_t pitch = (size_t)c->stride * c->elem_bytes;
    for (int i = 0; i < 19; ++i) {
        a->srcp[i] = (src && i < c->q) ? static_cast<const char*>(src) + i * pitch : nullptr;
        a->dstp[i] = (dst && i < c->q) ? static_cast<char*>(dst) + i * pitch : nullptr;
    }
}

bool has_force(const lbm_ctx* c) {
    return c->p.force_field || c->force[0] != 0.0 || c->force[1] != 0.0 || c->force[2] != 0.0;
}

enum Tag { T_D3Q19_F64, T_D3Q19_F32, T_D3Q19_F16, T_D3Q19_BF16, T_D3Q15_F64, T_D3Q15_F32, T_D3Q15_F16, T_D3Q15_BF16, T_D2Q9_F64, T_D2Q9_F32, T_NONE };

Tag tag_of(int q, int precision) {
    if (q == 19) {
        switch (precision) {
            case LBM_FP64: return T_D3Q19_F64;
            case LBM_FP32: return T_D3Q19_F32;
            case LBM_FP16S: return T_D3Q19_F16;
            case LBM_BF16S: return T_D3Q19_BF16;
        }
    } else if (q == 15) {
        switch (precision) {
            case LBM_FP64: return T_D3Q15_F64;
            case LBM_FP32: return T_D3Q15_F32;
            case LBM_FP16S: return T_D3Q15_F16;
            case LBM_BF16S: return T_D3Q15_BF16;
        }
    } else if (q == 9) {
        switch (precision) {
            case LBM_FP64: return T_D2Q9_F64;
            case LBM_FP32: return T_D2Q9_F32;
        }
    }
    return T_NONE;
}

// Several steps in one launch (float storage).  Returns cudaErrorNotSupported when the
// streamed form does not apply or (automatic schedule) is not expected to pay: a D2Q9 lattice,
// more than 2^22 nodes, or too few units to keep every resident block busy without waiting; the
// caller then launches step by step.
cudaError_t run_stream(lbm_ctx* c, int nsteps) {
    if (c->p.precision == LBM_FP64 || c->schedule == LBM_SCHEDULE_PER_STEP || c->halo)
        return cudaErrorNotSupported;
    // automatic schedule: 3D lattices of at most 2^22 nodes (measured on GB300: +7% on a 4.2M-node
    // channel, +17% on a 2.1M-node box, but -8% on a 7.1M-node box, -2% on a 2048^2 and -26% on a
    // 4096^2 D2Q9 lattice); the launchers also decline without enough units per resident block
    if (c->schedule == LBM_SCHEDULE_AUTO && (c->nz == 1 || c->N > (1LL << 22))) return cudaErrorNotSupported;
    // the stall check starts at step 1 of the launch: the neighbours' step 0 never runs
    const bool stall = c->schedule == LBM_SCHEDULE_STALL_CHECK;
    lbm::StepArgs<float> a0, a1;
    fill_args(c, &a0);
    a0.readout = 0;
    a0.S_out = a0.tau_out = a0.drho_out = a0.u_out = nullptr;
    a1 = a0;
    set_buffers(c, &a0, c->buf[c->cur], c->buf[1 - c->cur]);
    set_buffers(c, &a1, c->buf[1 - c->cur], c->buf[c->cur]);
    const lbm::StreamCtl ctl = {c->sync, nsteps, c->stream_rows, c->stream_tiles, stall ? 1 : 0, 0};
    const int force = has_force(c) ? 1 : 0, forced = (stall || c->schedule == LBM_SCHEDULE_STREAM) ? 1 : 0;
    const int cl = c->p.closure, fm = c->p.formula;
    if (stall) c->schedule = LBM_SCHEDULE_AUTO;
    switch (tag_of(c->q, c->p.precision)) {
        case T_D3Q19_F32: return lbm::stream_d3q19_f32(a0, a1, ctl, cl, fm, force, forced, c->stream);
        case T_D3Q19_F16: return lbm::stream_d3q19_f16(a0, a1, ctl, cl, fm, force, forced, c->stream);
        case T_D3Q19_BF16: return lbm::stream_d3q19_bf16(a0, a1, ctl, cl, fm, force, forced, c->stream);
        case T_D3Q15_F32: return lbm::stream_d3q15_f32(a0, a1, ctl, cl, fm, force, forced, c->stream);
        case T_D3Q15_F16: return lbm::stream_d3q15_f16(a0, a1, ctl, cl, fm, force, forced, c->stream);
        case T_D3Q15_BF16: return lbm::stream_d3q15_bf16(a0, a1, ctl, cl, fm, force, forced, c->stream);
        case T_D2Q9_F32: return lbm::stream_d2q9_f32(a0, a1, ctl, cl, fm, force, forced, c->stream);
        default: return cudaErrorNotSupported;
    }
}

// After a synchronisation: LBM_ERR_STATE (and the flag cleared) when a multi-step launch
// recorded that one of its dependency waits ran out.
int stream_flag(lbm_ctx* c) {
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, c->sync, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the multi-step status");
    if (flag) {
        cudaMemset(c->sync, 0, sizeof(int));
        return fail(c, LBM_ERR_STATE,
                    "a multi-step launch stopped: a wait for neighbouring units ran out; the state is invalid");
    }
    return LBM_OK;
}

// step or read-out launch through the right instantiation
cudaError_t run_step(lbm_ctx* c, int formula, int readout, void* S, void* tau, void* drho, void* u,
                     const void* src, void* dst) {
    const int force = has_force(c) ? 1 : 0;
    const Tag t = tag_of(c->q, c->p.precision);
    if (c->p.precision == LBM_FP64) {
        lbm::StepArgs<double> a;
        fill_args(c, &a);
        a.readout = readout;
        set_buffers(c, &a, src, dst);
        a.S_out = static_cast<double*>(S);
        a.tau_out = static_cast<double*>(tau);
        a.drho_out = static_cast<double*>(drho);
        a.u_out = static_cast<double*>(u);
        switch (t) {
            case T_D3Q19_F64: return lbm::step_d3q19_f64(a, c->p.closure, formula, force, c->stream);
            case T_D3Q15_F64: return lbm::step_d3q15_f64(a, c->p.closure, formula, force, c->stream);
            case T_D2Q9_F64: return lbm::step_d2q9_f64(a, c->p.closure, formula, force, c->stream);
            default: return cudaErrorInvalidValue;
        }
    }
    lbm::StepArgs<float> a;
    fill_args(c, &a);
    a.readout = readout;
    set_buffers(c, &a, src, dst);
    a.S_out = static_cast<float*>(S);
    a.tau_out = static_cast<float*>(tau);
    a.drho_out = static_cast<float*>(drho);
    a.u_out = static_cast<float*>(u);
    switch (t) {
        case T_D3Q19_F32: return lbm::step_d3q19_f32(a, c->p.closure, formula, force, c->stream);
        case T_D3Q19_F16: return lbm::step_d3q19_f16(a, c->p.closure, formula, force, c->stream);
        case T_D3Q19_BF16: return lbm::step_d3q19_bf16(a, c->p.closure, formula, force, c->stream);
        case T_D3Q15_F32: return lbm::step_d3q15_f32(a, c->p.closure, formula, force, c->stream);
        case T_D3Q15_F16: return lbm::step_d3q15_f16(a, c->p.closure, formula, force, c->stream);
        case T_D3Q15_BF16: return lbm::step_d3q15_bf16(a, c->p.closure, formula, force, c->stream);
        case T_D2Q9_F32: return lbm::step_d2q9_f32(a, c->p.closure, formula, force, c->stream);
        default: return cudaErrorInvalidValue;
    }
}

// n steps from the current buffer (which alternates): several per launch where the schedule
// allows, one launch per step otherwise.  A multi-step launch runs at most STREAM_CHUNK steps
// (and keeps its ticket count below 2^31), so that no single kernel runs for minutes.
// *launches counts the step kernels launched.
constexpr int STREAM_CHUNK = 4096;

cudaError_t advance(lbm_ctx* c, int n, long long* launches) {
    int it = 0;
    if (n >= 2) {
        const long long units = (long long)c->nz * c->stream_tiles;
        const int chunk = (int)std::min<long long>(std::min(n, STREAM_CHUNK), 0x7fffffffLL / units);
        while (n - it >= 2 && chunk >= 2) {
            const int k = std::min(chunk, n - it);
            cudaError_t e = run_stream(c, k);
            if (e == cudaErrorNotSupported) break;
            if (e != cudaSuccess) return e;
            if (k & 1) c->cur = 1 - c->cur;
            it += k;
            ++*launches;
        }
    }
    for (; it < n; ++it) {
        cudaError_t e = run_step(c, c->p.formula, 0, nullptr, nullptr, nullptr, nullptr, c->buf[c->cur], c->buf[1 - c->cur]);
        if (e != cudaSuccess) return e;
        c->cur = 1 - c->cur;
        ++*launches;
    }
    return cudaSuccess;
}

int check_bound(lbm_ctx* c) {
    if (!c) return LBM_ERR_ARG;
    if (!c->bound) return fail(c, LBM_ERR_STATE, "no buffers bound (call lbm_bind first)");
    if (c->p.closure == LBM_SMAG_LAGGED && !c->tau_field)
        return fail(c, LBM_ERR_STATE, "the lagged closure needs its tau field (call lbm_bind_tau first)");
    return LBM_OK;
}


// Global sums of the current state into out[0..d] (HOST), synchronising the bound stream:
// LBM_ERR_CUDA, LBM_ERR_STATE (a multi-step launch's wait ran out), LBM_ERR_NONFINITE (out
// filled) or LBM_OK.
int sums_now(lbm_ctx* c, double* out, const char* who) {
    cudaError_t e;
    const Tag t = tag_of(c->q, c->p.precision);
    if (c->p.precision == LBM_FP64) {
        lbm::StepArgs<double> a;
        fill_args(c, &a);
        set_buffers(c, &a, c->buf[c->cur], nullptr);
        switch (t) {
            case T_D3Q19_F64: e = lbm::sums_d3q19_f64(a, c->partial, c->result, c->stream); break;
            case T_D3Q15_F64: e = lbm::sums_d3q15_f64(a, c->partial, c->result, c->stream); break;
            case T_D2Q9_F64: e = lbm::sums_d2q9_f64(a, c->partial, c->result, c->stream); break;
            default: e = cudaErrorInvalidValue;
        }
    } else {
        lbm::StepArgs<float> a;
        fill_args(c, &a);
        set_buffers(c, &a, c->buf[c->cur], nullptr);
        switch (t) {
            case T_D3Q19_F32: e = lbm::sums_d3q19_f32(a, c->partial, c->result, c->stream); break;
            case T_D3Q19_F16: e = lbm::sums_d3q19_f16(a, c->partial, c->result, c->stream); break;
            case T_D3Q19_BF16: e = lbm::sums_d3q19_bf16(a, c->partial, c->result, c->stream); break;
            case T_D3Q15_F32: e = lbm::sums_d3q15_f32(a, c->partial, c->result, c->stream); break;
            case T_D3Q15_F16: e = lbm::sums_d3q15_f16(a, c->partial, c->result, c->stream); break;
            case T_D3Q15_BF16: e = lbm::sums_d3q15_bf16(a, c->partial, c->result, c->stream); break;
            case T_D2Q9_F32: e = lbm::sums_d2q9_f32(a, c->partial, c->result, c->stream); break;
            default: e = cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return cuda_fail(c, e, who);
    e = cudaMemcpyAsync(out, c->result, sizeof(double) * (1 + c->d), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, who);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, who);
    int rc = stream_flag(c);
    if (rc) return rc;
    for (int k = 0; k <= c->d; ++k)
        if (!is_finite(out[k])) return fail(c, LBM_ERR_NONFINITE, "%s: non-finite sum %d (%g)", who, k, out[k]);
    return LBM_OK;
}

// The watchdog's test of sums s taken after step c->n_steps: the total mass stays at the
// reference, and on an all-periodic lattice without a force field each momentum component grows
// by N F per step from the reference (halfway bounce-back walls exchange momentum with the
// fluid, and a per-node force field's total is not known to the library); bound tol * N * rho0.
int watch_check(lbm_ctx* c, const double* s) {
    const double bound = c->watch_tol * (double)c->N * c->p.rho0;
    const long long k = c->n_steps - c->watch_ref_step;
    const double dm = s[0] - c->watch_ref[0];
    if (!(std::fabs(dm) <= bound))
        return fail(c, LBM_ERR_DRIFT, "watchdog: total mass changed by %.6g over %lld steps (bound %.6g)", dm, k, bound);
    bool periodic = true;
    for (int f = 0; f < 2 * c->d; ++f) periodic = periodic && c->p.bc[f] == LBM_PERIODIC;
    if (periodic && !c->p.force_field) {
        for (int a = 0; a < c->d; ++a) {
            const double dj = s[1 + a] - (c->watch_ref[1 + a] + (double)k * (double)c->N * c->force[a]);
            if (!(std::fabs(dj) <= bound))
                return fail(c, LBM_ERR_DRIFT,
                            "watchdog: total momentum %d is %.6g away from its balance over %lld steps (bound %.6g)", a,
                            dj, k, bound);
        }
    }
    return LBM_OK;
}

// lbm_step(n) under the watchdog: chunks of at most watch_every steps, the sums checked after each
int step_watched(lbm_ctx* c, int n) {
    if (!c->watch_ref_ok) {
        int rc = sums_now(c, c->watch_ref, "watchdog reference");
        if (rc) return rc;
        c->watch_ref_ok = 1;
        c->watch_ref_step = c->n_steps;
    }
    for (int done = 0; done < n;) {
        const int k = std::min(c->watch_every, n - done);
        long long launches = 0;
        cudaError_t e = advance(c, k, &launches);
        if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step");
        c->n_steps += k;
        c->n_step_launches += launches;
        done += k;
        double s[4];
        int rc = sums_now(c, s, "watchdog");
        if (rc) return rc;
        rc = watch_check(c, s);
        if (rc) return rc;
    }
    return LBM_OK;
}

// ------------------------------------------------------------------------------------------
// adjoint driver helpers

struct AdjLayout {
    int ncp = 0, nseg = 0, nblocks = 0;
    size_t state = 0, lam = 0, dF = 0, partial = 0;
    size_t off_cp = 0, off_seg = 0, off_lam = 0, off_dF = 0, off_partial = 0, total = 0;
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int adjoint_check(lbm_ctx* c, int T, int seg) {
    if (c->q != 19) return fail(c, LBM_ERR_ARG, "lbm_adjoint: D3Q19 only");
    if (c->halo) return fail(c, LBM_ERR_ARG, "lbm_adjoint: not for a lattice with halo faces");
    if (c->p.precision != LBM_FP32 && c->p.precision != LBM_FP64)
        return fail(c, LBM_ERR_ARG, "lbm_adjoint: FP32 or FP64 populations only");
    if (c->p.closure != LBM_NEWTON && c->p.closure != LBM_SMAG)
        return fail(c, LBM_ERR_ARG, "lbm_adjoint: Newtonian or Smagorinsky closure only");
    for (int f = 0; f < 6; ++f)
        if (c->p.bc[f] != LBM_PERIODIC) return fail(c, LBM_ERR_ARG, "lbm_adjoint: periodic faces only");
    if (!c->p.force_field) return fail(c, LBM_ERR_ARG, "lbm_adjoint: needs a bound force field (the gradient's variable)");
    if (T < 0 || seg < 1) return fail(c, LBM_ERR_ARG, "lbm_adjoint: T >= 0 and seg >= 1 required");
    return LBM_OK;
}

AdjLayout adjoint_layout(const lbm_ctx* c, int T, int seg) {
    AdjLayout L;
    const size_t comp = c->p.precision == LBM_FP64 ? 8 : 4;
    L.ncp = T > 0 ? (T + seg - 1) / seg : 0;
    L.nseg = T > 0 ? (seg < T ? seg : T) - 1 : 0;
    L.nblocks = lbm::functional_blocks(c->nx, c->ny, c->nz);
    L.state = align256((size_t)c->q * c->stride * c->elem_bytes);
    L.lam = align256((size_t)c->q * c->stride * comp);
    L.dF = align256((size_t)3 * c->N * comp);
    L.partial = align256((size_t)(L.nblocks + 1) * sizeof(double));
    L.off_cp = 0;
    L.off_seg = L.off_cp + L.ncp * L.state;
    L.off_lam = L.off_seg + L.nseg * L.state;
    L.off_dF = L.off_lam + 2 * L.lam;
    L.off_partial = L.off_dF + L.dF;
    L.total = L.off_partial + L.partial;
    return L;
}

template <class R>
cudaError_t adjoint_run(lbm_ctx* c, int T, int seg, char* work, const AdjLayout& L, double* dLdg, double* loss) {
    cudaStream_t s = c->stream;
    cudaError_t e;
    const size_t state_bytes = (size_t)c->q * c->stride * c->elem_bytes;
    auto cp = [&](int k) { return static_cast<void*>(work + L.off_cp + k * L.state); };
    auto sg = [&](int k) { return static_cast<void*>(work + L.off_seg + k * L.state); };
    R* lam[2] = {reinterpret_cast<R*>(work + L.off_lam), reinterpret_cast<R*>(work + L.off_lam + L.lam)};
    R* dF = reinterpret_cast<R*>(work + L.off_dF);
    double* partial = reinterpret_cast<double*>(work + L.off_partial);
    double* result = partial + L.nblocks;
    constexpr bool F64 = std::is_same<R, double>::value;
    auto fold = [&](R* acc) {
        if constexpr (F64)
            return lbm::adj_fold_f64(acc, dLdg, c->p.rho0, 3LL * c->N, s);
        else
            return lbm::adj_fold_f32(acc, dLdg, c->p.rho0, 3LL * c->N, s);
    };

    const long long ring = (long long)(L.state / c->elem_bytes);  // elements between segment states
    const int forced = c->schedule == LBM_SCHEDULE_STREAM ? 1 : 0;
    // states 1 .. m - 1 of segment sgi into the segment buffers sg(0 .. m - 2), from its checkpoint:
    // the first step from the checkpoint, the rest (FP32, where the schedule allows) in one ring
    // launch that writes each step to the next state buffer
    auto fill_segment = [&](int sgi, int m) -> cudaError_t {
        cudaError_t err;
        int i = 1;
        if (m >= 2) {
            err = run_step(c, c->p.formula, 0, nullptr, nullptr, nullptr, nullptr, cp(sgi), sg(0));
            if (err != cudaSuccess) return err;
            i = 2;
        }
        if constexpr (!F64) {
            if (m - 2 >= 2 && c->schedule != LBM_SCHEDULE_PER_STEP) {
                lbm::StepArgs<float> ra;
                fill_args(c, &ra);
                ra.readout = 0;
                ra.S_out = ra.tau_out = ra.drho_out = ra.u_out = nullptr;
                set_buffers(c, &ra, sg(0), sg(1));
                const lbm::StreamCtl ctl = {c->sync, m - 2, c->stream_rows, c->stream_tiles, 0, ring};
                err = lbm::stream_ring_d3q19_f32(ra, ctl, c->p.closure, c->p.formula, has_force(c) ? 1 : 0, forced, s);
                if (err == cudaSuccess)
                    i = m;
                else if (err != cudaErrorNotSupported)
                    return err;
            }
        }
        for (; i < m; ++i) {
            err = run_step(c, c->p.formula, 0, nullptr, nullptr, nullptr, nullptr, sg(i - 2), sg(i - 1));
            if (err != cudaSuccess) return err;
        }
        return cudaSuccess;
    };

    // forward T steps from the current state, keeping every seg-th state: per segment, the first
    // step reads the checkpoint into a context buffer, the middle steps ping-pong between the two
    // context buffers (several per launch where the schedule allows), and the last step writes the
    // next checkpoint.  The last segment writes its states straight into the segment buffers the
    // reverse sweep reads (so it needs no recomputation there) and its last step the final state
    // into a context buffer.
    const void* fcur = c->buf[c->cur];
    bool last_filled = false;
    if (T > 0) {
        e = cudaMemcpyAsync(cp(0), c->buf[c->cur], state_bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        for (int k0 = 0; k0 < T; k0 += seg) {
            const int k1 = (k0 + seg < T) ? k0 + seg : T;
            const bool to_cp = k1 < T;
            if (to_cp && k1 - k0 == 1) {  // one-step segments: checkpoint to checkpoint
                e = run_step(c, c->p.formula, 0, nullptr, nullptr, nullptr, nullptr, cp(k0 / seg), cp(k1 / seg));
                if (e != cudaSuccess) return e;
                continue;
            }
            if (!to_cp && k1 - k0 >= 2) {  // the last segment
                e = fill_segment(k0 / seg, k1 - k0);
                if (e != cudaSuccess) return e;
                e = run_step(c, c->p.formula, 0, nullptr, nullptr, nullptr, nullptr, sg(k1 - k0 - 2), c->buf[0]);
                if (e != cudaSuccess) return e;
                c->cur = 0;
                last_filled = true;
                continue;
            }
            e = run_step(c, c->p.formula, 0, nullptr, nullptr, nullptr, nullptr, cp(k0 / seg), c->buf[0]);
            if (e != cudaSuccess) return e;
            c->cur = 0;
            long long launches = 0;
            e = advance(c, k1 - k0 - 1 - (to_cp ? 1 : 0), &launches);
            if (e != cudaSuccess) return e;
            if (to_cp) {
                e = run_step(c, c->p.formula, 0, nullptr, nullptr, nullptr, nullptr, c->buf[c->cur], cp(k1 / seg));
                if (e != cudaSuccess) return e;
            }
        }
        fcur = c->buf[c->cur];
    }

    lbm::AdjArgs<R> a;
    fill_args(c, &a.st);
    a.dF = dF;
    a.partial = partial;
    // the functional at f^T: loss partials, lambda_T, dF
    set_buffers(c, &a.st, fcur, nullptr);
    lbm::set_lambda(&a, static_cast<const R*>(nullptr), lam[0]);
    int nb = 0;
    if constexpr (F64)
        e = lbm::adj_functional_f64(a, c->p.closure, s, &nb);
    else
        e = lbm::adj_functional_f32(a, c->p.closure, s, &nb);
    if (e != cudaSuccess) return e;
    lbm::k_sums_final<<<1, 256, 0, s>>>(partial, nb, 1, result);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(dLdg, 0, sizeof(double) * 3 * c->N, s);
    if (e != cudaSuccess) return e;

    // reverse sweep, segment by segment from the last, recomputing the states of every segment but
    // the last
    int lc = 0;
    for (int sgi = L.ncp - 1; sgi >= 0; --sgi) {
        const int k0 = sgi * seg, k1 = (k0 + seg < T) ? k0 + seg : T, m = k1 - k0;
        const void* states[1024];
        states[0] = cp(sgi);
        for (int i = 1; i < m; ++i) states[i] = sg(i - 1);
        // recompute the segment's states (the last segment's are still there from the forward sweep)
        if (!(sgi == L.ncp - 1 && last_filled)) {
            e = fill_segment(sgi, m);
            if (e != cudaSuccess) return e;
        }
        // reverse steps k1 - 1 .. k0 + 1 (states sg(m - 2) down to sg(0), equally spaced) in one
        // launch where the schedule allows, the rest one launch per step
        int n = k1 - 1;
        if constexpr (!F64) {
            if (m - 1 >= 2 && c->schedule != LBM_SCHEDULE_PER_STEP) {
                lbm::AdjArgs<R> b0 = a, b1 = a;
                set_buffers(c, &b0.st, states[m - 1], nullptr);
                set_buffers(c, &b1.st, states[m - 1], nullptr);
                lbm::set_lambda(&b0, static_cast<const R*>(lam[lc]), lam[1 - lc]);
                lbm::set_lambda(&b1, static_cast<const R*>(lam[1 - lc]), lam[lc]);
                const lbm::StreamCtl ctl = {c->sync, m - 1, c->stream_rows, c->stream_tiles, 0, ring};
                e = lbm::adj_stream_f32(b0, b1, ctl, c->p.closure, forced, s);
                if (e == cudaSuccess) {
                    n = k0;
                    if ((m - 1) & 1) lc = 1 - lc;
                } else if (e != cudaErrorNotSupported) {
                    return e;
                }
            }
        }
        for (; n >= k0; --n) {
            set_buffers(c, &a.st, states[n - k0], nullptr);
            lbm::set_lambda(&a, static_cast<const R*>(lam[lc]), lam[1 - lc]);
            if constexpr (F64)
                e = lbm::adj_step_f64(a, c->p.closure, s);
            else
                e = lbm::adj_step_f32(a, c->p.closure, s);
            if (e != cudaSuccess) return e;
            lc = 1 - lc;
        }
        e = fold(dF);
        if (e != cudaSuccess) return e;
    }
    if (L.ncp == 0) {  // T = 0: only the functional's direct term
        e = fold(dF);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemcpyAsync(loss, result, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace

namespace lbm {
__global__ void k_sums_final(const double* __restrict__ partial, int nblocks, int width, double* __restrict__ out) {
    // one block of 256 threads: thread t adds rows t, t + 256, ... of each column, then a fixed
    // shared-memory tree (the order never changes, so the result is reproducible)
    __shared__ double red[256];
    for (int c = 0; c < width; ++c) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[b * width + c];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = red[0];
        __syncthreads();
    }
}
}  // namespace lbm

namespace {

// the halo copy of the current buffer: lo / hi are the halo buffers (send for a pack, receive for
// an unpack)
lbm::HaloArgs halo_args(const lbm_ctx* c, void* lo, void* hi) {
    lbm::HaloArgs h;
    std::memset(&h, 0, sizeof(h));
    h.buf = static_cast<char*>(c->buf[c->cur]);
    h.pitch = c->stride * c->elem_bytes;
    h.plane = (long long)c->nx * c->ny;
    h.pops = c->hpops;
    for (int k = 0; k < c->hpops; ++k) {
        h.up[k] = c->hpop_up[k];
        h.dn[k] = c->hpop_dn[k];
    }
    h.z_lo = c->z0;                // bottom own plane
    h.z_hi = c->z0 + c->nzc - 1;   // top own plane
    h.lo = static_cast<char*>(lo);
    h.hi = static_cast<char*>(hi);
    return h;
}

}  // namespace

extern "C" {

void lbm_default_params(lbm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->precision = LBM_FP32;
    p->closure = LBM_NEWTON;
    p->formula = LBM_YU;
    p->smag_iters = 6;
    p->pl_max_iter = 64;
    for (int f = 0; f < 6; ++f) p->bc[f] = LBM_PERIODIC;
    p->force_field = 0;
    p->rho0 = 1.0;
    p->smag_cs = 0.0;
    p->pl_n = 1.0;
    p->pl_k = 0.0;
    p->pl_tau_min = 0.505;
    p->pl_tau_max = 5.0;
    p->pl_tol = -1.0;  // resolved by lbm_create from the precision
}

int lbm_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, const double* rates, const double* force,
               const lbm_params* pin) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_ctx* c = new (std::nothrow) lbm_ctx;
    if (!c) return LBM_ERR_NOMEM;
    std::memset(c, 0, sizeof(*c));
    auto bad = [&](const char* what) {
        snprintf(create_err, sizeof(create_err), "lbm_create: invalid %s", what);
        delete c;
        return LBM_ERR_ARG;
    };
    create_err[0] = '\0';
    if (lattice != LBM_D3Q19 && lattice != LBM_D3Q15 && lattice != LBM_D2Q9) return bad("lattice");
    c->q = lattice;
    c->d = lattice == LBM_D2Q9 ? 2 : 3;
    c->ns = lattice == LBM_D2Q9 ? 3 : 6;
    if (nx < 1 || ny < 1 || nz < 1) return bad("dims");
    if (c->d == 2 && nz != 1) return bad("nz");
    if (!rates) return bad("rates");
    if (pin)
        c->p = *pin;
    else
        lbm_default_params(&c->p);
    lbm_params& p = c->p;
    // halo faces (z only, both): the context holds a ghost plane beyond each
    c->halo = (c->d == 3 && p.bc[4] == LBM_HALO && p.bc[5] == LBM_HALO) ? 1 : 0;
    const int nzb = c->halo ? nz + 2 : nz;
    if (ny > 65535 || nzb > 65535) return bad("ny/nz");
    const long long N = (long long)nx * ny * nzb;
    if (N >= (1LL << 31)) return bad("N");
    c->nx = nx;
    c->ny = ny;
    c->nz = nzb;
    c->z0 = c->halo ? 1 : 0;
    c->nzc = nz;
    c->N = N;
    c->stride = (N + 127) / 128 * 128;
    c->hpops = 0;
    for (int i = 0; i < c->q && c->d == 3; ++i) {
        const int cz = c->q == 19 ? lbm::D3Q19::c(i, 2) : lbm::D3Q15::c(i, 2);
        if (cz == 1) c->hpop_up[c->hpops++] = i;
    }
    for (int i = 0, k = 0; i < c->q && c->d == 3; ++i) {
        const int cz = c->q == 19 ? lbm::D3Q19::c(i, 2) : lbm::D3Q15::c(i, 2);
        if (cz == -1) c->hpop_dn[k++] = i;
    }
    for (int k = 0; k < c->q; ++k) {
        const double s = rates[k];
        if (!is_finite(s)) return bad("rate");
        if (is_conserved(c->q, k)) {
            if (s != 0.0) return bad("conserved rate");
        } else if (!(s > 0.0 && s < 2.0)) {
            return bad("rate range");
        }
        c->rates[k] = s;
    }
    for (int d = 0; d < 3; ++d) c->force[d] = (force && d < c->d) ? force[d] : 0.0;
    for (int d = 0; d < 3; ++d)
        if (!is_finite(c->force[d])) return bad("force");
    switch (p.precision) {
        case LBM_FP64: c->elem_bytes = 8; break;
        case LBM_FP32: c->elem_bytes = 4; break;
        case LBM_FP16S:
        case LBM_BF16S: c->elem_bytes = 2; break;
        default: return bad("precision");
    }
    if (tag_of(c->q, p.precision) == T_NONE) return bad("lattice/precision");
    if (p.closure < LBM_NEWTON || p.closure > LBM_SMAG_DEV) return bad("closure");
    if ((p.precision == LBM_FP16S || p.precision == LBM_BF16S) && p.closure != LBM_NEWTON && p.closure != LBM_SMAG)
        return bad("closure for 16-bit storage");
    if (p.formula != LBM_YU && p.formula != LBM_CHAI) return bad("formula");
    if ((p.closure != LBM_NEWTON || p.formula == LBM_YU) && !viscous_rates_equal(c)) return bad("viscous rates");
    if (!(p.rho0 > 0.0) || !is_finite(p.rho0)) return bad("rho0");
    if (p.smag_iters < 1 || p.smag_iters > 64) return bad("smag_iters");
    if (p.pl_max_iter < 1 || p.pl_max_iter > 1000) return bad("pl_max_iter");
    if (!is_finite(p.smag_cs) || p.smag_cs < 0.0) return bad("smag_cs");
    if (p.closure == LBM_POWERLAW) {
        if (!(p.pl_n > 0.0) || !is_finite(p.pl_n) || !(p.pl_k >= 0.0) || !is_finite(p.pl_k)) return bad("power law");
        if (!(p.pl_tau_min > 0.5) || !(p.pl_tau_max >= p.pl_tau_min) || !is_finite(p.pl_tau_max)) return bad("clamp");
    }
    if (p.pl_tol < 0.0) p.pl_tol = p.precision == LBM_FP64 ? 1e-13 : 1e-6;
    if (!is_finite(p.pl_tol)) return bad("pl_tol");
    for (int a = 0; a < c->d; ++a) {
        const int f0 = p.bc[2 * a], f1 = p.bc[2 * a + 1];
        if (a == 2 && (f0 == LBM_HALO || f1 == LBM_HALO)) {
            if (f0 != f1) return bad("bc pair");
            continue;
        }
        if (f0 < LBM_PERIODIC || f0 > LBM_LID || f1 < LBM_PERIODIC || f1 > LBM_LID) return bad("bc");
        if ((f0 == LBM_PERIODIC) != (f1 == LBM_PERIODIC)) return bad("bc pair");
    }
    if (c->d == 2) p.bc[4] = p.bc[5] = LBM_PERIODIC;
    for (int f = 0; f < 6; ++f)
        for (int k = 0; k < 3; ++k)
            if (!is_finite(p.lid_u[f][k])) return bad("lid");
    if (p.force_field != 0 && p.force_field != 1) return bad("force_field");

    // units of the multi-step launch: one z plane times enough rows for about 1024 nodes
    c->stream_rows = nx >= 1024 ? 1 : std::min(ny, 1024 / nx);
    c->stream_tiles = (ny + c->stream_rows - 1) / c->stream_rows;
    c->schedule = LBM_SCHEDULE_AUTO;

    // library-owned scratch for the global sums and the multi-step launch
    cudaError_t e = cudaMalloc(&c->partial, sizeof(double) * (size_t)lbm::SUM_BLOCKS * (1 + c->d));
    if (e == cudaSuccess) e = cudaMalloc(&c->result, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->sync, sizeof(int) * (2 + (size_t)c->nz * c->stream_tiles));
    if (e == cudaSuccess) e = cudaMemset(c->sync, 0, sizeof(int));
    if (e != cudaSuccess) {
        snprintf(create_err, sizeof(create_err), "lbm_create: scratch allocation failed: %s", cudaGetErrorString(e));
        cudaFree(c->partial);
        cudaFree(c->result);
        cudaFree(c->sync);
        delete c;
        return e == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA;
    }
    c->err[0] = '\0';
    *out = c;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_OK;
    cudaFree(c->partial);
    cudaFree(c->result);
    cudaFree(c->sync);
    delete c;
    return LBM_OK;
}

int lbm_stats(const lbm_ctx* c, int64_t* steps, int64_t* step_launches) {
    if (!c) return LBM_ERR_ARG;
    if (steps) *steps = c->n_steps;
    if (step_launches) *step_launches = c->n_step_launches;
    return LBM_OK;
}

int lbm_set_schedule(lbm_ctx* c, int schedule) {
    if (!c) return LBM_ERR_ARG;
    if (schedule != LBM_SCHEDULE_AUTO && schedule != LBM_SCHEDULE_PER_STEP && schedule != LBM_SCHEDULE_STREAM &&
        schedule != LBM_SCHEDULE_STALL_CHECK)
        return fail(c, LBM_ERR_ARG, "lbm_set_schedule: unknown schedule %d", schedule);
    c->schedule = schedule;
    return LBM_OK;
}

int lbm_set_watchdog(lbm_ctx* c, int every, double tol) {
    if (!c) return LBM_ERR_ARG;
    if (every < 0) return fail(c, LBM_ERR_ARG, "lbm_set_watchdog: every < 0");
    if (every > 0 && c->halo) return fail(c, LBM_ERR_ARG, "lbm_set_watchdog: a slab's own totals change by the flux through its halo faces");
    if (every > 0 && !(tol >= 0.0 && is_finite(tol))) return fail(c, LBM_ERR_ARG, "lbm_set_watchdog: tol");
    c->watch_every = every;
    c->watch_tol = tol;
    c->watch_ref_ok = 0;
    return LBM_OK;
}

int lbm_status(lbm_ctx* c) {
    if (!c) return LBM_ERR_ARG;
    if (!c->bound) return LBM_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_status");
    return stream_flag(c);
}

int lbm_layout(const lbm_ctx* c, int* q, int64_t* stride, int* elem_bytes) {
    if (!c) return LBM_ERR_ARG;
    if (q) *q = c->q;
    if (stride) *stride = c->stride;
    if (elem_bytes) *elem_bytes = c->elem_bytes;
    return LBM_OK;
}

int lbm_bind(lbm_ctx* c, void* f_a, void* f_b, const void* force_field, void* stream) {
    if (!c) return LBM_ERR_ARG;
    if (!f_a || !f_b || f_a == f_b) return fail(c, LBM_ERR_ARG, "lbm_bind: need two distinct buffers");
    if (((uintptr_t)f_a | (uintptr_t)f_b) & 15) return fail(c, LBM_ERR_ARG, "lbm_bind: buffers must be 16-byte aligned");
    if (c->p.force_field && !force_field) return fail(c, LBM_ERR_ARG, "lbm_bind: force field required");
    c->buf[0] = f_a;
    c->buf[1] = f_b;
    c->force_field = c->p.force_field ? force_field : nullptr;
    c->stream = static_cast<cudaStream_t>(stream);
    c->bound = 1;
    c->cur = 0;
    c->watch_ref_ok = 0;
    c->err[0] = '\0';
    return LBM_OK;
}

int lbm_bind_tau(lbm_ctx* c, void* tau_field) {
    if (!c) return LBM_ERR_ARG;
    if (!tau_field) return fail(c, LBM_ERR_ARG, "lbm_bind_tau: tau field required");
    if ((uintptr_t)tau_field & (c->p.precision == LBM_FP64 ? 7 : 3))
        return fail(c, LBM_ERR_ARG, "lbm_bind_tau: misaligned tau field");
    c->tau_field = tau_field;
    c->err[0] = '\0';
    return LBM_OK;
}

int lbm_init(lbm_ctx* c, const double* drho, const double* u, const double* grad_u) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!drho || !u) return fail(c, LBM_ERR_ARG, "lbm_init: drho and u are required");
    lbm::StepArgs<double> a;
    fill_args(c, &a);
    set_buffers(c, &a, nullptr, c->buf[c->cur]);
    cudaError_t e;
    void* tf = c->p.closure == LBM_SMAG_LAGGED ? c->tau_field : nullptr;  // only the lagged closure keeps taus
    const Tag t = tag_of(c->q, c->p.precision);
    switch (t) {
        case T_D3Q19_F64:
            e = lbm::init_d3q19_f64(a, c->p.closure, drho, u, grad_u, static_cast<const double*>(c->force_field),
                                    static_cast<double*>(tf), c->stream);
            break;
        case T_D3Q15_F64:
            e = lbm::init_d3q15_f64(a, c->p.closure, drho, u, grad_u, static_cast<const double*>(c->force_field),
                                    static_cast<double*>(tf), c->stream);
            break;
        case T_D3Q15_F32:
            e = lbm::init_d3q15_f32(a, c->p.closure, drho, u, grad_u, static_cast<const float*>(c->force_field),
                                    static_cast<float*>(tf), c->stream);
            break;
        case T_D2Q9_F64:
            e = lbm::init_d2q9_f64(a, c->p.closure, drho, u, grad_u, static_cast<const double*>(c->force_field),
                                    static_cast<double*>(tf), c->stream);
            break;
        case T_D3Q19_F32:
            e = lbm::init_d3q19_f32(a, c->p.closure, drho, u, grad_u, static_cast<const float*>(c->force_field),
                                    static_cast<float*>(tf), c->stream);
            break;
        case T_D3Q19_F16:
            e = lbm::init_d3q19_f16(a, c->p.closure, drho, u, grad_u, static_cast<const float*>(c->force_field),
                                    static_cast<float*>(tf), c->stream);
            break;
        case T_D3Q19_BF16:
            e = lbm::init_d3q19_bf16(a, c->p.closure, drho, u, grad_u, static_cast<const float*>(c->force_field),
                                    static_cast<float*>(tf), c->stream);
            break;
        case T_D3Q15_F16:
            e = lbm::init_d3q15_f16(a, c->p.closure, drho, u, grad_u, static_cast<const float*>(c->force_field),
                                    static_cast<float*>(tf), c->stream);
            break;
        case T_D3Q15_BF16:
            e = lbm::init_d3q15_bf16(a, c->p.closure, drho, u, grad_u, static_cast<const float*>(c->force_field),
                                    static_cast<float*>(tf), c->stream);
            break;
        case T_D2Q9_F32:
            e = lbm::init_d2q9_f32(a, c->p.closure, drho, u, grad_u, static_cast<const float*>(c->force_field),
                                    static_cast<float*>(tf), c->stream);
            break;
        default: return fail(c, LBM_ERR_ARG, "lbm_init: unsupported lattice/precision");
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_init");
    c->watch_ref_ok = 0;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (n < 0) return fail(c, LBM_ERR_ARG, "lbm_step: n < 0");
    if (c->halo && n > 1)
        return fail(c, LBM_ERR_ARG, "lbm_step: a lattice with halo faces takes one step per call (exchange between steps)");
    if (c->watch_every > 0 && n > 0) return step_watched(c, n);
    long long launches = 0;
    cudaError_t e = advance(c, n, &launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step");
    c->n_steps += n;
    c->n_step_launches += launches;
    return LBM_OK;
}

int lbm_strain_rate(lbm_ctx* c, int formula, void* S_out, void* tau_out) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (formula != LBM_YU && formula != LBM_CHAI) return fail(c, LBM_ERR_ARG, "lbm_strain_rate: formula");
    if (!S_out) return fail(c, LBM_ERR_ARG, "lbm_strain_rate: S_out is required");
    if (formula == LBM_YU && !viscous_rates_equal(c))
        return fail(c, LBM_ERR_ARG, "lbm_strain_rate: Yu's formula needs equal viscous rates");
    cudaError_t e = run_step(c, formula, 1, S_out, tau_out, nullptr, nullptr, c->buf[c->cur], nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_strain_rate");
    return LBM_OK;
}

int lbm_macroscopic(lbm_ctx* c, void* drho_out, void* u_out) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!drho_out && !u_out) return LBM_OK;
    cudaError_t e = run_step(c, c->p.formula, 1, nullptr, nullptr, drho_out, u_out, c->buf[c->cur], nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_macroscopic");
    return LBM_OK;
}

int lbm_sums(lbm_ctx* c, double* out) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!out) return fail(c, LBM_ERR_ARG, "lbm_sums: out is required");
    return sums_now(c, out, "lbm_sums");
}

int lbm_get_state(lbm_ctx* c, void* dst) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!dst) return fail(c, LBM_ERR_ARG, "lbm_get_state: dst");
    const size_t row = (size_t)c->N * c->elem_bytes, pitch = (size_t)c->stride * c->elem_bytes;
    cudaError_t e = row == pitch  // contiguous populations: one linear copy
                        ? cudaMemcpyAsync(dst, c->buf[c->cur], row * c->q, cudaMemcpyDefault, c->stream)
                        : cudaMemcpy2DAsync(dst, row, c->buf[c->cur], pitch, row, c->q, cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_get_state");
    return LBM_OK;
}

int lbm_set_state(lbm_ctx* c, const void* src) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!src) return fail(c, LBM_ERR_ARG, "lbm_set_state: src");
    const size_t row = (size_t)c->N * c->elem_bytes, pitch = (size_t)c->stride * c->elem_bytes;
    cudaError_t e = row == pitch
                        ? cudaMemcpyAsync(c->buf[c->cur], src, row * c->q, cudaMemcpyDefault, c->stream)
                        : cudaMemcpy2DAsync(c->buf[c->cur], pitch, src, row, row, c->q, cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_set_state");
    c->watch_ref_ok = 0;
    return LBM_OK;
}

int lbm_halo_layout(const lbm_ctx* c, int* pops, int64_t* elems) {
    if (!c || !c->halo) return LBM_ERR_ARG;
    if (pops) *pops = c->hpops;
    if (elems) *elems = (int64_t)c->hpops * c->nx * c->ny;
    return LBM_OK;
}

int lbm_halo_pack(lbm_ctx* c, void* send_lo, void* send_hi) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!c->halo) return fail(c, LBM_ERR_ARG, "lbm_halo_pack: the lattice has no halo faces");
    if (!send_lo || !send_hi) return fail(c, LBM_ERR_ARG, "lbm_halo_pack: two send buffers are required");
    cudaError_t e = lbm::halo_copy(halo_args(c, send_lo, send_hi), 1, c->elem_bytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_halo_pack");
    return LBM_OK;
}

int lbm_halo_unpack(lbm_ctx* c, const void* recv_lo, const void* recv_hi) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!c->halo) return fail(c, LBM_ERR_ARG, "lbm_halo_unpack: the lattice has no halo faces");
    if (!recv_lo || !recv_hi) return fail(c, LBM_ERR_ARG, "lbm_halo_unpack: two receive buffers are required");
    cudaError_t e = lbm::halo_copy(halo_args(c, const_cast<void*>(recv_lo), const_cast<void*>(recv_hi)), 0,
                                   c->elem_bytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_halo_unpack");
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : create_err; }

int lbm_adjoint_workspace(lbm_ctx* c, int T, int seg, int64_t* bytes) {
    if (!c || !bytes) return LBM_ERR_ARG;
    int rc = adjoint_check(c, T, seg);
    if (rc) return rc;
    if (seg > 1024) return fail(c, LBM_ERR_ARG, "lbm_adjoint: seg <= 1024");
    *bytes = (int64_t)adjoint_layout(c, T, seg).total;
    return LBM_OK;
}

int lbm_adjoint(lbm_ctx* c, int T, int seg, void* work, int64_t work_bytes, double* dLdg, double* loss) {
    int rc = check_bound(c);
    if (rc) return rc;
    rc = adjoint_check(c, T, seg);
    if (rc) return rc;
    if (seg > 1024) return fail(c, LBM_ERR_ARG, "lbm_adjoint: seg <= 1024");
    if (!work || !dLdg || !loss) return fail(c, LBM_ERR_ARG, "lbm_adjoint: work, dLdg and loss are required");
    if ((uintptr_t)work & 255) return fail(c, LBM_ERR_ARG, "lbm_adjoint: workspace must be 256-byte aligned");
    const AdjLayout L = adjoint_layout(c, T, seg);
    if (work_bytes < (int64_t)L.total) return fail(c, LBM_ERR_ARG, "lbm_adjoint: workspace too small");
    cudaError_t e = c->p.precision == LBM_FP64
                        ? adjoint_run<double>(c, T, seg, static_cast<char*>(work), L, dLdg, loss)
                        : adjoint_run<float>(c, T, seg, static_cast<char*>(work), L, dLdg, loss);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_adjoint");
    c->watch_ref_ok = 0;  // the current state is now the one after T steps
    if (!is_finite(*loss)) return fail(c, LBM_ERR_NONFINITE, "lbm_adjoint: non-finite functional");
    return LBM_OK;
}

}  // extern "C"
