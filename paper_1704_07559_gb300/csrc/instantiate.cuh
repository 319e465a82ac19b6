// instantiate.cuh -- defines the launch entry points of launch.h for one (lattice, storage)
// pair.  Included by one small translation unit per pair so the kernels compile in parallel.
#pragma once

#include "launch.h"
#include "step.cuh"
#include "step_pair.cuh"

namespace lbm {

// Step kernel selection: one node per thread (k_step), except 16-bit storage with nx even and no
// read-out, which runs two x-adjacent nodes per thread in packed FP32-pair arithmetic
// (k_step_pair_seq, step_pair.cuh: the 16-bit step is issue-bound, and the shared pull and the
// pair instructions halve its arithmetic per node).  FP32 storage stays one node per thread: its
// step already runs at the HBM bound, and it keeps the delta form, whose FP32 rounding acts on
// the collision increment only; FP64 is bound by its arithmetic.
template <class L, class ST, int C, int F, bool FO>
cudaError_t launch_form(const StepArgs<typename Store<ST>::R>& a, cudaStream_t s) {
    if constexpr (sizeof(ST) == 2) {
        if (!a.readout && a.nx % 2 == 0) {
            dim3 g, b;
            lattice_grid(a.nx / 2, a.ny, a.nzc, &g, &b);
            return launch_pdl(k_step_pair_seq<L, ST, C, F, FO>, g, b, s, a);
        }
    }
    dim3 g, b;
    lattice_grid(a.nx, a.ny, a.nzc, &g, &b);
    return launch_pdl(k_step<L, ST, C, F, FO>, g, b, s, a);
}

template <class L, class ST, int C, int F>
cudaError_t launch_step_cf(const StepArgs<typename Store<ST>::R>& a, int force, cudaStream_t s) {
    return force ? launch_form<L, ST, C, F, true>(a, s) : launch_form<L, ST, C, F, false>(a, s);
}

// EXTRA_CLOSURES: the power law and the two Smagorinsky variants (lagged, deviatoric) are
// instantiated (FP32 and FP64 storage); 16-bit storage builds Newtonian and Smagorinsky only.
template <class L, class ST, bool EXTRA_CLOSURES>
cudaError_t launch_step(const StepArgs<typename Store<ST>::R>& a, int closure, int formula, int force,
                        cudaStream_t s) {
    const bool yu = formula == F_YU;
    switch (closure) {
        case CL_NEWTON:
            return yu ? launch_step_cf<L, ST, CL_NEWTON, F_YU>(a, force, s)
                      : launch_step_cf<L, ST, CL_NEWTON, F_CHAI>(a, force, s);
        case CL_SMAG:
            return yu ? launch_step_cf<L, ST, CL_SMAG, F_YU>(a, force, s)
                      : launch_step_cf<L, ST, CL_SMAG, F_CHAI>(a, force, s);
        case CL_POWERLAW:
            if constexpr (EXTRA_CLOSURES)
                return yu ? launch_step_cf<L, ST, CL_POWERLAW, F_YU>(a, force, s)
                          : launch_step_cf<L, ST, CL_POWERLAW, F_CHAI>(a, force, s);
            return cudaErrorNotSupported;
        case CL_SMAG_LAGGED:
            if constexpr (EXTRA_CLOSURES)
                return yu ? launch_step_cf<L, ST, CL_SMAG_LAGGED, F_YU>(a, force, s)
                          : launch_step_cf<L, ST, CL_SMAG_LAGGED, F_CHAI>(a, force, s);
            return cudaErrorNotSupported;
        case CL_SMAG_DEV:
            if constexpr (EXTRA_CLOSURES)
                return yu ? launch_step_cf<L, ST, CL_SMAG_DEV, F_YU>(a, force, s)
                          : launch_step_cf<L, ST, CL_SMAG_DEV, F_CHAI>(a, force, s);
            return cudaErrorNotSupported;
        default:
            return cudaErrorInvalidValue;
    }
}

template <class L, class ST>
cudaError_t launch_init(const StepArgs<double>& a, int closure, const double* drho, const double* u, const double* gu,
                        const typename Store<ST>::R* ffield, typename Store<ST>::R* tau_field, cudaStream_t s) {
    dim3 g, b;
    lattice_grid(a.nx, a.ny, a.nzc, &g, &b);
    k_init<L, ST><<<g, b, 0, s>>>(a, closure, drho, u, gu, ffield, tau_field);
    return cudaGetLastError();
}

template <class L, class ST>
cudaError_t launch_sums(const StepArgs<typename Store<ST>::R>& a, double* partial, double* out, cudaStream_t s) {
    k_sums<L, ST><<<SUM_BLOCKS, SUM_THREADS, 0, s>>>(a, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sums_final<<<1, 256, 0, s>>>(partial, SUM_BLOCKS, 1 + L::D, out);
    return cudaGetLastError();
}

}  // namespace lbm

#define LBM_DEFINE_ENTRY(TAG, L, ST, EXTRA_CLOSURES)                                                         \
    namespace lbm {                                                                                          \
    cudaError_t step_##TAG(const StepArgs<Store<ST>::R>& a, int closure, int formula, int force,             \
                           cudaStream_t s) {                                                                 \
        return launch_step<L, ST, EXTRA_CLOSURES>(a, closure, formula, force, s);                            \
    }                                                                                                        \
    cudaError_t init_##TAG(const StepArgs<double>& a, int closure, const double* drho, const double* u,      \
                           const double* gu, const Store<ST>::R* ffield, Store<ST>::R* tau_field,            \
                           cudaStream_t s) {                                                                 \
        return launch_init<L, ST>(a, closure, drho, u, gu, ffield, tau_field, s);                            \
    }                                                                                                        \
    cudaError_t sums_##TAG(const StepArgs<Store<ST>::R>& a, double* partial, double* out, cudaStream_t s) {  \
        return launch_sums<L, ST>(a, partial, out, s);                                                       \
    }                                                                                                        \
    }
