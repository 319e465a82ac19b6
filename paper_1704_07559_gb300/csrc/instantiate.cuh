// instantiate.cuh -- defines the launch entry points of launch.h for one (lattice, storage)
// pair.  Included by one small translation unit per pair so the kernels compile in parallel.
#pragma once

#include "launch.h"
#include "step.cuh"

namespace lbm {

// The packed two-node form (VW = 2: float compute, nx even so each thread's pair is 8-byte
// aligned) executes about 0.63x the instructions of the one-node form but needs ~140 registers,
// and at that occupancy it is latency-bound and no faster on GB300; it is compiled out until the
// loads are decoupled from the registers.  One node per thread is dispatched.
constexpr bool kDispatchPairs = false;
template <class ST>
constexpr bool has_pairs() {
    return kDispatchPairs && std::is_same<typename Store<ST>::R, float>::value;
}

template <class L, class ST, int C, int F>
cudaError_t launch_step_cf(const StepArgs<typename Store<ST>::R>& a, int force, cudaStream_t s) {
    dim3 g, b;
    if constexpr (has_pairs<ST>()) {
        if (a.nx % 2 == 0) {
            lattice_grid(a.nx / 2, a.ny, a.nz, &g, &b);
            if (force)
                k_step<L, ST, C, F, true, 2><<<g, b, 0, s>>>(a);
            else
                k_step<L, ST, C, F, false, 2><<<g, b, 0, s>>>(a);
            return cudaGetLastError();
        }
    }
    lattice_grid(a.nx, a.ny, a.nz, &g, &b);
    if (force)
        k_step<L, ST, C, F, true, 1><<<g, b, 0, s>>>(a);
    else
        k_step<L, ST, C, F, false, 1><<<g, b, 0, s>>>(a);
    return cudaGetLastError();
}

template <class L, class ST, bool POWERLAW_BUILT>
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
            if constexpr (POWERLAW_BUILT)
                return yu ? launch_step_cf<L, ST, CL_POWERLAW, F_YU>(a, force, s)
                          : launch_step_cf<L, ST, CL_POWERLAW, F_CHAI>(a, force, s);
            return cudaErrorNotSupported;
        default:
            return cudaErrorInvalidValue;
    }
}

template <class L, class ST>
cudaError_t launch_init(const StepArgs<double>& a, int closure, const double* drho, const double* u, const double* gu,
                        const typename Store<ST>::R* ffield, cudaStream_t s) {
    dim3 g, b;
    lattice_grid(a.nx, a.ny, a.nz, &g, &b);
    k_init<L, ST><<<g, b, 0, s>>>(a, closure, drho, u, gu, ffield);
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

#define LBM_DEFINE_ENTRY(TAG, L, ST, POWERLAW_BUILT)                                                         \
    namespace lbm {                                                                                          \
    cudaError_t step_##TAG(const StepArgs<Store<ST>::R>& a, int closure, int formula, int force,             \
                           cudaStream_t s) {                                                                 \
        return launch_step<L, ST, POWERLAW_BUILT>(a, closure, formula, force, s);                            \
    }                                                                                                        \
    cudaError_t init_##TAG(const StepArgs<double>& a, int closure, const double* drho, const double* u,      \
                           const double* gu, const Store<ST>::R* ffield, cudaStream_t s) {                   \
        return launch_init<L, ST>(a, closure, drho, u, gu, ffield, s);                                       \
    }                                                                                                        \
    cudaError_t sums_##TAG(const StepArgs<Store<ST>::R>& a, double* partial, double* out, cudaStream_t s) {  \
        return launch_sums<L, ST>(a, partial, out, s);                                                       \
    }                                                                                                        \
    }
