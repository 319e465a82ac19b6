// instantiate.cuh -- defines the launch entry points of launch.h for one (lattice, storage)
// pair.  Included by one small translation unit per pair so the kernels compile in parallel.
#pragma once

#include "launch.h"
#include "step.cuh"
#include "step_async.cuh"

namespace lbm {

// Step kernel selection for the float compute types (FP32, FP16S, BF16S):
//   LBM_STEP_FORM 0: one node per thread, direct loads (k_step, VW = 1); for 16-bit storage with
//                    nx even, k_step_pair_seq (form 6) instead;
//   LBM_STEP_FORM 1: persistent double-buffered k_step_async, one node per thread;
//   LBM_STEP_FORM 2: persistent double-buffered k_step_async, two nodes per thread in packed
//                    FP32 pairs when nx is even (one node per thread otherwise);
//   LBM_STEP_FORM 3: persistent k_step_prefetch (next node's loads in registers), one node;
//   LBM_STEP_FORM 4: persistent k_step_prefetch, two nodes per thread when nx is even;
//   LBM_STEP_FORM 5: k_step_pair, two nodes per thread in packed FP32 pairs when nx is even;
//   LBM_STEP_FORM 6: k_step_pair_seq, two nodes per thread sharing the pull, collided one after
//                    the other in scalar arithmetic, when nx is even.
// FP64 always uses k_step (its arithmetic, not its loads, bounds it).
#ifndef LBM_STEP_FORM
#define LBM_STEP_FORM 0
#endif

template <class ST>
constexpr bool float_compute() {
    return std::is_same<typename Store<ST>::R, float>::value;
}

template <class L, class ST, int C, int F, bool FO, int VW, bool PREFETCH>
cudaError_t launch_async(const StepArgs<typename Store<ST>::R>& a, cudaStream_t s) {
    const int nseg = (a.nx + ASYNC_THREADS * VW - 1) / (ASYNC_THREADS * VW);
    const long long tiles = (long long)nseg * a.ny * a.nz;
    const int smem = PREFETCH ? 0 : 2 * L::Q * ASYNC_THREADS * slot_bytes<ST, VW>();
    static int per_sm = 0, sms = 0;  // occupancy of this instantiation, found once
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (PREFETCH)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_prefetch<L, ST, C, F, FO, VW>, ASYNC_THREADS, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_async<L, ST, C, F, FO, VW>, ASYNC_THREADS, smem);
        if (per_sm < 1) per_sm = 1;
    }
    const long long want = (long long)per_sm * sms;
    const int grid = (int)(tiles < want ? tiles : want);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    if constexpr (PREFETCH)
        k_step_prefetch<L, ST, C, F, FO, VW><<<grid, ASYNC_THREADS, 0, s>>>(a, nseg, (int)tiles);
    else
        k_step_async<L, ST, C, F, FO, VW><<<grid, ASYNC_THREADS, smem, s>>>(a, nseg, (int)tiles);
    return cudaGetLastError();
}

template <class L, class ST, int C, int F, bool FO>
cudaError_t launch_form(const StepArgs<typename Store<ST>::R>& a, cudaStream_t s) {
    // 16-bit storage (issue-bound): two nodes per thread sharing the pull when nx is even
    // (measured 3-12% faster than one node per thread; slower for FP32, which stays one per thread)
    if constexpr (sizeof(ST) == 2 && LBM_STEP_FORM == 0) {
        if (!a.readout && a.nx % 2 == 0) {
            dim3 g, b;
            lattice_grid(a.nx / 2, a.ny, a.nz, &g, &b);
            return launch_pdl(k_step_pair_seq<L, ST, C, F, FO>, g, b, s, a);
        }
    }
    if constexpr (float_compute<ST>() && LBM_STEP_FORM != 0) {
        if (LBM_STEP_FORM == 5 && !a.readout && a.nx % 2 == 0) {
            dim3 g, b;
            lattice_grid(a.nx / 2, a.ny, a.nz, &g, &b);
            return launch_pdl(k_step_pair<L, ST, C, F, FO>, g, b, s, a);
        }
        if (LBM_STEP_FORM == 6 && !a.readout && a.nx % 2 == 0) {
            dim3 g, b;
            lattice_grid(a.nx / 2, a.ny, a.nz, &g, &b);
            return launch_pdl(k_step_pair_seq<L, ST, C, F, FO>, g, b, s, a);
        }
        if (LBM_STEP_FORM < 5 && !a.readout) {
            constexpr bool PF = LBM_STEP_FORM >= 3;
            constexpr bool PAIRS = LBM_STEP_FORM == 2 || LBM_STEP_FORM == 4;
            if (PAIRS && a.nx % 2 == 0) return launch_async<L, ST, C, F, FO, 2, PF>(a, s);
            return launch_async<L, ST, C, F, FO, 1, PF>(a, s);
        }
    }
    dim3 g, b;
    lattice_grid(a.nx, a.ny, a.nz, &g, &b);
    return launch_pdl(k_step<L, ST, C, F, FO, 1>, g, b, s, a);
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
    lattice_grid(a.nx, a.ny, a.nz, &g, &b);
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
