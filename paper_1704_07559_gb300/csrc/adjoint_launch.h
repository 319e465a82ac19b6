// adjoint_launch.h -- host entry points of the adjoint kernels (k_adjoint.cu).
#pragma once

#include <cuda_runtime.h>

#include "launch.h"

namespace lbm {

template <class R>
struct AdjArgs;

int functional_blocks(int nx, int ny, int nz);
cudaError_t adj_functional_f32(const AdjArgs<float>& a, int closure, cudaStream_t s, int* nblocks);
cudaError_t adj_functional_f64(const AdjArgs<double>& a, int closure, cudaStream_t s, int* nblocks);
cudaError_t adj_step_f32(const AdjArgs<float>& a, int closure, cudaStream_t s);
cudaError_t adj_step_f64(const AdjArgs<double>& a, int closure, cudaStream_t s);
// several reverse steps per launch (FP32; see k_adjoint_stream); cudaErrorNotSupported when the
// schedule's policy declines, the caller then launches step by step
cudaError_t adj_stream_f32(const AdjArgs<float>& a0, const AdjArgs<float>& a1, const StreamCtl& c, int closure,
                           int force_stream, cudaStream_t s);
cudaError_t adj_fold_f32(float* dF, double* dLdg, double rho0, long long n, cudaStream_t s);
cudaError_t adj_fold_f64(double* dF, double* dLdg, double rho0, long long n, cudaStream_t s);

}  // namespace lbm
