// adjoint_launch.h -- host entry points of the adjoint kernels (k_adjoint.cu).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

template <class R>
struct AdjArgs;

int functional_blocks(int nx, int ny, int nz);
cudaError_t adj_functional_f32(const AdjArgs<float>& a, int closure, cudaStream_t s, int* nblocks);
cudaError_t adj_functional_f64(const AdjArgs<double>& a, int closure, cudaStream_t s, int* nblocks);
cudaError_t adj_step_f32(const AdjArgs<float>& a, int closure, cudaStream_t s);
cudaError_t adj_step_f64(const AdjArgs<double>& a, int closure, cudaStream_t s);
cudaError_t adj_fold_f32(float* dF, double* dLdg, double rho0, long long n, cudaStream_t s);
cudaError_t adj_fold_f64(double* dF, double* dLdg, double rho0, long long n, cudaStream_t s);

}  // namespace lbm
