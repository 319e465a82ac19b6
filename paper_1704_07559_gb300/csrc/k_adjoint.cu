// Adjoint kernel instantiations: D3Q19 with FP32 (FP64 accumulation of the force gradient)
// and FP64 populations, Newtonian and Smagorinsky closures.
#include "adjoint.cuh"
#include "adjoint_launch.h"
#include "launch.h"

namespace lbm {

template <class ST>
static cudaError_t functional_impl(const AdjArgs<typename Store<ST>::R>& a, int closure, cudaStream_t s, int* nblocks) {
    dim3 g, b;
    lattice_grid(a.st.nx, a.st.ny, a.st.nz, &g, &b);
    *nblocks = g.x * g.y * g.z;
    if (closure == CL_SMAG)
        k_functional<ST, CL_SMAG><<<g, b, 0, s>>>(a);
    else
        k_functional<ST, CL_NEWTON><<<g, b, 0, s>>>(a);
    return cudaGetLastError();
}

template <class ST>
static cudaError_t step_impl(const AdjArgs<typename Store<ST>::R>& a, int closure, cudaStream_t s) {
    dim3 g, b;
    lattice_grid(a.st.nx, a.st.ny, a.st.nz, &g, &b);
    if (closure == CL_SMAG) return launch_pdl(k_adjoint_step<ST, CL_SMAG>, g, b, s, a);
    return launch_pdl(k_adjoint_step<ST, CL_NEWTON>, g, b, s, a);
}

template <class R>
static cudaError_t fold_impl(R* dF, double* dLdg, double rho0, long long n, cudaStream_t s) {
    k_fold<R><<<4 * 152, 256, 0, s>>>(dF, dLdg, rho0, n);
    return cudaGetLastError();
}

int functional_blocks(int nx, int ny, int nz) {
    dim3 g, b;
    lattice_grid(nx, ny, nz, &g, &b);
    return g.x * g.y * g.z;
}

cudaError_t adj_functional_f32(const AdjArgs<float>& a, int closure, cudaStream_t s, int* nb) {
    return functional_impl<float>(a, closure, s, nb);
}
cudaError_t adj_functional_f64(const AdjArgs<double>& a, int closure, cudaStream_t s, int* nb) {
    return functional_impl<double>(a, closure, s, nb);
}
cudaError_t adj_step_f32(const AdjArgs<float>& a, int closure, cudaStream_t s) { return step_impl<float>(a, closure, s); }
cudaError_t adj_step_f64(const AdjArgs<double>& a, int closure, cudaStream_t s) { return step_impl<double>(a, closure, s); }
cudaError_t adj_fold_f32(float* dF, double* dLdg, double rho0, long long n, cudaStream_t s) {
    return fold_impl<float>(dF, dLdg, rho0, n, s);
}
cudaError_t adj_fold_f64(double* dF, double* dLdg, double rho0, long long n, cudaStream_t s) {
    return fold_impl<double>(dF, dLdg, rho0, n, s);
}

}  // namespace lbm
