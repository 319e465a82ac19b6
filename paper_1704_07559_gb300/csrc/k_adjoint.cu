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

// several adjoint steps per launch, with the forward multi-step launch's policy: lattices up to
// 2^23 nodes with enough units that no block waits, unless forced
template <int CLOSURE>
static cudaError_t stream_impl(const AdjArgs<float>& a0, const AdjArgs<float>& a1, const StreamCtl& c,
                               bool force_stream, cudaStream_t s) {
    const long long N = (long long)a0.st.nx * a0.st.ny * a0.st.nz;
    if (!force_stream && N > (1LL << 23)) return cudaErrorNotSupported;
    static const int resident = resident_blocks(k_adjoint_stream<float, CLOSURE>);
    StreamCtl u;
    if (!pick_units(c, a0.st.ny, a0.st.nz, resident, &u) && !force_stream) return cudaErrorNotSupported;
    const long long total = (long long)a0.st.nz * u.tiles_y * u.steps;
    if (total >= (1LL << 31) || u.steps < 1) return cudaErrorInvalidValue;
    const int grid = (int)(total < resident ? total : resident);
    cudaError_t e = cudaMemsetAsync(u.sync + 1, 0, sizeof(int) * (1 + (size_t)a0.st.nz * u.tiles_y), s);
    if (e != cudaSuccess) return e;
    k_adjoint_stream<float, CLOSURE><<<grid, 128, 0, s>>>(a0, a1, u);
    return cudaGetLastError();
}

cudaError_t adj_stream_f32(const AdjArgs<float>& a0, const AdjArgs<float>& a1, const StreamCtl& c, int closure,
                           int force_stream, cudaStream_t s) {
    if (closure == CL_SMAG) return stream_impl<CL_SMAG>(a0, a1, c, force_stream != 0, s);
    if (closure == CL_NEWTON) return stream_impl<CL_NEWTON>(a0, a1, c, force_stream != 0, s);
    return cudaErrorNotSupported;
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
