// noalloc.cu -- lbm_sums_noalloc: the global mass / momentum sums without any allocation.
//
// The regular lbm_sums needs a context from lbm_create, which allocates its partial-sum scratch
// with cudaMalloc.  Some callers cannot allocate device memory when they need the sums: code
// whose device memory is owned by another allocator (a framework's caching pool that must not
// be bypassed), or a time-stepping loop with a latency budget, where cudaMalloc / cudaFree can
// synchronise the device and take unbounded time.  This entry point runs the same sum kernels
// on caller-owned inputs, and keeps its scratch in a fixed static device array instead.
//
// Scratch: one static __device__ array per GPU that loads this library, held until the process
// exits.  It holds at most LBM_NOALLOC_MAX_BLOCKS partial rows of up to four doubles plus the
// four-double result.  Every call writes each slot it later reads, so nothing needs clearing
// between calls; but all calls share the one array, so calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/lbm.h"
#include "launch.h"
#include "step.cuh"

namespace {

constexpr int ROWS_PER_BLOCK = LBM_NOALLOC_MAX_ROWS / LBM_NOALLOC_MAX_BLOCKS;
constexpr int MAX_BLOCKS = LBM_NOALLOC_MAX_BLOCKS;
constexpr int WIDTH = 4;  // 1 + d for the widest lattice

// the scratch: partial rows, then the final row of sums
static __device__ __align__(256) double g_noalloc_scratch[MAX_BLOCKS * WIDTH + WIDTH];

// Device address of the static scratch on the current device.  In host code the array's name is
// only a host-side stand-in, so the address is looked up, on every call: the lookup allocates
// nothing and costs little, and an address kept from an earlier call could be stale after a
// device reset (the module, and with it the array, is loaded again in the new context).
cudaError_t scratch_for_current_device(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

template <class L, class ST>
cudaError_t run(const lbm::StepArgs<typename lbm::Store<ST>::R>& a, int blocks, double* scratch, cudaStream_t s) {
    lbm::k_sums<L, ST><<<blocks, lbm::SUM_THREADS, 0, s>>>(a, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lbm::k_sums_final<<<1, 256, 0, s>>>(scratch, blocks, 1 + L::D, scratch + MAX_BLOCKS * WIDTH);
    return cudaGetLastError();
}

template <class R>
void fill(lbm::StepArgs<R>* a, int q, int nx, int ny, int nz, const lbm_params* p, const double* force,
          const void* f, int64_t stride, int elem, const void* ffield) {
    *a = lbm::StepArgs<R>{};
    a->nx = nx;
    a->ny = ny;
    a->nz = nz;
    a->z0 = 0;
    a->nzc = nz;
    a->stride = stride;
    a->src = f;
    for (int i = 0; i < q; ++i) a->srcp[i] = static_cast<const char*>(f) + (size_t)i * stride * elem;
    const int d = q == LBM_D2Q9 ? 2 : 3;
    for (int k = 0; k < 3; ++k) a->F[k] = R((force && k < d) ? force[k] : 0.0);
    a->rho0 = R(p->rho0);
    a->inv_rho0 = R(1.0 / p->rho0);
    int wall = 0, lid = 0;
    for (int fc = 0; fc < 2 * d; ++fc) {
        if (p->bc[fc] != LBM_PERIODIC) wall |= 1 << fc;
        if (p->bc[fc] == LBM_LID) lid |= 1 << fc;
        for (int k = 0; k < 3; ++k) a->lid[fc][k] = R(p->lid_u[fc][k]);
    }
    a->wall_mask = wall;
    a->lid_mask = lid;
    a->force_field = static_cast<const R*>(ffield);
}

}  // namespace

extern "C" int lbm_sums_noalloc(int lattice, int nx, int ny, int nz, const lbm_params* p, const double* force,
                                const void* f, int64_t stride, const void* force_field, double* out, void* stream) {
    // argument checks first: a rejected call touches no CUDA state
    if ((lattice != LBM_D3Q19 && lattice != LBM_D3Q15 && lattice != LBM_D2Q9) || !p || !f || !out) return LBM_ERR_ARG;
    const int d = lattice == LBM_D2Q9 ? 2 : 3;
    if (nx < 1 || ny < 1 || nz < 1 || (d == 2 && nz != 1) || ny > 65535 || nz > 65535) return LBM_ERR_ARG;
    const long long N = (long long)nx * ny * nz;
    if (N >= (1LL << 31) || stride < N) return LBM_ERR_ARG;
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) return LBM_ERR_ARG;
    for (int a = 0; a < d; ++a)
        if (force && !std::isfinite(force[a])) return LBM_ERR_ARG;
    for (int fc = 0; fc < 2 * d; ++fc)
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(p->lid_u[fc][k])) return LBM_ERR_ARG;
    for (int a = 0; a < d; ++a) {
        const int f0 = p->bc[2 * a], f1 = p->bc[2 * a + 1];
        if (f0 < LBM_PERIODIC || f0 > LBM_LID || f1 < LBM_PERIODIC || f1 > LBM_LID) return LBM_ERR_ARG;
        if ((f0 == LBM_PERIODIC) != (f1 == LBM_PERIODIC)) return LBM_ERR_ARG;
    }
    const long long rows = (long long)ny * nz;
    const long long blocks = (rows + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
    if (blocks > MAX_BLOCKS) return LBM_ERR_ARG;  // more than LBM_NOALLOC_MAX_ROWS rows (ny * nz)
    int elem;
    switch (p->precision) {
        case LBM_FP64: elem = 8; break;
        case LBM_FP32: elem = 4; break;
        case LBM_FP16S:
        case LBM_BF16S: elem = 2; break;
        default: return LBM_ERR_ARG;
    }
    if (lattice == LBM_D2Q9 && elem == 2) return LBM_ERR_ARG;

    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return LBM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const int nb = (int)blocks;
    if (p->precision == LBM_FP64) {
        lbm::StepArgs<double> a;
        fill(&a, lattice, nx, ny, nz, p, force, f, stride, elem, force_field);
        e = lattice == LBM_D3Q19   ? run<lbm::D3Q19, double>(a, nb, scratch, s)
            : lattice == LBM_D3Q15 ? run<lbm::D3Q15, double>(a, nb, scratch, s)
                                   : run<lbm::D2Q9, double>(a, nb, scratch, s);
    } else {
        lbm::StepArgs<float> a;
        fill(&a, lattice, nx, ny, nz, p, force, f, stride, elem, force_field);
        if (lattice == LBM_D2Q9)
            e = run<lbm::D2Q9, float>(a, nb, scratch, s);
        else if (lattice == LBM_D3Q15)
            e = p->precision == LBM_FP32    ? run<lbm::D3Q15, float>(a, nb, scratch, s)
                : p->precision == LBM_FP16S ? run<lbm::D3Q15, __half>(a, nb, scratch, s)
                                            : run<lbm::D3Q15, __nv_bfloat16>(a, nb, scratch, s);
        else if (p->precision == LBM_FP32)
            e = run<lbm::D3Q19, float>(a, nb, scratch, s);
        else if (p->precision == LBM_FP16S)
            e = run<lbm::D3Q19, __half>(a, nb, scratch, s);
        else
            e = run<lbm::D3Q19, __nv_bfloat16>(a, nb, scratch, s);
    }
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    e = cudaMemcpyAsync(out, scratch + MAX_BLOCKS * WIDTH, sizeof(double) * (1 + d), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    for (int k = 0; k <= d; ++k)
        if (!(out[k] == out[k]) || out[k] - out[k] != 0.0) return LBM_ERR_NONFINITE;
    return LBM_OK;
}
