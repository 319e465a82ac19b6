// launch.h -- host-side entry points into the kernel instantiations, one set per
// (lattice, storage precision).  Each returns the CUDA status of its launches.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

template <class R>
struct StepArgs;

// geometry of a lattice launch: 128-thread blocks covering x (and several y rows when nx is small)
inline void lattice_grid(int nx, int ny, int nz, dim3* grid, dim3* block) {
    const int bx = nx <= 32 ? 32 : (nx <= 64 ? 64 : 128);
    const int by = 128 / bx;
    *block = dim3(bx, by, 1);
    *grid = dim3((nx + bx - 1) / bx, (ny + by - 1) / by, nz);
}

// Programmatic dependent launch of a step (or adjoint step) kernel: consecutive steps overlap launch and block
// scheduling with the previous step's tail (the kernel waits for the previous one before its
// first load).
template <class K, class A>
cudaError_t launch_pdl(K kernel, dim3 g, dim3 b, cudaStream_t s, const A& a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

// Several steps in one launch (step_stream.cuh): the library-owned synchronisation words and the
// unit geometry.  sync[0] is a sticky error flag (a dependency wait ran out), sync[1] the ticket
// counter and sync[2 + z * tiles_y + ty] the number of steps unit (z, ty) has completed (room for
// nz * tiles_y units at the given rows); the launcher zeroes sync[1 ..] before each launch.
struct StreamCtl {
    int* sync;
    int steps;       // steps in this launch
    int rows;        // lattice rows (y) per unit (the launcher may take a multiple)
    int tiles_y;     // units per z plane: ceil(ny / rows)
    int first_step;  // 0; 1 only for the diagnostic that makes every dependency wait run out
    long long ring;  // 0: two buffers; else step k's buffers are the first ones shifted by k * ring elements
};

constexpr int SUM_BLOCKS = 608;  // 4 blocks per SM on 152 SMs; partial rows in scratch

// The populations crossing the z faces of a slab (k_halo.cu): population up[k] (c_z = +1) of the
// top own plane z_hi and population dn[k] (c_z = -1) of the bottom own plane z_lo, each plane
// `plane` elements; lo / hi hold pops * plane elements.  A pack copies the own planes into hi (up)
// and lo (dn); an unpack copies lo into population up[k] of ghost plane z_lo - 1 and hi into
// population dn[k] of ghost plane z_hi + 1.
struct HaloArgs {
    char* buf;         // population buffer
    long long pitch;   // bytes between population arrays
    long long plane;   // elements of one z plane (nx ny)
    int pops;          // populations crossing each face
    int up[5], dn[5];
    int z_lo, z_hi;    // bottom and top own planes
    char* lo;
    char* hi;
};
// pack (1) or unpack (0), elements of elem_bytes bytes
cudaError_t halo_copy(const HaloArgs& h, int pack, int elem_bytes, cudaStream_t s);

#define LBM_DECLARE_ENTRY(TAG, R)                                                                         \
    cudaError_t step_##TAG(const StepArgs<R>& a, int closure, int formula, int force, cudaStream_t s);   \
    cudaError_t init_##TAG(const StepArgs<double>& a, int closure, const double* drho, const double* u, \
                           const double* gu, const R* ffield, R* tau_field, cudaStream_t s);             \
    cudaError_t sums_##TAG(const StepArgs<R>& a, double* partial, double* out, cudaStream_t s);

#define LBM_DECLARE_STREAM_ENTRY(TAG, R)                                                                      \
    cudaError_t stream_##TAG(const StepArgs<R>& a0, const StepArgs<R>& a1, const StreamCtl& c, int closure, \
                             int formula, int force, int force_stream, cudaStream_t s);
LBM_DECLARE_STREAM_ENTRY(d3q19_f32, float)
LBM_DECLARE_STREAM_ENTRY(d3q19_f16, float)
LBM_DECLARE_STREAM_ENTRY(d3q19_bf16, float)
LBM_DECLARE_STREAM_ENTRY(d3q15_f32, float)
LBM_DECLARE_STREAM_ENTRY(d3q15_f16, float)
LBM_DECLARE_STREAM_ENTRY(d3q15_bf16, float)
LBM_DECLARE_STREAM_ENTRY(d2q9_f32, float)
#undef LBM_DECLARE_STREAM_ENTRY
// ring launches (each step writes a buffer of its own): D3Q19 FP32, Newtonian and Smagorinsky
cudaError_t stream_ring_d3q19_f32(const StepArgs<float>& a, const StreamCtl& c, int closure, int formula, int force,
                                  int force_stream, cudaStream_t s);

LBM_DECLARE_ENTRY(d3q19_f64, double)
LBM_DECLARE_ENTRY(d3q19_f32, float)
LBM_DECLARE_ENTRY(d3q19_f16, float)
LBM_DECLARE_ENTRY(d3q19_bf16, float)
LBM_DECLARE_ENTRY(d3q15_f64, double)
LBM_DECLARE_ENTRY(d3q15_f32, float)
LBM_DECLARE_ENTRY(d3q15_f16, float)
LBM_DECLARE_ENTRY(d3q15_bf16, float)
LBM_DECLARE_ENTRY(d2q9_f64, double)
LBM_DECLARE_ENTRY(d2q9_f32, float)

#undef LBM_DECLARE_ENTRY

}  // namespace lbm
