// Kernel instantiations for lattice D3Q19 with __nv_bfloat16 population storage.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d3q19_bf16, lbm::D3Q19, __nv_bfloat16, false)
