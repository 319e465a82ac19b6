// Kernel instantiations for lattice D3Q15 with bfloat16 storage of the delta-rho populations.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d3q15_bf16, lbm::D3Q15, __nv_bfloat16, false)
