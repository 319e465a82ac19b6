// Kernel instantiations for lattice D3Q19 with __half population storage.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d3q19_f16, lbm::D3Q19, __half, false)
