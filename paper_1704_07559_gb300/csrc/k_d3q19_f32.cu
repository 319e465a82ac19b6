// Kernel instantiations for lattice D3Q19 with float population storage.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d3q19_f32, lbm::D3Q19, float, true)
