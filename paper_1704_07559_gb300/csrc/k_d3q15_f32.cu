// Kernel instantiations for lattice D3Q15 with float population storage.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d3q15_f32, lbm::D3Q15, float, true)
