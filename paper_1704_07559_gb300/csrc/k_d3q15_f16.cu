// Kernel instantiations for lattice D3Q15 with IEEE half storage of the delta-rho populations.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d3q15_f16, lbm::D3Q15, __half, false)
