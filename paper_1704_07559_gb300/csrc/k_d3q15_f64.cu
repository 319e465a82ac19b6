// Kernel instantiations for lattice D3Q15 with double population storage.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d3q15_f64, lbm::D3Q15, double, true)
