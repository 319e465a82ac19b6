// Kernel instantiations for lattice D3Q19 with double population storage.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d3q19_f64, lbm::D3Q19, double, true)
