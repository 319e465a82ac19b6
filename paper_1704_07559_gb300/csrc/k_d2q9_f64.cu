// Kernel instantiations for lattice D2Q9 with double population storage.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d2q9_f64, lbm::D2Q9, double, true)
