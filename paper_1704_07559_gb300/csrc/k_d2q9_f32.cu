// Kernel instantiations for lattice D2Q9 with float population storage.
#include "instantiate.cuh"
LBM_DEFINE_ENTRY(d2q9_f32, lbm::D2Q9, float, true)
