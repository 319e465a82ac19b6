// Multi-step (streamed) kernel instantiations for lattice D2Q9 with float population storage.
#include "step_stream.cuh"
LBM_DEFINE_STREAM_ENTRY(d2q9_f32, lbm::D2Q9, float, true)
