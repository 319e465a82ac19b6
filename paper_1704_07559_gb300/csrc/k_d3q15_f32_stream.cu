// Multi-step (streamed) kernel instantiations for lattice D3Q15 with float population storage.
#include "step_stream.cuh"
LBM_DEFINE_STREAM_ENTRY(d3q15_f32, lbm::D3Q15, float, true)
