// Multi-step (streamed) kernel instantiations for lattice D3Q19 with float population storage.
#include "step_stream.cuh"
LBM_DEFINE_STREAM_ENTRY(d3q19_f32, lbm::D3Q19, float, true)
LBM_DEFINE_STREAM_RING_ENTRY(d3q19_f32, lbm::D3Q19, float)
