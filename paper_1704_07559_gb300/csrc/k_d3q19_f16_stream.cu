// Multi-step (streamed) kernel instantiations for lattice D3Q19 with __half population storage.
#include "step_stream.cuh"
LBM_DEFINE_STREAM_ENTRY(d3q19_f16, lbm::D3Q19, __half, false)
