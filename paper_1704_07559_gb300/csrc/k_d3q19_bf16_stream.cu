// Multi-step (streamed) kernel instantiations for lattice D3Q19 with __nv_bfloat16 population storage.
#include "step_stream.cuh"
LBM_DEFINE_STREAM_ENTRY(d3q19_bf16, lbm::D3Q19, __nv_bfloat16, false)
