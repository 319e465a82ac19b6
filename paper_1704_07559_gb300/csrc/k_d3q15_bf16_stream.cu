// Multi-step (streamed) kernel instantiations for lattice D3Q15 with __nv_bfloat16 population storage.
#include "step_stream.cuh"
LBM_DEFINE_STREAM_ENTRY(d3q15_bf16, lbm::D3Q15, __nv_bfloat16, false)
