// k_halo.cu -- the exchange copies of a z-slab (lbm_halo_pack / lbm_halo_unpack): the
// post-collision populations that the neighbouring slabs pull across the two z faces.
#include <cuda_runtime.h>

#include <stdint.h>

#include "launch.h"

namespace lbm {

// blockIdx.y: the crossing population k; blockIdx.z: 0 the lower face (dn / lo), 1 the upper
// face (up / hi)
template <class E>
__global__ void __launch_bounds__(256) k_halo(const HaloArgs h, int pack) {
    const int k = blockIdx.y;
    const bool upper = blockIdx.z == 1;
    const int pop = upper ? h.up[k] : h.dn[k];
    // own plane (pack source) or ghost plane (unpack destination)
    const int z = pack ? (upper ? h.z_hi : h.z_lo) : (upper ? h.z_lo - 1 : h.z_hi + 1);
    // an unpack writes lo (the lower neighbour's upper face) into the lower ghost plane and hi
    // into the upper one
    const bool lo_buf = pack ? !upper : upper;
    E* plane = reinterpret_cast<E*>(h.buf + pop * h.pitch) + z * h.plane;
    E* halo = reinterpret_cast<E*>(lo_buf ? h.lo : h.hi) + k * h.plane;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < h.plane;
         i += (long long)gridDim.x * blockDim.x) {
        if (pack)
            halo[i] = plane[i];
        else
            plane[i] = halo[i];
    }
}

cudaError_t halo_copy(const HaloArgs& h, int pack, int elem_bytes, cudaStream_t s) {
    const long long blocks = (h.plane + 255) / 256;
    const dim3 grid((unsigned)(blocks < 1024 ? blocks : 1024), h.pops, 2);
    switch (elem_bytes) {
        case 2: k_halo<uint16_t><<<grid, 256, 0, s>>>(h, pack); break;
        case 4: k_halo<uint32_t><<<grid, 256, 0, s>>>(h, pack); break;
        case 8: k_halo<uint64_t><<<grid, 256, 0, s>>>(h, pack); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbm
