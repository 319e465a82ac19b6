// step_async.cuh -- the fused step as a persistent, double-buffered kernel.
//
// The step is bound by how many loads each SM keeps in flight: a thread that loads its 19 pulled
// populations into registers holds them (and its issue slots) idle for a memory latency.  Here
// each CTA walks a sequence of tiles (row segments of 128 * VW nodes); while it computes tile t,
// the loads of tile t + gridDim.x are already travelling as asynchronous global-to-shared copies
// (cp.async), which occupy no registers.  Each thread copies into, and later reads from, only its
// own shared-memory slots, so the pipeline needs no block-wide barrier: cp.async.wait_group on the
// thread's own copy groups is the only wait (a hardware completion wait, not a spin loop).
//
// Nodes next to a wall or moving wall take the general pull with direct loads; every other node
// (periodic faces included) takes the copied path.  The collision is step_body, unchanged.
#pragma once

#include "step.cuh"

namespace lbm {

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

constexpr int ASYNC_THREADS = 128;

// bytes of one thread's slot for one population
template <class ST, int VW>
__host__ __device__ constexpr int slot_bytes() {
    return sizeof(ST) == 2 ? 4 * VW : static_cast<int>(sizeof(ST)) * VW;
}

// geometry of the node (pair) a thread owns in a tile, and whether it takes the copied path
struct TileNode {
    int x, y, z, node;
    bool active, fast;
    int dxm, dxp, dy[3], dz[3];  // source offsets: c_x = +1 / -1 (first node), c_y, c_z = -1, 0, +1
};

template <class RS, int VW>
__device__ __forceinline__ TileNode tile_node(const StepArgs<RS>& a, int t, int nseg) {
    TileNode n;
    const int seg = t % nseg, row = t / nseg;
    n.y = row % a.ny;
    n.z = row / a.ny;
    n.x = (seg * ASYNC_THREADS + static_cast<int>(threadIdx.x)) * VW;
    n.active = n.x < a.nx;
    const int nx = a.nx, nxy = a.nx * a.ny;
    n.node = n.z * nxy + n.y * nx + n.x;
    const int xl = n.x + VW - 1;  // last node of the thread
    const bool wx0 = n.x == 0 && (a.wall_mask & 1), wx1 = xl == nx - 1 && (a.wall_mask & 2);
    const bool wy0 = n.y == 0 && (a.wall_mask & 4), wy1 = n.y == a.ny - 1 && (a.wall_mask & 8);
    const bool wz0 = n.z == 0 && (a.wall_mask & 16), wz1 = n.z == a.nz - 1 && (a.wall_mask & 32);
    n.fast = n.active && !(wx0 || wx1 || wy0 || wy1 || wz0 || wz1);
    n.dxm = n.x == 0 ? nx - 1 : -1;                        // first node, c_x = +1: x - 1 (wrapped)
    n.dxp = xl == nx - 1 ? VW - nx : VW;                    // last node, c_x = -1: x + 1 (wrapped)
    // pull source of c_y = +1 is y - 1, of c_y = -1 is y + 1 (index by c + 1)
    n.dy[2] = n.y == 0 ? (a.ny - 1) * nx : -nx;
    n.dy[1] = 0;
    n.dy[0] = n.y == a.ny - 1 ? -(a.ny - 1) * nx : nx;
    n.dz[2] = n.z == 0 ? (a.nz - 1) * nxy : -nxy;
    n.dz[1] = 0;
    n.dz[0] = n.z == a.nz - 1 ? -(a.nz - 1) * nxy : nxy;
    return n;
}

// issue the copies of one tile into `stage`; returns the parity bits of 16-bit sources
template <class L, class ST, int VW, class RS>
__device__ __forceinline__ uint64_t issue_copies(const StepArgs<RS>& a, const TileNode& n, unsigned char* stage) {
    uint64_t par = 0;
    if (!n.fast) return par;
    constexpr int SB = slot_bytes<ST, VW>();
    sfor<L::Q>([&](auto i) {
        constexpr int cx = L::c(CV(i), 0), cy = L::c(CV(i), 1), cz = L::c(CV(i), 2);
        const ST* base = static_cast<const ST*>(a.srcp[CV(i)]);
        const int row = n.node + n.dy[cy + 1] + n.dz[cz + 1];
        unsigned char* slot = stage + (CV(i) * ASYNC_THREADS + threadIdx.x) * SB;
        if constexpr (VW == 1) {
            const int off = row + (cx > 0 ? n.dxm : (cx < 0 ? n.dxp : 0));
            if constexpr (sizeof(ST) == 2) {
                cp_async4(slot, base + (off & ~1));
                par |= uint64_t(off & 1) << CV(i);
            } else if constexpr (sizeof(ST) == 4) {
                cp_async4(slot, base + off);
            } else {
                cp_async8(slot, base + off);
            }
        } else {
            // two nodes x, x + 1 (x even): c_x = 0 is one aligned pair, otherwise two sources
            if constexpr (cx == 0) {
                if constexpr (sizeof(ST) == 2)
                    cp_async4(slot, base + row);
                else
                    cp_async8(slot, base + row);
            } else {
                const int o0 = row + (cx > 0 ? n.dxm : 1);
                const int o1 = row + (cx > 0 ? 0 : n.dxp);
                if constexpr (sizeof(ST) == 2) {
                    cp_async4(slot, base + (o0 & ~1));
                    cp_async4(slot + 4, base + (o1 & ~1));
                    par |= uint64_t(o0 & 1) << (2 * CV(i));
                    par |= uint64_t(o1 & 1) << (2 * CV(i) + 1);
                } else {
                    cp_async4(slot, base + o0);
                    cp_async4(slot + 4, base + o1);
                }
            }
        }
    });
    return par;
}

__device__ __forceinline__ float half_of(uint32_t w, int hi, __half) {
    const unsigned short b = hi ? static_cast<unsigned short>(w >> 16) : static_cast<unsigned short>(w & 0xffffu);
    return __half2float(__ushort_as_half(b));
}
__device__ __forceinline__ float half_of(uint32_t w, int hi, __nv_bfloat16) {
    const unsigned short b = hi ? static_cast<unsigned short>(w >> 16) : static_cast<unsigned short>(w & 0xffffu);
    return __bfloat162float(__ushort_as_bfloat16(b));
}

// read one tile's populations back from `stage`
template <class L, class ST, int VW, class R>
__device__ __forceinline__ void read_copies(const unsigned char* stage, uint64_t par, R (&f)[L::Q]) {
    constexpr int SB = slot_bytes<ST, VW>();
    sfor<L::Q>([&](auto i) {
        const unsigned char* slot = stage + (CV(i) * ASYNC_THREADS + threadIdx.x) * SB;
        if constexpr (VW == 1) {
            if constexpr (sizeof(ST) == 2) {
                const uint32_t w = *reinterpret_cast<const uint32_t*>(slot);
                f[i] = half_of(w, int((par >> CV(i)) & 1), ST());
            } else {
                f[i] = *reinterpret_cast<const ST*>(slot);
            }
        } else {
            constexpr int cx = L::c(CV(i), 0);
            if constexpr (sizeof(ST) == 2) {
                if constexpr (cx == 0) {
                    const uint32_t w = *reinterpret_cast<const uint32_t*>(slot);
                    f[i] = F2(half_of(w, 0, ST()), half_of(w, 1, ST()));
                } else {
                    const uint2 w = *reinterpret_cast<const uint2*>(slot);
                    f[i] = F2(half_of(w.x, int((par >> (2 * CV(i))) & 1), ST()),
                              half_of(w.y, int((par >> (2 * CV(i) + 1)) & 1), ST()));
                }
            } else {
                f[i] = F2(*reinterpret_cast<const float2*>(slot));
            }
        }
    });
}

template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE, int VW>
__global__ void __launch_bounds__(ASYNC_THREADS) k_step_async(const StepArgs<typename Store<ST>::R> a, int nseg,
                                                                 int tiles) {
    using RS = typename Store<ST>::R;
    using R = std::conditional_t<VW == 2, F2, RS>;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int STAGE = L::Q * ASYNC_THREADS * slot_bytes<ST, VW>();
    int t = blockIdx.x;
    int s = 0;
    uint64_t par[2] = {0, 0};
    if (t < tiles) par[0] = issue_copies<L, ST, VW>(a, tile_node<RS, VW>(a, t, nseg), smem);
    cp_commit();
    for (; t < tiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        if (tn < tiles) par[s ^ 1] = issue_copies<L, ST, VW>(a, tile_node<RS, VW>(a, tn, nseg), smem + (s ^ 1) * STAGE);
        cp_commit();
        cp_wait_all_but_one();
        const TileNode n = tile_node<RS, VW>(a, t, nseg);
        if (n.active) {
            R f[L::Q];
            if (n.fast) {
                read_copies<L, ST, VW>(smem + s * STAGE, par[s], f);
            } else if constexpr (VW == 2) {
                pull2<L, ST>(a, n.x, n.y, n.z, f);
            } else {
                pull<L, ST>(a, n.x, n.y, n.z, f);
            }
            step_body<L, ST, CLOSURE, FORMULA, FORCE, VW>(a, f, n.node);
        }
        s ^= 1;
    }
}

// ------------------------------------------------------------------------------------------
// persistent loop with the next node's loads in flight in registers while the current one is
// computed (the loop is unrolled by two so the two register sets swap roles without copies)

template <class L, class ST, int VW, class RS, class R>
__device__ __forceinline__ void load_node(const StepArgs<RS>& a, const TileNode& n, R (&f)[L::Q]) {
    if (!n.active) return;
    if (!n.fast) {
        if constexpr (VW == 2)
            pull2<L, ST>(a, n.x, n.y, n.z, f);
        else
            pull<L, ST>(a, n.x, n.y, n.z, f);
        return;
    }
    sfor<L::Q>([&](auto i) {
        constexpr int cx = L::c(CV(i), 0), cy = L::c(CV(i), 1), cz = L::c(CV(i), 2);
        const ST* base = static_cast<const ST*>(a.srcp[CV(i)]);
        const int row = n.node + n.dy[cy + 1] + n.dz[cz + 1];
        if constexpr (VW == 1) {
            f[i] = Store<ST>::ld(base + row + (cx > 0 ? n.dxm : (cx < 0 ? n.dxp : 0)));
        } else {
            if constexpr (cx == 0)
                f[i] = Store<ST>::ld2(base + row);
            else if constexpr (cx > 0)
                f[i] = F2(Store<ST>::ld(base + row + n.dxm), Store<ST>::ld(base + row));
            else
                f[i] = F2(Store<ST>::ld(base + row + 1), Store<ST>::ld(base + row + n.dxp));
        }
    });
}

template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE, int VW>
__global__ void __launch_bounds__(ASYNC_THREADS) k_step_prefetch(const StepArgs<typename Store<ST>::R> a, int nseg,
                                                                    int tiles) {
    using RS = typename Store<ST>::R;
    using R = std::conditional_t<VW == 2, F2, RS>;
    const int G = gridDim.x;
    int t = blockIdx.x;
    R fa[L::Q], fb[L::Q];
    TileNode na = tile_node<RS, VW>(a, t < tiles ? t : 0, nseg), nb;
    na.active = na.active && t < tiles;
    load_node<L, ST, VW>(a, na, fa);
    while (t < tiles) {
        nb = tile_node<RS, VW>(a, t + G < tiles ? t + G : 0, nseg);
        nb.active = nb.active && t + G < tiles;
        load_node<L, ST, VW>(a, nb, fb);
        if (na.active) step_body<L, ST, CLOSURE, FORMULA, FORCE, VW>(a, fa, na.node);
        t += G;
        if (t >= tiles) break;
        na = tile_node<RS, VW>(a, t + G < tiles ? t + G : 0, nseg);
        na.active = na.active && t + G < tiles;
        load_node<L, ST, VW>(a, na, fa);
        if (nb.active) step_body<L, ST, CLOSURE, FORMULA, FORCE, VW>(a, fb, nb.node);
        t += G;
    }
}

}  // namespace lbm
