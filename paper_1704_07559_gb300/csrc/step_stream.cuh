// step_stream.cuh -- several time steps in one launch, scheduled tile by tile.
//
// A step launched on its own must wait for the whole previous step to finish: every SM drains
// at the end of each step and the memory system ramps up again at the start of the next, a fixed
// cost per step that is a tenth of a 4M-node step.  Here one launch runs `steps` steps.  The
// lattice is cut into units (one z plane times `rows` rows of y, all of x); a block takes tickets
// in order from a global counter, ticket t being step t / units at unit position t % units, and
// runs that unit once the nine units around it (z +-1, y tile +-1, wrapped) have completed the
// previous step.  Those nine cover both hazards of the two-buffer scheme: the populations the
// unit pulls were written by them in the previous step (read after write), and the buffer the
// unit writes was last read by them in the previous step (write after read).
//
// Forward progress: a block holds a ticket only while it is resident, every dependency of a
// ticket is an earlier ticket, and a block that takes its next ticket before publishing its
// current unit publishes it without waiting on any other block; so the earliest unfinished
// ticket can always run.  Units are
// visited in a zigzag order (0, n-1, 1, n-2, ...) along z and along the y tiles, so the first
// units of a step depend only on the first units of the previous step and the steps overlap
// without stalls once there are more units than resident blocks.
//
// Ordering: a unit's stores are published by a barrier and one release store of the unit's step
// count (cumulative over the block's stores); a waiting block acquires the counts of its
// neighbours and then passes a barrier before any load, and the populations are read through L2
// (ld.global.cg), never through the non-coherent path.  Every wait is bounded (about two seconds
// of global-timer time): on a timeout the block records an error flag, later blocks skip their
// work but still publish their counts, and the kernel ends; the host reads the flag.
#pragma once

#include "launch.h"
#include "step.cuh"
#include "step_pair.cuh"

namespace lbm {

__device__ __forceinline__ int zigzag(int p, int n) { return (p & 1) ? n - 1 - (p >> 1) : (p >> 1); }

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long STREAM_WAIT_NS = 2000000000ull;  // bound of one dependency wait
constexpr int STREAM_WAIT_ITERS = 1 << 25;                    // and of its polls

// Wait until *flag >= want.  Returns false (and sets *err) when the wait ran out, or at once
// when another block already recorded an error.
__device__ __noinline__ static bool wait_count(const int* flag, int want, int* err) {
    if (ld_acquire(flag) >= want) return true;
    const unsigned long long t0 = global_ns();
    for (int it = 0; it < STREAM_WAIT_ITERS; ++it) {
        __nanosleep(128);
        if (ld_acquire(flag) >= want) return true;
        if (ld_acquire(err) != 0) return false;
        if (global_ns() - t0 > STREAM_WAIT_NS) break;
    }
    atomicExch(err, 1);
    return false;
}

// One unit: rows [y0, y1) of plane z, one node per thread (PAIR false) or two x-adjacent nodes
// per thread in packed pair arithmetic (PAIR true, nx even).  es / ds shift the source / destination
// populations by that many elements (ring launches; one node per thread only).
template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE, bool PAIR>
__device__ __forceinline__ void stream_unit(const StepArgs<typename Store<ST>::R>& a, int z, int y0, int y1,
                                            long long es = 0, long long ds = 0) {
    using R = typename Store<ST>::R;
    for (int y = y0; y < y1; ++y) {
        if constexpr (PAIR) {
            for (int x = 2 * (int)threadIdx.x; x < a.nx; x += 2 * (int)blockDim.x) {
                F2 f2[L::Q];
                pull2<L, ST, true>(a, x, y, z, f2);
                step_pair<L, ST, CLOSURE, FORMULA, FORCE>(a, f2, (z * a.ny + y) * a.nx + x);
            }
        } else {
            for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
                R f[L::Q];
                pull<L, ST, true>(a, x, y, z, f, es);
                step_body<L, ST, CLOSURE, FORMULA, FORCE>(a, f, (z * a.ny + y) * a.nx + x, ds);
            }
        }
    }
}

// The scheduler: takes tickets until the launch's steps are exhausted and calls run(k, z, y0, y1)
// for step k (0-based within the launch) of unit (z, band) once its neighbours have finished step
// k - 1.  Every thread of the block calls it; run must not synchronise the block.  Two barriers
// per unit: after the dependency waits, and after the unit's work, before which thread 0 (its own
// share done) already takes the next ticket.  Everything the scheduler needs after the unit's
// work is in shared memory or recomputed from the launch's constants, so none of its values stays
// live in registers across the work (measured on the channel: FP32 Yu +1.4%, FP32 Chai +0.7%,
// FP16 Chai +1.7%, FP16 Yu -1.7%, against three barriers per unit and the values kept live).
template <class Run>
__device__ __forceinline__ void stream_schedule(int ny, int nz, const StreamCtl& c, Run&& run) {
    __shared__ int s_ticket, s_skip, s_unit, s_kp1;
    // c.sync[0]: the error flag; c.sync[1]: the ticket counter; c.sync[2 + unit]: the units' step counts
    if (threadIdx.x == 0) s_ticket = atomicAdd(c.sync + 1, 1) + c.first_step * nz * c.tiles_y;
    __syncthreads();
    for (;;) {
        int k, z, ty;
        {
            const int tiles = c.tiles_y, units = nz * tiles;
            const int t = s_ticket;
            if (t >= c.steps * units) return;  // the host keeps steps * units below 2^31
            k = t / units;
            const int p = t - k * units;
            const int pz = p / tiles, py = p - pz * tiles;
            z = zigzag(pz, nz);
            ty = zigzag(py, tiles);
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                bool ok = true;
                if (lane < 9) {
                    if (k > 0) {
                        int zz = z + lane / 3 - 1, yy = ty + lane % 3 - 1;
                        zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
                        yy = yy < 0 ? yy + tiles : (yy >= tiles ? yy - tiles : yy);
                        ok = wait_count(c.sync + 2 + zz * tiles + yy, k, c.sync);
                    }
                    if (ok && ld_acquire(c.sync) != 0) ok = false;
                }
                const bool bad = __any_sync(0xffffffffu, !ok);
                if (lane == 0) {
                    s_skip = bad ? 1 : 0;
                    s_unit = z * tiles + ty;
                    s_kp1 = k + 1;
                }
            }
        }
        __syncthreads();
        if (!s_skip) {
            const int y0 = ty * c.rows, y1 = min(ny, y0 + c.rows);
            run(k, z, y0, y1);
        }
        // every thread read s_ticket before the barrier above, so thread 0 may replace it now
        if (threadIdx.x == 0) s_ticket = atomicAdd(c.sync + 1, 1) + c.first_step * nz * c.tiles_y;
        __syncthreads();
        if (threadIdx.x == 0) st_release(c.sync + 2 + s_unit, s_kp1);
    }
}

// Two-buffer launches: a0 reads buffer A and writes B (even steps of the launch), a1 the reverse
// (odd steps).  Ring launches (c.ring != 0): step k reads a0's source and writes a0's
// destination, both shifted by k * c.ring elements (each step writes a buffer of its own).
template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE, bool PAIR>
__device__ __forceinline__ void stream_steps(const StepArgs<typename Store<ST>::R>& a0,
                                             const StepArgs<typename Store<ST>::R>& a1, const StreamCtl& c) {
    stream_schedule(a0.ny, a0.nz, c, [&](int k, int z, int y0, int y1) {
        if (k & 1)
            stream_unit<L, ST, CLOSURE, FORMULA, FORCE, PAIR>(a1, z, y0, y1);
        else
            stream_unit<L, ST, CLOSURE, FORMULA, FORCE, PAIR>(a0, z, y0, y1);
    });
}

// One node per thread.  9 resident blocks (56 registers, a few spilled values) for the Yu route
// with the Smagorinsky closure: against 8 blocks at 64 registers, D3Q15 channel +4%, 128^3 box
// +1%, the adjoint's forward sweep +4%, the D3Q19 channel unchanged (A/B on one box; 10 blocks on
// D3Q15 -1%).  9 blocks for D3Q15 Chai with the Smagorinsky closure too (56 registers, no spills:
// +4.6%).  8 blocks (64 registers) for the other Yu forms and for D3Q19 Chai with the Smagorinsky
// and power-law closures (Chai: measured 4.5% faster than 7 blocks at 72 registers on the channel,
// 1.8% faster than 9 blocks at 56), 7 for the other Chai forms (spills of 64-144 B at 64
// registers).  Unbounded, the unit loop costs 7-8 more registers and a block.
template <int CLOSURE, int FORMULA, int Q>
constexpr int stream_min_blocks() {
    if (CLOSURE == CL_SMAG && (FORMULA == F_YU || Q == 15)) return 9;
    return (FORMULA == F_YU || CLOSURE == CL_SMAG || CLOSURE == CL_POWERLAW) ? 8 : 7;
}

template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE>
__global__ void __launch_bounds__(128, stream_min_blocks<CLOSURE, FORMULA, L::Q>())
    k_step_stream(const StepArgs<typename Store<ST>::R> a0, const StepArgs<typename Store<ST>::R> a1,
                  const StreamCtl c) {
    stream_steps<L, ST, CLOSURE, FORMULA, FORCE, false>(a0, a1, c);
}

// Two nodes per thread in packed pair arithmetic (16-bit storage, nx even; step_pair.cuh): 7
// resident blocks, as the one-step pair kernel.
template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE>
__global__ void __launch_bounds__(128, PAIR_MIN_BLOCKS) k_step_stream_pair(const StepArgs<typename Store<ST>::R> a0,
                                                             const StepArgs<typename Store<ST>::R> a1,
                                                             const StreamCtl c) {
    stream_steps<L, ST, CLOSURE, FORMULA, FORCE, true>(a0, a1, c);
}

// Ring launch (see stream_steps), one node per thread; 9 resident blocks for the Yu route (the
// adjoint's recompute: its whole call 0.7% shorter than with 8).
template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE>
__global__ void __launch_bounds__(128, FORMULA == F_YU ? 9 : 7)
    k_step_stream_ring(const StepArgs<typename Store<ST>::R> a, const StreamCtl c) {
    stream_schedule(a.ny, a.nz, c, [&](int k, int z, int y0, int y1) {
        const long long sh = k * c.ring;
        stream_unit<L, ST, CLOSURE, FORMULA, FORCE, false>(a, z, y0, y1, sh, sh);
    });
}

template <class K>
int resident_blocks(K kernel) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0);
    return (per_sm < 1 ? 1 : per_sm) * sms;
}

// Unit height: c.rows (about 1024 nodes) times the largest m in {4, 2, 1} that still leaves more
// units than resident blocks plus the span of positions a unit's dependencies reach ahead of it
// (two planes of bands and two bands; no planes when nz = 1), so that no block waits; false when
// even m = 1 does not.
inline bool pick_units(const StreamCtl& base, int ny, int nz, int resident, StreamCtl* out) {
    for (int m = 4; m >= 1; m /= 2) {
        const int rows = base.rows * m < ny ? base.rows * m : ny;
        const int tiles = (ny + rows - 1) / rows;
        const long long units = (long long)nz * tiles;
        const long long span = (nz > 1 ? 2LL * tiles : 0) + 3;
        if (units >= resident + span) {
            *out = base;
            out->rows = rows;
            out->tiles_y = tiles;
            return true;
        }
    }
    *out = base;
    return false;
}

// Launch `c.steps` steps, after zeroing the ticket and the counts of the chosen units.  Not forced,
// the streamed form is taken only on lattices up to 2^23 nodes, where the fixed cost of a step
// boundary is a large share of a step (measured on GB300: +7% FP32 Yu and +10% FP32 Chai on a
// 4.2M-node channel, +17% on a 2.1M-node box; -5% on a 134M-node box, where the per-unit
// synchronisation costs more than the boundaries), and only when no block would wait;
// cudaErrorNotSupported tells the caller to launch step by step instead.
template <class L, class ST, int C, int F, bool FO>
cudaError_t launch_stream_form(const StepArgs<typename Store<ST>::R>& a0, const StepArgs<typename Store<ST>::R>& a1,
                               const StreamCtl& c, bool force_stream, cudaStream_t s) {
    const long long N = (long long)a0.nx * a0.ny * a0.nz;
    if (!force_stream && N > (1LL << 23)) return cudaErrorNotSupported;
    StreamCtl u;
    if constexpr (sizeof(ST) == 2) {
        if (a0.nx % 2 == 0) {
            static const int resident = resident_blocks(k_step_stream_pair<L, ST, C, F, FO>);
            if (!pick_units(c, a0.ny, a0.nz, resident, &u) && !force_stream) return cudaErrorNotSupported;
            const long long total = (long long)a0.nz * u.tiles_y * u.steps;
            if (total >= (1LL << 31) || u.steps < 1) return cudaErrorInvalidValue;
            const int grid = (int)(total < resident ? total : resident);
            cudaError_t e = cudaMemsetAsync(u.sync + 1, 0, sizeof(int) * (1 + (size_t)a0.nz * u.tiles_y), s);
            if (e != cudaSuccess) return e;
            k_step_stream_pair<L, ST, C, F, FO><<<grid, 128, 0, s>>>(a0, a1, u);
            return cudaGetLastError();
        }
    }
    static const int resident = resident_blocks(k_step_stream<L, ST, C, F, FO>);
    if (!pick_units(c, a0.ny, a0.nz, resident, &u) && !force_stream) return cudaErrorNotSupported;
    const long long total = (long long)a0.nz * u.tiles_y * u.steps;
    if (total >= (1LL << 31) || u.steps < 1) return cudaErrorInvalidValue;
    const int grid = (int)(total < resident ? total : resident);
    cudaError_t e = cudaMemsetAsync(u.sync + 1, 0, sizeof(int) * (1 + (size_t)a0.nz * u.tiles_y), s);
    if (e != cudaSuccess) return e;
    k_step_stream<L, ST, C, F, FO><<<grid, 128, 0, s>>>(a0, a1, u);
    return cudaGetLastError();
}

template <class L, class ST, int C, int F, bool FO>
cudaError_t launch_stream_ring_form(const StepArgs<typename Store<ST>::R>& a, const StreamCtl& c, bool force_stream,
                                    cudaStream_t s) {
    const long long N = (long long)a.nx * a.ny * a.nz;
    if (!force_stream && N > (1LL << 23)) return cudaErrorNotSupported;
    static const int resident = resident_blocks(k_step_stream_ring<L, ST, C, F, FO>);
    StreamCtl u;
    if (!pick_units(c, a.ny, a.nz, resident, &u) && !force_stream) return cudaErrorNotSupported;
    const long long total = (long long)a.nz * u.tiles_y * u.steps;
    if (total >= (1LL << 31) || u.steps < 1) return cudaErrorInvalidValue;
    const int grid = (int)(total < resident ? total : resident);
    cudaError_t e = cudaMemsetAsync(u.sync + 1, 0, sizeof(int) * (1 + (size_t)a.nz * u.tiles_y), s);
    if (e != cudaSuccess) return e;
    k_step_stream_ring<L, ST, C, F, FO><<<grid, 128, 0, s>>>(a, u);
    return cudaGetLastError();
}

template <class L, class ST, int C, int F>
cudaError_t launch_stream_cf(const StepArgs<typename Store<ST>::R>& a0, const StepArgs<typename Store<ST>::R>& a1,
                             const StreamCtl& c, int force, bool force_stream, cudaStream_t s) {
    return force ? launch_stream_form<L, ST, C, F, true>(a0, a1, c, force_stream, s)
                 : launch_stream_form<L, ST, C, F, false>(a0, a1, c, force_stream, s);
}

// FP64 stays step by step (its arithmetic, not the step boundaries, bounds it).
template <class L, class ST, bool EXTRA_CLOSURES>
cudaError_t launch_stream(const StepArgs<typename Store<ST>::R>& a0, const StepArgs<typename Store<ST>::R>& a1,
                          const StreamCtl& c, int closure, int formula, int force, bool force_stream,
                          cudaStream_t s) {
    const bool yu = formula == F_YU;
    switch (closure) {
        case CL_NEWTON:
            return yu ? launch_stream_cf<L, ST, CL_NEWTON, F_YU>(a0, a1, c, force, force_stream, s)
                      : launch_stream_cf<L, ST, CL_NEWTON, F_CHAI>(a0, a1, c, force, force_stream, s);
        case CL_SMAG:
            return yu ? launch_stream_cf<L, ST, CL_SMAG, F_YU>(a0, a1, c, force, force_stream, s)
                      : launch_stream_cf<L, ST, CL_SMAG, F_CHAI>(a0, a1, c, force, force_stream, s);
        case CL_POWERLAW:
            if constexpr (EXTRA_CLOSURES)
                return yu ? launch_stream_cf<L, ST, CL_POWERLAW, F_YU>(a0, a1, c, force, force_stream, s)
                          : launch_stream_cf<L, ST, CL_POWERLAW, F_CHAI>(a0, a1, c, force, force_stream, s);
            return cudaErrorNotSupported;
        case CL_SMAG_DEV:
            if constexpr (EXTRA_CLOSURES)
                return yu ? launch_stream_cf<L, ST, CL_SMAG_DEV, F_YU>(a0, a1, c, force, force_stream, s)
                          : launch_stream_cf<L, ST, CL_SMAG_DEV, F_CHAI>(a0, a1, c, force, force_stream, s);
            return cudaErrorNotSupported;
        case CL_SMAG_LAGGED:  // the stored tau is the node's own: its unit's previous step wrote it
            if constexpr (EXTRA_CLOSURES)
                return yu ? launch_stream_cf<L, ST, CL_SMAG_LAGGED, F_YU>(a0, a1, c, force, force_stream, s)
                          : launch_stream_cf<L, ST, CL_SMAG_LAGGED, F_CHAI>(a0, a1, c, force, force_stream, s);
            return cudaErrorNotSupported;
        default:
            return cudaErrorNotSupported;
    }
}

}  // namespace lbm

#define LBM_DEFINE_STREAM_RING_ENTRY(TAG, L, ST)                                                              \
    namespace lbm {                                                                                          \
    cudaError_t stream_ring_##TAG(const StepArgs<Store<ST>::R>& a, const StreamCtl& c, int closure,          \
                                  int formula, int force, int force_stream, cudaStream_t s) {                \
        const bool fs = force_stream != 0;                                                                   \
        const bool yu = formula == F_YU;                                                                     \
        if (closure == CL_SMAG) {                                                                            \
            if (yu)                                                                                          \
                return force ? launch_stream_ring_form<L, ST, CL_SMAG, F_YU, true>(a, c, fs, s)              \
                             : launch_stream_ring_form<L, ST, CL_SMAG, F_YU, false>(a, c, fs, s);            \
            return force ? launch_stream_ring_form<L, ST, CL_SMAG, F_CHAI, true>(a, c, fs, s)                \
                         : launch_stream_ring_form<L, ST, CL_SMAG, F_CHAI, false>(a, c, fs, s);              \
        }                                                                                                    \
        if (closure == CL_NEWTON) {                                                                          \
            if (yu)                                                                                          \
                return force ? launch_stream_ring_form<L, ST, CL_NEWTON, F_YU, true>(a, c, fs, s)            \
                             : launch_stream_ring_form<L, ST, CL_NEWTON, F_YU, false>(a, c, fs, s);          \
            return force ? launch_stream_ring_form<L, ST, CL_NEWTON, F_CHAI, true>(a, c, fs, s)              \
                         : launch_stream_ring_form<L, ST, CL_NEWTON, F_CHAI, false>(a, c, fs, s);            \
        }                                                                                                    \
        return cudaErrorNotSupported;                                                                        \
    }                                                                                                        \
    }

#define LBM_DEFINE_STREAM_ENTRY(TAG, L, ST, EXTRA_CLOSURES)                                                  \
    namespace lbm {                                                                                          \
    cudaError_t stream_##TAG(const StepArgs<Store<ST>::R>& a0, const StepArgs<Store<ST>::R>& a1,             \
                             const StreamCtl& c, int closure, int formula, int force, int force_stream,      \
                             cudaStream_t s) {                                                               \
        return launch_stream<L, ST, EXTRA_CLOSURES>(a0, a1, c, closure, formula, force, force_stream != 0,  \
                                                    s);                                                      \
    }                                                                                                        \
    }
