// bfs_common.cuh -- device helpers shared by the BFS kernels (sm_103a).
//
// Memory-model notes used throughout:
//  * Anything written by another CTA during the same launch (visited /
//    frontier bitmaps, queues, counters) is read with ld.global.cg (L2 only):
//    the per-SM L1 is not coherent, and a line cached at an earlier level
//    would be stale at a later one.
//  * The graph (row offsets, column ids, isolated-vertex bitmap) is read-only
//    for the life of a launch and goes through the non-coherent path (__ldg).
//  * Grid-wide ordering comes from grid_sync(): a bounded sense barrier
//    (release on arrival, acquire on departure) whose wait gives up after a
//    time limit, records BFS_DEV_TIMEOUT in the run's status word and lets
//    every CTA leave, so a missing CTA can never hang the GPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bfsk {

constexpr unsigned kDevOk = 0;
constexpr unsigned kDevTimeout = 1;
constexpr unsigned kDevOverflow = 2;

// Grid barrier + run status; the first member of every launch control block.
// `count` only grows during a launch: barrier k is complete once it reaches
// (k+1) * expected, so an arriving CTA needs one atomic and no separate
// generation word.  Bit 63 is the abort flag: set together with `status`, it
// releases every waiting CTA at once.
struct BarrierState {
    unsigned long long count;
    unsigned status;
    unsigned pad;
};
constexpr unsigned long long kAbortBit = 1ull << 63;

// Control block of one single-source launch: zeroed by the host
// (cudaMemsetAsync) before every launch.  Counters indexed [slot] rotate over
// levels (slot = level % 3).
struct Ctrl {
    BarrierState b;
    unsigned long long tail[3];      // length of the queue holding frontier `slot`
    unsigned long long accn[3];      // size of frontier `slot` (bottom-up producer)
    unsigned long long accm[3];      // degree sum of frontier `slot`
    unsigned long long scanned[3];   // bottom-up searchers of the level producing frontier `slot`
    unsigned long long examined[3];  // serial early-exit examinations of that level
    unsigned long long ntask[3];     // top-down edge-chunk tasks of that level
    unsigned long long nmiss[3];     // bottom-up first-probe misses left to phase B (miss-list length)
    unsigned long long nmiss_in[3];  // ... resolved by their chunk's warp in phase A
    unsigned long long dsum_out[3];  // directed graphs: out-degree sum of frontier `slot`
    unsigned long long dsum_in[3];   // directed graphs: in-degree sum of frontier `slot`
    unsigned long long heavy[3];     // top-down: vertices of frontier `slot` above the cluster-level degree cap
    // cluster levels (levels run by thread-block cluster 0 alone while the frontier is small)
    unsigned long long clu_gen;      // episodes finished: the waiting CTAs resume when it reaches theirs
    unsigned long long clu_prog;     // last level the cluster started (progress for the waiters' time limit)
    unsigned long long clu_spill;    // frontier entries that found no room in the cluster's shared memory
    long long clu_d, clu_nf, clu_mf, clu_mu, clu_reached, clu_done;   // state handed back to the grid
    long long num_levels;
    long long reached;
    unsigned long long t_enter;    // lead CTA's clock at kernel entry
    unsigned long long t_init;     // ... after the initialisation barrier
    unsigned long long t_levels;   // ... after the last level
    unsigned long long t_done;     // clock of the last CTA to finish the final pass
    unsigned long long done_ctas;  // CTAs through the final pass
};

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Counter reads after a grid barrier: the barrier already ordered them, so
// they need no acquire of their own and can be in flight together.
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_inclusive_scan(int v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide sum of up to 4 per-thread counters, then one atomicAdd each from
// thread 0 (per-level counters see one atomic per CTA, not per warp).
__device__ __forceinline__ void block_add4(unsigned long long a, unsigned long long b, unsigned long long c,
                                           unsigned long long d, unsigned long long* ga,
                                           unsigned long long* gb, unsigned long long* gc,
                                           unsigned long long* gd) {
    __shared__ unsigned long long red[4][32];
    const int lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    d = warp_sum(d);
    __syncthreads();
    if (lane == 0) {
        red[0][wid] = a;
        red[1][wid] = b;
        red[2][wid] = c;
        red[3][wid] = d;
    }
    __syncthreads();
    if (wid == 0) {
        unsigned long long x0 = lane < nw ? red[0][lane] : 0ull;
        unsigned long long x1 = lane < nw ? red[1][lane] : 0ull;
        unsigned long long x2 = lane < nw ? red[2][lane] : 0ull;
        unsigned long long x3 = lane < nw ? red[3][lane] : 0ull;
        x0 = warp_sum(x0);
        x1 = warp_sum(x1);
        x2 = warp_sum(x2);
        x3 = warp_sum(x3);
        if (lane == 0) {
            if (ga && x0) atomicAdd(ga, x0);
            if (gb && x1) atomicAdd(gb, x1);
            if (gc && x2) atomicAdd(gc, x2);
            if (gd && x3) atomicAdd(gd, x3);
        }
    }
}

// Record a launch failure for the host and release every CTA waiting at a
// grid barrier (they then leave their loops).
__device__ __forceinline__ void raise_status(BarrierState* c, unsigned code) {
    atomicMax(&c->status, code);
    atomicOr(&c->count, kAbortBit);
}

// Bounded grid barrier.  Every thread of every CTA calls it.  Returns false
// when the run has failed (this wait or another CTA's ran out of time, or a
// phase raised an error); the caller then leaves its loop.  `expected` is the
// number of CTAs (plus any deliberately missing arrivals in the timeout test).
// The arrival is one acquire-release atomic by thread 0 after the CTA barrier:
// it publishes the CTA's writes and, for the last arriver, acquires everyone
// else's; waiters acquire through their polling load.
__device__ __forceinline__ bool grid_sync(BarrierState* c, unsigned expected, uint64_t timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long old;
        asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], 1;" : "=l"(old) : "l"(&c->count) : "memory");
        const unsigned long long target = ((old & ~kAbortBit) / expected + 1ull) * expected;
        unsigned long long cur = old + 1ull;
        if (!(cur & kAbortBit) && cur < target) {
            const uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (true) {
                cur = ld_acquire64(&c->count);
                if ((cur & kAbortBit) || cur >= target) break;
                if (++spins > 32u) {
                    __nanosleep(32);
                    if ((spins & 63u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
                        raise_status(c, kDevTimeout);
                        cur = kAbortBit;
                        break;
                    }
                }
            }
        }
        s_ok = (cur & kAbortBit) ? 0 : 1;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace bfsk
