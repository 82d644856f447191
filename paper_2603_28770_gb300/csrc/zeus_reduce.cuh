// zeus_reduce.cuh -- deterministic (value, index) argmin across a block and
// across a grid (the best-of-swarm reduction of Alg. 7, also used for the
// PSO global best).  NaN counts as +inf; ties go to the lowest index.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "zeus_internal.h"

namespace zeus {

__device__ __forceinline__ bool better(double fa, long long ia, double fb, long long ib) {
    return fa < fb || (fa == fb && ia < ib);
}

__device__ __forceinline__ double nan_to_inf(double v) { return isnan(v) ? CUDART_INF : v; }

// Warp argmin of (f, idx); every lane returns the warp's winner.
__device__ __forceinline__ void warp_argmin(double& f, long long& idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double fo = __shfl_xor_sync(0xffffffffu, f, o);
        const long long io = __shfl_xor_sync(0xffffffffu, idx, o);
        if (better(fo, io, f, idx)) {
            f = fo;
            idx = io;
        }
    }
}

// Block argmin; the result is valid in thread 0.  Every thread of the
// block must call it.  `scratch` holds 32 ArgPair entries.
__device__ __forceinline__ void block_argmin(double& f, long long& idx, ArgPair* scratch) {
    warp_argmin(f, idx);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
        scratch[w].f = f;
        scratch[w].idx = idx;
    }
    __syncthreads();
    if (w == 0) {
        f = (threadIdx.x < nw) ? scratch[threadIdx.x].f : CUDART_INF;
        idx = (threadIdx.x < nw) ? scratch[threadIdx.x].idx : 0x7fffffffffffffffll;
        warp_argmin(f, idx);
    }
    __syncthreads();
}

// Publishes this block's (f, idx) and reports whether the block is the last
// one of the grid to arrive (threadfence-reduction pattern).  Called by
// every thread; returns the same bool to all threads of the block.  The
// last block must reset ctrl->blocks_done to 0 when it has finished.
__device__ __forceinline__ bool publish_and_check_last(double f, long long idx, ArgPair* partials,
                                                       Ctrl* ctrl, int* s_last,
                                                       int block = -1, int nblocks = -1) {
    if (block < 0) {
        block = blockIdx.x;
        nblocks = gridDim.x;
    }
    if (threadIdx.x == 0) {
        partials[block].f = f;
        partials[block].idx = idx;
        __threadfence();
        const unsigned prev = atomicAdd(&ctrl->blocks_done, 1u);
        *s_last = (prev == (unsigned)nblocks - 1) ? 1 : 0;
    }
    __syncthreads();
    const bool last = *s_last != 0;
    if (last) __threadfence();
    return last;
}

// In the last block: reduce the gridDim.x partials; thread 0 gets the result.
__device__ __forceinline__ void reduce_partials(const ArgPair* partials, double& f, long long& idx,
                                                ArgPair* scratch, int nblocks = -1) {
    if (nblocks < 0) nblocks = gridDim.x;
    f = CUDART_INF;
    idx = 0x7fffffffffffffffll;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        volatile const ArgPair* p = partials + b;
        const double pf = p->f;
        const long long pi = p->idx;
        if (better(pf, pi, f, idx)) {
            f = pf;
            idx = pi;
        }
    }
    block_argmin(f, idx, scratch);
}

}  // namespace zeus
