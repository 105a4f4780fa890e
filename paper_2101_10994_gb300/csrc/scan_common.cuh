// Block-wide exclusive prefix sums shared by the ordering kernels (the
// tracers' ray-group handout, the batch's chunk order) and the point sort.
#pragma once

#include <cuda_runtime.h>

namespace nglod {

__device__ __forceinline__ int warp_inclusive_sum(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive prefix of v over the block (blockDim.x a multiple of 32, at most
// 1024); ws holds 33 ints of shared memory; total receives the block's sum.
// Every thread of the block calls it.
__device__ __forceinline__ int block_exclusive_sum(int v, int* ws, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int incl = warp_inclusive_sum(v, lane);
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int s = lane < nw ? ws[lane] : 0;
        const int si = warp_inclusive_sum(s, lane);
        if (lane < nw) ws[lane] = si - s;
        if (lane == 31) ws[32] = si;
    }
    __syncthreads();
    total = ws[32];
    const int r = ws[w] + incl - v;
    __syncthreads();   // ws may be reused right away
    return r;
}

}  // namespace nglod
