// nglod_sort_points: reorders sample points by the Morton code of the
// octree cell of a given depth that contains them (a counting sort), so
// that neighbouring samples share voxels and corner rows.  Eq. 4 sums over
// the samples, so their order changes no gradient beyond FP32 rounding;
// sorted batches let the tensor-core adjoint merge the corner updates of a
// warp (one atomic per corner and block of samples in the same voxel) and
// keep the corner rows of its gathers in L1.
//   k_sort_keys     key = Morton code of clamp(floor((x + 1) 2^(depth-1))),
//                   counted per key (atomics; keys of 3 depth bits);
//   k_scan_*        exclusive sum of the 2^(3 depth) counts (block sums,
//                   one block over them, block-local scans);
//   k_sort_scatter  every point to its key's next slot (the lanes of a
//                   warp with the same key share one atomic).
#include <cuda_runtime.h>

#include <algorithm>

#include "nglod_internal.cuh"
#include "scan_common.cuh"

namespace nglod {
namespace {

constexpr int kSortThreads = 256;
constexpr int kScanBlock = 1024;       // counts per block of the scan
constexpr int kMaxSortDepth = 7;       // 2^21 keys

__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t cell_key(const float* __restrict__ x, long long i, int depth) {
    const float sc = (float)(1 << (depth - 1));
    const int hi = (1 << depth) - 1;
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float q = __fmul_rn(__fadd_rn(x[3 * i + a], 1.0f), sc);
        // NaN and out-of-range points go to the nearest boundary cell
        const int v = q >= 0.0f ? (q < (float)hi ? (int)floorf(q) : hi) : 0;
        c[a] = (uint32_t)v;
    }
    return spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
}

__global__ void k_sort_keys(const float* __restrict__ x, long long Q, int depth, uint32_t* __restrict__ key,
                            int* __restrict__ count) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t k = cell_key(x, i, depth);
        key[i] = k;
        atomicAdd(&count[k], 1);
    }
}

// per block of kScanBlock counts: its sum
__global__ void k_scan_sums(const int* __restrict__ count, long long n, int* __restrict__ bsum) {
    __shared__ int ws[33];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    int total;
    block_exclusive_sum(i < n ? count[i] : 0, ws, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// exclusive sum of the block sums, in place (one block, sequential over chunks)
__global__ void k_scan_top(int* __restrict__ bsum, int nb) {
    __shared__ int ws[33];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += kScanBlock) {
        const int i = b0 + threadIdx.x;
        int total;
        const int e = block_exclusive_sum(i < nb ? bsum[i] : 0, ws, total);
        if (i < nb) bsum[i] = carry + e;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

// cursor[i] = exclusive prefix of count[i]
__global__ void k_scan_apply(const int* __restrict__ count, long long n, const int* __restrict__ bsum,
                             int* __restrict__ cursor) {
    __shared__ int ws[33];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    int total;
    const int e = block_exclusive_sum(i < n ? count[i] : 0, ws, total);
    if (i < n) cursor[i] = bsum[blockIdx.x] + e;
}

__global__ void k_sort_scatter(const float* __restrict__ x, const float* __restrict__ extra, long long Q,
                               const uint32_t* __restrict__ key, int* __restrict__ cursor, float* __restrict__ x_out,
                               float* __restrict__ extra_out, int32_t* __restrict__ perm) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < Q; i0 += stride) {
        const long long i = i0 + lane;
        const bool act = i < Q;
        const unsigned live = __ballot_sync(0xffffffffu, act);
        if (!act) continue;
        const uint32_t k = key[i];
        const unsigned peers = __match_any_sync(live, k);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&cursor[k], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        const long long pos = base + __popc(peers & ((1u << lane) - 1u));
        x_out[3 * pos] = x[3 * i];
        x_out[3 * pos + 1] = x[3 * i + 1];
        x_out[3 * pos + 2] = x[3 * i + 2];
        if (extra) extra_out[pos] = extra[i];
        if (perm) perm[pos] = (int32_t)i;
    }
}

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace nglod

using namespace nglod;

extern "C" size_t nglod_sort_points_workspace(int64_t Q, int depth) {
    if (Q < 0 || depth < 1 || depth > kMaxSortDepth) return 0;
    const size_t nk = (size_t)1 << (3 * depth);
    const size_t nb = (nk + kScanBlock - 1) / kScanBlock;
    return al256(sizeof(uint32_t) * (size_t)Q) + 2 * al256(sizeof(int) * nk) + al256(sizeof(int) * nb);
}

extern "C" int nglod_sort_points(const float* x, const float* extra, int64_t Q, int depth, float* x_out,
                                 float* extra_out, int32_t* perm, void* work, size_t work_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (Q < 0 || Q >= (1ll << 31)) return fail(NGLOD_ERR_INVALID_ARG, "nglod_sort_points: bad Q");
    if (depth < 1 || depth > kMaxSortDepth) return fail(NGLOD_ERR_INVALID_ARG, "nglod_sort_points: depth must lie in 1..7");
    if (Q == 0) return NGLOD_OK;
    if (!x || !x_out || !work || (extra && !extra_out)) return fail(NGLOD_ERR_INVALID_ARG, "nglod_sort_points: NULL argument");
    if (x == x_out || (extra && extra == extra_out)) return fail(NGLOD_ERR_INVALID_ARG, "nglod_sort_points: in place");
    if (work_bytes < nglod_sort_points_workspace(Q, depth))
        return fail(NGLOD_ERR_CAPACITY, "nglod_sort_points: workspace too small");
    const long long nk = 1ll << (3 * depth);
    const int nb = (int)((nk + kScanBlock - 1) / kScanBlock);
    char* w = static_cast<char*>(work);
    uint32_t* key = reinterpret_cast<uint32_t*>(w);
    int* count = reinterpret_cast<int*>(w + al256(sizeof(uint32_t) * (size_t)Q));
    int* cursor = reinterpret_cast<int*>(reinterpret_cast<char*>(count) + al256(sizeof(int) * (size_t)nk));
    int* bsum = reinterpret_cast<int*>(reinterpret_cast<char*>(cursor) + al256(sizeof(int) * (size_t)nk));
    NGLOD_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)nk, st));
    const int sms = device_sms();
    const int g = (int)std::max<long long>(1, std::min<long long>((Q + kSortThreads - 1) / kSortThreads, (long long)sms * 8));
    k_sort_keys<<<g, kSortThreads, 0, st>>>(x, Q, depth, key, count);
    k_scan_sums<<<nb, kScanBlock, 0, st>>>(count, nk, bsum);
    k_scan_top<<<1, kScanBlock, 0, st>>>(bsum, nb);
    k_scan_apply<<<nb, kScanBlock, 0, st>>>(count, nk, bsum, cursor);
    k_sort_scatter<<<g, kSortThreads, 0, st>>>(x, extra, Q, key, cursor, x_out, extra_out, perm);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}
