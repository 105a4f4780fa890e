// svo_build / svo_info / svo_free / nglod_last_error and the status plumbing.
//
// The octree (Sec. 3.2) arrives as sorted Morton keys per depth.  The build
// derives, on the device, everything the traversal and the feature query
// need: packed voxel coordinates, parent index, occupied-children mask and
// first-child index per voxel, and -- the initialisation step of Sec. 3.4 --
// the 8 corner ids per voxel, with corners shared between neighbours.
//
// Corner deduplication marks every corner in a bitmap over the Morton space
// of the (2^dp + 1)^3 corner lattice; a corner's id is the number of marked
// corners with a smaller Morton key (an exclusive scan of per-word popcounts
// plus a popcount inside the word), which is exactly its rank among the
// sorted unique corner keys.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nglod_internal.cuh"

namespace nglod {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int check_cuda(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? NGLOD_ERR_OOM : NGLOD_ERR_CUDA;
}

static std::atomic<long long> g_wait_polls{kDefaultWaitPolls};

long long mma_wait_polls() { return g_wait_polls.load(std::memory_order_relaxed); }

int device_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

namespace {

__device__ __forceinline__ uint32_t compact3(uint64_t x) {
    // keep bits 0, 3, 6, ... of x and pack them
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x001f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x001f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x00000000001fffffull;
    return (uint32_t)x;
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ int64_t lower_bound_dev(const uint64_t* keys, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Validates depth dp and fills its node records (parent, coords, first child).
__global__ void k_nodes(const uint64_t* __restrict__ keys, int64_t n, int dp,
                        const uint64_t* __restrict__ pkeys, int64_t pn,
                        const uint64_t* __restrict__ ckeys, int64_t cn,
                        Node* __restrict__ node, int* __restrict__ err) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[v];
        const uint64_t limit = dp == 0 ? 1ull : (1ull << (3 * dp));
        if (key >= limit || (v > 0 && keys[v - 1] >= key)) atomicExch(err, 1);
        Node nd;
        nd.ijk = pack_ijk(compact3(key), compact3(key >> 1), compact3(key >> 2));
        nd.childmask = 0u;
        nd.childbase = ckeys ? (int32_t)lower_bound_dev(ckeys, cn, key << 3) : 0;
        nd.parent = -1;
        if (dp > 0) {
            const int64_t p = lower_bound_dev(pkeys, pn, key >> 3);
            if (p >= pn || pkeys[p] != (key >> 3)) atomicExch(err, 2);
            else nd.parent = (int32_t)p;
        }
        node[v] = nd;
    }
}

// Sets the child-mask bit of each voxel's parent.
__global__ void k_childmask(const uint64_t* __restrict__ keys, int64_t n,
                            const Node* __restrict__ node, Node* __restrict__ pnode) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = node[v].parent;
        if (p >= 0) atomicOr(&pnode[p].childmask, 1u << (uint32_t)(keys[v] & 7u));
    }
}

__device__ __forceinline__ uint64_t corner_key(uint32_t ijk, int c) {
    return spread3(unpack_i(ijk) + (c & 1)) | (spread3(unpack_j(ijk) + ((c >> 1) & 1)) << 1) |
           (spread3(unpack_k(ijk) + ((c >> 2) & 1)) << 2);
}

__global__ void k_mark_corners(const Node* __restrict__ node, int64_t n,
                               uint32_t* __restrict__ bitmap) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * 8;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ck = corner_key(node[t >> 3].ijk, (int)(t & 7));
        atomicOr(&bitmap[ck >> 5], 1u << (uint32_t)(ck & 31u));
    }
}

__global__ void k_assign_corners(const Node* __restrict__ node, int64_t n,
                                 const uint32_t* __restrict__ bitmap,
                                 const uint32_t* __restrict__ prefix,
                                 int32_t* __restrict__ corners) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * 8;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ck = corner_key(node[t >> 3].ijk, (int)(t & 7));
        const uint32_t w = bitmap[ck >> 5];
        const uint32_t below = w & ((1u << (uint32_t)(ck & 31u)) - 1u);
        corners[t] = (int32_t)(prefix[ck >> 5] + (uint32_t)__popc(below));
    }
}

struct NodePtrs {
    const Node* node[kMaxDepth + 1];
};

// Ancestor table of depth d: the voxel ids at depths 3..d along the parent
// chain, so a query reads all of them with one 32-byte load.
__global__ void k_ancestors(NodePtrs np, int d, int64_t n, int32_t* __restrict__ anc) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t rec[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) rec[i] = -1;
        int32_t id = (int32_t)v;
        for (int dd = d; dd >= kFirstFeatureDepth; --dd) {
            rec[dd - kFirstFeatureDepth] = id;
            id = np.node[dd][id].parent;
        }
        int4* dst = reinterpret_cast<int4*>(anc + 8 * v);
        dst[0] = make_int4(rec[0], rec[1], rec[2], rec[3]);
        dst[1] = make_int4(rec[4], rec[5], rec[6], rec[7]);
    }
}

// Flat corner-id table of depth d: for voxel v the corner ids of its
// ancestors at depths 3..d, level by level (anc then corners, resolved once
// here so a query's ids are one load per level instead of two dependent ones).
struct CornerPtrs {
    const int32_t* corners[kMaxDepth + 1];
};

__global__ void k_flat_corners(CornerPtrs cp, int d, int64_t n, const int32_t* __restrict__ anc,
                               int32_t* __restrict__ cids) {
    const int nl = d - kFirstFeatureDepth + 1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nl * 8;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = t / (nl * 8);
        const int i = (int)((t / 8) % nl), c = (int)(t & 7);
        const int32_t a = anc[8 * v + i];
        cids[t] = cp.corners[kFirstFeatureDepth + i][8 * (int64_t)a + c];
    }
}

// ---- three-pass exclusive scan of per-word popcounts (build time only) ----
constexpr int kScanBlock = 1024;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums,
                                                         uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        warp_sums[lane] = si - s;
        if (lane == 31) warp_sums[32] = si;
    }
    __syncthreads();
    total = warp_sums[32];
    const uint32_t r = warp_sums[warp] + incl - v;
    __syncthreads();
    return r;
}

__global__ void k_popc_block_sums(const uint32_t* __restrict__ bitmap, int64_t nw,
                                  uint32_t* __restrict__ block_sums) {
    __shared__ uint32_t ws[33];
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const uint32_t v = i < nw ? (uint32_t)__popc(bitmap[i]) : 0u;
    uint32_t total;
    block_exclusive_scan(v, ws, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void k_scan_block_sums(uint32_t* __restrict__ sums, int64_t nb, uint32_t* __restrict__ grand) {
    __shared__ uint32_t ws[33];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, ws, total);
        if (i < nb) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_popc_prefix(const uint32_t* __restrict__ bitmap, int64_t nw,
                              const uint32_t* __restrict__ block_prefix,
                              uint32_t* __restrict__ prefix) {
    __shared__ uint32_t ws[33];
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const uint32_t v = i < nw ? (uint32_t)__popc(bitmap[i]) : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(v, ws, total);
    if (i < nw) prefix[i] = block_prefix[blockIdx.x] + ex;
}

int grid_for(int64_t n, int block = 256) {
    int64_t g = (n + block - 1) / block;
    const int64_t cap = (int64_t)device_sms() * 32;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

void destroy(nglod_svo* s, cudaStream_t st) {
    if (!s) return;
    for (int d = 0; d <= kMaxDepth; ++d) {
        if (s->node[d]) cudaFreeAsync(s->node[d], st);
        if (s->corners[d]) cudaFreeAsync(s->corners[d], st);
        if (s->anc[d]) cudaFreeAsync(s->anc[d], st);
        if (s->cids[d]) cudaFreeAsync(s->cids[d], st);
    }
    if (s->dstatus) cudaFreeAsync(s->dstatus, st);
    if (s->dscratch) cudaFreeAsync(s->dscratch, st);
    cudaStreamSynchronize(st);
    delete s;
}

}  // namespace
}  // namespace nglod

using namespace nglod;

extern "C" const char* nglod_last_error(void) { return g_last_error.c_str(); }

extern "C" int nglod_set_wait_polls(int64_t polls) {
    g_wait_polls.store(polls < 0 ? kDefaultWaitPolls : (long long)polls, std::memory_order_relaxed);
    return NGLOD_OK;
}

extern "C" int svo_build(const uint64_t* const* h_keys, const int64_t* h_counts, int num_depths,
                         void* stream, nglod_svo** out) {
    if (!out) return fail(NGLOD_ERR_INVALID_ARG, "svo_build: out is NULL");
    *out = nullptr;
    if (!h_keys || !h_counts) return fail(NGLOD_ERR_INVALID_ARG, "svo_build: NULL keys/counts");
    if (num_depths < kFirstFeatureDepth + 1 || num_depths > kMaxDepth + 1)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_build: num_depths must be in [4, 11]");
    if (h_counts[0] != 1 || !h_keys[0] || h_keys[0][0] != 0ull)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_build: depth 0 must hold exactly the root key 0");
    for (int d = 0; d < num_depths; ++d) {
        if (h_counts[d] < 1 || h_counts[d] > (int64_t)1 << (3 * d) || (h_counts[d] > 0 && !h_keys[d]))
            return fail(NGLOD_ERR_INVALID_ARG, "svo_build: bad voxel count at depth " + std::to_string(d));
        if (h_counts[d] >= ((int64_t)1 << 31) / 8)
            return fail(NGLOD_ERR_NOT_SUPPORTED, "svo_build: too many voxels at one depth");
    }
    cudaStream_t st = (cudaStream_t)stream;
    nglod_svo* s = new (std::nothrow) nglod_svo();
    if (!s) return fail(NGLOD_ERR_OOM, "svo_build: host allocation failed");
    s->num_depths = num_depths;
    s->num_sms = device_sms();
    cudaGetDevice(&s->device);

    std::vector<uint64_t*> dkeys(num_depths, nullptr);
    int* derr = nullptr;
    uint32_t* scratch = nullptr;
    int status = NGLOD_OK;
    auto cleanup_tmp = [&]() {
        for (auto p : dkeys) if (p) cudaFreeAsync(p, st);
        if (derr) cudaFreeAsync(derr, st);
        if (scratch) cudaFreeAsync(scratch, st);
        cudaStreamSynchronize(st);
    };
#define BUILD_CUDA(call)                                          \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) {                                  \
            status = check_cuda(_e, #call);                       \
            cleanup_tmp();                                        \
            destroy(s, st);                                       \
            return status;                                        \
        }                                                         \
    } while (0)

    BUILD_CUDA(cudaMallocAsync(&derr, sizeof(int), st));
    BUILD_CUDA(cudaMallocAsync(&s->dstatus, sizeof(int), st));
    BUILD_CUDA(cudaMemsetAsync(s->dstatus, 0, sizeof(int), st));
    BUILD_CUDA(cudaMallocAsync(&s->dscratch, sizeof(unsigned) * 16, st));
    BUILD_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
    for (int d = 0; d < num_depths; ++d) {
        s->n[d] = h_counts[d];
        BUILD_CUDA(cudaMallocAsync(&dkeys[d], sizeof(uint64_t) * h_counts[d], st));
        BUILD_CUDA(cudaMemcpyAsync(dkeys[d], h_keys[d], sizeof(uint64_t) * h_counts[d],
                                   cudaMemcpyHostToDevice, st));
        BUILD_CUDA(cudaMallocAsync(&s->node[d], sizeof(Node) * h_counts[d], st));
    }
    for (int d = 0; d < num_depths; ++d) {
        const bool has_child = d + 1 < num_depths;
        k_nodes<<<grid_for(s->n[d]), 256, 0, st>>>(
            dkeys[d], s->n[d], d, d > 0 ? dkeys[d - 1] : nullptr, d > 0 ? s->n[d - 1] : 0,
            has_child ? dkeys[d + 1] : nullptr, has_child ? s->n[d + 1] : 0, s->node[d], derr);
    }
    for (int d = 1; d < num_depths; ++d)
        k_childmask<<<grid_for(s->n[d]), 256, 0, st>>>(dkeys[d], s->n[d], s->node[d], s->node[d - 1]);
    BUILD_CUDA(cudaGetLastError());
    int herr = 0;
    BUILD_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
    BUILD_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        cleanup_tmp();
        destroy(s, st);
        return fail(NGLOD_ERR_INVALID_ARG, herr == 1 ? "svo_build: keys not strictly increasing or out of range"
                                                     : "svo_build: a voxel's parent is missing");
    }
    {
        NodePtrs np;
        for (int d = 0; d <= kMaxDepth; ++d) np.node[d] = d < num_depths ? s->node[d] : nullptr;
        for (int d = kFirstFeatureDepth; d < num_depths; ++d) {
            BUILD_CUDA(cudaMallocAsync(&s->anc[d], sizeof(int32_t) * 8 * s->n[d], st));
            k_ancestors<<<grid_for(s->n[d]), 256, 0, st>>>(np, d, s->n[d], s->anc[d]);
        }
    }
    for (int d = kFirstFeatureDepth; d < num_depths; ++d) {
        const int64_t nbits = (int64_t)1 << (3 * (d + 1));
        const int64_t nw = nbits >> 5;
        const int64_t nb = (nw + kScanBlock - 1) / kScanBlock;
        // bitmap | prefix | block sums | grand total
        BUILD_CUDA(cudaMallocAsync(&scratch, sizeof(uint32_t) * (2 * nw + nb + 1), st));
        uint32_t* bitmap = scratch;
        uint32_t* prefix = scratch + nw;
        uint32_t* bsums = prefix + nw;
        uint32_t* grand = bsums + nb;
        BUILD_CUDA(cudaMemsetAsync(bitmap, 0, sizeof(uint32_t) * nw, st));
        k_mark_corners<<<grid_for(s->n[d] * 8), 256, 0, st>>>(s->node[d], s->n[d], bitmap);
        k_popc_block_sums<<<(unsigned)nb, kScanBlock, 0, st>>>(bitmap, nw, bsums);
        k_scan_block_sums<<<1, kScanBlock, 0, st>>>(bsums, nb, grand);
        k_popc_prefix<<<(unsigned)nb, kScanBlock, 0, st>>>(bitmap, nw, bsums, prefix);
        BUILD_CUDA(cudaMallocAsync(&s->corners[d], sizeof(int32_t) * 8 * s->n[d], st));
        k_assign_corners<<<grid_for(s->n[d] * 8), 256, 0, st>>>(s->node[d], s->n[d], bitmap, prefix,
                                                               s->corners[d]);
        BUILD_CUDA(cudaGetLastError());
        uint32_t total = 0;
        BUILD_CUDA(cudaMemcpyAsync(&total, grand, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        BUILD_CUDA(cudaStreamSynchronize(st));
        s->nc[d] = total;
        cudaFreeAsync(scratch, st);
        scratch = nullptr;
    }
    {
        CornerPtrs cp;
        for (int d = 0; d <= kMaxDepth; ++d) cp.corners[d] = d < num_depths ? s->corners[d] : nullptr;
        for (int d = kFirstFeatureDepth; d < num_depths; ++d) {
            const int64_t cnt = s->n[d] * (d - kFirstFeatureDepth + 1) * 8;
            BUILD_CUDA(cudaMallocAsync(&s->cids[d], sizeof(int32_t) * cnt, st));
            k_flat_corners<<<grid_for(cnt), 256, 0, st>>>(cp, d, s->n[d], s->anc[d], s->cids[d]);
        }
        BUILD_CUDA(cudaGetLastError());
    }
    cleanup_tmp();
#undef BUILD_CUDA
    *out = s;
    return NGLOD_OK;
}

extern "C" int svo_info(const nglod_svo* s, int* h_num_depths, int64_t* h_voxels, int64_t* h_corners) {
    if (!s) return fail(NGLOD_ERR_INVALID_ARG, "svo_info: NULL handle");
    if (h_num_depths) *h_num_depths = s->num_depths;
    for (int d = 0; d < s->num_depths; ++d) {
        if (h_voxels) h_voxels[d] = s->n[d];
        if (h_corners && d >= kFirstFeatureDepth) h_corners[d - kFirstFeatureDepth] = s->nc[d];
    }
    return NGLOD_OK;
}

extern "C" int svo_device_arrays(const nglod_svo* s, int dp, const void** node, const int32_t** corners) {
    if (!s || dp < 0 || dp >= s->num_depths)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_device_arrays: bad handle or depth");
    if (node) *node = s->node[dp];
    if (corners) *corners = dp >= kFirstFeatureDepth ? s->corners[dp] : nullptr;
    return NGLOD_OK;
}

extern "C" int svo_read_arrays(const nglod_svo* s, int dp, void* h_node, int32_t* h_corners, int32_t* h_anc) {
    if (!s || dp < 0 || dp >= s->num_depths)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_read_arrays: bad handle or depth");
    if ((h_corners || h_anc) && dp < kFirstFeatureDepth)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_read_arrays: corners/ancestors exist for depth >= 3 only");
    const size_t V = (size_t)s->n[dp];
    if (h_node) NGLOD_CUDA(cudaMemcpy(h_node, s->node[dp], sizeof(Node) * V, cudaMemcpyDeviceToHost));
    if (h_corners) NGLOD_CUDA(cudaMemcpy(h_corners, s->corners[dp], sizeof(int32_t) * 8 * V, cudaMemcpyDeviceToHost));
    if (h_anc) NGLOD_CUDA(cudaMemcpy(h_anc, s->anc[dp], sizeof(int32_t) * 8 * V, cudaMemcpyDeviceToHost));
    return NGLOD_OK;
}

extern "C" void svo_free(nglod_svo* s) {
    if (!s) return;
    destroy(s, (cudaStream_t)0);
}
