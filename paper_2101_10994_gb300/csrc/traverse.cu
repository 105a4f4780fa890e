// svo_trace_rays: level-synchronous ray/octree intersection.
//
// Algorithm 1 of the paper runs, per octree level, Decide (one thread per
// ray/voxel pair), ExclusiveSum of the decisions, then Subdivide (write the
// hit voxels' occupied children, front to back) or, at the target level,
// Compactify (keep the hit pairs).  Here the three steps of one level are a
// single kernel: each CTA takes the next tile of the pair list (tiles are
// handed out in order by an atomic counter), decides its pairs, scans the
// decisions inside the CTA, obtains the tile's global offset with a
// decoupled look-back over the preceding tiles' published sums, and writes
// its children (or compacted hits) straight to their final positions.  The
// decisions and their prefix sums never touch memory, the list sizes stay on
// the device, and no host round trip happens between levels.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "nglod_internal.cuh"

namespace nglod {
namespace {

constexpr int kThreads = 256;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr long kSpinLimit = 1l << 22;   // ~0.1-1 s of waiting, then time out

struct Counters {
    long long count[kMaxDepth + 2];   // list length entering each depth
    long long max_pairs;
    int tile_ctr[kMaxDepth + 2];
    int status;                        // kStatus*
};

struct LevelParams {
    const RayPrep* rays;
    const Node* node;                  // voxels of depth dp
    const int2* in;                    // pairs entering depth dp (NULL at dp 0)
    int2* out;                         // children (dp < D)
    long long out_cap;
    int32_t* voxel_id;                 // dp == D outputs
    float2* t_range;
    int32_t* out_ray;
    long long hit_cap;
    Counters* ctr;
    unsigned long long* tile_state;
    int dp, D;
};

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive prefix of this tile among all tiles (decoupled look-back),
// computed by one whole warp: each poll reads the published states of the 32
// nearest unvisited predecessors at once, sums the aggregates up to the
// nearest one that already carries its inclusive prefix, and moves the
// window back only when none does.  Every wait is bounded; on expiry the
// status word records a timeout and the (then meaningless) partial prefix is
// returned.
__device__ long long tile_prefix_warp(unsigned long long* state, long long tile, long long agg, int* status) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_release(state, kFlagPre | (unsigned long long)agg);
        return 0;
    }
    if (lane == 0) st_release(state + tile, kFlagAgg | (unsigned long long)agg);
    long long excl = 0;
    long long end = tile - 1;          // nearest predecessor not yet summed
    long spins = 0;
    for (;;) {
        const long long j = end - lane;
        const unsigned long long s = j >= 0 ? ld_acquire(state + j) : kFlagPre;
        const unsigned long long flag = s & ~kValMask;
        if (__any_sync(0xffffffffu, flag == 0ull)) {
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicExch(status, kStatusTimeout);
                break;
            }
            if (spins > 16) __nanosleep(32);
            continue;
        }
        const unsigned pre = __ballot_sync(0xffffffffu, flag == kFlagPre);
        const int stop = pre ? __ffs(pre) - 1 : 31;
        long long v = lane <= stop ? (long long)(s & kValMask) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pre) break;
        end -= 32;
    }
    if (lane == 0) st_release(state + tile, kFlagPre | (unsigned long long)(excl + agg));
    return excl;
}

__device__ __forceinline__ int block_exclusive_sum(int v, int* warp_sums, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int s = lane < kThreads / 32 ? warp_sums[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = si - s;
        if (lane == kThreads / 32 - 1) warp_sums[kThreads / 32] = si;
    }
    __syncthreads();
    total = warp_sums[kThreads / 32];
    return warp_sums[warp] + incl - v;
}

__global__ void __launch_bounds__(kThreads) k_prep_rays(const float* __restrict__ o,
                                                        const float* __restrict__ d, long long R,
                                                        RayPrep* __restrict__ rays, Counters* ctr) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R;
         r += (long long)gridDim.x * blockDim.x) {
        RayPrep p;
        p.ox = o[3 * r];
        p.oy = o[3 * r + 1];
        p.oz = o[3 * r + 2];
        const float dd[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
        const float oo[3] = {p.ox, p.oy, p.oz};
        int ok = 1, par = 0;
        float inv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!isfinite(oo[a]) || !isfinite(dd[a])) ok = 0;
            const bool pa = fabsf(dd[a]) < 1.17549435e-38f;
            par |= pa ? (1 << a) : 0;
            inv[a] = pa ? 0.0f : __fdiv_rn(1.0f, dd[a]);
        }
        if (par == 7) ok = 0;
        p.ix = inv[0];
        p.iy = inv[1];
        p.iz = inv[2];
        p.par = par;
        p.valid = ok;
        rays[r] = p;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->count[0] = R;
}

// One level of the traversal, with Decide of the next level fused into
// Subdivide.  Input: the pairs (ray, voxel) of depth dp that Decide kept (at
// dp = 0 the implicit pairs (ray, root), which are decided here first).  For
// each input pair the thread tests the voxel's occupied children (their
// bounds follow from the parent's coordinates, no load needed), counts the
// hit ones (Decide of depth dp + 1), the CTA scans the counts
// (ExclusiveSum) and obtains its tile's global offset by decoupled
// look-back, and the hit children are written in front-to-back rank order
// (Subdivide).  When depth dp + 1 is the target depth the written list is
// the final one (Compactify): voxel ids, their (t_enter, t_exit) and the ray
// of each entry.  Output order and contents equal those of the unfused
// Decide / ExclusiveSum / Subdivide / Compactify sequence.
constexpr int kTileX = kThreads * 2;                 // parents per tile (2 per thread)
constexpr int kStageBytes = kTileX * 8 * 16;         // up to 8 children x 16 B per parent

__global__ void __launch_bounds__(kThreads) k_level(const LevelParams p) {
    constexpr int kIt = kTileX / kThreads;
    extern __shared__ __align__(16) unsigned char stage[];
    int2* stage_p = reinterpret_cast<int2*>(stage);
    int32_t* stage_i = reinterpret_cast<int32_t*>(stage);
    float2* stage_f = reinterpret_cast<float2*>(stage + kTileX * 8 * sizeof(int32_t));
    int32_t* stage_r = reinterpret_cast<int32_t*>(stage + kTileX * 8 * (sizeof(int32_t) + sizeof(float2)));
    __shared__ int warp_sums[kThreads / 32 + 1];
    __shared__ long long s_tile;
    __shared__ long long s_prefix;
    if (p.ctr->status != kStatusOk) return;
    const long long n = p.ctr->count[p.dp];
    const long long ntiles = (n + kTileX - 1) / kTileX;
    const int dc = p.dp + 1;                          // depth of the children
    const bool final_level = dc == p.D;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&p.ctr->tile_ctr[p.dp], 1);
        __syncthreads();
        const long long tile = s_tile;
        if (tile >= ntiles) break;
        const long long base = tile * kTileX + (long long)threadIdx.x * kIt;
        int2 pr[kIt];
        RayPrep ray[kIt];
        uint32_t cij[kIt];       // coordinates of child slot 0 (parent coords << 1)
        uint32_t mask[kIt];      // occupied children (slot bits)
        uint32_t hitr[kIt];      // hit children, by front-to-back rank
        uint32_t oct[kIt];
        int32_t cb[kIt];
        int sum = 0;
        if (p.dp > 0 && base + kIt <= n) {
            const int4 a = *reinterpret_cast<const int4*>(p.in + base);
            pr[0] = make_int2(a.x, a.y);
            pr[1] = make_int2(a.z, a.w);
        } else {
#pragma unroll
            for (int i = 0; i < kIt; ++i) {
                const long long idx = base + i;
                pr[i] = idx < n ? (p.dp == 0 ? make_int2((int)idx, 0) : p.in[idx]) : make_int2(-1, -1);
            }
        }
#pragma unroll
        for (int i = 0; i < kIt; ++i) {
            hitr[i] = 0;
            mask[i] = 0;
            oct[i] = 0;
            cb[i] = 0;
            cij[i] = 0;
            if (pr[i].x < 0) continue;
            ray[i] = p.rays[pr[i].x];
            const Node nd = p.node[pr[i].y];
            uint32_t o8;
            if (p.dp == 0) {
                // the root is the only undecided input; every other pair was kept by Decide
                float t0, t1;
                if (!ray[i].valid || !slab_test(ray[i], nd.ijk, 0, t0, t1, &o8)) continue;
            } else {
                o8 = origin_octant(ray[i], nd.ijk, p.dp);
            }
            mask[i] = nd.childmask;
            oct[i] = o8;
            cb[i] = nd.childbase;
            cij[i] = (nd.ijk << 1) & 0x3ffffffeu;
            uint32_t h = 0;
            for (uint32_t rm = rank_mask(nd.childmask, o8); rm; rm &= rm - 1u) {
                const uint32_t r = (uint32_t)(__ffs(rm) - 1);
                const uint32_t c = r ^ o8;
                const uint32_t ijk = cij[i] | pack_ijk(c & 1u, (c >> 1) & 1u, (c >> 2) & 1u);
                float a0, a1;
                if (slab_test(ray[i], ijk, dc, a0, a1)) h |= 1u << r;
            }
            hitr[i] = h;
            sum += __popc(h);
        }
        int tile_total;
        const int excl = block_exclusive_sum(sum, warp_sums, tile_total);
        if (threadIdx.x < 32) {
            const long long pre = tile_prefix_warp(p.tile_state, tile, tile_total, &p.ctr->status);
            if (threadIdx.x == 0) {
                s_prefix = pre;
                if (tile == ntiles - 1) {
                    const long long total = pre + tile_total;
                    p.ctr->count[dc] = total;
                    if (total > p.ctr->max_pairs) p.ctr->max_pairs = total;
                    if (total > (final_level ? p.hit_cap : p.out_cap))
                        atomicCAS(&p.ctr->status, kStatusOk, kStatusOverflow);
                }
            }
        }
        // stage this tile's output in shared memory at tile-local offsets ...
        int loc = excl;
#pragma unroll
        for (int i = 0; i < kIt; ++i) {
            for (uint32_t h = hitr[i]; h; h &= h - 1u) {
                const uint32_t c = (uint32_t)(__ffs(h) - 1) ^ oct[i];
                const int32_t child = cb[i] + __popc(mask[i] & ((1u << c) - 1u));
                if (final_level) {
                    float a0 = 0.f, a1 = 0.f;
                    slab_test(ray[i], cij[i] | pack_ijk(c & 1u, (c >> 1) & 1u, (c >> 2) & 1u), dc, a0, a1);
                    stage_i[loc] = child;
                    stage_f[loc] = make_float2(a0, a1);
                    stage_r[loc] = pr[i].x;
                } else {
                    stage_p[loc] = make_int2(pr[i].x, child);
                }
                ++loc;
            }
        }
        __syncthreads();
        // ... then write it to its global position with coalesced stores
        const long long off = s_prefix;
        if (final_level) {
            const long long lim = min((long long)tile_total, p.hit_cap - off);
            for (int i = threadIdx.x; i < lim; i += kThreads) {
                p.voxel_id[off + i] = stage_i[i];
                p.t_range[off + i] = stage_f[i];
                p.out_ray[off + i] = stage_r[i];
            }
        } else {
            const long long lim = min((long long)tile_total, p.out_cap - off);
            for (int i = threadIdx.x; i < lim; i += kThreads) p.out[off + i] = stage_p[i];
        }
        __syncthreads();   // s_tile / s_prefix / warp_sums / staging reuse
    }
}

// ray_offsets[r] = first list position whose ray is >= r (binary search).
__global__ void __launch_bounds__(kThreads) k_ray_offsets(const int32_t* __restrict__ out_ray,
                                                          const Counters* __restrict__ ctr, int D,
                                                          long long R, long long cap,
                                                          int32_t* __restrict__ offs) {
    const long long H = min(ctr->count[D], cap);   // never past what was written
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r <= R;
         r += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = H;
        while (lo < hi) {
            const long long mid = lo + ((hi - lo) >> 1);
            if (out_ray[mid] < r) lo = mid + 1; else hi = mid;
        }
        offs[r] = (int32_t)lo;
    }
}

size_t align_up(size_t v, size_t a = 256) { return (v + a - 1) / a * a; }

// Resident CTAs per SM of the level kernel with its staging buffer (the
// persistent grid is sized to exactly what fits).
int level_ctas_per_sm() {
    static int cached = 0;
    if (!cached) {
        cudaFuncSetAttribute(k_level, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBytes);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_level, kThreads, kStageBytes);
        cached = n > 0 ? n : 1;
    }
    return cached;
}

long long max_tiles(long long R, long long cap) {
    return (std::max(R, cap) + kTileX - 1) / kTileX + 1;
}

}  // namespace
}  // namespace nglod

using namespace nglod;

extern "C" size_t svo_trace_rays_workspace(int64_t R, int64_t pair_capacity) {
    if (R < 0 || pair_capacity < 0) return 0;
    return align_up(sizeof(Counters)) + align_up(sizeof(RayPrep) * (size_t)R) +
           2 * align_up(sizeof(int2) * (size_t)pair_capacity) +
           align_up(sizeof(unsigned long long) * (size_t)max_tiles(R, pair_capacity));
}

extern "C" int svo_trace_rays(const nglod_svo* svo, const float* o, const float* d, int64_t R,
                              int target_lod, void* work, size_t work_bytes, int64_t pair_capacity,
                              int32_t* ray_offsets, int32_t* voxel_id, float* t_range,
                              int64_t hit_capacity, int64_t* h_stats, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!svo) return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays: NULL octree");
    const int D = target_lod + kFirstFeatureDepth - 1;
    if (target_lod < 1 || D >= svo->num_depths)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays: target_lod outside 1.." +
                                               std::to_string(svo->num_depths - kFirstFeatureDepth));
    if (R < 0 || R >= (1ll << 31) - 1 || pair_capacity < 0 || hit_capacity < 0)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays: bad R or capacity");
    if (!ray_offsets) return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays: NULL ray_offsets");
    if (h_stats) h_stats[0] = h_stats[1] = 0;
    if (R == 0) {
        NGLOD_CUDA(cudaMemsetAsync(ray_offsets, 0, sizeof(int32_t), st));
        return NGLOD_OK;
    }
    if (!o || !d || !work) return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays: NULL input or workspace");
    if ((hit_capacity > 0 && (!voxel_id || !t_range)))
        return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays: NULL voxel_id / t_range");
    if (work_bytes < svo_trace_rays_workspace(R, pair_capacity))
        return fail(NGLOD_ERR_CAPACITY, "svo_trace_rays: workspace smaller than svo_trace_rays_workspace()");
    if (((uintptr_t)work & 255u) != 0) return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays: work must be 256-B aligned");

    char* w = (char*)work;
    Counters* ctr = (Counters*)w;
    w += align_up(sizeof(Counters));
    RayPrep* rays = (RayPrep*)w;
    w += align_up(sizeof(RayPrep) * (size_t)R);
    int2* buf[2];
    buf[0] = (int2*)w;
    w += align_up(sizeof(int2) * (size_t)pair_capacity);
    buf[1] = (int2*)w;
    w += align_up(sizeof(int2) * (size_t)pair_capacity);
    unsigned long long* tile_state = (unsigned long long*)w;
    const long long ntiles_max = max_tiles(R, pair_capacity);

    const int sms = svo->num_sms;
    NGLOD_CUDA(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
    k_prep_rays<<<std::min<long long>((R + kThreads - 1) / kThreads, (long long)sms * 16), kThreads, 0, st>>>(
        o, d, R, rays, ctr);
    for (int dp = 0; dp < D; ++dp) {
        NGLOD_CUDA(cudaMemsetAsync(tile_state, 0, sizeof(unsigned long long) * ntiles_max, st));
        LevelParams lp;
        lp.rays = rays;
        lp.node = svo->node[dp];
        lp.in = dp == 0 ? nullptr : buf[dp & 1];
        lp.out = buf[(dp + 1) & 1];
        lp.out_cap = pair_capacity;
        lp.voxel_id = voxel_id;
        lp.t_range = (float2*)t_range;
        lp.out_ray = (int32_t*)buf[(dp + 1) & 1];   // used when dp + 1 == D
        lp.hit_cap = std::min<long long>(hit_capacity, pair_capacity);
        lp.ctr = ctr;
        lp.tile_state = tile_state;
        lp.dp = dp;
        lp.D = D;
        const long long grid = std::min<long long>(ntiles_max, (long long)sms * level_ctas_per_sm());
        k_level<<<(unsigned)grid, kThreads, kStageBytes, st>>>(lp);
    }
    k_ray_offsets<<<std::min<long long>((R + kThreads) / kThreads, (long long)sms * 16), kThreads, 0, st>>>(
        (const int32_t*)buf[D & 1], ctr, D, R, std::min<long long>(hit_capacity, pair_capacity), ray_offsets);
    NGLOD_CUDA(cudaGetLastError());
    Counters h;
    NGLOD_CUDA(cudaMemcpyAsync(&h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    NGLOD_CUDA(cudaStreamSynchronize(st));
    const long long H = h.count[D];
    if (h_stats) {
        h_stats[0] = h.status == kStatusOk || H > 0 ? H : 0;
        h_stats[1] = h.max_pairs;
    }
    if (h.status == kStatusTimeout)
        return fail(NGLOD_ERR_TIMEOUT, "svo_trace_rays: scan look-back wait expired");
    if (h.status == kStatusOverflow) {
        long long need = 0;
        for (int dp = 1; dp < D; ++dp) need = std::max(need, h.count[dp]);
        if (h_stats) h_stats[1] = std::max<long long>(need, h.max_pairs);
        return fail(NGLOD_ERR_CAPACITY, "svo_trace_rays: list larger than capacity (pairs " +
                                            std::to_string(need) + ", hits " + std::to_string(H) + ")");
    }
    return NGLOD_OK;
}

// ---------------------------------------------------------------------------
// svo_trace_rays_noalloc: the same traversal with its workspace in a fixed
// device array compiled into this library, for callers that must not
// allocate device memory while they render.
//
// Who needs it: a renderer embedded in a host application that owns the
// GPU's memory budget (a viewer or engine plugin whose allocator hands out
// every byte), or a real-time frame loop that may not risk the implicit
// device-wide synchronisation cudaMalloc/cudaFree can cause in mid-frame.
// Such a caller passes only its inputs and outputs.
//
// The array below, kNoAllocScratchBytes (32 MiB) long, is created on every
// GPU that loads this library and stays there until the process exits.  Its
// host-side name is only a stand-in; the device address is looked up with
// cudaGetSymbolAddress once per device, the first time this entry point runs
// with that device current (make that first call before any stream
// capture).  All calls share the array and it keeps the previous call's
// contents: the traversal clears its own counters and scan state at the
// start of every call, but two calls that overlap on the GPU (different
// streams, or different host threads on one device) race on it.
// ---------------------------------------------------------------------------
#include <mutex>

namespace nglod {
namespace {
constexpr size_t kNoAllocScratchBytes = 32u << 20;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace
}  // namespace nglod

extern "C" int svo_trace_rays_noalloc(const nglod_svo* svo, const float* o, const float* d, int64_t R,
                                      int target_lod, int32_t* ray_offsets, int32_t* voxel_id,
                                      float* t_range, int64_t hit_capacity, int64_t* h_stats, void* stream) {
    using namespace nglod;
    if (R < 0) return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays_noalloc: R < 0");
    // the largest intermediate-list capacity whose workspace fits the array
    int64_t lo = 0, hi = (int64_t)(kNoAllocScratchBytes / sizeof(int2));
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (svo_trace_rays_workspace(R, mid) <= kNoAllocScratchBytes) lo = mid; else hi = mid - 1;
    }
    const int64_t pair_capacity = lo;
    if (R > 0 && pair_capacity < R)
        return fail(NGLOD_ERR_CAPACITY, "svo_trace_rays_noalloc: " + std::to_string(R) +
                                            " rays do not fit the fixed 32 MiB scratch (use svo_trace_rays with a "
                                            "caller-allocated workspace)");
    int dev = 0;
    NGLOD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(NGLOD_ERR_NOT_SUPPORTED, "svo_trace_rays_noalloc: device index out of range");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                return check_cuda(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                  "svo_trace_rays_noalloc: cudaGetSymbolAddress(scratch)");
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    const int rc = svo_trace_rays(svo, o, d, R, target_lod, scratch, kNoAllocScratchBytes, pair_capacity,
                                  ray_offsets, voxel_id, t_range, hit_capacity, h_stats, stream);
    if (rc == NGLOD_ERR_CAPACITY)
        set_error(std::string(nglod_last_error()) + " [svo_trace_rays_noalloc: the fixed 32 MiB scratch holds " +
                  std::to_string(pair_capacity) + " pairs per level for these rays]");
    return rc;
}
