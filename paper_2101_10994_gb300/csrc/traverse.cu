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
    int dp, D;
};

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
// dp = 0 the implicit pairs (ray, root), decided here first).  For each input
// pair a thread tests the voxel's occupied children (their bounds follow
// from the parent's coordinates, no load needed) and records which ones the
// ray hits (Decide of depth dp + 1).  The exclusive sum of the hit counts
// gives every pair its output position, and the hit children are written in
// front-to-back rank order (Subdivide); when depth dp + 1 is the target
// depth the written list is the final one (Compactify): voxel ids, their
// (t_enter, t_exit) and the ray of each entry.  Output order and contents
// equal those of the unfused Decide / ExclusiveSum / Subdivide / Compactify
// sequence.
//
// Scan structure: the launch is cooperative (every CTA resident) and each
// CTA owns one contiguous chunk of the input list.
//   pass 1  decide the chunk, store a 16-bit record per pair (hit children
//           by rank | octant << 8) and the chunk's hit count;
//   barrier one bounded grid-wide barrier; each CTA then sums the counts of
//           the chunks before it (the ExclusiveSum at chunk granularity);
//   pass 2  re-read the chunk (now L2-resident), scan inside each tile and
//           write the children at their final positions through shared
//           memory, coalesced.
// No CTA ever waits on another except at the single barrier.
constexpr int kTileX = kThreads * 2;                 // parents per pass-2 tile (2 per thread)
constexpr int kPass1 = 4;                            // parents per thread per pass-1 step
// staging: up to 8 children per parent, 8 B (pair) or 16 B (final entry) each
template <bool FINAL>
constexpr int stage_bytes() { return kTileX * 8 * (FINAL ? 16 : 8); }

struct LevelScratch {
    uint16_t* rec;          // [input pairs] hit-by-rank | octant << 8
    long long* chunk_cnt;   // [grid]
    unsigned* arrive;       // grid barrier counter (zeroed per level)
};

__device__ __forceinline__ bool grid_barrier(unsigned* arrive, unsigned nblocks, int* status) {
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(arrive, 1u);
        long spins = 0;
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(arrive) : "memory");
            if (v >= nblocks) break;
            if (++spins > kSpinLimit) {
                atomicExch(status, kStatusTimeout);
                ok = false;
                break;
            }
            if (spins > 32) __nanosleep(64);
        }
    }
    __syncthreads();
    return ok;
}

template <bool FINAL>
__global__ void __launch_bounds__(kThreads) k_level(const LevelParams p, const LevelScratch x) {
    constexpr int kIt = kTileX / kThreads;
    extern __shared__ __align__(16) unsigned char stage[];
    int2* stage_p = reinterpret_cast<int2*>(stage);
    int32_t* stage_i = reinterpret_cast<int32_t*>(stage);
    float2* stage_f = reinterpret_cast<float2*>(stage + kTileX * 8 * sizeof(int32_t));
    int32_t* stage_r = reinterpret_cast<int32_t*>(stage + kTileX * 8 * (sizeof(int32_t) + sizeof(float2)));
    __shared__ int warp_sums[kThreads / 32 + 1];
    __shared__ long long s_prefix;
    const bool skip = p.ctr->status != kStatusOk;     // uniform: earlier level failed
    const long long n = skip ? 0 : p.ctr->count[p.dp];
    const long long ntiles = (n + kTileX - 1) / kTileX;
    const long long per = (ntiles + gridDim.x - 1) / gridDim.x;
    const long long t_begin = min((long long)blockIdx.x * per, ntiles);
    const long long t_end = min(t_begin + per, ntiles);
    const int dc = p.dp + 1;                          // depth of the children
    constexpr bool final_level = FINAL;

    // ---- pass 1: Decide the children of every pair of the chunk ----
    long long mine = 0;
    const long long c_lo = t_begin * kTileX, c_hi = min(t_end * kTileX, n);
    for (long long base = c_lo + (long long)threadIdx.x * kPass1; base < c_hi; base += (long long)kThreads * kPass1) {
#pragma unroll
        for (int i = 0; i < kPass1; ++i) {
            const long long idx = base + i;
            if (idx >= c_hi) continue;
            const int2 pr = p.dp == 0 ? make_int2((int)idx, 0) : p.in[idx];
            const RayPrep ray = p.rays[pr.x];
            const Node nd = p.node[pr.y];
            uint32_t o8, h = 0;
            bool live = true;
            if (p.dp == 0) {
                float t0, t1;   // the root is the only undecided input
                live = ray.valid && slab_test(ray, nd.ijk, 0, t0, t1, &o8);
            } else {
                o8 = origin_octant(ray, nd.ijk, p.dp);
            }
            if (live && nd.childmask) {
                ChildSlabs cs;
                child_slabs(ray, nd.ijk, p.dp, cs);
                uint32_t hs = 0;   // by slot, all 8 tested without branches
#pragma unroll
                for (uint32_t c = 0; c < 8; ++c) {
                    float a0, a1;
                    hs |= child_hit(cs, c, a0, a1) ? (1u << c) : 0u;
                }
                h = rank_mask(hs & nd.childmask, o8);
            }
            x.rec[idx] = (uint16_t)(h | (live ? (o8 << 8) : 0u));
            mine += __popc(h);
        }
    }
    // chunk total -> scan of chunk totals (one bounded grid barrier)
    {
        int total;
        block_exclusive_sum((int)mine, warp_sums, total);
        if (threadIdx.x == 0) {
            asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(x.chunk_cnt + blockIdx.x),
                         "l"((unsigned long long)total)
                         : "memory");
        }
    }
    if (!grid_barrier(x.arrive, gridDim.x, &p.ctr->status)) return;
    if (threadIdx.x < 32) {
        long long acc = 0;
        for (unsigned b = threadIdx.x; b < blockIdx.x; b += 32) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(x.chunk_cnt + b) : "memory");
            acc += (long long)v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) {
            s_prefix = acc;
            if (blockIdx.x == gridDim.x - 1 && !skip) {
                unsigned long long mine_tot;
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(mine_tot) : "l"(x.chunk_cnt + blockIdx.x) : "memory");
                const long long total = acc + (long long)mine_tot;
                p.ctr->count[dc] = total;
                if (total > p.ctr->max_pairs) p.ctr->max_pairs = total;
                if (total > (final_level ? p.hit_cap : p.out_cap))
                    atomicCAS(&p.ctr->status, kStatusOk, kStatusOverflow);
            }
        }
    }
    __syncthreads();
    long long off = s_prefix;

    // ---- pass 2: positions inside each tile, then Subdivide / Compactify ----
    for (long long tile = t_begin; tile < t_end; ++tile) {
        const long long base = tile * kTileX + (long long)threadIdx.x * kIt;
        uint32_t rec[kIt];
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < kIt; ++i) {
            rec[i] = base + i < n ? x.rec[base + i] : 0u;
            cnt += __popc(rec[i] & 0xffu);
        }
        int tile_total;
        int loc = block_exclusive_sum(cnt, warp_sums, tile_total);
#pragma unroll
        for (int i = 0; i < kIt; ++i) {
            const uint32_t h0 = rec[i] & 0xffu;
            if (!h0) continue;
            const long long idx = base + i;
            const int2 pr = p.dp == 0 ? make_int2((int)idx, 0) : p.in[idx];
            const Node nd = p.node[pr.y];
            const uint32_t o8 = rec[i] >> 8;
            ChildSlabs cs;
            if (final_level) child_slabs(p.rays[pr.x], nd.ijk, p.dp, cs);
            for (uint32_t h = h0; h; h &= h - 1u) {
                const uint32_t c = (uint32_t)(__ffs(h) - 1) ^ o8;
                const int32_t child = nd.childbase + __popc(nd.childmask & ((1u << c) - 1u));
                if (final_level) {
                    float a0 = 0.f, a1 = 0.f;
                    child_hit(cs, c, a0, a1);
                    stage_i[loc] = child;
                    stage_f[loc] = make_float2(a0, a1);
                    stage_r[loc] = pr.x;
                } else {
                    stage_p[loc] = make_int2(pr.x, child);
                }
                ++loc;
            }
        }
        __syncthreads();
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
        off += tile_total;
        __syncthreads();   // staging and warp_sums reuse
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

constexpr int kMaxGrid = 4096;   // chunk-count slots (>= resident CTAs of the level kernel)

// Resident CTAs per SM of the level kernel with its staging buffer (the
// persistent grid is sized to exactly what fits).
template <bool FINAL>
int level_ctas_per_sm() {
    static int cached = 0;
    if (!cached) {
        cudaFuncSetAttribute(k_level<FINAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, stage_bytes<FINAL>());
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_level<FINAL>, kThreads, stage_bytes<FINAL>());
        cached = n > 0 ? n : 1;
    }
    return cached;
}


}  // namespace
}  // namespace nglod

using namespace nglod;

extern "C" size_t svo_trace_rays_workspace(int64_t R, int64_t pair_capacity) {
    if (R < 0 || pair_capacity < 0) return 0;
    const size_t n_in = (size_t)std::max<int64_t>(R, pair_capacity);
    return align_up(sizeof(Counters)) + align_up(sizeof(RayPrep) * (size_t)R) +
           2 * align_up(sizeof(int2) * (size_t)pair_capacity) +
           align_up(sizeof(unsigned long long) * kMaxGrid) + align_up(sizeof(unsigned) * (kMaxDepth + 2)) +
           align_up(sizeof(uint16_t) * n_in);
}

namespace nglod {
namespace {

// Enqueues the whole traversal on the stream (no host synchronisation).
int enqueue_traversal(const nglod_svo* svo, const float* o, const float* d, int64_t R, int target_lod, void* work,
                      size_t work_bytes, int64_t pair_capacity, int32_t* ray_offsets, int32_t* voxel_id,
                      float* t_range, int64_t hit_capacity, cudaStream_t st, const char* who) {
    const std::string w(who);
    if (!svo) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL octree");
    const int D = target_lod + kFirstFeatureDepth - 1;
    if (target_lod < 1 || D >= svo->num_depths)
        return fail(NGLOD_ERR_INVALID_ARG, w + ": target_lod outside 1.." +
                                               std::to_string(svo->num_depths - kFirstFeatureDepth));
    if (R < 0 || R >= (1ll << 31) - 1 || pair_capacity < 0 || hit_capacity < 0)
        return fail(NGLOD_ERR_INVALID_ARG, w + ": bad R or capacity");
    if (!ray_offsets) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL ray_offsets");
    if (!work) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL workspace");
    if (work_bytes < svo_trace_rays_workspace(R, pair_capacity))
        return fail(NGLOD_ERR_CAPACITY, w + ": workspace smaller than svo_trace_rays_workspace()");
    if (((uintptr_t)work & 255u) != 0) return fail(NGLOD_ERR_INVALID_ARG, w + ": work must be 256-B aligned");
    Counters* ctr = (Counters*)work;
    if (R == 0) {
        NGLOD_CUDA(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
        NGLOD_CUDA(cudaMemsetAsync(ray_offsets, 0, sizeof(int32_t), st));
        return NGLOD_OK;
    }
    if (!o || !d) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL rays");
    if ((hit_capacity > 0 && (!voxel_id || !t_range)))
        return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL voxel_id / t_range");

    char* wp = (char*)work;
    wp += align_up(sizeof(Counters));
    RayPrep* rays = (RayPrep*)wp;
    wp += align_up(sizeof(RayPrep) * (size_t)R);
    int2* buf[2];
    buf[0] = (int2*)wp;
    wp += align_up(sizeof(int2) * (size_t)pair_capacity);
    buf[1] = (int2*)wp;
    wp += align_up(sizeof(int2) * (size_t)pair_capacity);
    long long* chunk_cnt = (long long*)wp;
    wp += align_up(sizeof(unsigned long long) * kMaxGrid);
    unsigned* arrive = (unsigned*)wp;
    wp += align_up(sizeof(unsigned) * (kMaxDepth + 2));
    uint16_t* rec = (uint16_t*)wp;

    const int sms = svo->num_sms;
    NGLOD_CUDA(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
    NGLOD_CUDA(cudaMemsetAsync(arrive, 0, sizeof(unsigned) * (kMaxDepth + 2), st));
    k_prep_rays<<<std::min<long long>((R + kThreads - 1) / kThreads, (long long)sms * 16), kThreads, 0, st>>>(
        o, d, R, rays, ctr);
    for (int dp = 0; dp < D; ++dp) {
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
        lp.dp = dp;
        lp.D = D;
        LevelScratch xs;
        xs.rec = rec;
        xs.chunk_cnt = chunk_cnt;
        xs.arrive = arrive + dp;
        const bool fin = dp + 1 == D;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident (one grid barrier)
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.blockDim = dim3(kThreads);
        cfg.stream = st;
        if (fin) {
            cfg.gridDim = dim3(std::min(sms * level_ctas_per_sm<true>(), kMaxGrid));
            cfg.dynamicSmemBytes = stage_bytes<true>();
            NGLOD_CUDA(cudaLaunchKernelEx(&cfg, k_level<true>, lp, xs));
        } else {
            cfg.gridDim = dim3(std::min(sms * level_ctas_per_sm<false>(), kMaxGrid));
            cfg.dynamicSmemBytes = stage_bytes<false>();
            NGLOD_CUDA(cudaLaunchKernelEx(&cfg, k_level<false>, lp, xs));
        }
    }
    k_ray_offsets<<<std::min<long long>((R + kThreads) / kThreads, (long long)sms * 16), kThreads, 0, st>>>(
        (const int32_t*)buf[D & 1], ctr, D, R, std::min<long long>(hit_capacity, pair_capacity), ray_offsets);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

// Reads the counters of a finished traversal and maps them to a status.
int read_traversal(const void* work, int D, int64_t* h_stats, cudaStream_t st, const char* who) {
    Counters h;
    NGLOD_CUDA(cudaMemcpyAsync(&h, work, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    NGLOD_CUDA(cudaStreamSynchronize(st));
    const long long H = h.count[D];
    if (h_stats) {
        h_stats[0] = H;
        h_stats[1] = h.max_pairs;
    }
    if (h.status == kStatusTimeout)
        return fail(NGLOD_ERR_TIMEOUT, std::string(who) + ": grid barrier wait expired");
    if (h.status == kStatusOverflow) {
        long long need = 0;
        for (int dp = 1; dp < D; ++dp) need = std::max(need, h.count[dp]);
        if (h_stats) h_stats[1] = std::max<long long>(need, h.max_pairs);
        return fail(NGLOD_ERR_CAPACITY, std::string(who) + ": list larger than capacity (pairs " +
                                            std::to_string(need) + ", hits " + std::to_string(H) + ")");
    }
    return NGLOD_OK;
}

}  // namespace
}  // namespace nglod

extern "C" int svo_trace_rays(const nglod_svo* svo, const float* o, const float* d, int64_t R, int target_lod,
                              void* work, size_t work_bytes, int64_t pair_capacity, int32_t* ray_offsets,
                              int32_t* voxel_id, float* t_range, int64_t hit_capacity, int64_t* h_stats,
                              void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (h_stats) h_stats[0] = h_stats[1] = 0;
    int rc = enqueue_traversal(svo, o, d, R, target_lod, work, work_bytes, pair_capacity, ray_offsets, voxel_id,
                               t_range, hit_capacity, st, "svo_trace_rays");
    if (rc || R == 0) return rc;
    return read_traversal(work, target_lod + kFirstFeatureDepth - 1, h_stats, st, "svo_trace_rays");
}

extern "C" int svo_trace_rays_async(const nglod_svo* svo, const float* o, const float* d, int64_t R, int target_lod,
                                    void* work, size_t work_bytes, int64_t pair_capacity, int32_t* ray_offsets,
                                    int32_t* voxel_id, float* t_range, int64_t hit_capacity, void* stream) {
    return enqueue_traversal(svo, o, d, R, target_lod, work, work_bytes, pair_capacity, ray_offsets, voxel_id,
                             t_range, hit_capacity, (cudaStream_t)stream, "svo_trace_rays_async");
}

extern "C" int svo_trace_rays_check(const void* work, int target_lod, int64_t* h_stats, void* stream) {
    if (!work || target_lod < 1 || target_lod + kFirstFeatureDepth - 1 > kMaxDepth)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays_check: bad arguments");
    return read_traversal(work, target_lod + kFirstFeatureDepth - 1, h_stats, (cudaStream_t)stream,
                          "svo_trace_rays_check");
}

extern "C" int svo_trace_rays_sizes(const void* work, int64_t* h_sizes, int n, void* stream) {
    using namespace nglod;
    if (!work || !h_sizes || n < 1 || n > kMaxDepth + 2)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays_sizes: bad arguments");
    Counters h;
    NGLOD_CUDA(cudaMemcpyAsync(&h, work, sizeof(Counters), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    NGLOD_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    for (int i = 0; i < n; ++i) h_sizes[i] = h.count[i];
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
