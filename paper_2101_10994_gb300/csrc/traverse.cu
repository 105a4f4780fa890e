// svo_trace_rays: ray/octree intersection (Algorithm 1 of the paper).
//
// Algorithm 1 runs, per octree level, Decide (one thread per ray/voxel
// pair), ExclusiveSum of the decisions, then Subdivide (write the hit
// voxels' occupied children, front to back) or, at the target level,
// Compactify (keep the hit pairs).  Rays are independent, so the same
// level-by-level sweep is run here per tile of kTR consecutive rays, with
// the whole frontier of the tile kept in shared memory: Decide, the
// exclusive sum (a block scan) and Subdivide of every level happen on chip,
// and only the final, compacted entries ever reach device memory.
//   k_traverse  one persistent kernel takes tiles from an atomic ticket,
//               sweeps their levels and appends each tile's entries (in
//               ray order, front to back per ray) to a staging list at a
//               slot reserved with one atomic; it also stores the tile's
//               entry count and each ray's count;
//   k_tile_scan the exclusive sum of the tile counts (one CTA);
//   k_place     moves every tile's entries to their final CSR positions and
//               writes its rays' offsets.
// No CTA ever waits for another.  The output equals the global
// level-synchronous sequence entry for entry: within a tile the per-level
// scans keep pairs in (ray, front to back) order, and tiles are placed in
// ray order.
//
// A tile whose frontier would outgrow shared memory at some depth keeps the
// last level that fits (already decided) and continues from it in chunks of
// whole rays, each small enough for the rest of the pool; each chunk stages
// its entries as soon as its levels are done and records each ray's first
// staging slot, so nothing above that level is run twice.  A chunk that
// overflows again further down hands its rays (and the tile's later ones) to
// runs from the root over halving ray ranges; a single ray always fits,
// since a ray crosses at most 3 * 2^dp - 2 voxels of depth dp.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "nglod_internal.cuh"

namespace nglod {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTR = 128;                 // rays per tile
constexpr int kFCap = 4096;              // frontier capacity (pairs) of one buffer
static_assert(kFCap >= 3 * (1 << (kMaxDepth - 1)), "one ray's frontier must fit");
constexpr int kScanThreads = 1024;

struct Counters {
    long long count[kMaxDepth + 2];   // pairs kept at each depth (count[0] = R)
    long long max_pairs;               // filled on the host
    unsigned long long next_tile;      // tile ticket
    unsigned long long stage_top;      // staging slots handed out
    int status;                        // kStatus*
};

struct TileInfo {
    long long stage;                   // first staging slot of the tile's entries (-1: staged per
                                       // sub-range, each ray's first slot in ray_src)
    long long count;                   // entries of the tile
};

struct NodeTab {
    const Node* node[kMaxDepth + 1];
};

struct TileParams {
    NodeTab nt;
    const float* o;
    const float* d;
    long long R, ntiles, stage_cap;
    int D;
    int32_t* ray_cnt;                  // [R] entries per ray (k_place turns them into offsets)
    int32_t* ray_src;                  // [R] staging slot of each ray's first entry (sub-range tiles;
                                       // every tile's with first_all)
    bool first_all;                    // staged lists wanted (no placement follows)
    int32_t* stage_vid;                // [stage_cap] staged entries
    float2* stage_tr;                  // ... and their t ranges (null: not wanted)
    TileInfo* tiles;                   // [ntiles]
    Counters* ctr;
};

struct TileSmem {
    RayPrep ray[kTR];
    int32_t vox[2 * kFCap];            // frontier pool: voxel ids ...
    uint8_t rl[2 * kFCap];             // ... and the tile-local ray of each pair
    uint16_t rec[kFCap];               // decisions: hit children by rank | octant << 8
    int ray_cnt[kTR];                  // entries per ray at the target depth
    long long lvl[kMaxDepth + 2];      // level sizes of the current pass
    int warp_sums[kThreads / 32 + 1];
    int wtot[kThreads / 32];           // per-warp totals of a level ...
    int wbase[kThreads / 32 + 1];      // ... their exclusive prefix and sum
    long long tile;
    long long stage;
    // continuation after an overflow: per ray its children at the next depth
    // | its pairs at the kept depth << 16, and the chunks' first rays / pairs
    int ray_chpc[kTR];
    uint16_t chunk_pair[kTR + 1];
    uint8_t chunk_ray[kTR + 1];
    int nchunks;
    uint8_t rank_lut[8 * 256];         // rank_mask(m, oct) at [oct * 256 + m]
};
// four CTAs per SM: 4 x (shared memory + the 1 KB reserved per CTA) <= 228 KB
static_assert(sizeof(TileSmem) + 1024 <= 233472 / 4, "traversal tile state must allow 4 CTAs per SM");

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
    const int r = warp_sums[warp] + incl - v;
    __syncthreads();                   // warp_sums may be reused right away
    return r;
}

__device__ __forceinline__ RayPrep prep_ray(const float* o, const float* d, long long r) {
    return make_ray_prep(o[3 * r], o[3 * r + 1], o[3 * r + 2], d[3 * r], d[3 * r + 1], d[3 * r + 2]);
}

// The pairs [0, n) of a level are split into kWarps contiguous ranges, one
// per warp; lane l of a warp takes pairs w0 + 32 j + l (rows of 32), so
// neighbouring lanes read neighbouring shared-memory words and write
// neighbouring outputs, and a warp-wide scan per row keeps every output in
// pair order.
__device__ __forceinline__ void warp_range(int n, int& w0, int& w1) {
    const int q = ((n + kWarps - 1) / kWarps + 31) & ~31;   // whole rows: idle warps issue nothing
    w0 = min((int)(threadIdx.x >> 5) * q, n);
    w1 = min(w0 + q, n);
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// S.wbase[w] = exclusive prefix of the warps' totals; returns the sum.
__device__ __forceinline__ int warp_bases(TileSmem& S, int wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) S.wtot[warp] = wsum;
    __syncthreads();
    if (warp == 0) {
        const int v = lane < kWarps ? S.wtot[lane] : 0;
        const int incl = warp_incl_scan(v, lane);
        if (lane < kWarps) S.wbase[lane] = incl - v;
        if (lane == kWarps - 1) S.wbase[kWarps] = incl;
    }
    __syncthreads();
    return S.wbase[kWarps];
}

// Decide at depth dp for the n pairs at pool offset src: each pair's
// occupied children are slab-tested (all 8 from the 3 shared plane crossings
// per axis) and recorded by front-to-back rank in S.rec (hit ranks | origin
// octant << 8).  Returns the number of children hit; S.wbase holds each
// warp's first output position.
__device__ __forceinline__ int decide(TileSmem& S, const TileParams& p, int dp, int src, int n) {
    const int lane = threadIdx.x & 31;
    int w0, w1;
    warp_range(n, w0, w1);
    const Node* nodes = p.nt.node[dp];
    int cnt = 0;
    for (int rb = w0; rb < w1; rb += 32) {
        const int i = rb + lane;
        if (i < w1) {
            const Node nd = nodes[S.vox[src + i]];
            const RayPrep ray = S.ray[S.rl[src + i]];
            uint32_t o8 = 0, h = 0;
            bool live = true;
            if (dp == 0) {
                float t0, t1;   // the root is the only undecided input
                live = ray.valid && slab_test(ray, nd.ijk, 0, t0, t1, &o8);
            }
            if (live && nd.childmask) {
                const uint32_t hs = child_hits8<false>(ray, nd.ijk, dp, o8);
                h = S.rank_lut[(o8 << 8) | (hs & nd.childmask)];
            }
            // (the octant is read only where a child was hit)
            S.rec[i] = (uint16_t)(h | (o8 << 8));
            cnt += __popc(h);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    return warp_bases(S, cnt);
}

// Subdivide: the hit children of the n pairs at src, front to back, to dst.
__device__ __forceinline__ void subdivide(TileSmem& S, const TileParams& p, int dp, int src, int dst, int n) {
    const int lane = threadIdx.x & 31;
    int w0, w1;
    warp_range(n, w0, w1);
    const Node* nodes = p.nt.node[dp];
    int run = S.wbase[threadIdx.x >> 5];
    for (int rb = w0; rb < w1; rb += 32) {
        const int i = rb + lane;
        const uint32_t r = i < w1 ? S.rec[i] : 0u;
        const uint32_t h0 = r & 0xffu;
        const int c = __popc(h0);
        const int incl = warp_incl_scan(c, lane);
        int pos = run + incl - c;
        run += __shfl_sync(0xffffffffu, incl, 31);
        if (h0) {
            const Node nd = nodes[S.vox[src + i]];
            const uint32_t o8 = r >> 8;
            const uint8_t rl = S.rl[src + i];
            for (uint32_t h = h0; h; h &= h - 1u) {
                const uint32_t cs = (uint32_t)(__ffs(h) - 1) ^ o8;
                S.vox[dst + pos] = nd.childbase + __popc(nd.childmask & ((1u << cs) - 1u));
                S.rl[dst + pos] = rl;
                ++pos;
            }
        }
    }
}

// Compactify at the target depth: the hit children of the n pairs at src with their
// (t_enter, t_exit), written to their staging slots from `base` on, and each
// ray's entry count added to S.ray_cnt (pairs are grouped by ray, so the
// last lane of each run of one ray in a row adds the run's sum).
template <bool WT>
__device__ __forceinline__ void write_final(TileSmem& S, const TileParams& p, int dp, int src, int n,
                                            long long base) {
    const int lane = threadIdx.x & 31;
    int w0, w1;
    warp_range(n, w0, w1);
    const Node* nodes = p.nt.node[dp];
    long long run = base + S.wbase[threadIdx.x >> 5];
    for (int rb = w0; rb < w1; rb += 32) {
        const int i = rb + lane;
        const bool valid = i < w1;
        const uint32_t r = valid ? S.rec[i] : 0u;
        const int rl = valid ? (int)S.rl[src + i] : -1;
        const uint32_t h0 = r & 0xffu;
        const int c = __popc(h0);
        const int incl = warp_incl_scan(c, lane);
        long long pos = run + incl - c;
        run += __shfl_sync(0xffffffffu, incl, 31);
        // runs of equal rays in the row: heads, and each lane's run head
        const int rl_prev = __shfl_up_sync(0xffffffffu, rl, 1);
        const int rl_next = __shfl_down_sync(0xffffffffu, rl, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || rl_prev != rl);
        const int head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const int excl_head = __shfl_sync(0xffffffffu, incl - c, head);
        if (valid && (lane == 31 || rl_next != rl) && incl > excl_head) atomicAdd(&S.ray_cnt[rl], incl - excl_head);
        if (h0) {
            const Node nd = nodes[S.vox[src + i]];
            const uint32_t o8 = r >> 8;
            // the exact (t_enter, t_exit) of the hit children only (about one
            // per pair at the target depth), when the caller wants them
            ChildSlabs cs;
            if constexpr (WT) child_slabs(S.ray[rl], nd.ijk, dp, cs);
            for (uint32_t h = h0; h; h &= h - 1u) {
                const uint32_t cc = (uint32_t)(__ffs(h) - 1) ^ o8;
                if (pos < p.stage_cap) {
                    p.stage_vid[pos] = nd.childbase + __popc(nd.childmask & ((1u << cc) - 1u));
                    if constexpr (WT) {
                        float a0 = 0.f, a1 = 0.f;
                        child_hit(cs, cc, a0, a1);
                        p.stage_tr[pos] = make_float2(a0, a1);
                    }
                }
                ++pos;
            }
        }
    }
}

// Root pairs of the tile-local rays [r0, r0 + nr) at the pool's start.
__device__ __forceinline__ void init_roots(TileSmem& S, int r0, int nr) {
    for (int i = threadIdx.x; i < nr; i += kThreads) {
        S.vox[i] = 0;
        S.rl[i] = (uint8_t)(r0 + i);
    }
}

// Where a sweep of levels stopped: the n pairs of depth dp at pool offset
// src, decided (S.rec; S.wbase holds each warp's first output), and the
// number of pairs (or entries, at the target depth) their decisions make.
struct LevelRun {
    int src, n, dp, total;
};

// Decide / Subdivide from depth dp0 for the n pairs at pool offset a, the
// levels alternating between offsets a and b, each holding at most cap
// pairs.  Returns true at the target depth (lr: its decided pairs and the
// entry count) or false (block-uniform) when the Decide at depth lr.dp would
// make a frontier of lr.total > cap pairs (lr: that depth's pairs, kept in
// place).  S.lvl[dp + 1] receives the size every decided level makes.  The
// caller syncs after placing the first level's pairs.
__device__ bool run_from(TileSmem& S, const TileParams& p, int dp0, int a, int b, int n, int cap, LevelRun& lr) {
    for (int dp = dp0;; ++dp) {
        const int total = decide(S, p, dp, a, n);
        if (threadIdx.x == 0) S.lvl[dp + 1] = total;
        lr = LevelRun{a, n, dp, total};
        if (dp + 1 == p.D) {
            __syncthreads();
            return true;
        }
        if (total > cap) return false;
        subdivide(S, p, dp, a, b, n);
        __syncthreads();
        const int t = a;
        a = b;
        b = t;
        n = total;
    }
}

// Reserves n staging slots (one atomic, thread 0) into S.stage; flags an
// overflow of the staging capacity.  The caller syncs before reading S.stage.
__device__ __forceinline__ void reserve_stage(TileSmem& S, const TileParams& p, long long n) {
    if (threadIdx.x == 0) {
        const long long st = (long long)atomicAdd(&p.ctr->stage_top, (unsigned long long)n);
        S.stage = st;
        if (st + n > p.stage_cap) atomicCAS(&p.ctr->status, kStatusOk, kStatusOverflow);
    }
}

// Adds the level sizes S.lvl[lo..hi] of the last sweep to the counters.
__device__ __forceinline__ void commit_levels(TileSmem& S, const TileParams& p, int lo, int hi) {
    const int l = (int)threadIdx.x;
    if (l >= lo && l <= hi && S.lvl[l])
        atomicAdd((unsigned long long*)&p.ctr->count[l], (unsigned long long)S.lvl[l]);
}

// Stages the entries of a finished sweep whose decisions (at the target
// depth) are lr's, covering the tile-local rays [r_lo, r_hi): one
// reservation, the entries written, and each ray's first staging slot.
template <bool WT>
__device__ __forceinline__ void stage_sweep(TileSmem& S, const TileParams& p, long long ra, int r_lo, int r_hi,
                                            const LevelRun& lr) {
    reserve_stage(S, p, lr.total);
    __syncthreads();
    write_final<WT>(S, p, p.D - 1, lr.src, lr.n, S.stage);
    __syncthreads();                       // the rays' counts are complete
    const int j = (int)threadIdx.x, l = r_hi - r_lo;
    int sum;
    const int pre = block_exclusive_sum(j < l ? S.ray_cnt[r_lo + j] : 0, S.warp_sums, sum);
    if (j < l) p.ray_src[ra + r_lo + j] = (int32_t)(S.stage + pre);
}

// Runs the tile-local rays [r, nr) from the root over ranges that fit,
// halving a range that overflows and growing back after a success; level
// sizes from depth lmin on are counted.  Returns the entries staged.
template <bool WT>
__device__ long long sweep_halving(TileSmem& S, const TileParams& p, long long ra, int r, int nr, int lmin) {
    long long staged = 0;
    const int half = max(1, (nr - r) / 2);
    int len = half;
    while (r < nr) {
        const int l = min(len, nr - r);
        init_roots(S, r, l);
        __syncthreads();
        LevelRun lr;
        if (!run_from(S, p, 0, 0, kFCap, l, kFCap, lr)) {
            len = max(1, l / 2);
            __syncthreads();               // the pool is refilled next
            continue;
        }
        commit_levels(S, p, lmin, p.D);
        stage_sweep<WT>(S, p, ra, r, r + l, lr);
        staged += lr.total;
        r += l;
        len = min(half, 2 * len);
    }
    return staged;
}

// A tile whose frontier at depth lr0.dp + 1 would overflow.  The lr0.n pairs
// of depth lr0.dp (decided: S.rec) move to the pool's start and are split at
// ray boundaries into chunks whose pairs fit one of two buffers after them
// and whose children fit too (half a buffer where deeper frontiers follow);
// each chunk is decided again at that depth, swept down to the target depth
// in those buffers and staged.  Returns the tile's entry count.
template <bool WT>
__device__ long long sweep_chunks(TileSmem& S, const TileParams& p, long long ra, int nr, const LevelRun& lr0) {
    const int dp = lr0.dp, n = lr0.n;
    for (int i = threadIdx.x; i < kTR; i += kThreads) S.ray_chpc[i] = 0;
    __syncthreads();
    commit_levels(S, p, 1, dp + 1);        // those levels are complete for the tile
    for (int i = threadIdx.x; i < n; i += kThreads)
        atomicAdd(&S.ray_chpc[S.rl[lr0.src + i]], __popc(S.rec[i] & 0xffu) | (1 << 16));
    __syncthreads();
    if (lr0.src != 0) {                    // [kFCap, kFCap + n) -> [0, n): disjoint
        for (int i = threadIdx.x; i < n; i += kThreads) {
            S.vox[i] = S.vox[lr0.src + i];
            S.rl[i] = S.rl[lr0.src + i];
        }
    }
    const int F = min(kFCap, (2 * kFCap - n) / 2);     // >= kFCap / 2: a single ray always fits
    const int A = n, B = n + F;
    const int budget = dp + 2 == p.D ? F : F / 2;
    if (threadIdx.x == 0) {
        // a chunk's own pairs must fit one buffer too
        int nch = 0, acc = 0, pairs = 0, first = 0;
        S.chunk_ray[0] = 0;
        S.chunk_pair[0] = 0;
        for (int r = 0; r < nr; ++r) {
            const int v = S.ray_chpc[r];
            const int c = v & 0xffff, pc = v >> 16;
            if (r > first && (acc + c > budget || pairs + pc - (int)S.chunk_pair[nch] > F)) {
                ++nch;
                S.chunk_ray[nch] = (uint8_t)r;
                S.chunk_pair[nch] = (uint16_t)pairs;
                first = r;
                acc = 0;
            }
            acc += c;
            pairs += pc;
        }
        ++nch;
        S.chunk_ray[nch] = (uint8_t)nr;
        S.chunk_pair[nch] = (uint16_t)pairs;
        S.nchunks = nch;
    }
    __syncthreads();
    const int nch = S.nchunks;
    long long staged = 0;
    for (int k = 0; k < nch; ++k) {
        const int r_lo = S.chunk_ray[k], r_hi = S.chunk_ray[k + 1];
        const int pa = S.chunk_pair[k], m = (int)S.chunk_pair[k + 1] - pa;
        for (int i = threadIdx.x; i < m; i += kThreads) {
            S.vox[A + i] = S.vox[pa + i];
            S.rl[A + i] = S.rl[pa + i];
        }
        __syncthreads();
        LevelRun lr;
        if (!run_from(S, p, dp, A, B, m, F, lr)) {
            __syncthreads();
            return staged + sweep_halving<WT>(S, p, ra, r_lo, nr, dp + 2);
        }
        commit_levels(S, p, dp + 2, p.D);
        stage_sweep<WT>(S, p, ra, r_lo, r_hi, lr);
        staged += lr.total;
        __syncthreads();                   // the chunk's buffers are reused next
    }
    return staged;
}

// WT: the entries' t ranges are staged too (the caller asked for them).
template <bool WT>
__global__ void __launch_bounds__(kThreads, 4) k_traverse(const TileParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
    if (blockIdx.x == 0 && threadIdx.x == 0) p.ctr->count[0] = p.R;
    for (int i = threadIdx.x; i < 8 * 256; i += kThreads) S.rank_lut[i] = (uint8_t)rank_mask(i & 255, i >> 8);
    for (;;) {
        if (threadIdx.x == 0) S.tile = (long long)atomicAdd(&p.ctr->next_tile, 1ull);
        __syncthreads();
        const long long t = S.tile;
        if (t >= p.ntiles) break;
        const long long ra = t * kTR;
        const int nr = (int)min((long long)kTR, p.R - ra);
        for (int i = threadIdx.x; i < kTR; i += kThreads) {
            if (i < nr) S.ray[i] = prep_ray(p.o, p.d, ra + i);
            S.ray_cnt[i] = 0;
        }
        init_roots(S, 0, nr);
        __syncthreads();
        LevelRun lr;
        const bool whole = run_from(S, p, 0, 0, kFCap, nr, kFCap, lr);
        if (whole) {
            commit_levels(S, p, 1, p.D);
            reserve_stage(S, p, lr.total);
            if (threadIdx.x == 0) p.tiles[t] = TileInfo{S.stage, (long long)lr.total};
            __syncthreads();
            write_final<WT>(S, p, p.D - 1, lr.src, lr.n, S.stage);
        } else {
            __syncthreads();               // S.lvl of the overflowing level
            const long long staged = sweep_chunks<WT>(S, p, ra, nr, lr);
            if (threadIdx.x == 0) p.tiles[t] = TileInfo{-1, staged};
        }
        __syncthreads();                   // per-ray counts complete
        if (!p.first_all) {
            if ((int)threadIdx.x < nr) p.ray_cnt[ra + threadIdx.x] = S.ray_cnt[threadIdx.x];
        } else {
            // staged lists: each ray's first staging slot (a tile staged in one
            // piece holds its rays in order; sub-range tiles recorded theirs
            // while staging).  A list that does not lie whole inside the
            // staging capacity (the staging list overflowed: the status says
            // so) gets no entries, so a reader sees a miss, never an unwritten
            // slot.
            long long first = 0;
            if (whole) {
                int sum;
                const int pre = block_exclusive_sum((int)threadIdx.x < nr ? S.ray_cnt[threadIdx.x] : 0,
                                                    S.warp_sums, sum);
                first = S.stage + pre;
            } else if ((int)threadIdx.x < nr) {
                first = p.ray_src[ra + threadIdx.x];
            }
            if ((int)threadIdx.x < nr) {
                const int c = S.ray_cnt[threadIdx.x];
                const bool inside = first >= 0 && first + c <= p.stage_cap;
                p.ray_cnt[ra + threadIdx.x] = inside ? c : 0;
                p.ray_src[ra + threadIdx.x] = inside ? (int32_t)first : 0;
            }
        }
        __syncthreads();   // shared state is reused by the next tile
    }
}

// Exclusive sum of the tile counts, in place over TileInfo::count (one CTA):
// chunks of kScanChunk tiles staged in shared memory with coalesced loads,
// kScanPer consecutive tiles a thread.
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanThreads * kScanPer;

__device__ __forceinline__ long long warp_incl_scan_ll(long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_scan(TileInfo* __restrict__ tiles, long long ntiles,
                                                            Counters* __restrict__ ctr, long long hit_cap, int D) {
    __shared__ long long buf[kScanChunk];
    __shared__ long long warp_sums[kScanThreads / 32 + 1];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long b0 = 0; b0 < ntiles; b0 += kScanChunk) {
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const long long i = b0 + j * kScanThreads + threadIdx.x;
            buf[j * kScanThreads + threadIdx.x] = i < ntiles ? tiles[i].count : 0;
        }
        __syncthreads();
        long long c[kScanPer], sum = 0;
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            c[j] = buf[threadIdx.x * kScanPer + j];
            sum += c[j];
        }
        const long long incl = warp_incl_scan_ll(sum, lane);
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const long long s = warp_sums[lane];
            const long long si = warp_incl_scan_ll(s, lane);
            warp_sums[lane] = si - s;
            if (lane == 31) warp_sums[32] = si;
        }
        __syncthreads();
        long long run = carry + warp_sums[warp] + incl - sum;
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            buf[threadIdx.x * kScanPer + j] = run;
            run += c[j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const long long i = b0 + j * kScanThreads + threadIdx.x;
            if (i < ntiles) tiles[i].count = buf[j * kScanThreads + threadIdx.x];   // now the exclusive prefix
        }
        if (threadIdx.x == 0) carry += warp_sums[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (carry != ctr->count[D]) atomicCAS(&ctr->status, kStatusOk, kStatusBadIndex);
        if (carry > hit_cap) atomicCAS(&ctr->status, kStatusOk, kStatusOverflow);
    }
}

// One CTA per tile: its rays' CSR offsets (exclusive sum of their counts
// after the tile's prefix) and its staged entries copied to their final
// positions (coalesced, four independent copies in flight per thread).
constexpr int kPlaceThreads = 256;

__global__ void __launch_bounds__(kPlaceThreads) k_place(const TileInfo* __restrict__ tiles, const TileParams p,
                                                        const int32_t* __restrict__ ray_cnt,
                                                        int32_t* __restrict__ ray_offsets,
                                                        int32_t* __restrict__ voxel_id, float2* __restrict__ t_range) {
    __shared__ int warp_sums[kTR / 32 + 1];
    __shared__ int ray_pre[kTR + 1];                // sub-range tiles: each ray's first entry in the tile
    __shared__ int32_t ray_from[kTR];               // ... and its first staging slot
    if (p.ctr->status != kStatusOk) {
        // overflow: no lists are placed, so every ray's list is left empty
        // (a reader sees misses, never stale offsets)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= p.R;
             i += (long long)gridDim.x * blockDim.x)
            ray_offsets[i] = 0;
        return;
    }
    for (long long t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
        const long long ra = t * kTR;
        const int nr = (int)min((long long)kTR, p.R - ra);
        const long long off = tiles[t].count;           // exclusive prefix (k_tile_scan)
        const long long st = tiles[t].stage;
        long long my_dst = 0;                           // this thread's ray's first final position
        if (threadIdx.x < kTR) {
            const int v = (int)threadIdx.x < nr ? ray_cnt[ra + threadIdx.x] : 0;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) warp_sums[warp] = incl;
            asm volatile("bar.sync 1, %0;" ::"r"(kTR));   // the kTR scanning threads only
            if (threadIdx.x == 0) {
                int a = 0;
                for (int w = 0; w < kTR / 32; ++w) {
                    const int x = warp_sums[w];
                    warp_sums[w] = a;
                    a += x;
                }
                warp_sums[kTR / 32] = a;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kTR));
            my_dst = off + warp_sums[warp] + incl - v;
            if ((int)threadIdx.x < nr) ray_offsets[ra + threadIdx.x] = (int32_t)my_dst;
        }
        __syncthreads();
        // staged entries -> final positions (within both capacities: the
        // status checked above covers the staging list and H <= hit_cap)
        const int cnt = warp_sums[kTR / 32];
        if (t == p.ntiles - 1 && threadIdx.x == 0) ray_offsets[p.R] = (int32_t)(off + cnt);
        if (st < 0) {
            // staged per sub-range: entry e of the tile belongs to the ray j
            // with ray_pre[j] <= e < ray_pre[j + 1] and sits at staging slot
            // ray_from[j] + e - ray_pre[j]; the threads take consecutive
            // entries (coalesced writes), each finding its ray by bisection
            if ((int)threadIdx.x < kTR) {
                ray_pre[threadIdx.x] = (int)threadIdx.x < nr ? (int)(my_dst - off) : cnt;
                ray_from[threadIdx.x] = (int)threadIdx.x < nr ? p.ray_src[ra + threadIdx.x] : 0;
            }
            if (threadIdx.x == 0) ray_pre[kTR] = cnt;
            __syncthreads();
            for (int e = threadIdx.x; e < cnt; e += kPlaceThreads) {
                int lo = 0, hi = nr - 1;          // the last ray j with ray_pre[j] <= e
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (ray_pre[mid] <= e) lo = mid; else hi = mid - 1;
                }
                const long long src = (long long)ray_from[lo] + (e - ray_pre[lo]);
                voxel_id[off + e] = p.stage_vid[src];
                if (t_range) t_range[off + e] = p.stage_tr[src];
            }
            __syncthreads();
            continue;
        }
        if (t_range) {
            for (int i0 = threadIdx.x; i0 < cnt; i0 += 4 * kPlaceThreads) {
                int32_t v[4];
                float2 tr[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * kPlaceThreads;
                    if (i < cnt) {
                        v[u] = p.stage_vid[st + i];
                        tr[u] = p.stage_tr[st + i];
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * kPlaceThreads;
                    if (i < cnt) {
                        voxel_id[off + i] = v[u];
                        t_range[off + i] = tr[u];
                    }
                }
            }
        } else {
            for (int i0 = threadIdx.x; i0 < cnt; i0 += 8 * kPlaceThreads) {
                int32_t v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u * kPlaceThreads;
                    if (i < cnt) v[u] = p.stage_vid[st + i];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u * kPlaceThreads;
                    if (i < cnt) voxel_id[off + i] = v[u];
                }
            }
        }
        __syncthreads();
    }
}

size_t align_up(size_t v, size_t a = 256) { return (v + a - 1) / a * a; }

long long num_tiles(long long R) { return (R + kTR - 1) / kTR; }

// Resident traversal CTAs per SM, found (and the shared-memory opt-in set)
// once per device.
int traverse_ctas_per_sm() {
    static std::atomic<int> cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int>& c = cached[dev & 63];
    if (!c.load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(k_traverse<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSmem));
        cudaFuncSetAttribute(k_traverse<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSmem));
        int n = 0, n2 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_traverse<true>, kThreads, sizeof(TileSmem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, k_traverse<false>, kThreads, sizeof(TileSmem));
        n = std::min(n, n2);
        c.store(n > 0 ? n : 1, std::memory_order_release);
    }
    return c.load(std::memory_order_acquire);
}

}  // namespace
}  // namespace nglod

using namespace nglod;

extern "C" size_t svo_trace_rays_workspace(int64_t R, int64_t pair_capacity) {
    if (R < 0 || pair_capacity < 0) return 0;
    return align_up(sizeof(Counters)) + align_up(sizeof(TileInfo) * (size_t)(num_tiles(R) + 1)) +
           2 * align_up(sizeof(int32_t) * (size_t)(R + 1)) + align_up(sizeof(int32_t) * (size_t)pair_capacity) +
           align_up(sizeof(float2) * (size_t)pair_capacity);
}

namespace nglod {
namespace {

// Enqueues the whole traversal on the stream (no host synchronisation).
// The workspace's regions (svo_trace_rays_workspace).
struct TraversalWs {
    Counters* ctr;
    TileInfo* tiles;
    int32_t* ray_cnt;
    int32_t* ray_src;
    int32_t* stage_vid;
    float2* stage_tr;
};

TraversalWs traversal_ws(void* work, int64_t R, int64_t pair_capacity) {
    TraversalWs w;
    char* wp = (char*)work;
    w.ctr = (Counters*)wp;
    wp += align_up(sizeof(Counters));
    w.tiles = (TileInfo*)wp;
    wp += align_up(sizeof(TileInfo) * (size_t)(num_tiles(R) + 1));
    w.ray_cnt = (int32_t*)wp;
    wp += align_up(sizeof(int32_t) * (size_t)(R + 1));
    w.ray_src = (int32_t*)wp;
    wp += align_up(sizeof(int32_t) * (size_t)(R + 1));
    w.stage_vid = (int32_t*)wp;
    wp += align_up(sizeof(int32_t) * (size_t)pair_capacity);
    w.stage_tr = (float2*)wp;
    return w;
}

// staged: the lists stay in the staging list (svo_trace_rays_staged_async):
// no placement, every ray's first staging slot recorded, no CSR outputs.
int enqueue_traversal(const nglod_svo* svo, const float* o, const float* d, int64_t R, int target_lod, void* work,
                      size_t work_bytes, int64_t pair_capacity, int32_t* ray_offsets, int32_t* voxel_id,
                      float* t_range, int64_t hit_capacity, cudaStream_t st, const char* who, int ctas_per_sm = 0,
                      bool staged = false) {
    const std::string w(who);
    if (!svo) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL octree");
    const int D = target_lod + kFirstFeatureDepth - 1;
    if (target_lod < 1 || D >= svo->num_depths)
        return fail(NGLOD_ERR_INVALID_ARG, w + ": target_lod outside 1.." +
                                               std::to_string(svo->num_depths - kFirstFeatureDepth));
    if (R < 0 || R >= (1ll << 31) - 1 || pair_capacity < 0 || pair_capacity >= (1ll << 31) - 1 ||
        hit_capacity < 0)
        return fail(NGLOD_ERR_INVALID_ARG, w + ": bad R or capacity");
    if (!ray_offsets && !staged) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL ray_offsets");
    if (!work) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL workspace");
    if (work_bytes < svo_trace_rays_workspace(R, pair_capacity))
        return fail(NGLOD_ERR_CAPACITY, w + ": workspace smaller than svo_trace_rays_workspace()");
    if (((uintptr_t)work & 255u) != 0) return fail(NGLOD_ERR_INVALID_ARG, w + ": work must be 256-B aligned");
    Counters* ctr = (Counters*)work;
    if (R == 0) {
        NGLOD_CUDA(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
        if (!staged) NGLOD_CUDA(cudaMemsetAsync(ray_offsets, 0, sizeof(int32_t), st));
        return NGLOD_OK;
    }
    if (!o || !d) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL rays");
    if (!staged && hit_capacity > 0 && !voxel_id) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL voxel_id");

    const long long ntiles = num_tiles(R);
    const TraversalWs ws = traversal_ws(work, R, pair_capacity);
    TileInfo* tiles = ws.tiles;
    int32_t* ray_cnt = ws.ray_cnt;
    int32_t* ray_src = ws.ray_src;
    int32_t* stage_vid = ws.stage_vid;
    float2* stage_tr = ws.stage_tr;
    NGLOD_CUDA(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
    TileParams p;
    for (int dp = 0; dp <= kMaxDepth; ++dp) p.nt.node[dp] = dp < svo->num_depths ? svo->node[dp] : nullptr;
    p.o = o;
    p.d = d;
    p.R = R;
    p.ntiles = ntiles;
    p.stage_cap = pair_capacity;
    p.D = D;
    p.ray_cnt = ray_cnt;
    p.ray_src = ray_src;
    p.first_all = staged;
    p.stage_vid = stage_vid;
    p.stage_tr = t_range && !staged ? stage_tr : nullptr;
    p.tiles = tiles;
    p.ctr = ctr;
    const int sms = svo->num_sms;
    const int occ = traverse_ctas_per_sm();
    const long long grid = std::min<long long>(ntiles, (long long)sms * (ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ));
    if (p.stage_tr)
        k_traverse<true><<<(unsigned)grid, kThreads, sizeof(TileSmem), st>>>(p);
    else
        k_traverse<false><<<(unsigned)grid, kThreads, sizeof(TileSmem), st>>>(p);
    if (staged) {
        NGLOD_CUDA(cudaGetLastError());
        return NGLOD_OK;
    }
    k_tile_scan<<<1, kScanThreads, 0, st>>>(tiles, ntiles, ctr, hit_capacity, D);
    k_place<<<(unsigned)std::min<long long>(ntiles, (long long)sms * 8), kPlaceThreads, 0, st>>>(
        tiles, p, ray_cnt, ray_offsets, voxel_id, (float2*)t_range);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

// Reads the counters of a finished traversal and maps them to a status.
int read_traversal(const void* work, int D, int64_t* h_stats, cudaStream_t st, const char* who) {
    Counters h;
    NGLOD_CUDA(cudaMemcpyAsync(&h, work, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    NGLOD_CUDA(cudaStreamSynchronize(st));
    const long long H = h.count[D];
    long long mx = 0;
    for (int dp = 1; dp <= D; ++dp) mx = std::max(mx, h.count[dp]);
    if (h_stats) {
        h_stats[0] = H;
        h_stats[1] = mx;
    }
    if (h.status == kStatusOverflow)
        return fail(NGLOD_ERR_CAPACITY, std::string(who) + ": " + std::to_string(H) +
                                            " hits exceed hit_capacity or pair_capacity");
    if (h.status != kStatusOk)
        return fail(NGLOD_ERR_CUDA, std::string(who) + ": inconsistent traversal counters");
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

extern "C" int svo_trace_rays_async_width(const nglod_svo* svo, const float* o, const float* d, int64_t R,
                                          int target_lod, void* work, size_t work_bytes, int64_t pair_capacity,
                                          int32_t* ray_offsets, int32_t* voxel_id, float* t_range,
                                          int64_t hit_capacity, int ctas_per_sm, void* stream) {
    if (ctas_per_sm < 0 || ctas_per_sm > 4)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays_async_width: ctas_per_sm must lie in 0..4");
    return enqueue_traversal(svo, o, d, R, target_lod, work, work_bytes, pair_capacity, ray_offsets, voxel_id,
                             t_range, hit_capacity, (cudaStream_t)stream, "svo_trace_rays_async_width", ctas_per_sm);
}

extern "C" int svo_trace_rays_staged_async(const nglod_svo* svo, const float* o, const float* d, int64_t R,
                                           int target_lod, void* work, size_t work_bytes, int64_t pair_capacity,
                                           int ctas_per_sm, const int32_t** ray_first, const int32_t** ray_count,
                                           const int32_t** voxel_id, void* stream) {
    if (ctas_per_sm < 0 || ctas_per_sm > 4)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays_staged_async: ctas_per_sm must lie in 0..4");
    if (!ray_first || !ray_count || !voxel_id)
        return fail(NGLOD_ERR_INVALID_ARG, "svo_trace_rays_staged_async: NULL output pointer");
    const int rc = enqueue_traversal(svo, o, d, R, target_lod, work, work_bytes, pair_capacity, nullptr, nullptr,
                                     nullptr, 0, (cudaStream_t)stream, "svo_trace_rays_staged_async", ctas_per_sm,
                                     true);
    if (rc) return rc;
    const TraversalWs ws = traversal_ws(work, R, pair_capacity);
    *ray_first = ws.ray_src;
    *ray_count = ws.ray_cnt;
    *voxel_id = ws.stage_vid;
    return NGLOD_OK;
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
// cudaGetSymbolAddress with the device current -- on the first call on each
// device and on every call made outside a stream capture (make the first
// call on a device before any stream capture; a capture reuses the address
// of the last lookup, so a device reset followed directly by a capture is
// not supported).  All calls share the array and it keeps the previous call's
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
    // the fixed part of the workspace (counters, tile records, per-ray
    // counts) must fit the array; the rest is the staging-list capacity
    if (svo_trace_rays_workspace(R, 0) > kNoAllocScratchBytes)
        return fail(NGLOD_ERR_CAPACITY, "svo_trace_rays_noalloc: " + std::to_string(R) +
                                            " rays need more workspace than the fixed 32 MiB scratch (use "
                                            "svo_trace_rays with a caller-allocated workspace)");
    int64_t lo = 0, hi = (int64_t)(kNoAllocScratchBytes / (sizeof(int32_t) + sizeof(float2)));
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (svo_trace_rays_workspace(R, mid) <= kNoAllocScratchBytes) lo = mid; else hi = mid - 1;
    }
    const int64_t pair_capacity = lo;
    int dev = 0;
    NGLOD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(NGLOD_ERR_NOT_SUPPORTED, "svo_trace_rays_noalloc: device index out of range");
    // outside a stream capture the address is looked up on every call (cheap),
    // so a device reset, after which the runtime loads the module again,
    // cannot leave a stale address behind; inside a capture the address of
    // the last lookup on this device is used
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NGLOD_CUDA(cudaStreamIsCapturing((cudaStream_t)stream, &cap));
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
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
        set_error(std::string(nglod_last_error()) + " [svo_trace_rays_noalloc: the fixed 32 MiB scratch stages " +
                  std::to_string(pair_capacity) + " entries for these rays]");
    return rc;
}
