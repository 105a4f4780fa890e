// Ray state and stepping rules of the sphere tracer (Sec. 3.4 "Adaptive Ray
// Stepping", supplementary Sec. A.4) shared by the FP32 and BF16 kernels,
// plus the FP32 decoder evaluated from shared-memory weights.
#pragma once

#include "nglod_internal.cuh"
#include "query_common.cuh"

namespace nglod {

// FP32 decoder staged in shared memory.  Row h of W1 is stored reordered as
// [z_0..z_31, x_0, x_1, x_2, 0] (K4 = 32 or 36 floats) so that the input
// vector splits into aligned float4s; every thread of a warp reads the same
// row (a broadcast), so each 16-byte shared load feeds four FFMAs.
constexpr int kK4Max = 36;
struct SmemDecoder {
    float W1[kHidden * kK4Max];
    float2 bw[kHidden];        // (b1[h], W2[h])
};

template <int IN>
__device__ __forceinline__ void stage_decoder(SmemDecoder& sd, const float* __restrict__ W1,
                                              const float* __restrict__ b1, const float* __restrict__ W2) {
    constexpr int OFF = IN - kFeatDim;
    constexpr int K4 = OFF ? 36 : 32;
    for (int i = threadIdx.x; i < kHidden * K4; i += blockDim.x) {
        const int h = i / K4, k = i - h * K4;
        float w;
        if (k < kFeatDim) w = W1[h * IN + OFF + k];
        else if (k < kFeatDim + OFF) w = W1[h * IN + (k - kFeatDim)];
        else w = 0.0f;
        sd.W1[i] = w;
    }
    for (int h = threadIdx.x; h < kHidden; h += blockDim.x) sd.bw[h] = make_float2(b1[h], W2[h]);
}

// d = W2 . relu(W1 [x, z] + b1) + b2 for the lane's own slot, z read from
// its staged row (Eq. 2).
template <int IN, bool MASK = false>
__device__ __forceinline__ float mlp_f32(const SmemDecoder& sd, float b2, const float* zrow, float x0,
                                         float x1, float x2, uint4* mask = nullptr) {
    constexpr int OFF = IN - kFeatDim;
    constexpr int K4 = OFF ? 36 : 32;
    float v[K4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 a = reinterpret_cast<const float4*>(zrow)[j];
        v[4 * j] = a.x;
        v[4 * j + 1] = a.y;
        v[4 * j + 2] = a.z;
        v[4 * j + 3] = a.w;
    }
    if constexpr (OFF == 3) {
        v[32] = x0;
        v[33] = x1;
        v[34] = x2;
        v[35] = 0.0f;
    }
    float out = b2;
    uint32_t m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
        uint32_t bits = 0u;
#pragma unroll 2
        for (int hh = 0; hh < 32; ++hh) {
            const int h = c * 32 + hh;
            const float4* w = reinterpret_cast<const float4*>(sd.W1 + h * K4);
            // two partial sums as one packed pair (each lane rounded once, as fmaf)
            float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < K4 / 4; ++j) {
                const float4 ww = w[j];
                a = __ffma2_rn(make_float2(ww.x, ww.y), make_float2(v[4 * j], v[4 * j + 1]), a);
                a = __ffma2_rn(make_float2(ww.z, ww.w), make_float2(v[4 * j + 2], v[4 * j + 3]), a);
            }
            const float2 bw = sd.bw[h];
            const float pre = a.x + a.y + bw.x;
            out = fmaf(bw.y, fmaxf(pre, 0.0f), out);
            if constexpr (MASK) bits |= (pre > 0.0f ? 1u : 0u) << hh;
        }
        if constexpr (MASK) {
            m0 = c == 0 ? bits : m0;
            m1 = c == 1 ? bits : m1;
            m2 = c == 2 ? bits : m2;
            m3 = c == 3 ? bits : m3;
        }
    }
    if constexpr (MASK) *mask = make_uint4(m0, m1, m2, m3);
    return out;
}

// Position of the k-th (0-based) set bit of m; k < popc(m).
__device__ __forceinline__ int kth_set_bit(unsigned m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

struct TraceArgs {
    const float* o;
    const float* d;
    long long R;
    int D;
    float eps, far_t;
    int max_steps, osc;
    // the rays' voxel lists (CSR); each entry's interval [t_enter, t_exit]
    // is recomputed from its voxel by the traversal's slab test (same bits)
    const int32_t* offs;
    const int32_t* vid;
    // with cnt, the lists as the traversal staged them: ray r's entries are
    // vid[offs[r] .. offs[r] + cnt[r]) (each ray's contiguous, front to
    // back; rays in no particular order), and offs has R entries
    const int32_t* cnt = nullptr;
    float* t_hit;
    uint8_t* hit;
    int32_t* steps;       // nullable
    int32_t* hit_vox;     // workspace: voxel of the hit (for normals)
    int* queue;           // workspace: next unstarted ray
    int* hit_count;       // workspace: number of rays in hit_list
    int32_t* hit_list;    // workspace: ids of the rays that hit (any order)
    // workspace: the order in which 32-ray groups are handed out (null:
    // index order); longest-working groups first shortens the frame's tail
    const int32_t* order = nullptr;
    // workspace: the ReLU mask (bit h: pre_h > 0) of each hit's last decode,
    // indexed by ray (null: not recorded); the normals need no forward pass
    // then
    uint4* hit_mask = nullptr;
    uint4* hit_mask2 = nullptr;   // level blending: the second decoder's masks
    // workspace: the normals' masked-sum operand (B fragments of diag(W2) W1,
    // rebuilt for each decoder by launch_normals*)
    uint2* wfrag = nullptr;
    int ctas_per_sm = 0;          // launch width of the persistent trace (0: the most that fit)
    // workspace (null: not prepared): per ray its first list entry as
    // (t_enter bits, t_exit bits, voxel id, packed ijk), written by the
    // handout-order pass, so a ray starts with one round of independent loads
    const int4* start = nullptr;
};

// One ray being traced: its list cursor [cur, end) with the current entry's
// interval [tin, tout], the current voxel, t, the decode count and the
// previous distance (oscillation rule).
struct RaySlot {
    int ray;
    int hit_ray;          // id of a ray this slot just finished as a hit, else -1
    int job;              // batched tracing: the job the ray belongs to
    float ox, oy, oz, dx, dy, dz;
    float t, tin, tout, dprev;
    int cur, end, k, vox;
    uint32_t ijk;
    // the next list entry's voxel (cur + 1 < end), loaded ahead so that moving
    // on costs no list read; its packed ijk once nijk_ok
    int nvox;
    uint32_t nijk;
    bool nijk_ok;
};

// The current entry's interval from its voxel S.ijk at depth D.
__device__ __forceinline__ void entry_interval(RaySlot& S, int D) {
    voxel_interval(S.ox, S.oy, S.oz, S.dx, S.dy, S.dz, S.ijk, D, S.tin, S.tout);
}

// Warp-uniform batch of ray indices taken from the global queue.
struct RayQueue {
    int next, end;
    bool exhausted;
    __device__ __forceinline__ void init() {
        next = end = 0;
        exhausted = false;
    }
};

__device__ __forceinline__ void finish(RaySlot& S, const TraceArgs& A, bool hit) {
    A.t_hit[S.ray] = hit ? S.t : __int_as_float(0x7f800000);
    A.hit[S.ray] = hit ? 1 : 0;
    if (A.steps) A.steps[S.ray] = S.k;
    A.hit_vox[S.ray] = hit ? S.vox : -1;
    if (hit) S.hit_ray = S.ray;
    S.ray = -1;
}

// Appends the rays this warp just finished as hits to the hit list (one
// atomic per warp and step).  Called by the whole warp, converged.
__device__ __forceinline__ void publish_hits(RaySlot& S, const TraceArgs& A, int lane,
                                             uint4 mask = make_uint4(0u, 0u, 0u, 0u),
                                             uint4 mask2 = make_uint4(0u, 0u, 0u, 0u)) {
    const unsigned m = __ballot_sync(0xffffffffu, S.hit_ray >= 0);
    if (m) {
        int base = 0;
        if (lane == 0) base = atomicAdd(A.hit_count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (S.hit_ray >= 0) {
            const int pos = base + __popc(m & ((1u << lane) - 1u));
            A.hit_list[pos] = S.hit_ray;
            if (A.hit_mask) A.hit_mask[S.hit_ray] = mask;
            if (A.hit_mask2) A.hit_mask2[S.hit_ray] = mask2;
        }
    }
    S.hit_ray = -1;
}

// Issues the load of the list entry after the current one (consumed by a
// later advance, so its latency hides behind the next decode).
__device__ __forceinline__ void load_next(RaySlot& S, const TraceArgs& A) {
    if (S.cur + 1 < S.end) S.nvox = A.vid[S.cur + 1];
    S.nijk_ok = false;
}

// The packed ijk of the next entry's voxel (its id arrived during the last
// decode); called between the gather and the decoder, so it is in a register
// before the ray can move on.
__device__ __forceinline__ void prefetch_next_ijk(RaySlot& S, const TraceArgs& A, const Tables& tb) {
    if (S.ray >= 0 && !S.nijk_ok && S.cur + 1 < S.end) {
        S.nijk = tb.node[A.D][S.nvox].ijk;
        S.nijk_ok = true;
    }
}

// Moves the cursor past entries that end before t (the ray is discarded when
// the list runs out), then jumps t to the current entry's start (Sec. 3.4).
__device__ __forceinline__ void advance(RaySlot& S, const TraceArgs& A, const Tables& tb) {
    bool first = true;
    while (S.t > S.tout) {
        if (++S.cur >= S.end) {
            finish(S, A, false);
            return;
        }
        S.vox = S.nvox;
        S.ijk = first && S.nijk_ok ? S.nijk : tb.node[A.D][S.vox].ijk;
        first = false;
        load_next(S, A);
        entry_interval(S, A.D);
    }
    if (S.t < S.tin) S.t = S.tin;
    if (S.t > A.far_t) finish(S, A, false);
}

__device__ __forceinline__ void start_ray(RaySlot& S, int r, const TraceArgs& A, const Tables& tb) {
    S.ray = r;
    S.k = 0;
    S.t = 0.0f;
    S.vox = -1;
    S.cur = A.offs[r];
    S.end = A.cnt ? S.cur + A.cnt[r] : A.offs[r + 1];
    int4 first = make_int4(0, 0, 0, 0);
    if (A.start) first = A.start[r];      // independent of the offsets: one round of loads
    if (S.cur >= S.end) {
        finish(S, A, false);
        return;
    }
    S.ox = A.o[3 * r];
    S.oy = A.o[3 * r + 1];
    S.oz = A.o[3 * r + 2];
    S.dx = A.d[3 * r];
    S.dy = A.d[3 * r + 1];
    S.dz = A.d[3 * r + 2];
    if (A.start) {
        S.tin = __int_as_float(first.x);
        S.tout = __int_as_float(first.y);
        S.vox = first.z;
        S.ijk = (uint32_t)first.w;
    } else {
        S.vox = A.vid[S.cur];
        S.ijk = tb.node[A.D][S.vox].ijk;
        entry_interval(S, A.D);
    }
    S.t = S.tin;
    S.dprev = __int_as_float(0x7fc00000);
    load_next(S, A);
    if (S.t > A.far_t) finish(S, A, false);
}

// Gives every lane without a ray the next unstarted ray (rays with an empty
// list are finished on the spot).  The batch is shared by the warp: one
// atomic per 32 rays, and neighbouring lanes get neighbouring rays.
__device__ __forceinline__ void refill(RaySlot& S, RayQueue& Qu, const TraceArgs& A, const Tables& tb,
                                       int lane) {
    for (;;) {
        const unsigned need = __ballot_sync(0xffffffffu, S.ray < 0);
        if (need == 0u || Qu.exhausted) return;
        if (Qu.next >= Qu.end) {
            int s = 0;
            if (lane == 0) s = atomicAdd(A.queue, 32);
            s = __shfl_sync(0xffffffffu, s, 0);
            if ((long long)s >= A.R) {
                Qu.exhausted = true;
                return;
            }
            if (A.order) s = A.order[s >> 5] << 5;
            Qu.next = s;
            Qu.end = (int)min((long long)s + 32, A.R);
        }
        const int rank = __popc(need & ((1u << lane) - 1u));
        const int avail = Qu.end - Qu.next;
        if (S.ray < 0 && rank < avail) start_ray(S, Qu.next + rank, A, tb);
        Qu.next += min(__popc(need), avail);
    }
}

// One sphere-tracing step after a decode returned dhat (Sec. A.4 rules).
__device__ __forceinline__ void step_update(RaySlot& S, float dhat, const TraceArgs& A, const Tables& tb) {
    ++S.k;
    if (dhat < A.eps) {
        finish(S, A, true);
        return;
    }
    if (A.osc && S.k > 1 && fabsf(dhat - S.dprev) < 6.0f * A.eps) {
        finish(S, A, fabsf(dhat) < 6.0f * A.eps);
        return;
    }
    S.dprev = dhat;
    S.t += dhat;
    if (S.t > A.far_t || S.k >= A.max_steps) {
        finish(S, A, false);
        return;
    }
    advance(S, A, tb);
}

// ---------------------------------------------------------------------------
// Batched tracing: many (octree, features, rays) jobs in one persistent
// launch.  Jobs sharing a decoder form a group; the kernel traces the groups
// one after another (staging each group's decoder once), and inside a group
// one ray queue spans all of its jobs' rays.
// ---------------------------------------------------------------------------
struct TraceJob {
    TraceArgs A;             // per-job rays, lists, outputs, workspace words
    Tables tb;               // per-job octree and feature tables
    long long ray_base;      // index of the job's first ray in its group's queue (a multiple of 32)
};

struct JobGroup {
    int j0, j1;              // jobs [j0, j1)
    long long nrays;         // queue length: the jobs' rays, each job padded to a multiple of 32
    const float* W1;
    const float* b1;
    const float* W2;
    const float* b2;         // one float (device)
    float z_scale;           // FP8 decode
    int* queue;
    const int32_t* order;    // handout order of the group's 32-ray chunks (longest list first)
};

// Gives every idle lane the next ray of the group (finishing empty-list rays
// on the spot); a lane's job is found by binary search over the jobs' bases.
__device__ __forceinline__ void refill_batch(RaySlot& S, RayQueue& Qu, const JobGroup& G,
                                             const TraceJob* __restrict__ jobs, int lane) {
    for (;;) {
        const unsigned need = __ballot_sync(0xffffffffu, S.ray < 0);
        if (need == 0u || Qu.exhausted) return;
        if (Qu.next >= Qu.end) {
            int s = 0;
            if (lane == 0) s = atomicAdd(G.queue, 32);
            s = __shfl_sync(0xffffffffu, s, 0);
            if ((long long)s >= G.nrays) {
                Qu.exhausted = true;
                return;
            }
            if (G.order) s = G.order[s >> 5] << 5;
            Qu.next = s;
            Qu.end = (int)min((long long)s + 32, G.nrays);
        }
        const int rank = __popc(need & ((1u << lane) - 1u));
        const int avail = Qu.end - Qu.next;
        if (S.ray < 0 && rank < avail) {
            const long long gi = Qu.next + rank;
            int lo = G.j0, hi = G.j1 - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].ray_base <= gi) lo = mid; else hi = mid - 1;
            }
            const long long local = gi - jobs[lo].ray_base;
            if (local < jobs[lo].A.R) {      // else: the padding after the job's last ray
                S.job = lo;
                start_ray(S, (int)local, jobs[lo].A, jobs[lo].tb);
            }
        }
        Qu.next += min(__popc(need), avail);
    }
}

// Appends finished hits to their own job's hit list.
__device__ __forceinline__ void publish_hits_batch(RaySlot& S, const TraceJob* __restrict__ jobs,
                                                   uint4 mask = make_uint4(0u, 0u, 0u, 0u)) {
    if (S.hit_ray >= 0) {
        const TraceArgs& A = jobs[S.job].A;
        const int pos = atomicAdd(A.hit_count, 1);
        A.hit_list[pos] = S.hit_ray;
        if (A.hit_mask) A.hit_mask[S.hit_ray] = mask;
    }
    S.hit_ray = -1;
}

// Host-side entry points implemented per translation unit.
// summed_ok: the caller only queries points inside voxels of LOD `lod` and
// so may take a summed corner table (nglod_features.summed_lod = lod).
int fill_tables(const nglod_svo* svo, const nglod_features* f, int lod, Tables& tb, bool summed_ok = false);
int check_decoder(const nglod_decoder* dec);
int launch_trace_fp32(const nglod_decoder* dec, const Tables& tb, const TraceArgs& A, bool f16, int sms,
                      cudaStream_t st);
int launch_normals(const nglod_decoder* dec, const Tables& tb, const TraceArgs& A, float* normal, bool f16,
                   int sms, cudaStream_t st);
// Central-difference normals of the hit rays (step h), plain and blended.
int launch_normals_fd(const nglod_decoder* dec, const Tables& tb, const TraceArgs& A, float h, float* normal,
                      bool f16, int sms, cudaStream_t st);
int launch_normals_blend_fd(const nglod_decoder* lo, const nglod_decoder* hi, float alpha, const Tables& tb,
                            const TraceArgs& A, float h, float* normal, bool f16, int sms, cudaStream_t st);
int check_normal_params(const nglod_trace_params* params, const char* who);
// Workspace layout of sphere_trace: [0, 256) header {queue, status, hit
// count}, then int32 hit voxel per ray, then int32 hit list.
inline size_t trace_ws_hit_vox_offset() { return 256; }
inline size_t trace_ws_hit_list_offset(long long R) { return 256 + ((sizeof(int32_t) * (size_t)R + 255) / 256) * 256; }
// ... then the ray-group order: int32 order[G], uint8 key[G] (G = ceil(R / 32))
// and the 2 x kOrderBuckets counters of its counting sort.
constexpr int kOrderBuckets = 256;
inline size_t trace_ws_align(size_t v) { return (v + 255) / 256 * 256; }
inline size_t trace_ws_order_offset(long long R) {
    return trace_ws_hit_list_offset(R) + trace_ws_align(sizeof(int32_t) * (size_t)R);
}
inline size_t trace_ws_key_offset(long long R) {
    return trace_ws_order_offset(R) + trace_ws_align(sizeof(int32_t) * (size_t)((R + 31) / 32));
}
inline size_t trace_ws_count_offset(long long R) { return trace_ws_key_offset(R) + trace_ws_align((size_t)((R + 31) / 32)); }
// ... then the hits' ReLU masks (16 B per ray); header word 3
// is nonzero when the last trace recorded them
inline size_t trace_ws_mask_offset(long long R) {
    return trace_ws_count_offset(R) + trace_ws_align(2 * kOrderBuckets * sizeof(int));
}
// ... then, per ray, its first list entry (16 B; the handout-order pass writes it)
inline size_t trace_ws_start_offset(long long R) { return trace_ws_mask_offset(R) + trace_ws_align(32 * (size_t)R); }
// ... then the normals' masked-sum operand: 3 splits x 8 K steps x 5 N tiles x 32 lanes x 8 B
constexpr size_t kWsFragBytes = 3 * 8 * 5 * 32 * 8;
inline size_t trace_ws_wfrag_offset(long long R) { return trace_ws_align(trace_ws_start_offset(R) + 16 * (size_t)R); }
inline size_t trace_ws_size(long long R) { return trace_ws_wfrag_offset(R) + kWsFragBytes; }
// header word 3: 1 = one mask per hit (plain traces), 2 = two (blended: the
// lower LOD's at [0, R), the upper's at [R, 2R)), 0 = none
constexpr int kWsMaskFlagWord = 3;
// Points A at the workspace's mask region(s) and marks them as recorded.
int enable_hit_masks(TraceArgs& A, void* work, cudaStream_t st, bool two = false);
// Rewrites the finished trace's hit list (hit_count ids) in ray order from
// the per-ray hit flags A.hit, so that the normals visit neighbouring hits
// together (the ray-order scratch of the workspace holds the block counts).
int enqueue_hit_order(const TraceArgs& A, void* work, cudaStream_t st);
// Enqueues the work-ordered ray-group handout of a trace (sets A.order) and
// the rays' first-entry records (sets A.start; node_D = the nodes of the
// lists' depth).
int enqueue_ray_order(TraceArgs& A, void* work, const Node* node_D, cudaStream_t st);
// split = true: the FP32-accurate decode (three-term BF16 splits, six products)
int launch_trace_bf16(const nglod_svo* svo, const nglod_decoder* dec, const Tables& tb, const TraceArgs& A,
                      bool f16, float fp8_z_absmax, cudaStream_t st, bool split = false);
int launch_query_bf16(const nglod_svo* svo, const Tables& tb, const nglod_decoder* dec, const float* x,
                      long long Q, int D, float* sdf, int8_t* deepest, bool f16, float fp8_z_absmax,
                      cudaStream_t st, bool split = false);
int launch_trace_batch_tc(const TraceJob* jobs, const JobGroup* groups, int ngroups, int in_dim, bool f16, bool fp8,
                          int ctas_per_sm, int sms, int* err, cudaStream_t st);
int launch_trace_blend_f32(const nglod_decoder* lo, const nglod_decoder* hi, float alpha, const Tables& tb,
                           const TraceArgs& A, bool f16, int sms, cudaStream_t st);
int launch_query_blend_f32(const nglod_decoder* lo, const nglod_decoder* hi, float alpha, const Tables& tb,
                           const float* x, long long Q, int D, float* sdf, bool f16, int sms, cudaStream_t st);
int launch_normals_blend(const nglod_decoder* lo, const nglod_decoder* hi, float alpha, const Tables& tb,
                         const TraceArgs& A, float* normal, bool f16, int sms, cudaStream_t st);
int launch_trace_blend_bf16(const nglod_svo* svo, const nglod_decoder* lo, const nglod_decoder* hi, float alpha,
                            const Tables& tb, const TraceArgs& A, bool f16, cudaStream_t st);
int launch_query_blend_bf16(const nglod_svo* svo, const nglod_decoder* lo, const nglod_decoder* hi, float alpha,
                            const Tables& tb, const float* x, long long Q, int D, float* sdf, bool f16,
                            cudaStream_t st);
int launch_trace_batch_f32(const TraceJob* jobs, const JobGroup* groups, int ngroups, int in_dim, bool f16,
                           int ctas_per_sm, int sms, cudaStream_t st);

}  // namespace nglod
