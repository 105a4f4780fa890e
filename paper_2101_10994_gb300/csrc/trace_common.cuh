// Ray state and stepping rules of the sphere tracer (Sec. 3.4 "Adaptive Ray
// Stepping", supplementary Sec. A.4) shared by the FP32 and BF16 kernels,
// plus the FP32 decoder evaluated with constant-bank weights.
#pragma once

#include "nglod_internal.cuh"
#include "query_common.cuh"

namespace nglod {

// The whole FP32 decoder as a kernel parameter block (constant bank).
struct DecParams {
    float W1[kHidden * 35];   // [hidden][in_dim], row stride = in_dim
    float b1[kHidden];
    float W2[kHidden];
    float b2;
};

// d = W2 . relu(W1 [x, z] + b1) + b2 for the lane's own slot, z read from
// its staged row.  Fully unrolled: each weight is an immediate operand.
template <int IN>
__device__ __forceinline__ float mlp_f32(const DecParams& P, const float* zrow, float x0, float x1,
                                         float x2) {
    constexpr int OFF = IN - kFeatDim;
    float v[IN];
    if constexpr (OFF == 3) {
        v[0] = x0;
        v[1] = x1;
        v[2] = x2;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 a = reinterpret_cast<const float4*>(zrow)[j];
        v[OFF + 4 * j] = a.x;
        v[OFF + 4 * j + 1] = a.y;
        v[OFF + 4 * j + 2] = a.z;
        v[OFF + 4 * j + 3] = a.w;
    }
    float out = P.b2;
#pragma unroll
    for (int h = 0; h < kHidden; ++h) {
        float acc = P.b1[h];
#pragma unroll
        for (int k = 0; k < IN; ++k) acc = fmaf(P.W1[h * IN + k], v[k], acc);
        out = fmaf(P.W2[h], fmaxf(acc, 0.0f), out);
    }
    return out;
}

struct TraceArgs {
    const float* o;
    const float* d;
    long long R;
    int D;
    float eps, far_t;
    int max_steps, osc;
    const int32_t* offs;
    const int32_t* vid;
    const float2* tr;
    float* t_hit;
    uint8_t* hit;
    int32_t* steps;       // nullable
    int32_t* hit_vox;     // workspace: voxel of the hit (for normals)
    int* queue;           // workspace: next unstarted ray
};

// One ray being traced: its list cursor [cur, end) with the current entry's
// interval [tin, tout], the current voxel, t, the decode count and the
// previous distance (oscillation rule).
struct RaySlot {
    int ray;
    float ox, oy, oz, dx, dy, dz;
    float t, tin, tout, dprev;
    int cur, end, k, vox;
    uint32_t ijk;
};

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
    S.ray = -1;
}

// Moves the cursor past entries that end before t (the ray is discarded when
// the list runs out), then jumps t to the current entry's start (Sec. 3.4).
__device__ __forceinline__ void advance(RaySlot& S, const TraceArgs& A, const Tables& tb) {
    bool moved = false;
    while (S.t > S.tout) {
        if (++S.cur >= S.end) {
            finish(S, A, false);
            return;
        }
        const float2 tr = A.tr[S.cur];
        S.tin = tr.x;
        S.tout = tr.y;
        moved = true;
    }
    if (moved) {
        S.vox = A.vid[S.cur];
        S.ijk = tb.node[A.D][S.vox].ijk;
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
    S.end = A.offs[r + 1];
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
    const float2 tr = A.tr[S.cur];
    S.tin = tr.x;
    S.tout = tr.y;
    S.t = tr.x;
    S.dprev = __int_as_float(0x7fc00000);
    S.vox = A.vid[S.cur];
    S.ijk = tb.node[A.D][S.vox].ijk;
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

// Host-side entry points implemented per translation unit.
int fill_tables(const nglod_svo* svo, const nglod_features* f, int lod, Tables& tb);
int fill_dec_params(const nglod_decoder* dec, DecParams& P, cudaStream_t st);
int launch_trace_fp32(const nglod_decoder* dec, const DecParams& P, const Tables& tb, const TraceArgs& A,
                      bool f16, int sms, cudaStream_t st);
int launch_normals(const nglod_decoder* dec, const Tables& tb, const TraceArgs& A, float* normal, bool f16,
                   int sms, cudaStream_t st);
int launch_trace_bf16(const nglod_svo* svo, const nglod_decoder* dec, const Tables& tb, const TraceArgs& A,
                      bool f16, cudaStream_t st);
int launch_query_bf16(const nglod_svo* svo, const Tables& tb, const nglod_decoder* dec, const float* x,
                      long long Q, int D, float* sdf, int8_t* deepest, bool f16, cudaStream_t st);

}  // namespace nglod
