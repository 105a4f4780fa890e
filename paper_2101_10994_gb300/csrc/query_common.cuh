// Device building blocks of the feature query (Sec. 3.2) shared by the
// sdf_query, sphere_trace and gradient kernels.
//
// Work layout: a warp owns 32 query "slots" (one per lane: the lane holds the
// slot's point, voxel and, in the tracer, its ray state).  Feature gathers
// are cooperative: in gather_slot the warp splits into 4 groups of 8 lanes
// and each group interpolates one slot at a time, lane l covering channels
// 4l..4l+3, so one warp-wide 16-byte load fetches 4 whole 128-byte corner
// rows (FP32); gather_slot4 (the sphere tracers) uses 8 groups of 4 lanes, 8
// channels a lane, so a warp interpolates 8 slots per round and needs half
// the rounds (measured ~10 % faster traces).  The interpolated z of the 32
// slots is staged in shared memory (or the MMA's operand tile), where each
// lane reads back its own slot's 32 channels for the decoder.
#pragma once

#include <cuda_fp16.h>

#include "nglod_internal.cuh"

namespace nglod {

constexpr int kZStride = 36;   // floats per staged z row (16-B aligned, 4-way banks)

struct Tables {
    const void* feats[kMaxLods];             // LOD l at index l - 1
    // first depth whose table is gathered: kFirstFeatureDepth, or the
    // queried depth for a summed corner table (it already holds the
    // coarser levels' sum at its corners)
    int first_depth;
    const int32_t* corners[kMaxDepth + 1];   // [V_dp, 8]
    const int32_t* anc[kMaxDepth + 1];       // [V_dp, 8]
    const int32_t* cids[kMaxDepth + 1];      // [V_dp, dp - 2, 8]: corner ids of every level (svo_build)
    const Node* node[kMaxDepth + 1];
};

template <typename T>
struct FeatLoad;

template <>
struct FeatLoad<float> {
    // channels 4l..4l+3 of feature row `row`
    static __device__ __forceinline__ float4 load(const void* base, int row, int l) {
        return __ldg(reinterpret_cast<const float4*>(base) + (size_t)row * 8 + l);
    }
};

template <>
struct FeatLoad<__half> {
    static __device__ __forceinline__ float4 load(const void* base, int row, int l) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(base) + (size_t)row * 8 + l);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};

__device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.0f), 1.0f); }

// Trilinear weights w_c = prod_a (c_a ? u_a : 1 - u_a), c = cx | cy<<1 | cz<<2.
__device__ __forceinline__ void trilinear_weights(float u0, float u1, float u2, float w[8]) {
    const float a0 = 1.0f - u0, a1 = 1.0f - u1, a2 = 1.0f - u2;
    const float p00 = a1 * a2, p10 = u1 * a2, p01 = a1 * u2, p11 = u1 * u2;
    w[0] = a0 * p00; w[1] = u0 * p00;
    w[2] = a0 * p10; w[3] = u0 * p10;
    w[4] = a0 * p01; w[5] = u0 * p01;
    w[6] = a0 * p11; w[7] = u0 * p11;
}

// Group-cooperative z for one slot: the slot's voxel at depth dd is `vox`
// with packed coordinates ijk; q = x + 1 in FP32.  Returns this lane's four
// channels of sum_{dp=3..dd} psi_dp(x).  All 8 lanes of the group must call
// it together (gmask = the group's lanes, gbase = its first lane).
template <typename T>
__device__ __forceinline__ float4 gather_slot(const Tables& tb, int dd, int vox, uint32_t ijk,
                                              float q0, float q1, float q2, unsigned gmask,
                                              int gbase, int l) {
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int a = (l <= dd - kFirstFeatureDepth) ? __ldg(tb.anc[dd] + (size_t)vox * 8 + l) : -1;
#pragma unroll 1
    for (int dp = tb.first_depth; dp <= dd; ++dp) {
        const int v = __shfl_sync(gmask, a, gbase + dp - kFirstFeatureDepth);
        const int cid = __ldg(tb.corners[dp] + (size_t)v * 8 + l);
        const int sh = dd - dp;
        const float sc = pow2f(dp - 1);
        const float u0 = clamp01(__fsub_rn(__fmul_rn(q0, sc), (float)(unpack_i(ijk) >> sh)));
        const float u1 = clamp01(__fsub_rn(__fmul_rn(q1, sc), (float)(unpack_j(ijk) >> sh)));
        const float u2 = clamp01(__fsub_rn(__fmul_rn(q2, sc), (float)(unpack_k(ijk) >> sh)));
        float w[8];
        trilinear_weights(u0, u1, u2, w);
        const void* fb = tb.feats[dp - kFirstFeatureDepth];
        float4 r[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) r[c] = FeatLoad<T>::load(fb, __shfl_sync(gmask, cid, gbase + c), l);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            z.x = fmaf(w[c], r[c].x, z.x);
            z.y = fmaf(w[c], r[c].y, z.y);
            z.z = fmaf(w[c], r[c].z, z.z);
            z.w = fmaf(w[c], r[c].w, z.w);
        }
    }
    return z;
}

// Channels 8 l4 .. 8 l4 + 7 of feature row `row` (4 lanes cover the 32).
template <typename T>
struct FeatLoad8;

// FP32 rows: one 32-byte load per lane (the 4 lanes read the 128-byte row
// with a single instruction; rows are 128-byte aligned).
template <>
struct FeatLoad8<float> {
    static __device__ __forceinline__ void load(const void* base, int row, int l4, float4& a, float4& b) {
        const float* p = reinterpret_cast<const float*>(base) + (size_t)row * 32 + 8 * l4;
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
            : "l"(p));
    }
};

template <>
struct FeatLoad8<__half> {
    static __device__ __forceinline__ void load(const void* base, int row, int l4, float4& a, float4& b) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(base) + (size_t)row * 4 + l4);
        const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        const float2 f2 = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
        const float2 f3 = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
        a = make_float4(f0.x, f0.y, f1.x, f1.y);
        b = make_float4(f2.x, f2.y, f3.x, f3.y);
    }
};

// FP32 fused multiply-add of two lanes at once (a packed pair, each
// component rounded once exactly as fmaf): z += w * r.
__device__ __forceinline__ float2 fma2(float w, float2 r, float2 z) {
    return __ffma2_rn(make_float2(w, w), r, z);
}

// One warp-level tensor-core MMA, D = A B + D, m16n8k16, BF16 operands and
// FP32 accumulation.  With g = lane / 4 and c = 2 (lane % 4): a0 holds
// A[g][c..c+1], a1 A[g+8][c..c+1], a2 A[g][c+8..c+9], a3 A[g+8][c+8..c+9]
// (two BF16, the lower column in the lower half); b.x holds B[c..c+1][g],
// b.y B[c+8..c+9][g]; c[0..1] = D[g][c..c+1], c[2..3] = D[g+8][c..c+1].
__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint2 b) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b.x), "r"(b.y));
}

// gather_slot with 4-lane groups: lane l4 of the group owns channels
// 8 l4 .. 8 l4 + 7, so a warp interpolates 8 slots at a time.  The corner
// ids of a level come from the flat table (one 8-byte load per lane: two
// corners each, shared within the group), and the next level's ids are in
// flight while this level's rows are loaded.  Every channel sums the same
// terms in the same order as gather_slot (levels ascending, corners 0..7;
// packed FMAs round each lane exactly as fmaf), so the result is
// bit-identical to it.
// This lane's pair of corner ids (corners 2 l4, 2 l4 + 1) at depth dp of the
// depth-dd voxel vox, from the flat table.
__device__ __forceinline__ const int2* corner_ids(const Tables& tb, int dd, int vox, int dp, int l4) {
    return reinterpret_cast<const int2*>(tb.cids[dd] + ((size_t)vox * (dd - kFirstFeatureDepth + 1) +
                                                        (dp - kFirstFeatureDepth)) * 8) + l4;
}

// The first depth a gather over depths dfirst..dlast reads.
__device__ __forceinline__ int gather_first_depth(const Tables& tb, int dfirst = kFirstFeatureDepth) {
    return max(dfirst, tb.first_depth);
}

// gather_slot4 with the first level's corner ids already loaded by the
// caller (first_ids = *corner_ids(tb, dd, vox, gather_first_depth(tb,
// dfirst), l4)), so that a loop over slots can fetch the next slot's ids
// while this one is gathered.
template <typename T>
__device__ __forceinline__ void gather_slot4_ids(const Tables& tb, int dd, int vox, uint32_t ijk, float q0, float q1,
                                                 float q2, unsigned gmask, int gbase, int l4, float4& za, float4& zb,
                                                 int2 first_ids, int dlast = kMaxDepth,
                                                 int dfirst = kFirstFeatureDepth) {
    float2 z[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const int top = min(dd, dlast);     // only depths dfirst..dlast (level blending, Eq. 3)
    int dp = gather_first_depth(tb, dfirst);
    // lane l4's pair of corner ids at level i: ids[4 i]
    const int2* ids = reinterpret_cast<const int2*>(tb.cids[dd] + (size_t)vox * (dd - kFirstFeatureDepth + 1) * 8) + l4;
    int2 cc = first_ids;
#pragma unroll 1
    for (; dp <= top; ++dp) {
        const int i = dp - kFirstFeatureDepth;
        const int2 cur = cc;
        if (dp < top) cc = __ldg(ids + 4 * (i + 1));
        const int sh = dd - dp;
        const float sc = pow2f(dp - 1);
        const float u0 = clamp01(__fsub_rn(__fmul_rn(q0, sc), (float)(unpack_i(ijk) >> sh)));
        const float u1 = clamp01(__fsub_rn(__fmul_rn(q1, sc), (float)(unpack_j(ijk) >> sh)));
        const float u2 = clamp01(__fsub_rn(__fmul_rn(q2, sc), (float)(unpack_k(ijk) >> sh)));
        float w[8];
        trilinear_weights(u0, u1, u2, w);
        const void* fb = tb.feats[i];
        float4 ra[8], rb[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int cid = __shfl_sync(gmask, (c & 1) ? cur.y : cur.x, gbase + (c >> 1));
            FeatLoad8<T>::load(fb, cid, l4, ra[c], rb[c]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            z[0] = fma2(w[c], make_float2(ra[c].x, ra[c].y), z[0]);
            z[1] = fma2(w[c], make_float2(ra[c].z, ra[c].w), z[1]);
            z[2] = fma2(w[c], make_float2(rb[c].x, rb[c].y), z[2]);
            z[3] = fma2(w[c], make_float2(rb[c].z, rb[c].w), z[3]);
        }
    }
    za = make_float4(z[0].x, z[0].y, z[1].x, z[1].y);
    zb = make_float4(z[2].x, z[2].y, z[3].x, z[3].y);
}

template <typename T>
__device__ __forceinline__ void gather_slot4(const Tables& tb, int dd, int vox, uint32_t ijk, float q0, float q1,
                                             float q2, unsigned gmask, int gbase, int l4, float4& za, float4& zb,
                                             int dlast = kMaxDepth, int dfirst = kFirstFeatureDepth) {
    const int dp = gather_first_depth(tb, dfirst);
    const int2 first = dp <= min(dd, dlast) ? __ldg(corner_ids(tb, dd, vox, dp, l4)) : make_int2(0, 0);
    gather_slot4_ids<T>(tb, dd, vox, ijk, q0, q1, q2, gmask, gbase, l4, za, zb, first, dlast, dfirst);
}

// Locates x by descending from the root through the child masks (the voxels
// V_1..V_L containing x, Sec. 3.2): q = fl32(x + 1), coordinates at depth D
// clamp(floor(q 2^(D-1)), 0, 2^D - 1), shifted for shallower depths.  Returns
// the deepest depth reached (-1 if x is outside [-1,1]^3 or NaN) with that
// voxel's id and packed coordinates.
__device__ __forceinline__ int locate_descend(const Tables& tb, int D, float x0, float x1, float x2,
                                              int& vox, uint32_t& ijk) {
    vox = -1;
    ijk = 0;
    if (!(x0 >= -1.0f && x0 <= 1.0f && x1 >= -1.0f && x1 <= 1.0f && x2 >= -1.0f && x2 <= 1.0f))
        return -1;
    const float sc = pow2f(D - 1);
    const int hi = (1 << D) - 1;
    const int c0 = min(max((int)floorf(__fmul_rn(__fadd_rn(x0, 1.0f), sc)), 0), hi);
    const int c1 = min(max((int)floorf(__fmul_rn(__fadd_rn(x1, 1.0f), sc)), 0), hi);
    const int c2 = min(max((int)floorf(__fmul_rn(__fadd_rn(x2, 1.0f), sc)), 0), hi);
    int v = 0, dd = 0;
    for (int dp = 1; dp <= D; ++dp) {
        const int sh = D - dp;
        const uint32_t slot = ((c0 >> sh) & 1) | (((c1 >> sh) & 1) << 1) | (((c2 >> sh) & 1) << 2);
        const Node nd = tb.node[dp - 1][v];
        if (!((nd.childmask >> slot) & 1u)) break;
        v = nd.childbase + __popc(nd.childmask & ((1u << slot) - 1u));
        dd = dp;
    }
    vox = v;
    const int sh = D - dd;
    ijk = pack_ijk((uint32_t)(c0 >> sh), (uint32_t)(c1 >> sh), (uint32_t)(c2 >> sh));
    return dd;
}

}  // namespace nglod
