// Device building blocks of the feature query (Sec. 3.2) shared by the
// sdf_query, sphere_trace and gradient kernels.
//
// Work layout: a warp owns 32 query "slots" (one per lane: the lane holds the
// slot's point, voxel and, in the tracer, its ray state).  Feature gathers
// are cooperative: the warp splits into 4 groups of 8 lanes and each group
// interpolates one slot at a time, lane l covering channels 4l..4l+3, so one
// warp-wide 16-byte load fetches 4 whole 128-byte corner rows (FP32) and the
// rows of neighbouring slots share cache lines.  The interpolated z of the
// 32 slots is staged in shared memory, where each lane reads back its own
// slot's 32 channels for the decoder.
#pragma once

#include <cuda_fp16.h>

#include "nglod_internal.cuh"

namespace nglod {

constexpr int kZStride = 36;   // floats per staged z row (16-B aligned, 4-way banks)

struct Tables {
    const void* feats[kMaxLods];             // LOD l at index l - 1
    const int32_t* corners[kMaxDepth + 1];   // [V_dp, 8]
    const int32_t* anc[kMaxDepth + 1];       // [V_dp, 8]
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
    for (int dp = kFirstFeatureDepth; dp <= dd; ++dp) {
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

// gather_slot restricted to the levels dfirst..dlast (3 <= dfirst, dlast <=
// dd): this lane's four channels of sum_{dp=dfirst..dlast} psi_dp(x).  Used
// by level blending (Eq. 3), which decodes the sums up to two consecutive
// LODs.  All 8 lanes of the group must call it together.
template <typename T>
__device__ __forceinline__ float4 gather_levels(const Tables& tb, int dd, int dfirst, int dlast, int vox,
                                                uint32_t ijk, float q0, float q1, float q2, unsigned gmask,
                                                int gbase, int l) {
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int a = (l <= dd - kFirstFeatureDepth) ? __ldg(tb.anc[dd] + (size_t)vox * 8 + l) : -1;
#pragma unroll 1
    for (int dp = dfirst; dp <= dlast; ++dp) {
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

// One slot of a warp as seen by the gather: its voxel at depth dd (dd < 3:
// no feature level, z = 0), packed coordinates and q = fl32(x + 1).
struct GSlot {
    int dd, vox;
    uint32_t ijk;
    float q0, q1, q2;
};

// Software-pipelined cooperative z of a warp's 32 slots.  As in gather_slot,
// each 8-lane group interpolates one slot per round (lane l: channels
// 4l..4l+3) over 8 rounds, but the three dependent loads of a level
// (ancestor -> corner ids -> feature rows) no longer run back to back:
// round r+1's corner ids of every level are copied into the warp's shared
// buffer with cp.async (no registers held while in flight) and round r+2's
// ancestors are loaded while round r's feature rows load, so a round waits
// on its feature loads only.  A group reads a level's 8 corner ids as two
// broadcast 16-byte shared loads.
//   cidbuf             per-warp shared int[2][kMaxLods][32], 16-byte aligned
//   slot(s)            GSlot of slot s (called converged by the whole warp)
//   store(r, zlo, z)   z = sum over depths 3..min(dd, dcap); zlo = the sum
//                      over 3..min(dd, dcap, dsplit)
constexpr int kCidBufInts = 2 * kMaxLods * 32;

__device__ __forceinline__ void cp_async4(int* dst, const int* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename T, typename SlotFn, typename StoreFn>
__device__ __forceinline__ void gather_warp(const Tables& tb, int dsplit, int dcap, int* __restrict__ cidbuf,
                                            SlotFn slot, StoreFn store, unsigned gmask, int gbase, int g, int l) {
    const int lane = gbase + l;
    auto anc_of = [&](const GSlot& S) -> int {
        return (S.dd >= kFirstFeatureDepth && l <= S.dd - kFirstFeatureDepth)
                   ? __ldg(tb.anc[S.dd] + (size_t)S.vox * 8 + l) : -1;
    };
    // lane l copies corner l of every level of slot S into buf[level][lane]
    auto issue_cids = [&](const GSlot& S, int a, int* buf) {
        const int top = min(S.dd, dcap);
#pragma unroll 1
        for (int dp = kFirstFeatureDepth; dp <= top; ++dp) {
            const int v = __shfl_sync(gmask, a, gbase + dp - kFirstFeatureDepth);
            cp_async4(buf + (dp - kFirstFeatureDepth) * 32 + lane, tb.corners[dp] + (size_t)v * 8 + l);
        }
        cp_async_commit();
    };
    GSlot S0 = slot(g), S1 = slot(4 + g);
    int a1 = anc_of(S1);
    issue_cids(S0, anc_of(S0), cidbuf);
#pragma unroll 1
    for (int r = 0; r < 8; ++r) {
        GSlot S2 = slot(min(r + 2, 7) * 4 + g);
        if (r + 2 > 7) S2.dd = -1;
        const int a2 = anc_of(S2);
        issue_cids(S1, a1, cidbuf + ((r + 1) & 1) * kMaxLods * 32);
        cp_async_wait<1>();                 // this lane's copies for round r are in
        __syncwarp();                       // ... and every other lane's
        const int* buf = cidbuf + (r & 1) * kMaxLods * 32;
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f), zlo = z;
        const int top = min(S0.dd, dcap);
#pragma unroll 1
        for (int dp = kFirstFeatureDepth; dp <= top; ++dp) {
            const int4 ca = *reinterpret_cast<const int4*>(buf + (dp - kFirstFeatureDepth) * 32 + gbase);
            const int4 cb = *reinterpret_cast<const int4*>(buf + (dp - kFirstFeatureDepth) * 32 + gbase + 4);
            const int sh = S0.dd - dp;
            const float sc = pow2f(dp - 1);
            const float u0 = clamp01(__fsub_rn(__fmul_rn(S0.q0, sc), (float)(unpack_i(S0.ijk) >> sh)));
            const float u1 = clamp01(__fsub_rn(__fmul_rn(S0.q1, sc), (float)(unpack_j(S0.ijk) >> sh)));
            const float u2 = clamp01(__fsub_rn(__fmul_rn(S0.q2, sc), (float)(unpack_k(S0.ijk) >> sh)));
            float w[8];
            trilinear_weights(u0, u1, u2, w);
            const void* fb = tb.feats[dp - kFirstFeatureDepth];
            const int cid[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
            float4 rr[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) rr[c] = FeatLoad<T>::load(fb, cid[c], l);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                z.x = fmaf(w[c], rr[c].x, z.x);
                z.y = fmaf(w[c], rr[c].y, z.y);
                z.z = fmaf(w[c], rr[c].z, z.z);
                z.w = fmaf(w[c], rr[c].w, z.w);
            }
            if (dp == dsplit) zlo = z;
        }
        if (dsplit >= top) zlo = z;
        store(r, zlo, z);
        __syncwarp();                       // buf is refilled two rounds on
        S0 = S1;
        S1 = S2;
        a1 = a2;
    }
    cp_async_wait<0>();
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
