// Internal declarations shared by the CUDA translation units of libnglod.
// Nothing here is part of the public C ABI (see include/nglod.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/nglod.h"

namespace nglod {

constexpr int kFirstFeatureDepth = 3;   // LOD 1 = resolution 8 = depth 3
constexpr int kMaxDepth = 10;           // packed voxel coords use 10 bits/axis
constexpr int kMaxLods = kMaxDepth - kFirstFeatureDepth + 1;
constexpr int kFeatDim = 32;            // m (Sec. 4)
constexpr int kHidden = 128;            // h (Sec. 4)

// Per-voxel record at one depth: packed coordinates (i | j << 10 | k << 20),
// index of the first child at depth + 1, 8-bit occupied-children mask and
// parent index (-1 for the root).  One 16-byte load per voxel.
struct __align__(16) Node {
    uint32_t ijk;
    int32_t childbase;
    uint32_t childmask;
    int32_t parent;
};

}  // namespace nglod

struct nglod_svo {
    int num_depths = 0;                                  // Dmax + 1
    int64_t n[nglod::kMaxDepth + 1] = {};                 // voxels per depth
    int64_t nc[nglod::kMaxDepth + 1] = {};                // corners per depth
    nglod::Node* node[nglod::kMaxDepth + 1] = {};         // device
    int32_t* corners[nglod::kMaxDepth + 1] = {};          // device [V * 8]
    // anc[d][8 v + i] = id of the depth-(3 + i) voxel containing voxel v of
    // depth d, for i = 0..d-3 (i = d-3 is v itself); unused entries are -1.
    int32_t* anc[nglod::kMaxDepth + 1] = {};
    int device = 0;
    int num_sms = 0;
};

namespace nglod {

// ---------------------------------------------------------------------------
// Host-side status plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int check_cuda(cudaError_t e, const char* what);
int device_sms();

#define NGLOD_CUDA(call)                                         \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return ::nglod::check_cuda(_e, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t pack_ijk(uint32_t i, uint32_t j, uint32_t k) {
    return i | (j << 10) | (k << 20);
}
__host__ __device__ __forceinline__ uint32_t unpack_i(uint32_t p) { return p & 1023u; }
__host__ __device__ __forceinline__ uint32_t unpack_j(uint32_t p) { return (p >> 10) & 1023u; }
__host__ __device__ __forceinline__ uint32_t unpack_k(uint32_t p) { return (p >> 20) & 1023u; }

// 2^e as a float for -126 <= e <= 127 (exact).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// A ray prepared once for every slab test: origin, IEEE reciprocal of each
// direction component, and a bit per axis whose direction component is
// below FLT_MIN in magnitude (such an axis is treated as parallel).
struct __align__(16) RayPrep {
    float ox, oy, oz;
    int valid;                // 0: NaN/Inf component or zero direction
    float ix, iy, iz;
    int par;                  // bit a set: axis a parallel
};

// FP32 slab test of a prepared ray against voxel (i,j,k) at depth dp, all in
// round-to-nearest with no contraction.  Voxel bounds -1 + i 2^(1-dp) are
// exact.  hit iff max(t_near, 0) <= t_far; [tin, tout] = [max(t_near,0),
// t_far].  Written to agree bit-for-bit with any IEEE implementation of the
// same formula.
__device__ __forceinline__ bool slab_test(const RayPrep& r, uint32_t ijk, int dp,
                                          float& tin, float& tout) {
    const float s = pow2f(1 - dp);
    float tn = -INFINITY, tf = INFINITY;
    const float o[3] = {r.ox, r.oy, r.oz};
    const float inv[3] = {r.ix, r.iy, r.iz};
    const uint32_t c[3] = {unpack_i(ijk), unpack_j(ijk), unpack_k(ijk)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = __fsub_rn(__fmul_rn((float)c[a], s), 1.0f);
        const float hi = __fsub_rn(__fmul_rn((float)(c[a] + 1u), s), 1.0f);
        if ((r.par >> a) & 1) {
            if (!(lo <= o[a] && o[a] <= hi)) return false;
            continue;
        }
        const float t0 = __fmul_rn(__fsub_rn(lo, o[a]), inv[a]);
        const float t1 = __fmul_rn(__fsub_rn(hi, o[a]), inv[a]);
        const float mn = t0 < t1 ? t0 : t1;
        const float mx = t0 < t1 ? t1 : t0;
        if (mn > tn) tn = mn;
        if (mx < tf) tf = mx;
    }
    const float te = tn > 0.0f ? tn : 0.0f;
    if (!(te <= tf)) return false;
    tin = te;
    tout = tf;
    return true;
}

// Octant of the ray origin relative to the centre of voxel (i,j,k) at depth
// dp: bit a set iff o_a >= centre_a.  The front-to-back rank of child slot c
// is c ^ octant (ordering depends only on the origin octant).
__device__ __forceinline__ uint32_t origin_octant(const RayPrep& r, uint32_t ijk, int dp) {
    const float h = pow2f(-dp);
    const float cx = __fsub_rn(__fmul_rn((float)(2u * unpack_i(ijk) + 1u), h), 1.0f);
    const float cy = __fsub_rn(__fmul_rn((float)(2u * unpack_j(ijk) + 1u), h), 1.0f);
    const float cz = __fsub_rn(__fmul_rn((float)(2u * unpack_k(ijk) + 1u), h), 1.0f);
    return (r.ox >= cx ? 1u : 0u) | (r.oy >= cy ? 2u : 0u) | (r.oz >= cz ? 4u : 0u);
}

// Kernel-side error status words (device memory, caller workspace).
enum : int { kStatusOk = 0, kStatusOverflow = 1, kStatusTimeout = 2, kStatusBadIndex = 3 };

}  // namespace nglod
