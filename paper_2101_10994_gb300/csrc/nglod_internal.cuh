// Internal declarations shared by the CUDA translation units of libnglod.
// Nothing here is part of the public C ABI (see include/nglod.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
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
    // cids[d][(v (d - 2) + i) 8 + c] = corner id, at depth 3 + i, of corner c
    // of the depth-(3 + i) voxel containing voxel v of depth d (i = 0..d-3):
    // every corner id a query in voxel v gathers, one 32-byte record per level
    int32_t* cids[nglod::kMaxDepth + 1] = {};
    int* dstatus = nullptr;                               // device status word
    unsigned* dscratch = nullptr;                         // 16 device words (reductions)
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

// Bounded tensor-core waits: the poll budget of the wait for each tile's
// MMA (nglod_set_wait_polls changes it, for tests of the expiry path); the
// wait that drains an MMA after an expiry always keeps the default, so no
// MMA is still in flight when its tensor memory is freed.
constexpr long long kDefaultWaitPolls = 1ll << 24;
long long mma_wait_polls();

// Runs f once for each device it is called on (the device current at the
// call): kernel attributes such as cudaFuncSetAttribute apply to the current
// device only, so a process that launches on several devices must set them
// on each.  Two threads may both run f for one device; f must be idempotent.
template <class F>
inline void once_per_device(std::atomic<unsigned long long>& done, F&& f) {
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load(std::memory_order_acquire) & bit)) {
        f();
        done.fetch_or(bit, std::memory_order_acq_rel);
    }
}

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

// Prepares a ray: IEEE reciprocals of the direction components (0 for an
// axis below FLT_MIN in magnitude, which is then parallel) and the validity
// flag (finite components, not all axes parallel).
__device__ __forceinline__ RayPrep make_ray_prep(float ox, float oy, float oz, float dx, float dy, float dz) {
    RayPrep p;
    p.ox = ox;
    p.oy = oy;
    p.oz = oz;
    const float dd[3] = {dx, dy, dz};
    const float oo[3] = {ox, oy, oz};
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
    return p;
}

// FP32 slab test of a prepared ray against voxel (i,j,k) at depth dp, all in
// round-to-nearest with no contraction of the rounded steps.  Voxel bounds
// lo = -1 + i 2^(1-dp) and hi = lo + 2^(1-dp) are exact (a single fused
// multiply-add of exact terms rounds nothing), as is the centre lo + 2^(-dp).
// Per axis t0 = (lo - o) * inv, t1 = (hi - o) * inv, each rounded after the
// subtraction and after the product.  hit iff max(t_near, 0) <= t_far;
// [tin, tout] = [max(t_near, 0), t_far].  *oct (if non-null) receives the
// origin octant relative to the voxel centre (bit a set iff o_a >= centre_a),
// which orders the children front to back: rank r visits slot r ^ oct.
__device__ __forceinline__ bool slab_test(const RayPrep& r, uint32_t ijk, int dp, float& tin, float& tout,
                                          uint32_t* oct = nullptr) {
    const float s = pow2f(1 - dp);
    const float hs = pow2f(-dp);
    float tn = -INFINITY, tf = INFINITY;
    const float o[3] = {r.ox, r.oy, r.oz};
    const float inv[3] = {r.ix, r.iy, r.iz};
    const uint32_t c[3] = {unpack_i(ijk), unpack_j(ijk), unpack_k(ijk)};
    uint32_t octant = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = __fmaf_rn((float)c[a], s, -1.0f);
        const float hi = __fadd_rn(lo, s);
        if (oct) octant |= (o[a] >= __fadd_rn(lo, hs)) ? (1u << a) : 0u;
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
    if (oct) *oct = octant;
    return true;
}

// [t_enter, t_exit] of ray (o, d) in voxel (i,j,k) at depth dp by the slab
// test above -- the bits the traversal writes for a listed voxel (its
// child_slabs + child_hit are equal to slab_test bit for bit); an interval
// that does not hit (never the case for a listed voxel) comes back empty.
__device__ __forceinline__ void voxel_interval(float ox, float oy, float oz, float dx, float dy, float dz,
                                               uint32_t ijk, int dp, float& tin, float& tout) {
    const RayPrep r = make_ray_prep(ox, oy, oz, dx, dy, dz);
    if (!slab_test(r, ijk, dp, tin, tout)) {
        tin = INFINITY;
        tout = -INFINITY;
    }
}

// Octant of the ray origin relative to the centre lo + 2^(-dp) of voxel
// (i,j,k) at depth dp, computed exactly as inside slab_test.
__device__ __forceinline__ uint32_t origin_octant(const RayPrep& r, uint32_t ijk, int dp) {
    const float s = pow2f(1 - dp);
    const float hs = pow2f(-dp);
    const float cx = __fadd_rn(__fmaf_rn((float)unpack_i(ijk), s, -1.0f), hs);
    const float cy = __fadd_rn(__fmaf_rn((float)unpack_j(ijk), s, -1.0f), hs);
    const float cz = __fadd_rn(__fmaf_rn((float)unpack_k(ijk), s, -1.0f), hs);
    return (r.ox >= cx ? 1u : 0u) | (r.oy >= cy ? 2u : 0u) | (r.oz >= cz ? 4u : 0u);
}

// Slab tests of all 8 children of voxel (i,j,k) at depth dp at once.  A
// child's bounds along axis a are (lo, mid) or (mid, hi) with lo, mid, hi the
// parent's low face, centre and high face -- the very values slab_test
// computes for the child (lo = fma(2i, 2^-dp, -1) = parent lo, hi = lo +
// 2^-dp), so each crossing t = (plane - o) * inv is computed once per plane
// and the results equal eight separate slab_test calls bit for bit.
// Returns the hit mask by child slot; tin/tout[c] hold the hit intervals.
struct ChildSlabs {
    float tn[3][2], tf[3][2];   // per axis, per side (0 low child, 1 high child)
    bool in[3][2];              // parallel axes: origin inside that side's slab
};

__device__ __forceinline__ void child_slabs(const RayPrep& r, uint32_t ijk, int dp, ChildSlabs& cs) {
    const float s = pow2f(1 - dp);
    const float hs = pow2f(-dp);
    const float o[3] = {r.ox, r.oy, r.oz};
    const float inv[3] = {r.ix, r.iy, r.iz};
    const uint32_t c[3] = {unpack_i(ijk), unpack_j(ijk), unpack_k(ijk)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = __fmaf_rn((float)c[a], s, -1.0f);
        const float mid = __fadd_rn(lo, hs);
        const float hi = __fadd_rn(mid, hs);
        if ((r.par >> a) & 1) {
            cs.in[a][0] = lo <= o[a] && o[a] <= mid;
            cs.in[a][1] = mid <= o[a] && o[a] <= hi;
            cs.tn[a][0] = cs.tn[a][1] = -INFINITY;
            cs.tf[a][0] = cs.tf[a][1] = INFINITY;
            continue;
        }
        cs.in[a][0] = cs.in[a][1] = true;
        const float t_lo = __fmul_rn(__fsub_rn(lo, o[a]), inv[a]);
        const float t_mid = __fmul_rn(__fsub_rn(mid, o[a]), inv[a]);
        const float t_hi = __fmul_rn(__fsub_rn(hi, o[a]), inv[a]);
        cs.tn[a][0] = t_lo < t_mid ? t_lo : t_mid;
        cs.tf[a][0] = t_lo < t_mid ? t_mid : t_lo;
        cs.tn[a][1] = t_mid < t_hi ? t_mid : t_hi;
        cs.tf[a][1] = t_mid < t_hi ? t_hi : t_mid;
    }
}

// Hit test of child slot c from its per-axis intervals (same max / min and
// closed-interval rule as slab_test).
__device__ __forceinline__ bool child_hit(const ChildSlabs& cs, uint32_t c, float& tin, float& tout) {
    const bool x = c & 1u, y = (c >> 1) & 1u, z = (c >> 2) & 1u;
    if (!((x ? cs.in[0][1] : cs.in[0][0]) && (y ? cs.in[1][1] : cs.in[1][0]) && (z ? cs.in[2][1] : cs.in[2][0])))
        return false;
    float tn = x ? cs.tn[0][1] : cs.tn[0][0];
    float tf = x ? cs.tf[0][1] : cs.tf[0][0];
    const float tn1 = y ? cs.tn[1][1] : cs.tn[1][0], tf1 = y ? cs.tf[1][1] : cs.tf[1][0];
    const float tn2 = z ? cs.tn[2][1] : cs.tn[2][0], tf2 = z ? cs.tf[2][1] : cs.tf[2][0];
    if (tn1 > tn) tn = tn1;
    if (tf1 < tf) tf = tf1;
    if (tn2 > tn) tn = tn2;
    if (tf2 < tf) tf = tf2;
    const float te = tn > 0.0f ? tn : 0.0f;
    if (!(te <= tf)) return false;
    tin = te;
    tout = tf;
    return true;
}

// All 8 children of voxel (i,j,k) at depth dp in one pass: the same values
// and comparisons as child_slabs + child_hit (hence as 8 slab_test calls),
// with the per-axis near/far terms combined pairwise -- the (x, y) pair once
// for both z sides -- in the order child_hit uses (x, then y, then z; a later
// axis replaces the running value only when strictly larger / smaller, so
// even the sign of a zero result is the same).  Returns the hit mask by slot
// and the origin octant (as origin_octant); with WANT_T the hit children's
// (t_enter, t_exit) land in tin / tout by slot.
template <bool WANT_T>
__device__ __forceinline__ uint32_t child_hits8(const RayPrep& r, uint32_t ijk, int dp, uint32_t& oct,
                                                float* tin = nullptr, float* tout = nullptr) {
    const float s = pow2f(1 - dp);
    const float hs = pow2f(-dp);
    const float o[3] = {r.ox, r.oy, r.oz};
    const float inv[3] = {r.ix, r.iy, r.iz};
    const uint32_t c[3] = {unpack_i(ijk), unpack_j(ijk), unpack_k(ijk)};
    float nr[3][2], fr[3][2];
    uint32_t allow = 0xffu;
    oct = 0;
    constexpr uint32_t kSide[3][2] = {{0x55u, 0xaau}, {0x33u, 0xccu}, {0x0fu, 0xf0u}};
    // the planes and crossings of x and y as packed pairs (each lane
    // rounded once, as the scalar operations)
    const float2 lo_xy = __ffma2_rn(make_float2((float)c[0], (float)c[1]), make_float2(s, s), make_float2(-1.0f, -1.0f));
    const float2 mid_xy = __fadd2_rn(lo_xy, make_float2(hs, hs));
    const float2 hi_xy = __fadd2_rn(mid_xy, make_float2(hs, hs));
    const float lo_z = __fmaf_rn((float)c[2], s, -1.0f);
    const float mid_z = __fadd_rn(lo_z, hs);
    const float hi_z = __fadd_rn(mid_z, hs);
    const float2 no_xy = make_float2(-o[0], -o[1]), inv_xy = make_float2(inv[0], inv[1]);
    const float2 tlo_xy = __fmul2_rn(__fadd2_rn(lo_xy, no_xy), inv_xy);
    const float2 tmid_xy = __fmul2_rn(__fadd2_rn(mid_xy, no_xy), inv_xy);
    const float2 thi_xy = __fmul2_rn(__fadd2_rn(hi_xy, no_xy), inv_xy);
    const float2 tlm_z = __fmul2_rn(__fadd2_rn(make_float2(lo_z, mid_z), make_float2(-o[2], -o[2])),
                                    make_float2(inv[2], inv[2]));
    const float thi_z = __fmul_rn(__fsub_rn(hi_z, o[2]), inv[2]);
    const float LO[3] = {lo_xy.x, lo_xy.y, lo_z}, MID[3] = {mid_xy.x, mid_xy.y, mid_z}, HI[3] = {hi_xy.x, hi_xy.y, hi_z};
    const float TLO[3] = {tlo_xy.x, tlo_xy.y, tlm_z.x}, TMID[3] = {tmid_xy.x, tmid_xy.y, tlm_z.y},
                THI[3] = {thi_xy.x, thi_xy.y, thi_z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = LO[a], mid = MID[a], hi = HI[a];
        oct |= (o[a] >= mid) ? (1u << a) : 0u;
        if ((r.par >> a) & 1) {
            allow &= ((lo <= o[a] && o[a] <= mid) ? kSide[a][0] : 0u) | ((mid <= o[a] && o[a] <= hi) ? kSide[a][1] : 0u);
            nr[a][0] = nr[a][1] = -INFINITY;
            fr[a][0] = fr[a][1] = INFINITY;
            continue;
        }
        const float t_lo = TLO[a], t_mid = TMID[a], t_hi = THI[a];
        if (WANT_T) {
            nr[a][0] = t_lo < t_mid ? t_lo : t_mid;
            fr[a][0] = t_lo < t_mid ? t_mid : t_lo;
            nr[a][1] = t_mid < t_hi ? t_mid : t_hi;
            fr[a][1] = t_mid < t_hi ? t_hi : t_mid;
        } else {
            nr[a][0] = fminf(t_lo, t_mid);
            fr[a][0] = fmaxf(t_lo, t_mid);
            nr[a][1] = fminf(t_mid, t_hi);
            fr[a][1] = fmaxf(t_mid, t_hi);
        }
    }
    uint32_t hit = 0;
    if (WANT_T) {
#pragma unroll
        for (int xy = 0; xy < 4; ++xy) {
            const int x = xy & 1, y = xy >> 1;
            float n2 = nr[0][x], f2 = fr[0][x];
            if (nr[1][y] > n2) n2 = nr[1][y];
            if (fr[1][y] < f2) f2 = fr[1][y];
#pragma unroll
            for (int z = 0; z < 2; ++z) {
                float tn = n2, tf = f2;
                if (nr[2][z] > tn) tn = nr[2][z];
                if (fr[2][z] < tf) tf = fr[2][z];
                const float te = tn > 0.0f ? tn : 0.0f;
                const int slot = xy | (z << 2);
                if (te <= tf) hit |= 1u << slot;
                tin[slot] = te;
                tout[slot] = tf;
            }
        }
    } else {
        // only the decision t_enter <= t_exit is needed: fmaxf / fminf give
        // the same values up to the sign of a zero (no operand is NaN: every
        // t is a finite or infinite product of finite factors), which no
        // comparison can see; the 0 of t_enter = max(t_near, 0) joins the z
        // terms
        const float nz0 = fmaxf(nr[2][0], 0.0f), nz1 = fmaxf(nr[2][1], 0.0f);
#pragma unroll
        for (int xy = 0; xy < 4; ++xy) {
            const int x = xy & 1, y = xy >> 1;
            const float n2 = fmaxf(nr[0][x], nr[1][y]), f2 = fminf(fr[0][x], fr[1][y]);
            if (fmaxf(n2, nz0) <= fminf(f2, fr[2][0])) hit |= 1u << xy;
            if (fmaxf(n2, nz1) <= fminf(f2, fr[2][1])) hit |= 1u << (xy | 4);
        }
    }
    return hit & allow;
}

// Child-slot mask re-indexed by front-to-back rank: bit r is set iff slot
// r ^ oct is occupied (an XOR permutation of the 8 bits, by conditional swaps
// of adjacent bits, bit pairs and nibbles).
__device__ __forceinline__ uint32_t rank_mask(uint32_t m, uint32_t oct) {
    if (oct & 1u) m = ((m & 0x55u) << 1) | ((m >> 1) & 0x55u);
    if (oct & 2u) m = ((m & 0x33u) << 2) | ((m >> 2) & 0x33u);
    if (oct & 4u) m = ((m & 0x0fu) << 4) | ((m >> 4) & 0x0fu);
    return m;
}

// Kernel-side error status words (device memory, caller workspace).
enum : int { kStatusOk = 0, kStatusOverflow = 1, kStatusTimeout = 2, kStatusBadIndex = 3 };

}  // namespace nglod
