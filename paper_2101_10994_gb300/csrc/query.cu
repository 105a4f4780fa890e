// sdf_query, sphere_trace (FP32 decode) and the analytic-gradient kernel.
//
// Decoder (Eq. 2) on CUDA cores: one thread per query evaluates the whole
// 35(32) -> 128 -> 1 MLP with the decoder staged once per CTA in shared
// memory; all lanes of a warp read the same weight row, so the loads are
// broadcasts and each 16-byte load feeds four FFMAs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "nglod_internal.cuh"
#include "query_common.cuh"
#include "scan_common.cuh"
#include "trace_common.cuh"

namespace nglod {

int fill_tables(const nglod_svo* svo, const nglod_features* f, int lod, Tables& tb, bool summed_ok) {
    const int D = lod + kFirstFeatureDepth - 1;
    if (!f) return fail(NGLOD_ERR_INVALID_ARG, "NULL features");
    if (f->m != kFeatDim) return fail(NGLOD_ERR_NOT_SUPPORTED, "only m = 32 features are built");
    if (f->dtype != NGLOD_F32 && f->dtype != NGLOD_F16)
        return fail(NGLOD_ERR_NOT_SUPPORTED, "features must be F32 or F16");
    if (f->num_lods < lod) return fail(NGLOD_ERR_INVALID_ARG, "features do not cover the requested LOD");
    if (f->summed_lod != 0) {
        if (!summed_ok)
            return fail(NGLOD_ERR_NOT_SUPPORTED,
                        "a summed corner table only serves sphere_trace (analytic normals) and trace_normals");
        if (f->summed_lod != lod)
            return fail(NGLOD_ERR_INVALID_ARG, "a summed corner table serves only its own LOD");
        if (f->dtype != NGLOD_F32) return fail(NGLOD_ERR_NOT_SUPPORTED, "summed corner tables are F32");
    }
    const int first = f->summed_lod != 0 ? lod : 1;
    tb.first_depth = first + kFirstFeatureDepth - 1;
    for (int l = 0; l < kMaxLods; ++l) tb.feats[l] = nullptr;
    for (int l = first; l <= lod; ++l) {
        if (!f->feats[l - 1]) return fail(NGLOD_ERR_INVALID_ARG, "NULL feature table for a LOD <= lod");
        // FP32 rows are read with 32-byte vector loads, FP16 rows with 16-byte ones
        if ((reinterpret_cast<uintptr_t>(f->feats[l - 1]) & (f->dtype == NGLOD_F32 ? 31u : 15u)) != 0)
            return fail(NGLOD_ERR_INVALID_ARG, "feature tables must be 32-byte (FP32) or 16-byte (FP16) aligned");
        tb.feats[l - 1] = f->feats[l - 1];
    }
    for (int d = 0; d <= kMaxDepth; ++d) {
        const bool ok = d < svo->num_depths && d <= D;
        tb.node[d] = ok ? svo->node[d] : nullptr;
        tb.corners[d] = ok ? svo->corners[d] : nullptr;
        tb.anc[d] = ok ? svo->anc[d] : nullptr;
        tb.cids[d] = ok && d >= kFirstFeatureDepth ? svo->cids[d] : nullptr;
    }
    return NGLOD_OK;
}

int check_decoder(const nglod_decoder* dec) {
    if (!dec) return fail(NGLOD_ERR_INVALID_ARG, "NULL decoder");
    if (dec->hidden != kHidden) return fail(NGLOD_ERR_NOT_SUPPORTED, "only hidden = 128 is built");
    if (dec->in_dim != 32 && dec->in_dim != 35) return fail(NGLOD_ERR_NOT_SUPPORTED, "in_dim must be 32 or 35");
    if (!dec->W1 || !dec->b1 || !dec->W2 || !dec->b2) return fail(NGLOD_ERR_INVALID_ARG, "NULL decoder weights");
    return NGLOD_OK;
}

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// ---------------------------------------------------------------------------
// sdf_query (FP32 decode)
// ---------------------------------------------------------------------------
struct DecPtrs {
    const float* W1;
    const float* b1;
    const float* W2;
    const float* b2;      // one float, read by the kernel at launch time
};

// Finite-difference normals (supplementary Sec. A.4 takes the normals by
// finite differences): at each hit point x = o + t d the SDF is evaluated at
// x + h e_a and x - h e_a (a = 0..2, FP32 coordinates), exactly as sdf_query
// evaluates a point, and n = normalise(d(x + h e_a) - d(x - h e_a))_a.  A
// warp holds 5 hit rays x 6 points in lanes 0..29 (lane 6 i + 2 a + s: ray
// i, axis a, sign s) and forms the normals with shuffles.
struct FDArgs {
    const float* o;
    const float* d;
    const float* t_hit;
    const int* hit_count;     // device: number of entries in hit_list
    const int32_t* hit_list;  // ray ids of the hits
    float h;
    float* normal;            // [R, 3], indexed by ray
};

constexpr int kFDRaysPerWarp = 5;

__device__ __forceinline__ bool fd_point(const FDArgs& F, long long c, int lane, long long nh, float& x0,
                                         float& x1, float& x2, int& ray) {
    const long long i = c * kFDRaysPerWarp + lane / 6;
    if (lane >= 6 * kFDRaysPerWarp || i >= nh) return false;
    ray = F.hit_list[i];
    const float t = F.t_hit[ray];
    x0 = fmaf(t, F.d[3 * ray], F.o[3 * ray]);
    x1 = fmaf(t, F.d[3 * ray + 1], F.o[3 * ray + 1]);
    x2 = fmaf(t, F.d[3 * ray + 2], F.o[3 * ray + 2]);
    const int k = lane % 6;
    const float dh = (k & 1) ? -F.h : F.h;
    if (k < 2) x0 = __fadd_rn(x0, dh);
    else if (k < 4) x1 = __fadd_rn(x1, dh);
    else x2 = __fadd_rn(x2, dh);
    return true;
}

__device__ __forceinline__ void fd_write(const FDArgs& F, int lane, bool act, int ray, float f) {
    const int b = min(lane / 6, kFDRaysPerWarp - 1) * 6;
    float g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        g[a] = __fsub_rn(__shfl_sync(0xffffffffu, f, b + 2 * a), __shfl_sync(0xffffffffu, f, b + 2 * a + 1));
    if (act && lane % 6 == 0) {
        const float nn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const float inv = nn > 0.f ? 1.0f / nn : 0.f;
        F.normal[3 * (size_t)ray] = g[0] * inv;
        F.normal[3 * (size_t)ray + 1] = g[1] * inv;
        F.normal[3 * (size_t)ray + 2] = g[2] * inv;
    }
}

// FD = false: Q points from x.  FD = true: the points of fd_point (Q, x,
// sdf, deepest unused) and the normals of fd_write.
template <typename T, int IN, bool FD>
__global__ void __launch_bounds__(kThreads) k_sdf_query(const DecPtrs dp, const Tables tb,
                                                        const float* __restrict__ x, long long Q, int D,
                                                        float* __restrict__ sdf, int8_t* __restrict__ deepest,
                                                        const FDArgs F) {
    __shared__ __align__(16) float zbuf[kWarps][32 * kZStride];
    __shared__ __align__(16) SmemDecoder sd;
    stage_decoder<IN>(sd, dp.W1, dp.b1, dp.W2);
    __syncthreads();
    const float b2 = __ldg(dp.b2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;
    float* zb = zbuf[warp];
    const long long nh = FD ? (long long)*F.hit_count : 0;
    const long long nchunks = FD ? (nh + kFDRaysPerWarp - 1) / kFDRaysPerWarp : (Q + 31) / 32;
    for (long long c = (long long)blockIdx.x * kWarps + warp; c < nchunks; c += (long long)gridDim.x * kWarps) {
        const long long qi = c * 32 + lane;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        int ray = -1;
        bool act;
        if constexpr (FD) {
            act = fd_point(F, c, lane, nh, x0, x1, x2, ray);
        } else {
            act = qi < Q;
            if (act) {
                x0 = x[3 * qi];
                x1 = x[3 * qi + 1];
                x2 = x[3 * qi + 2];
            }
        }
        int vox;
        uint32_t ijk;
        const int dd = act ? locate_descend(tb, D, x0, x1, x2, vox, ijk) : -1;
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
#pragma unroll 1
        for (int r = 0; r < 4; ++r) {
            const int s = r * 8 + g4;
            const int sdd = __shfl_sync(0xffffffffu, dd, s);
            const int svox = __shfl_sync(0xffffffffu, vox, s);
            const uint32_t sijk = __shfl_sync(0xffffffffu, ijk, s);
            const float s0 = __shfl_sync(0xffffffffu, q0, s);
            const float s1 = __shfl_sync(0xffffffffu, q1, s);
            const float s2 = __shfl_sync(0xffffffffu, q2, s);
            float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zc = za;
            if (sdd >= kFirstFeatureDepth) gather_slot4<T>(tb, sdd, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zc);
            float4* zr = reinterpret_cast<float4*>(zb + s * kZStride + 8 * l4);
            zr[0] = za;
            zr[1] = zc;
        }
        __syncwarp();
        const float out = mlp_f32<IN>(sd, b2, zb + lane * kZStride, x0, x1, x2);
        if constexpr (FD) {
            fd_write(F, lane, act, ray, out);
        } else if (act) {
            sdf[qi] = out;
            if (deepest) deepest[qi] = (int8_t)(dd >= kFirstFeatureDepth ? dd - kFirstFeatureDepth + 1 : 0);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Analytic gradient d sdf / dx (FP32): sdf_query(grad) and trace normals.
//
// d sdf/dx = W1x^T g + J^T W1z^T g with g_h = W2_h [pre_h > 0] and J = dz/dx
// (chain rule through Eq. 2 and the trilinear weights of Sec. 3.2).  Per warp
// of 32 items: (A) without a recorded ReLU mask, 4-lane groups gather z into
// shared memory and each lane runs its item's forward pass for the mask;
// (B) v = sum_h g_h W1[h], either as tensor-core MMAs of the mask matrix
// with the split-BF16 W' below, or per lane in the loop over hidden units
// (each W1 row read once as broadcast 16-byte loads); (C) 4-lane groups apply
// the trilinear derivative weights to v's z part, corner by corner, and
// reduce.  The trace normals run over the ray-ordered list of hit rays the
// tracer recorded.
// ---------------------------------------------------------------------------
// The masked sum v = sum_h W2_h [mask_h] W1[h] of the normals as a product
// of the warp's 32 x 128 mask matrix A (entries 0 or 1, exact in BF16) with
// W' = diag(W2) W1 (128 x 8 NT, the z columns and, for in_dim 35, the x
// columns), W' split into three BF16 terms (w0 + w1 + w2 = W' exactly):
// every product is exact and the sums are FP32, as in the CUDA-core form.
// Warp-level tensor-core MMAs (m16n8k16, FP32 accumulate): the operands
// live in registers, so no block barrier and no shared memory.
// B fragments in the order the MMA wants them: entry ((s * 8 + ks) * NT +
// nt) * 32 + lane holds lane's (b0, b1) for split s, K step ks (hidden units
// 16 ks ..), N tile nt: b0 = (W'_s[k0][n], W'_s[k0 + 1][n]), b1 = the same
// at k0 + 8, with k0 = 16 ks + 2 (lane % 4), n = 8 nt + lane / 4.
constexpr int kFragSplits = 3;
constexpr int kFragKSteps = kHidden / 16;
constexpr int kFragNTMax = 5;                   // in_dim 35: 35 columns in 5 tiles of 8
static_assert(sizeof(uint2) * kFragSplits * kFragKSteps * kFragNTMax * 32 == kWsFragBytes, "workspace region");

// Two mask bits as a pair of BF16 (lower bit in the lower half): 1.0 or 0.
__device__ __forceinline__ uint32_t bits_bf16x2(uint32_t m, int j) {
    return (((m >> j) & 1u) ? 0x3f80u : 0u) | (((m >> (j + 1)) & 1u) ? 0x3f800000u : 0u);
}

struct GradArgs {
    const float* x;        // mode 0: [Q, 3] points
    const float* o;        // mode 1: rays
    const float* d;
    const float* t_hit;
    const int32_t* hit_vox;
    const int* hit_count;  // mode 1: number of entries in hit_list
    const int32_t* hit_list;
    const uint4* hit_mask;  // modes 1, 2: the tracer's ReLU mask per ray (used if *mask_flag)
    const uint2* wfrag;     // with masks: B operand of the masked sum (k_wfrag), in fragment order
    const int* mask_flag;
    long long n;           // mode 0: Q
    int D;
    int mode;              // 0 query gradient, 1 normalised trace normal, 2 out[ray] += w * gradient
    float* out;            // [n, 3] (modes 1, 2: indexed by ray)
    int dcap;              // > 0: only depths 3..dcap enter z (level blending, Eq. 3)
    float w;               // mode 2 weight
};

template <typename T, int IN>
__global__ void __launch_bounds__(kThreads) k_grad(const DecPtrs dp, const Tables tb, const GradArgs A) {
    constexpr int OFF = IN - kFeatDim;
    constexpr int K4 = OFF ? 36 : 32;
    __shared__ __align__(16) float zbuf[kWarps][32 * kZStride];
    __shared__ __align__(16) float gxs[kWarps][32 * 4];
    __shared__ __align__(16) SmemDecoder sd;
    stage_decoder<IN>(sd, dp.W1, dp.b1, dp.W2);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* zb = zbuf[warp];
    float* gb = gxs[warp];
    const long long n = A.mode >= 1 ? (long long)*A.hit_count : A.n;
    const int dcap = A.dcap > 0 ? A.dcap : kMaxDepth;
    // trace normals after a tracer that recorded its hits' ReLU masks: no z
    // gather and no forward pass, v = sum_h W2_h [mask_h] W1[h] directly
    const bool use_mask = A.hit_mask != nullptr && A.wfrag != nullptr &&
                          ((A.mode == 1 && *A.mask_flag == 1) || (A.mode == 2 && *A.mask_flag == 2));
    for (long long base = ((long long)blockIdx.x * kWarps + warp) * 32; base < n;
         base += (long long)gridDim.x * kWarps * 32) {
        const long long it = base + lane;
        const bool act = it < n;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        int dd = -1, vox = -1, ray = -1;
        uint32_t ijk = 0;
        if (act) {
            if (A.mode >= 1) {
                ray = A.hit_list[it];
                const float t = A.t_hit[ray];
                x0 = fmaf(t, A.d[3 * ray], A.o[3 * ray]);
                x1 = fmaf(t, A.d[3 * ray + 1], A.o[3 * ray + 1]);
                x2 = fmaf(t, A.d[3 * ray + 2], A.o[3 * ray + 2]);
                dd = A.D;
                vox = A.hit_vox[ray];
                ijk = tb.node[dd][vox].ijk;
            } else {
                x0 = A.x[3 * it];
                x1 = A.x[3 * it + 1];
                x2 = A.x[3 * it + 2];
                dd = locate_descend(tb, A.D, x0, x1, x2, vox, ijk);
            }
        }
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
        // (A) z of the 32 items (4-lane groups, 8 channels a lane)
        const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
        const unsigned gm4 = 0xfu << gb4;
#pragma unroll 1
        for (int r = 0; r < (use_mask ? 0 : 4); ++r) {
            const int s = r * 8 + g4;
            const int sdd = __shfl_sync(0xffffffffu, dd, s);
            const int svox = __shfl_sync(0xffffffffu, vox, s);
            const uint32_t sijk = __shfl_sync(0xffffffffu, ijk, s);
            const float s0 = __shfl_sync(0xffffffffu, q0, s);
            const float s1 = __shfl_sync(0xffffffffu, q1, s);
            const float s2 = __shfl_sync(0xffffffffu, q2, s);
            float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zc = za;
            if (sdd >= kFirstFeatureDepth)
                gather_slot4<T>(tb, sdd, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zc, dcap);
            float4* zr = reinterpret_cast<float4*>(zb + s * kZStride + 8 * l4);
            zr[0] = za;
            zr[1] = zc;
        }
        __syncwarp();
        // (B) forward pass and v = sum_h W2_h [pre_h > 0] W1[h] for this lane's item
        float v[K4], gv[K4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 a = reinterpret_cast<const float4*>(zb + lane * kZStride)[j];
            v[4 * j] = a.x; v[4 * j + 1] = a.y; v[4 * j + 2] = a.z; v[4 * j + 3] = a.w;
        }
        if constexpr (OFF == 3) {
            v[32] = x0; v[33] = x1; v[34] = x2; v[35] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < K4; ++k) gv[k] = 0.0f;
        // the normals (modes 1, 2) form v by MMAs from the recorded masks, or
        // from the masks of an FP32 forward pass run here for them
        const bool mma_sum = A.wfrag != nullptr && A.mode >= 1;
        if (mma_sum) {
            uint4 mk = make_uint4(0u, 0u, 0u, 0u);
            if (use_mask) {
                if (act) mk = A.hit_mask[ray];
            } else {
                uint32_t m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    uint32_t bits = 0u;
#pragma unroll 2
                    for (int hh = 0; hh < 32; ++hh) {
                        const int h = c * 32 + hh;
                        const float4* w = reinterpret_cast<const float4*>(sd.W1 + h * K4);
                        // the two partial sums as one packed pair (each lane rounded once, as fmaf)
                        float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int j = 0; j < K4 / 4; ++j) {
                            const float4 ww = w[j];
                            a = __ffma2_rn(make_float2(ww.x, ww.y), make_float2(v[4 * j], v[4 * j + 1]), a);
                            a = __ffma2_rn(make_float2(ww.z, ww.w), make_float2(v[4 * j + 2], v[4 * j + 3]), a);
                        }
                        bits |= ((a.x + a.y + sd.bw[h].x) > 0.0f ? 1u : 0u) << hh;
                    }
                    m0 = c == 0 ? bits : m0;
                    m1 = c == 1 ? bits : m1;
                    m2 = c == 2 ? bits : m2;
                    m3 = c == 3 ? bits : m3;
                }
                if (act) mk = make_uint4(m0, m1, m2, m3);
            }
            // v of the warp's 32 items by MMAs (see mma_bf16_16816): item i's
            // mask is lane i's; the accumulators c[mt][nt] hold rows 16 mt +
            // lane / 4 (+ 8) and columns 8 nt + 2 (lane % 4) (+ 1) of v
            constexpr int NT = OFF ? 5 : 4;
            const int g = lane >> 2, cq = 2 * (lane & 3);
            float acc[2][NT][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
#pragma unroll 1
            for (int w = 0; w < 4; ++w) {
                const uint32_t word = w == 0 ? mk.x : w == 1 ? mk.y : w == 2 ? mk.z : mk.w;
                uint32_t m0[2], m1[2];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    m0[mt] = __shfl_sync(0xffffffffu, word, 16 * mt + g);
                    m1[mt] = __shfl_sync(0xffffffffu, word, 16 * mt + g + 8);
                }
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int ks = 2 * w + half, sh = 16 * half;
                    uint2 bf[kFragSplits][NT];
#pragma unroll
                    for (int sp = 0; sp < kFragSplits; ++sp)
#pragma unroll
                        for (int nt = 0; nt < NT; ++nt)
                            bf[sp][nt] = __ldg(A.wfrag + ((sp * kFragKSteps + ks) * NT + nt) * 32 + lane);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        const uint32_t r0 = m0[mt] >> sh, r1 = m1[mt] >> sh;
                        const uint32_t a0 = bits_bf16x2(r0, cq), a1 = bits_bf16x2(r1, cq);
                        const uint32_t a2 = bits_bf16x2(r0, cq + 8), a3 = bits_bf16x2(r1, cq + 8);
#pragma unroll
                        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                            for (int sp = kFragSplits - 1; sp >= 0; --sp)   // smallest terms first
                                mma_bf16_16816(acc[mt][nt], a0, a1, a2, a3, bf[sp][nt]);
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int col = 8 * nt + cq;
                    if (col < kZStride) {
                        *reinterpret_cast<float2*>(zb + (16 * mt + g) * kZStride + col) =
                            make_float2(acc[mt][nt][0], acc[mt][nt][1]);
                        *reinterpret_cast<float2*>(zb + (16 * mt + g + 8) * kZStride + col) =
                            make_float2(acc[mt][nt][2], acc[mt][nt][3]);
                    }
                }
            __syncwarp();
        }
#pragma unroll 1
        for (int h = 0; h < (mma_sum ? 0 : kHidden); ++h) {
            const float4* w = reinterpret_cast<const float4*>(sd.W1 + h * K4);
            // the two partial sums as one packed pair (each lane rounded once, as fmaf)
            float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < K4 / 4; ++j) {
                const float4 ww = w[j];
                a = __ffma2_rn(make_float2(ww.x, ww.y), make_float2(v[4 * j], v[4 * j + 1]), a);
                a = __ffma2_rn(make_float2(ww.z, ww.w), make_float2(v[4 * j + 2], v[4 * j + 3]), a);
            }
            const float2 bw = sd.bw[h];
            const float gh = (a.x + a.y + bw.x) > 0.0f ? bw.y : 0.0f;
#pragma unroll
            for (int j = 0; j < K4 / 4; ++j) {
                const float4 ww = w[j];
                const float2 lo = fma2(gh, make_float2(ww.x, ww.y), make_float2(gv[4 * j], gv[4 * j + 1]));
                const float2 hi = fma2(gh, make_float2(ww.z, ww.w), make_float2(gv[4 * j + 2], gv[4 * j + 3]));
                gv[4 * j] = lo.x;
                gv[4 * j + 1] = lo.y;
                gv[4 * j + 2] = hi.x;
                gv[4 * j + 3] = hi.y;
            }
        }
        if (!mma_sum) {
            __syncwarp();
#pragma unroll
            for (int j = 0; j < K4 / 4; ++j)
                reinterpret_cast<float4*>(zb + lane * kZStride)[j] =
                    make_float4(gv[4 * j], gv[4 * j + 1], gv[4 * j + 2], gv[4 * j + 3]);
            __syncwarp();
        }
        // (C) J^T v_z: the trilinear derivative weights of every level and corner
        // (4-lane groups: lane l4 dots its 8 channels of each corner row with v_z)
#pragma unroll 1
        for (int r = 0; r < 4; ++r) {
            const int s = r * 8 + g4;
            const int sdd = __shfl_sync(0xffffffffu, dd, s);
            const int svox = __shfl_sync(0xffffffffu, vox, s);
            const uint32_t sijk = __shfl_sync(0xffffffffu, ijk, s);
            const float sq[3] = {__shfl_sync(0xffffffffu, q0, s), __shfl_sync(0xffffffffu, q1, s),
                                 __shfl_sync(0xffffffffu, q2, s)};
            float part[3] = {0.f, 0.f, 0.f};
            if (sdd >= kFirstFeatureDepth) {
                const float4 ga = *reinterpret_cast<const float4*>(zb + s * kZStride + 8 * l4);
                const float4 gc = *reinterpret_cast<const float4*>(zb + s * kZStride + 8 * l4 + 4);
                // corner ids from the flat table, the next level's in flight
                const int top2 = min(sdd, dcap);
                const int2* ids = reinterpret_cast<const int2*>(
                                      tb.cids[sdd] + (size_t)svox * (sdd - kFirstFeatureDepth + 1) * 8) + l4;
                int2 cn = tb.first_depth <= top2 ? __ldg(ids + 4 * (tb.first_depth - kFirstFeatureDepth))
                                                 : make_int2(0, 0);
                for (int dp2 = tb.first_depth; dp2 <= top2; ++dp2) {
                    const int i = dp2 - kFirstFeatureDepth;
                    const int2 cc = cn;
                    if (dp2 < top2) cn = __ldg(ids + 4 * (i + 1));
                    const int sh = sdd - dp2;
                    const float sc = pow2f(dp2 - 1);
                    const uint32_t ci[3] = {unpack_i(sijk) >> sh, unpack_j(sijk) >> sh, unpack_k(sijk) >> sh};
                    float u[3];
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa) u[aa] = clamp01(__fsub_rn(__fmul_rn(sq[aa], sc), (float)ci[aa]));
                    const void* fb = tb.feats[i];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float4 ra, rc;
                        FeatLoad8<T>::load(fb, __shfl_sync(gm4, (c & 1) ? cc.y : cc.x, gb4 + (c >> 1)), l4, ra, rc);
                        const float pc = ra.x * ga.x + ra.y * ga.y + ra.z * ga.z + ra.w * ga.w +
                                         rc.x * gc.x + rc.y * gc.y + rc.z * gc.z + rc.w * gc.w;
                        float f[3], df[3];
#pragma unroll
                        for (int aa = 0; aa < 3; ++aa) {
                            const bool up = (c >> aa) & 1;
                            f[aa] = up ? u[aa] : 1.0f - u[aa];
                            df[aa] = up ? sc : -sc;
                        }
                        part[0] = fmaf(df[0] * f[1] * f[2], pc, part[0]);
                        part[1] = fmaf(f[0] * df[1] * f[2], pc, part[1]);
                        part[2] = fmaf(f[0] * f[1] * df[2], pc, part[2]);
                    }
                }
            }
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) {
                part[aa] += __shfl_xor_sync(0xffffffffu, part[aa], 1);
                part[aa] += __shfl_xor_sync(0xffffffffu, part[aa], 2);
            }
            if (l4 == 0) {
                gb[s * 4] = part[0];
                gb[s * 4 + 1] = part[1];
                gb[s * 4 + 2] = part[2];
            }
        }
        __syncwarp();
        if (act) {
            float gx[3] = {gb[lane * 4], gb[lane * 4 + 1], gb[lane * 4 + 2]};
            if constexpr (OFF == 3) {   // the x columns of v (x concatenated in Eq. 2)
                gx[0] += zb[lane * kZStride + 32];
                gx[1] += zb[lane * kZStride + 33];
                gx[2] += zb[lane * kZStride + 34];
            }
            const long long oi = A.mode >= 1 ? (long long)ray : it;
            if (A.mode == 2) {
                A.out[3 * oi] += A.w * gx[0];
                A.out[3 * oi + 1] += A.w * gx[1];
                A.out[3 * oi + 2] += A.w * gx[2];
            } else {
                if (A.mode == 1) {
                    const float nn = sqrtf(gx[0] * gx[0] + gx[1] * gx[1] + gx[2] * gx[2]);
                    const float inv = nn > 0.f ? 1.0f / nn : 0.f;
                    gx[0] *= inv;
                    gx[1] *= inv;
                    gx[2] *= inv;
                }
                A.out[3 * oi] = gx[0];
                A.out[3 * oi + 1] = gx[1];
                A.out[3 * oi + 2] = gx[2];
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Sphere tracing with adaptive stepping, FP32 decode (Sec. 3.4, A.4)
// ---------------------------------------------------------------------------
template <typename T, int IN>
__global__ void __launch_bounds__(kThreads, 2) k_trace_f32(const DecPtrs dp, const Tables tb, const TraceArgs A) {
    __shared__ __align__(16) float zbuf[kWarps][32 * kZStride];
    __shared__ __align__(16) SmemDecoder sd;
    stage_decoder<IN>(sd, dp.W1, dp.b1, dp.W2);
    __syncthreads();
    const float b2 = __ldg(dp.b2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* zb = zbuf[warp];
    RaySlot S;
    S.ray = -1;
    S.hit_ray = -1;
    RayQueue Qu;
    Qu.init();
    for (;;) {
        refill(S, Qu, A, tb, lane);
        if (__ballot_sync(0xffffffffu, S.ray >= 0) == 0u) break;
        const bool act = S.ray >= 0;
        const float x0 = fmaf(S.t, S.dx, S.ox), x1 = fmaf(S.t, S.dy, S.oy), x2 = fmaf(S.t, S.dz, S.oz);
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
        {
            const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
            const unsigned gm4 = 0xfu << gb4;
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {
                const int s = r * 8 + g4;
                const int sact = __shfl_sync(0xffffffffu, act ? 1 : 0, s);
                const int svox = __shfl_sync(0xffffffffu, S.vox, s);
                const uint32_t sijk = __shfl_sync(0xffffffffu, S.ijk, s);
                const float s0 = __shfl_sync(0xffffffffu, q0, s);
                const float s1 = __shfl_sync(0xffffffffu, q1, s);
                const float s2 = __shfl_sync(0xffffffffu, q2, s);
                float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zc = za;
                if (sact) gather_slot4<T>(tb, A.D, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zc);
                float4* zr = reinterpret_cast<float4*>(zb + s * kZStride + 8 * l4);
                zr[0] = za;
                zr[1] = zc;
            }
        }
        prefetch_next_ijk(S, A, tb);
        __syncwarp();
        uint4 mask;
        const float dhat = mlp_f32<IN, true>(sd, b2, zb + lane * kZStride, x0, x1, x2, &mask);
        __syncwarp();
        if (act) step_update(S, dhat, A, tb);
        publish_hits(S, A, lane, mask);
    }
}

DecPtrs dec_ptrs(const nglod_decoder* dec) { return DecPtrs{dec->W1, dec->b1, dec->W2, dec->b2}; }

// Batched tracing, FP32 decode: groups of jobs sharing a decoder, each warp
// drains a group's ray queue independently (no CTA-wide barrier inside a group).
template <typename T, int IN>
__global__ void __launch_bounds__(kThreads, 3) k_trace_batch_f32(const TraceJob* __restrict__ jobs,
                                                                  const JobGroup* __restrict__ groups, int ngroups) {
    __shared__ __align__(16) float zbuf[kWarps][32 * kZStride];
    __shared__ __align__(16) SmemDecoder sd;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;
    float* zb = zbuf[warp];
    for (int gi = 0; gi < ngroups; ++gi) {
        const JobGroup G = groups[gi];
        __syncthreads();
        stage_decoder<IN>(sd, G.W1, G.b1, G.W2);
        __syncthreads();
        const float b2 = __ldg(G.b2);
        RaySlot S;
        S.ray = -1;
        S.hit_ray = -1;
        S.job = G.j0;
        RayQueue Qu;
        Qu.init();
        for (;;) {
            refill_batch(S, Qu, G, jobs, lane);
            if (__ballot_sync(0xffffffffu, S.ray >= 0) == 0u) break;
            const bool act = S.ray >= 0;
            const float x0 = fmaf(S.t, S.dx, S.ox), x1 = fmaf(S.t, S.dy, S.oy), x2 = fmaf(S.t, S.dz, S.oz);
            const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {
                const int s = r * 8 + g4;
                const int sact = __shfl_sync(0xffffffffu, act ? 1 : 0, s);
                const int sjob = __shfl_sync(0xffffffffu, S.job, s);
                const int svox = __shfl_sync(0xffffffffu, S.vox, s);
                const uint32_t sijk = __shfl_sync(0xffffffffu, S.ijk, s);
                const float s0 = __shfl_sync(0xffffffffu, q0, s);
                const float s1 = __shfl_sync(0xffffffffu, q1, s);
                const float s2 = __shfl_sync(0xffffffffu, q2, s);
                float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zc = za;
                if (sact)
                    gather_slot4<T>(jobs[sjob].tb, jobs[sjob].A.D, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zc);
                float4* zr = reinterpret_cast<float4*>(zb + s * kZStride + 8 * l4);
                zr[0] = za;
                zr[1] = zc;
            }
            if (S.ray >= 0) prefetch_next_ijk(S, jobs[S.job].A, jobs[S.job].tb);
            __syncwarp();
            uint4 mask;
            const float dhat = mlp_f32<IN, true>(sd, b2, zb + lane * kZStride, x0, x1, x2, &mask);
            __syncwarp();
            if (act) step_update(S, dhat, jobs[S.job].A, jobs[S.job].tb);
            publish_hits_batch(S, jobs, mask);
        }
    }
}

template <typename T, int IN>
void launch_trace_f32(const DecPtrs& P, const Tables& tb, const TraceArgs& A, int grid, cudaStream_t st) {
    k_trace_f32<T, IN><<<grid, kThreads, 0, st>>>(P, tb, A);
}

template <typename T, int IN>
void launch_query(const DecPtrs& P, const Tables& tb, const float* x, long long Q, int D, float* sdf,
                  int8_t* deepest, int grid, cudaStream_t st) {
    k_sdf_query<T, IN, false><<<grid, kThreads, 0, st>>>(P, tb, x, Q, D, sdf, deepest, FDArgs{});
}

template <typename T, int IN>
void launch_fd(const DecPtrs& P, const Tables& tb, int D, const FDArgs& F, int grid, cudaStream_t st) {
    k_sdf_query<T, IN, true><<<grid, kThreads, 0, st>>>(P, tb, nullptr, 0, D, nullptr, nullptr, F);
}

template <typename T, int IN>
void launch_grad(const nglod_decoder* dec, const Tables& tb, const GradArgs& A, int grid, cudaStream_t st) {
    k_grad<T, IN><<<grid, kThreads, 0, st>>>(dec_ptrs(dec), tb, A);
}

int grid_items(long long n, int per_cta, int sms, int ctas_per_sm) {
    const long long g = (n + per_cta - 1) / per_cta;
    return (int)std::max<long long>(1, std::min<long long>(g, (long long)sms * ctas_per_sm));
}

int run_grad(const nglod_decoder* dec, const Tables& tb, const GradArgs& A, bool f16, int sms,
             cudaStream_t st) {
    const int grid = grid_items(A.n, kThreads, sms, 2);
    if (dec->in_dim == 35) {
        if (f16) launch_grad<__half, 35>(dec, tb, A, grid, st); else launch_grad<float, 35>(dec, tb, A, grid, st);
    } else {
        if (f16) launch_grad<__half, 32>(dec, tb, A, grid, st); else launch_grad<float, 32>(dec, tb, A, grid, st);
    }
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

// ---------------------------------------------------------------------------
// Level blending (Sec. 3.2, Eq. 3), FP32 decode.  The slots' z over depths
// 3..D-1 is decoded with LOD L*'s decoder; then the depth-D level is added
// to the staged rows and decoded with LOD L*+1's; the result is
// (1 - alpha) d_lo + alpha d_hi.  Two staged decoders do not fit beside the
// z rows in static shared memory, so both live in dynamic shared memory.
// ---------------------------------------------------------------------------
constexpr size_t kBlendF32Smem = 2 * sizeof(SmemDecoder) + sizeof(float) * kWarps * 32 * kZStride;

template <typename T, int IN>
__global__ void __launch_bounds__(kThreads, 2) k_trace_blend_f32(const DecPtrs lo, const DecPtrs hi, float alpha,
                                                                  const Tables tb, const TraceArgs A) {
    extern __shared__ __align__(16) unsigned char blend_smem[];
    SmemDecoder& slo = *reinterpret_cast<SmemDecoder*>(blend_smem);
    SmemDecoder& shi = *reinterpret_cast<SmemDecoder*>(blend_smem + sizeof(SmemDecoder));
    stage_decoder<IN>(slo, lo.W1, lo.b1, lo.W2);
    stage_decoder<IN>(shi, hi.W1, hi.b1, hi.W2);
    __syncthreads();
    const float b2lo = __ldg(lo.b2), b2hi = __ldg(hi.b2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;
    float* zb = reinterpret_cast<float*>(blend_smem + 2 * sizeof(SmemDecoder)) + warp * 32 * kZStride;
    RaySlot S;
    S.ray = -1;
    S.hit_ray = -1;
    RayQueue Qu;
    Qu.init();
    for (;;) {
        refill(S, Qu, A, tb, lane);
        if (__ballot_sync(0xffffffffu, S.ray >= 0) == 0u) break;
        const bool act = S.ray >= 0;
        const float x0 = fmaf(S.t, S.dx, S.ox), x1 = fmaf(S.t, S.dy, S.oy), x2 = fmaf(S.t, S.dz, S.oz);
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
        float dlo = 0.0f, dhi = 0.0f;
        uint4 mlo = make_uint4(0u, 0u, 0u, 0u), mhi = mlo;
        prefetch_next_ijk(S, A, tb);
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            // pass 0: depths 3..D-1 into the rows; pass 1: add depth D
            const int d0 = pass ? A.D : kFirstFeatureDepth, d1 = pass ? A.D : A.D - 1;
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {
                const int s = r * 8 + g4;
                const int sact = __shfl_sync(0xffffffffu, act ? 1 : 0, s);
                const int svox = __shfl_sync(0xffffffffu, S.vox, s);
                const uint32_t sijk = __shfl_sync(0xffffffffu, S.ijk, s);
                const float s0 = __shfl_sync(0xffffffffu, q0, s);
                const float s1 = __shfl_sync(0xffffffffu, q1, s);
                const float s2 = __shfl_sync(0xffffffffu, q2, s);
                float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zc = za;
                if (sact) gather_slot4<T>(tb, A.D, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zc, d1, d0);
                float4* row = reinterpret_cast<float4*>(zb + s * kZStride + 8 * l4);
                if (pass) {
                    const float4 p = row[0], q = row[1];
                    za = make_float4(p.x + za.x, p.y + za.y, p.z + za.z, p.w + za.w);
                    zc = make_float4(q.x + zc.x, q.y + zc.y, q.z + zc.z, q.w + zc.w);
                }
                row[0] = za;
                row[1] = zc;
            }
            __syncwarp();
            uint4 mk;
            const float dv = mlp_f32<IN, true>(pass ? shi : slo, pass ? b2hi : b2lo, zb + lane * kZStride, x0,
                                               x1, x2, &mk);
            if (pass) {
                dhi = dv;
                mhi = mk;
            } else {
                dlo = dv;
                mlo = mk;
            }
            __syncwarp();
        }
        const float dhat = fmaf(alpha, dhi - dlo, dlo);
        if (act) step_update(S, dhat, A, tb);
        publish_hits(S, A, lane, mlo, mhi);
    }
}

template <typename T, int IN, bool FD>
__global__ void __launch_bounds__(kThreads, 2) k_query_blend_f32(const DecPtrs lo, const DecPtrs hi, float alpha,
                                                                  const Tables tb, const float* __restrict__ x,
                                                                  long long Q, int D, float* __restrict__ sdf,
                                                                  const FDArgs F) {
    extern __shared__ __align__(16) unsigned char blend_smem[];
    SmemDecoder& slo = *reinterpret_cast<SmemDecoder*>(blend_smem);
    SmemDecoder& shi = *reinterpret_cast<SmemDecoder*>(blend_smem + sizeof(SmemDecoder));
    stage_decoder<IN>(slo, lo.W1, lo.b1, lo.W2);
    stage_decoder<IN>(shi, hi.W1, hi.b1, hi.W2);
    __syncthreads();
    const float b2lo = __ldg(lo.b2), b2hi = __ldg(hi.b2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;
    float* zb = reinterpret_cast<float*>(blend_smem + 2 * sizeof(SmemDecoder)) + warp * 32 * kZStride;
    const long long nh = FD ? (long long)*F.hit_count : 0;
    const long long nchunks = FD ? (nh + kFDRaysPerWarp - 1) / kFDRaysPerWarp : (Q + 31) / 32;
    for (long long c = (long long)blockIdx.x * kWarps + warp; c < nchunks; c += (long long)gridDim.x * kWarps) {
        const long long qi = c * 32 + lane;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        int ray = -1;
        bool act;
        if constexpr (FD) {
            act = fd_point(F, c, lane, nh, x0, x1, x2, ray);
        } else {
            act = qi < Q;
            if (act) {
                x0 = x[3 * qi];
                x1 = x[3 * qi + 1];
                x2 = x[3 * qi + 2];
            }
        }
        int vox;
        uint32_t ijk;
        const int dd = act ? locate_descend(tb, D, x0, x1, x2, vox, ijk) : -1;
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
        float dlo = 0.0f, dhi = 0.0f;
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {
                const int s = r * 8 + g4;
                const int sdd = __shfl_sync(0xffffffffu, dd, s);
                const int svox = __shfl_sync(0xffffffffu, vox, s);
                const uint32_t sijk = __shfl_sync(0xffffffffu, ijk, s);
                const float s0 = __shfl_sync(0xffffffffu, q0, s);
                const float s1 = __shfl_sync(0xffffffffu, q1, s);
                const float s2 = __shfl_sync(0xffffffffu, q2, s);
                float4* row = reinterpret_cast<float4*>(zb + s * kZStride + 8 * l4);
                if (pass == 0) {
                    float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zc = za;
                    if (sdd >= kFirstFeatureDepth)
                        gather_slot4<T>(tb, sdd, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zc, D - 1);
                    row[0] = za;
                    row[1] = zc;
                } else if (sdd == D) {
                    // the depth-D level exists only where x's depth-D voxel does
                    float4 za, zc;
                    gather_slot4<T>(tb, sdd, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zc, D, D);
                    const float4 p = row[0], q = row[1];
                    row[0] = make_float4(p.x + za.x, p.y + za.y, p.z + za.z, p.w + za.w);
                    row[1] = make_float4(q.x + zc.x, q.y + zc.y, q.z + zc.z, q.w + zc.w);
                }
            }
            __syncwarp();
            const float dv = mlp_f32<IN>(pass ? shi : slo, pass ? b2hi : b2lo, zb + lane * kZStride, x0, x1, x2);
            if (pass) dhi = dv;
            else dlo = dv;
            __syncwarp();
        }
        const float db = fmaf(alpha, dhi - dlo, dlo);
        if constexpr (FD) fd_write(F, lane, act, ray, db);
        else if (act) sdf[qi] = db;
    }
}

template <typename K>
void allow_blend_smem(K kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlendF32Smem);
}

template <typename T, int IN>
void go_blend_f32(bool trace, const DecPtrs& lo, const DecPtrs& hi, float alpha, const Tables& tb,
                  const TraceArgs* A, const float* x, long long Q, int D, float* sdf, const FDArgs* F, int grid,
                  cudaStream_t st) {
    if (trace) {
        static std::atomic<unsigned long long> done{0};
        once_per_device(done, [] { allow_blend_smem(k_trace_blend_f32<T, IN>); });
        k_trace_blend_f32<T, IN><<<grid, kThreads, kBlendF32Smem, st>>>(lo, hi, alpha, tb, *A);
    } else if (F) {
        static std::atomic<unsigned long long> done{0};
        once_per_device(done, [] { allow_blend_smem(k_query_blend_f32<T, IN, true>); });
        k_query_blend_f32<T, IN, true><<<grid, kThreads, kBlendF32Smem, st>>>(lo, hi, alpha, tb, nullptr, 0, D,
                                                                                nullptr, *F);
    } else {
        static std::atomic<unsigned long long> done{0};
        once_per_device(done, [] { allow_blend_smem(k_query_blend_f32<T, IN, false>); });
        k_query_blend_f32<T, IN, false><<<grid, kThreads, kBlendF32Smem, st>>>(lo, hi, alpha, tb, x, Q, D, sdf,
                                                                                 FDArgs{});
    }
}

void go_blend_f32_any(bool trace, int in_dim, bool f16, const DecPtrs& lo, const DecPtrs& hi, float alpha,
                      const Tables& tb, const TraceArgs* A, const float* x, long long Q, int D, float* sdf,
                      int grid, cudaStream_t st, const FDArgs* F = nullptr) {
    if (in_dim == 35) {
        if (f16) go_blend_f32<__half, 35>(trace, lo, hi, alpha, tb, A, x, Q, D, sdf, F, grid, st);
        else go_blend_f32<float, 35>(trace, lo, hi, alpha, tb, A, x, Q, D, sdf, F, grid, st);
    } else {
        if (f16) go_blend_f32<__half, 32>(trace, lo, hi, alpha, tb, A, x, Q, D, sdf, F, grid, st);
        else go_blend_f32<float, 32>(trace, lo, hi, alpha, tb, A, x, Q, D, sdf, F, grid, st);
    }
}

FDArgs fd_args(const TraceArgs& A, float h, float* normal) {
    FDArgs F;
    F.o = A.o;
    F.d = A.d;
    F.t_hit = A.t_hit;
    F.hit_count = A.hit_count;
    F.hit_list = A.hit_list;
    F.h = h;
    F.normal = normal;
    return F;
}

// Normalises the accumulated blended gradients of the hit rays.
__global__ void k_normalise_hits(const int* __restrict__ hit_count, const int32_t* __restrict__ hit_list,
                                 float* __restrict__ normal) {
    const long long n = *hit_count;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float* v = normal + 3 * (size_t)hit_list[i];
        const float nn = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const float inv = nn > 0.f ? 1.0f / nn : 0.f;
        v[0] *= inv;
        v[1] *= inv;
        v[2] *= inv;
    }
}

// B fragments of W' = diag(W2) W1 for the normals' masked sum (layout at
// mma_bf16_16816): one thread per (split, K step, N tile, lane) entry.
__device__ __forceinline__ float wprime(const float* __restrict__ W1, const float* __restrict__ W2, int in_dim, int h,
                                        int n) {
    const int off = in_dim - kFeatDim;
    if (n < kFeatDim) return W2[h] * W1[h * in_dim + off + n];
    if (n < kFeatDim + off) return W2[h] * W1[h * in_dim + (n - kFeatDim)];
    return 0.0f;
}

// Term sp of the three-term BF16 split of v (v = t0 + t1 + t2; each
// difference exact in FP32), as raw bits.
__device__ __forceinline__ uint32_t split_bits(float v, int sp) {
    const __nv_bfloat16 t0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(t0);
    const __nv_bfloat16 t1 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 t2 = __float2bfloat16_rn(r1 - __bfloat162float(t1));
    const __nv_bfloat16 t = sp == 0 ? t0 : sp == 1 ? t1 : t2;
    return (uint32_t)*reinterpret_cast<const unsigned short*>(&t);
}

__global__ void k_wfrag(const float* __restrict__ W1, const float* __restrict__ W2, int in_dim,
                        uint2* __restrict__ out) {
    const int NT = in_dim == 35 ? 5 : 4;
    const int total = kFragSplits * kFragKSteps * NT * 32;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int lane = e & 31, rest = e >> 5;
        const int nt = rest % NT, ks = (rest / NT) % kFragKSteps, sp = rest / (NT * kFragKSteps);
        const int n = 8 * nt + (lane >> 2), k0 = 16 * ks + 2 * (lane & 3);
        const uint32_t b0 = split_bits(wprime(W1, W2, in_dim, k0, n), sp) |
                            (split_bits(wprime(W1, W2, in_dim, k0 + 1, n), sp) << 16);
        const uint32_t b1 = split_bits(wprime(W1, W2, in_dim, k0 + 8, n), sp) |
                            (split_bits(wprime(W1, W2, in_dim, k0 + 9, n), sp) << 16);
        out[e] = make_uint2(b0, b1);
    }
}

// The masked-sum operand of decoder dec for the normals of a trace whose
// workspace holds one.
int enqueue_wfrag(const nglod_decoder* dec, const TraceArgs& A, cudaStream_t st) {
    if (!A.wfrag) return NGLOD_OK;
    k_wfrag<<<(kFragSplits * kFragKSteps * kFragNTMax * 32 + 255) / 256, 256, 0, st>>>(
        static_cast<const float*>(dec->W1), static_cast<const float*>(dec->W2), dec->in_dim, A.wfrag);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

}  // namespace

int launch_trace_fp32(const nglod_decoder* dec, const Tables& tb, const TraceArgs& A, bool f16, int sms,
                      cudaStream_t st) {
    const int grid = sms * (A.ctas_per_sm > 0 ? std::min(A.ctas_per_sm, 2) : 2);
    const DecPtrs P = dec_ptrs(dec);
    if (dec->in_dim == 35) {
        if (f16) launch_trace_f32<__half, 35>(P, tb, A, grid, st); else launch_trace_f32<float, 35>(P, tb, A, grid, st);
    } else {
        if (f16) launch_trace_f32<__half, 32>(P, tb, A, grid, st); else launch_trace_f32<float, 32>(P, tb, A, grid, st);
    }
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

int launch_trace_batch_f32(const TraceJob* jobs, const JobGroup* groups, int ngroups, int in_dim, bool f16,
                           int ctas_per_sm, int sms, cudaStream_t st) {
    const int grid = sms * std::max(1, std::min(ctas_per_sm > 0 ? ctas_per_sm : 3, 3));
    if (in_dim == 35) {
        if (f16) k_trace_batch_f32<__half, 35><<<grid, kThreads, 0, st>>>(jobs, groups, ngroups);
        else k_trace_batch_f32<float, 35><<<grid, kThreads, 0, st>>>(jobs, groups, ngroups);
    } else {
        if (f16) k_trace_batch_f32<__half, 32><<<grid, kThreads, 0, st>>>(jobs, groups, ngroups);
        else k_trace_batch_f32<float, 32><<<grid, kThreads, 0, st>>>(jobs, groups, ngroups);
    }
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

int launch_normals(const nglod_decoder* dec, const Tables& tb, const TraceArgs& A, float* normal, bool f16,
                   int sms, cudaStream_t st) {
    // misses get zero normals; the kernel writes the hits from the hit list
    NGLOD_CUDA(cudaMemsetAsync(normal, 0, sizeof(float) * 3 * (size_t)A.R, st));
    GradArgs G{};
    G.o = A.o;
    G.d = A.d;
    G.t_hit = A.t_hit;
    G.hit_vox = A.hit_vox;
    G.hit_count = A.hit_count;
    G.hit_list = A.hit_list;
    G.hit_mask = A.hit_mask;
    G.wfrag = A.wfrag;
    G.mask_flag = A.hit_count + (kWsMaskFlagWord - 2);
    G.n = A.R;
    G.D = A.D;
    G.mode = 1;
    G.out = normal;
    if (int rc = enqueue_wfrag(dec, A, st)) return rc;
    return run_grad(dec, tb, G, f16, sms, st);
}

int check_normal_params(const nglod_trace_params* params, const char* who) {
    if (params->normal_mode != NGLOD_NORMALS_ANALYTIC && params->normal_mode != NGLOD_NORMALS_FD)
        return fail(NGLOD_ERR_INVALID_ARG, std::string(who) + ": normal_mode must be ANALYTIC or FD");
    if (params->normal_mode == NGLOD_NORMALS_FD && !(params->fd_h > 0.0f && params->fd_h < 1.0f))
        return fail(NGLOD_ERR_INVALID_ARG, std::string(who) + ": fd_h must lie in (0, 1)");
    return NGLOD_OK;
}

int launch_normals_fd(const nglod_decoder* dec, const Tables& tb, const TraceArgs& A, float h, float* normal,
                      bool f16, int sms, cudaStream_t st) {
    NGLOD_CUDA(cudaMemsetAsync(normal, 0, sizeof(float) * 3 * (size_t)A.R, st));
    const FDArgs F = fd_args(A, h, normal);
    const int grid = grid_items((A.R + kFDRaysPerWarp - 1) / kFDRaysPerWarp * 32, kThreads, sms, 2);
    const DecPtrs P = dec_ptrs(dec);
    if (dec->in_dim == 35) {
        if (f16) launch_fd<__half, 35>(P, tb, A.D, F, grid, st); else launch_fd<float, 35>(P, tb, A.D, F, grid, st);
    } else {
        if (f16) launch_fd<__half, 32>(P, tb, A.D, F, grid, st); else launch_fd<float, 32>(P, tb, A.D, F, grid, st);
    }
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

int launch_normals_blend_fd(const nglod_decoder* lo, const nglod_decoder* hi, float alpha, const Tables& tb,
                            const TraceArgs& A, float h, float* normal, bool f16, int sms, cudaStream_t st) {
    NGLOD_CUDA(cudaMemsetAsync(normal, 0, sizeof(float) * 3 * (size_t)A.R, st));
    const FDArgs F = fd_args(A, h, normal);
    go_blend_f32_any(false, lo->in_dim, f16, dec_ptrs(lo), dec_ptrs(hi), alpha, tb, nullptr, nullptr, 0, A.D,
                     nullptr, grid_items((A.R + kFDRaysPerWarp - 1) / kFDRaysPerWarp * 32, kThreads, sms, 2), st, &F);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

int launch_trace_blend_f32(const nglod_decoder* lo, const nglod_decoder* hi, float alpha, const Tables& tb,
                           const TraceArgs& A, bool f16, int sms, cudaStream_t st) {
    go_blend_f32_any(true, lo->in_dim, f16, dec_ptrs(lo), dec_ptrs(hi), alpha, tb, &A, nullptr, 0, A.D, nullptr,
                     sms * (A.ctas_per_sm > 0 ? std::min(A.ctas_per_sm, 2) : 2), st);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

int launch_query_blend_f32(const nglod_decoder* lo, const nglod_decoder* hi, float alpha, const Tables& tb,
                           const float* x, long long Q, int D, float* sdf, bool f16, int sms, cudaStream_t st) {
    go_blend_f32_any(false, lo->in_dim, f16, dec_ptrs(lo), dec_ptrs(hi), alpha, tb, nullptr, x, Q, D, sdf,
                     grid_items(Q, kThreads, sms, 2), st);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

// Normals of the blended field: the normalised (1 - alpha) grad d_lo +
// alpha grad d_hi at each hit point (d_lo over depths 3..D-1 of the hit
// voxel's ancestors, d_hi over 3..D).
int launch_normals_blend(const nglod_decoder* lo, const nglod_decoder* hi, float alpha, const Tables& tb,
                         const TraceArgs& A, float* normal, bool f16, int sms, cudaStream_t st) {
    NGLOD_CUDA(cudaMemsetAsync(normal, 0, sizeof(float) * 3 * (size_t)A.R, st));
    GradArgs G{};
    G.o = A.o;
    G.d = A.d;
    G.t_hit = A.t_hit;
    G.hit_vox = A.hit_vox;
    G.hit_count = A.hit_count;
    G.hit_list = A.hit_list;
    G.n = A.R;
    G.D = A.D;
    G.mode = 2;
    G.out = normal;
    G.dcap = A.D - 1;
    G.w = 1.0f - alpha;
    G.hit_mask = A.hit_mask;                 // the lower LOD's masks, if the trace recorded them
    G.wfrag = A.wfrag;
    G.mask_flag = A.hit_count + (kWsMaskFlagWord - 2);
    int rc = enqueue_wfrag(lo, A, st);
    if (rc || (rc = run_grad(lo, tb, G, f16, sms, st))) return rc;
    G.dcap = A.D;
    G.w = alpha;
    G.hit_mask = A.hit_mask2;
    if ((rc = enqueue_wfrag(hi, A, st)) || (rc = run_grad(hi, tb, G, f16, sms, st))) return rc;
    k_normalise_hits<<<std::max(1, (int)std::min<long long>((A.R + 255) / 256, (long long)sms * 8)), 256, 0, st>>>(
        A.hit_count, A.hit_list, normal);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

}  // namespace nglod

using namespace nglod;

extern "C" int sdf_query(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* dec,
                         const float* x, int64_t Q, int lod, int decode_dtype, float* sdf, int8_t* deepest,
                         float* grad, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!svo) return fail(NGLOD_ERR_INVALID_ARG, "sdf_query: NULL octree");
    const int D = lod + kFirstFeatureDepth - 1;
    if (lod < 1 || D >= svo->num_depths) return fail(NGLOD_ERR_INVALID_ARG, "sdf_query: lod out of range");
    if (Q < 0) return fail(NGLOD_ERR_INVALID_ARG, "sdf_query: Q < 0");
    if (Q == 0) return NGLOD_OK;
    if (!x || !sdf) return fail(NGLOD_ERR_INVALID_ARG, "sdf_query: NULL x or sdf");
    Tables tb;
    int rc = fill_tables(svo, feats, lod, tb);
    if (rc) return rc;
    const bool f16 = feats->dtype == NGLOD_F16;
    if (decode_dtype == NGLOD_BF16 || decode_dtype == NGLOD_FP8E4M3 || decode_dtype == NGLOD_F32_SPLIT) {
        rc = check_decoder(dec);
        if (rc) return rc;
        if (grad) return fail(NGLOD_ERR_NOT_SUPPORTED, "sdf_query: grad needs the FP32 decode");
        const bool fp8 = decode_dtype == NGLOD_FP8E4M3;
        if (fp8 && !(feats->fp8_z_absmax > 0.0f))
            return fail(NGLOD_ERR_INVALID_ARG, "sdf_query: the FP8 decode needs feats->fp8_z_absmax > 0");
        rc = launch_query_bf16(svo, tb, dec, x, Q, D, sdf, deepest, f16, fp8 ? feats->fp8_z_absmax : 0.0f, st,
                               decode_dtype == NGLOD_F32_SPLIT);
        if (rc) return rc;
        return NGLOD_OK;
    }
    if (decode_dtype != NGLOD_F32) return fail(NGLOD_ERR_NOT_SUPPORTED, "sdf_query: decode_dtype");
    rc = check_decoder(dec);
    if (rc) return rc;
    const DecPtrs P = dec_ptrs(dec);
    const int grid = grid_items(Q, kThreads, svo->num_sms, 4);
    if (dec->in_dim == 35) {
        if (f16) launch_query<__half, 35>(P, tb, x, Q, D, sdf, deepest, grid, st);
        else launch_query<float, 35>(P, tb, x, Q, D, sdf, deepest, grid, st);
    } else {
        if (f16) launch_query<__half, 32>(P, tb, x, Q, D, sdf, deepest, grid, st);
        else launch_query<float, 32>(P, tb, x, Q, D, sdf, deepest, grid, st);
    }
    NGLOD_CUDA(cudaGetLastError());
    if (grad) {
        GradArgs G{};
        G.x = x;
        G.n = Q;
        G.D = D;
        G.mode = 0;
        G.out = grad;
        rc = run_grad(dec, tb, G, f16, svo->num_sms, st);
        if (rc) return rc;
    }
    return NGLOD_OK;
}

namespace nglod {
namespace {

// Ray-group handout order of the persistent tracers.  Rays are taken from the
// queue 32 at a time; a group whose longest voxel list is long tends to
// hold a slot for many steps, and started last it leaves the frame with a
// tail of nearly empty tiles.  The groups are therefore handed out by
// decreasing longest-list length (a counting sort over kOrderBuckets
// lengths, clamped), which changes only the schedule: every ray's outputs
// are those of the index-order trace.
// Also writes each ray's first list entry (t_enter, t_exit, voxel, packed
// ijk; the interval by the traversal's slab test at depth D) to start[r], so
// the tracer starts a ray with independent loads only.
__global__ void k_group_keys(const int32_t* __restrict__ offs, const int32_t* __restrict__ cnt, long long R,
                             uint8_t* __restrict__ key,
                             int* __restrict__ hist, const float* __restrict__ o, const float* __restrict__ d,
                             const int32_t* __restrict__ vid, const Node* __restrict__ node_D, int D,
                             int4* __restrict__ start) {
    __shared__ int h[kOrderBuckets];
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long G = (R + 31) / 32;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long g = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < G; g += nw) {
        const long long r = g * 32 + lane;
        const int c0 = r < R ? offs[r] : 0;
        const int len = r < R ? (cnt ? cnt[r] : offs[r + 1] - c0) : 0;
        if (len > 0) {
            const int v = vid[c0];
            const uint32_t ijk = node_D[v].ijk;
            float tin, tout;
            voxel_interval(o[3 * r], o[3 * r + 1], o[3 * r + 2], d[3 * r], d[3 * r + 1], d[3 * r + 2], ijk, D, tin,
                           tout);
            start[r] = make_int4(__float_as_int(tin), __float_as_int(tout), v, (int)ijk);
        }
        const int m = __reduce_max_sync(0xffffffffu, len);
        if (lane == 0) {
            const int b = kOrderBuckets - 1 - min(max(m, 0), kOrderBuckets - 1);   // longest first
            key[g] = (uint8_t)b;
            atomicAdd(&h[b], 1);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// cursor[b] = sum of hist[0..b) (one block of kOrderBuckets threads per
// histogram; block i scans histogram i).
__global__ void k_order_scan(const int* __restrict__ hist, int* __restrict__ cursor) {
    __shared__ int ws[33];
    int total;
    const int i = blockIdx.x * kOrderBuckets + threadIdx.x;
    cursor[i] = block_exclusive_sum(hist[i], ws, total);
}

// Places every group at its bucket's cursor; lanes of a warp with the same
// key share one atomic (most groups fall in a few buckets).
__global__ void k_order_scatter(const uint8_t* __restrict__ key, long long G, int* __restrict__ cursor,
                                int32_t* __restrict__ order) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); g0 < G; g0 += stride) {
        const long long g = g0 + lane;
        const bool act = g < G;
        const unsigned live = __ballot_sync(0xffffffffu, act);
        if (!act) continue;
        const int k = key[g];
        const unsigned peers = __match_any_sync(live, k);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&cursor[k], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        order[base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)g;
    }
}

}  // namespace

int enable_hit_masks(TraceArgs& A, void* work, cudaStream_t st, bool two) {
    A.hit_mask = reinterpret_cast<uint4*>(static_cast<char*>(work) + trace_ws_mask_offset(A.R));
    A.hit_mask2 = two ? A.hit_mask + A.R : nullptr;
    NGLOD_CUDA(cudaMemsetAsync(static_cast<int*>(work) + kWsMaskFlagWord, two ? 2 : 1, 1, st));
    return NGLOD_OK;
}

namespace {

// Hit list in ray order: blocks of kHitBlock rays, 16 consecutive rays a
// thread; k_hit_counts counts each block's hits, k_hit_scan turns the
// counts into block offsets, k_hit_place writes the hit rays' ids.
constexpr int kHitThreads = 256;
constexpr int kHitPerThread = 16;
constexpr long long kHitBlock = (long long)kHitThreads * kHitPerThread;

// Bit j of the result is set iff ray r0 + j (< R) hit; one 16-byte load
// where the 16 flags are aligned and in range.
__device__ __forceinline__ uint32_t thread_hit_bits(const uint8_t* __restrict__ hit, long long R, long long r0) {
    uint32_t bits = 0u;
    if (r0 + kHitPerThread <= R && ((reinterpret_cast<uintptr_t>(hit + r0) & 15u) == 0)) {
        const uint4 v = *reinterpret_cast<const uint4*>(hit + r0);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int b = 0; b < 4; ++b) bits |= (((w[q] >> (8 * b)) & 0xffu) ? 1u : 0u) << (4 * q + b);
    } else {
#pragma unroll
        for (int j = 0; j < kHitPerThread; ++j) bits |= (r0 + j < R && hit[r0 + j]) ? (1u << j) : 0u;
    }
    return bits;
}

__global__ void __launch_bounds__(kHitThreads) k_hit_counts(const uint8_t* __restrict__ hit, long long R,
                                                            int* __restrict__ cnt) {
    __shared__ int ws[33];
    const long long r0 = (long long)blockIdx.x * kHitBlock + (long long)threadIdx.x * kHitPerThread;
    int total;
    block_exclusive_sum(__popc(thread_hit_bits(hit, R, r0)), ws, total);
    if (threadIdx.x == 0) cnt[blockIdx.x] = total;
}

// Exclusive prefix of the n block counts, in place (one block).
__global__ void __launch_bounds__(1024) k_hit_scan(int* __restrict__ cnt, long long n) {
    __shared__ int ws[33];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < n; b0 += blockDim.x) {
        const long long i = b0 + threadIdx.x;
        const int v = i < n ? cnt[i] : 0;
        int total;
        const int e = block_exclusive_sum(v, ws, total);
        if (i < n) cnt[i] = carry + e;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kHitThreads) k_hit_place(const uint8_t* __restrict__ hit, long long R,
                                                           const int* __restrict__ off, int32_t* __restrict__ list) {
    __shared__ int ws[33];
    const long long r0 = (long long)blockIdx.x * kHitBlock + (long long)threadIdx.x * kHitPerThread;
    int total;
    uint32_t bits = thread_hit_bits(hit, R, r0);
    int pos = off[blockIdx.x] + block_exclusive_sum(__popc(bits), ws, total);
    for (; bits; bits &= bits - 1u) list[pos++] = (int32_t)(r0 + __ffs(bits) - 1);
}

}  // namespace

int enqueue_hit_order(const TraceArgs& A, void* work, cudaStream_t st) {
    const long long R = A.R;
    if (R <= 0) return NGLOD_OK;
    const long long nb = (R + kHitBlock - 1) / kHitBlock;
    // the ray-group order of the finished trace is no longer needed: its
    // region (R / 32 ints) holds the block counts
    int* cnt = reinterpret_cast<int*>(static_cast<char*>(work) + trace_ws_order_offset(R));
    k_hit_counts<<<(unsigned)nb, kHitThreads, 0, st>>>(A.hit, R, cnt);
    k_hit_scan<<<1, 1024, 0, st>>>(cnt, nb);
    k_hit_place<<<(unsigned)nb, kHitThreads, 0, st>>>(A.hit, R, cnt, A.hit_list);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

int enqueue_ray_order(TraceArgs& A, void* work, const Node* node_D, cudaStream_t st) {
    const long long R = A.R, G = (R + 31) / 32;
    char* w = static_cast<char*>(work);
    int32_t* order = reinterpret_cast<int32_t*>(w + trace_ws_order_offset(R));
    uint8_t* key = reinterpret_cast<uint8_t*>(w + trace_ws_key_offset(R));
    int* hist = reinterpret_cast<int*>(w + trace_ws_count_offset(R));
    int* cursor = hist + kOrderBuckets;
    NGLOD_CUDA(cudaMemsetAsync(hist, 0, kOrderBuckets * sizeof(int), st));
    const int sms = device_sms();
    const int gk = (int)std::max<long long>(1, std::min<long long>((G + 7) / 8, (long long)sms * 4));
    int4* start = reinterpret_cast<int4*>(w + trace_ws_start_offset(R));
    k_group_keys<<<gk, 256, 0, st>>>(A.offs, A.cnt, R, key, hist, A.o, A.d, A.vid, node_D, A.D, start);
    k_order_scan<<<1, kOrderBuckets, 0, st>>>(hist, cursor);
    const int gs = (int)std::max<long long>(1, std::min<long long>((G + 255) / 256, (long long)sms * 4));
    k_order_scatter<<<gs, 256, 0, st>>>(key, G, cursor, order);
    NGLOD_CUDA(cudaGetLastError());
    A.order = order;
    A.start = start;
    return NGLOD_OK;
}

}  // namespace nglod

extern "C" size_t sphere_trace_workspace(int64_t R) {
    if (R < 0) return 0;
    return trace_ws_size(R);
}

extern "C" int sphere_trace(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* dec,
                            const float* o, const float* d, int64_t R, int lod,
                            const nglod_trace_params* params, const int32_t* ray_offsets,
                            const int32_t* voxel_id, const float* t_range, void* work, size_t work_bytes,
                            float* t_hit, uint8_t* hit, int32_t* steps, float* normal, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!svo || !params) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace: NULL octree or params");
    const int D = lod + kFirstFeatureDepth - 1;
    if (lod < 1 || D >= svo->num_depths) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace: lod out of range");
    if (R < 0 || R >= (1ll << 31) - 64) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace: bad R");
    if (!(params->eps > 0.0f) || !(params->far_t > 0.0f) || params->max_steps < 1)
        return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace: eps, far_t and max_steps must be positive");
    if (int e = check_normal_params(params, "sphere_trace")) return e;
    if (params->ctas_per_sm < 0 || params->ctas_per_sm > 4)
        return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace: ctas_per_sm must lie in 0..4");
    if (R == 0) return NGLOD_OK;
    if (!o || !d || !ray_offsets || !t_hit || !hit || !work)
        return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace: NULL argument");
    if (work_bytes < sphere_trace_workspace(R)) return fail(NGLOD_ERR_CAPACITY, "sphere_trace: workspace too small");
    if (((uintptr_t)work & 255u) != 0) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace: work must be 256-B aligned");
    Tables tb;
    // FD normals evaluate the field off the hit voxel: per-LOD tables only
    const bool fd = normal && params->want_normals && params->normal_mode == NGLOD_NORMALS_FD;
    int rc = fill_tables(svo, feats, lod, tb, !fd);
    if (rc) return rc;
    if (!dec || dec->hidden != kHidden || (dec->in_dim != 32 && dec->in_dim != 35))
        return fail(NGLOD_ERR_NOT_SUPPORTED, "sphere_trace: decoder must be 32|35 -> 128 -> 1");
    const bool f16 = feats->dtype == NGLOD_F16;
    TraceArgs A;
    A.o = o;
    A.d = d;
    A.R = R;
    A.D = D;
    A.eps = params->eps;
    A.far_t = params->far_t;
    A.max_steps = params->max_steps;
    A.osc = params->osc_check;
    A.offs = ray_offsets;
    A.cnt = params->ray_counts;
    A.vid = voxel_id;
    A.t_hit = t_hit;
    A.hit = hit;
    A.steps = steps;
    A.queue = (int*)work;
    A.hit_count = (int*)work + 2;
    A.hit_vox = (int32_t*)((char*)work + trace_ws_hit_vox_offset());
    A.hit_list = (int32_t*)((char*)work + trace_ws_hit_list_offset(R));
    A.wfrag = (uint2*)((char*)work + trace_ws_wfrag_offset(R));
    A.ctas_per_sm = params->ctas_per_sm;
    NGLOD_CUDA(cudaMemsetAsync(work, 0, 256, st));
    rc = check_decoder(dec);
    if (rc) return rc;
    if ((rc = enqueue_ray_order(A, work, svo->node[D], st))) return rc;
    // the FP8 decode's ReLU masks are not recorded: with z rounded to four
    // significant bits a pre-activation can round to zero or flip sign (a
    // read-out unit pair at z = 0 would give a zero gradient), so its
    // normals recompute the forward pass in FP32
    if (params->decode_dtype != NGLOD_FP8E4M3 && (rc = enable_hit_masks(A, work, st))) return rc;
    if (params->decode_dtype == NGLOD_F32) {
        rc = launch_trace_fp32(dec, tb, A, f16, svo->num_sms, st);
    } else if (params->decode_dtype == NGLOD_BF16 || params->decode_dtype == NGLOD_FP8E4M3 ||
               params->decode_dtype == NGLOD_F32_SPLIT) {
        const bool fp8 = params->decode_dtype == NGLOD_FP8E4M3;
        if (fp8 && !(feats->fp8_z_absmax > 0.0f))
            return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace: the FP8 decode needs feats->fp8_z_absmax > 0");
        rc = launch_trace_bf16(svo, dec, tb, A, f16, fp8 ? feats->fp8_z_absmax : 0.0f, st,
                               params->decode_dtype == NGLOD_F32_SPLIT);
    } else {
        return fail(NGLOD_ERR_NOT_SUPPORTED, "sphere_trace: decode_dtype must be F32, BF16, FP8E4M3 or F32_SPLIT");
    }
    if (rc) return rc;
    if ((rc = enqueue_hit_order(A, work, st))) return rc;
    if (normal && params->want_normals) {
        rc = params->normal_mode == NGLOD_NORMALS_FD
                 ? launch_normals_fd(dec, tb, A, params->fd_h, normal, f16, svo->num_sms, st)
                 : launch_normals(dec, tb, A, normal, f16, svo->num_sms, st);
        if (rc) return rc;
    }
    return NGLOD_OK;
}

namespace {
int normals_common(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* dec, const float* o,
                   const float* d, int64_t R, int lod, const void* work, size_t work_bytes, const float* t_hit,
                   const uint8_t* hit, float* normal, float fd_h, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!svo) return fail(NGLOD_ERR_INVALID_ARG, "trace_normals: NULL octree");
    if (fd_h != 0.0f && !(fd_h > 0.0f && fd_h < 1.0f))
        return fail(NGLOD_ERR_INVALID_ARG, "trace_normals_fd: fd_h must lie in (0, 1)");
    const int D = lod + kFirstFeatureDepth - 1;
    if (lod < 1 || D >= svo->num_depths) return fail(NGLOD_ERR_INVALID_ARG, "trace_normals: lod out of range");
    if (R < 0) return fail(NGLOD_ERR_INVALID_ARG, "trace_normals: bad R");
    if (R == 0) return NGLOD_OK;
    if (!o || !d || !work || !t_hit || !hit || !normal)
        return fail(NGLOD_ERR_INVALID_ARG, "trace_normals: NULL argument");
    if (work_bytes < sphere_trace_workspace(R)) return fail(NGLOD_ERR_CAPACITY, "trace_normals: workspace too small");
    if (!dec || dec->hidden != kHidden || (dec->in_dim != 32 && dec->in_dim != 35))
        return fail(NGLOD_ERR_NOT_SUPPORTED, "trace_normals: decoder must be 32|35 -> 128 -> 1");
    Tables tb;
    int rc = fill_tables(svo, feats, lod, tb, fd_h == 0.0f);
    if (rc) return rc;
    TraceArgs A{};
    A.o = o;
    A.d = d;
    A.R = R;
    A.D = D;
    A.t_hit = const_cast<float*>(t_hit);
    A.hit = const_cast<uint8_t*>(hit);
    A.hit_count = (int*)const_cast<void*>(work) + 2;
    A.hit_vox = (int32_t*)((char*)work + trace_ws_hit_vox_offset());
    A.hit_list = (int32_t*)((char*)work + trace_ws_hit_list_offset(R));
    // the masked-sum operand is scratch of the normals themselves
    A.wfrag = (uint2*)((char*)const_cast<void*>(work) + trace_ws_wfrag_offset(R));
    A.hit_mask = (uint4*)((char*)work + trace_ws_mask_offset(R));   // used if the header flag says recorded
    const bool f16 = feats->dtype == NGLOD_F16;
    return fd_h > 0.0f ? launch_normals_fd(dec, tb, A, fd_h, normal, f16, svo->num_sms, st)
                       : launch_normals(dec, tb, A, normal, f16, svo->num_sms, st);
}
}  // namespace

extern "C" int trace_normals(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* dec,
                             const float* o, const float* d, int64_t R, int lod, const void* work,
                             size_t work_bytes, const float* t_hit, const uint8_t* hit, float* normal,
                             void* stream) {
    return normals_common(svo, feats, dec, o, d, R, lod, work, work_bytes, t_hit, hit, normal, 0.0f, stream);
}

extern "C" int trace_normals_fd(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* dec,
                                const float* o, const float* d, int64_t R, int lod, const void* work,
                                size_t work_bytes, const float* t_hit, const uint8_t* hit, float fd_h,
                                float* normal, void* stream) {
    if (!(fd_h > 0.0f && fd_h < 1.0f))
        return fail(NGLOD_ERR_INVALID_ARG, "trace_normals_fd: fd_h must lie in (0, 1)");
    return normals_common(svo, feats, dec, o, d, R, lod, work, work_bytes, t_hit, hit, normal, fd_h, stream);
}

extern "C" int sphere_trace_status(const void* work, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!work) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_status: NULL workspace");
    int h[2] = {0, 0};
    NGLOD_CUDA(cudaMemcpyAsync(h, work, sizeof(h), cudaMemcpyDeviceToHost, st));
    NGLOD_CUDA(cudaStreamSynchronize(st));
    if (h[1] == kStatusTimeout)
        return fail(NGLOD_ERR_TIMEOUT, "sphere_trace: a tensor-core wait expired; results are invalid");
    return NGLOD_OK;
}

namespace nglod {
namespace {
template <typename T>
__global__ void k_absmax(const T* __restrict__ a, long long n, unsigned* __restrict__ out) {
    float m = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf((float)a[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));   // non-negative: bit order = value order
}
}  // namespace
}  // namespace nglod

extern "C" int nglod_features_absmax(const nglod_svo* svo, const nglod_features* feats, int lod, float* h_out,
                                     void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!svo || !feats || !h_out || lod < 1 || lod > feats->num_lods || lod > svo->num_depths - kFirstFeatureDepth)
        return fail(NGLOD_ERR_INVALID_ARG, "nglod_features_absmax: bad arguments");
    if (feats->dtype != NGLOD_F32 && feats->dtype != NGLOD_F16)
        return fail(NGLOD_ERR_NOT_SUPPORTED, "nglod_features_absmax: features must be F32 or F16");
    if (feats->summed_lod != 0 && (feats->summed_lod != lod || feats->dtype != NGLOD_F32))
        return fail(NGLOD_ERR_INVALID_ARG, "nglod_features_absmax: a summed table serves only its own LOD (F32)");
    NGLOD_CUDA(cudaMemsetAsync(svo->dscratch, 0, sizeof(unsigned) * 16, st));
    const int first = feats->summed_lod != 0 ? lod : 1;   // a summed table bounds z alone
    for (int l = first; l <= lod; ++l) {
        if (!feats->feats[l - 1]) return fail(NGLOD_ERR_INVALID_ARG, "nglod_features_absmax: NULL table");
        const long long n = svo->nc[l + kFirstFeatureDepth - 1] * (long long)feats->m;
        const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)svo->num_sms * 8));
        if (feats->dtype == NGLOD_F16)
            k_absmax<__half><<<grid, 256, 0, st>>>((const __half*)feats->feats[l - 1], n, svo->dscratch + l);
        else
            k_absmax<float><<<grid, 256, 0, st>>>((const float*)feats->feats[l - 1], n, svo->dscratch + l);
    }
    NGLOD_CUDA(cudaGetLastError());
    unsigned h[16];
    NGLOD_CUDA(cudaMemcpyAsync(h, svo->dscratch, sizeof(h), cudaMemcpyDeviceToHost, st));
    NGLOD_CUDA(cudaStreamSynchronize(st));
    float sum = 0.0f;
    for (int l = first; l <= lod; ++l) {
        float v;
        memcpy(&v, &h[l], sizeof(float));
        sum += v;
    }
    *h_out = sum;
    return NGLOD_OK;
}
