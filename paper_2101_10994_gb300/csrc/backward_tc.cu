// sdf_l2_backward_bf16 / sdf_backward_bf16: the adjoint of the summed
// per-LOD objective of Eq. 4 (the same gradients as backward.cu) with the
// decoder's three contractions on the fifth-generation tensor cores, BF16
// operands and FP32 accumulation (mixed-precision training).
//
// A CTA owns 128 queries at a time (thread i <-> row i <-> TMEM lane i):
//   (A) 4-lane groups gather z (Sec. 3.2) and write v = [z | x | 0] as BF16
//       into the K-major tile A1 (128 x KV);
//   (B) MMA1: P = v W1^T (M = 128 queries, N = 128 hidden units, K = KV);
//   (C) epilogue (row per thread, FP32): pre = P + b1 (+ W1x x in FP32),
//       the prediction d and g (given, or 2 s (d - target) in L2 mode),
//       dpre_h = g W2_h [pre_h > 0] written as BF16 into the K-major tile A2
//       (128 x 128); db1, dW2 reduced over the rows by butterfly shuffles;
//   (D) MMA2: gv = dpre W1 (A2 K-major, W1 read transposed, i.e. MN-major)
//       and MMA3: dW1 += dpre^T v (A2 and A1 both read MN-major), the latter
//       accumulating in tensor memory over all of the CTA's tiles;
//   (E) 4-lane groups scatter w_c * gz (gz = the z part of gv) onto every
//       level's 8 corners with 16-byte vector atomic adds; the groups of a
//       warp whose slots share a voxel at a level first sum their
//       contributions (a butterfly over the groups), so spatially sorted
//       points (nglod_sort_points) need one atomic per corner and block.
// One tile layout serves each operand both ways: an MN-major view of a
// K-major tile takes LBO = the stride between core matrices adjacent along
// K and SBO = the stride between those adjacent along M/N.  The x columns
// of W1 stay FP32 (added in the epilogue); x enters A1 only for dW1's x
// columns.  Every tensor-core wait is bounded (status NGLOD_ERR_TIMEOUT).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "nglod_internal.cuh"
#include "query_common.cuh"
#include "tcgen05.cuh"
#include "trace_common.cuh"

namespace nglod {
namespace {

constexpr int kTQ = 128;                         // queries per tile = threads per CTA
constexpr uint32_t kColP = 0, kColG = 128, kColW = 192, kTmemCols = 256;

template <int KV>
struct TcSmem {
    alignas(1024) unsigned char A1[kTQ * KV * 2];        // v, bf16, K-major (query rows)
    alignas(1024) unsigned char W1[kHidden * KV * 2];    // W1 z columns (x columns 0), bf16, K-major (unit rows)
    alignas(1024) unsigned char A2[kTQ * kHidden * 2];   // dpre, bf16, K-major; then gz staging (FP32)
    float4 epi[kHidden];                                 // (b1, W2, W1x_0, W1x_1)
    float wx2[kHidden];                                  // W1x_2
    uint64_t bar;
    uint32_t taddr;
};
static_assert(kTQ * kZStride * 4 <= kTQ * kHidden * 2, "gz staging must fit in A2");

struct TcArgs {
    const float* W1;
    const float* b1;
    const float* W2;
    const float* b2;         // one float (device)
    const float* x;          // [Q, 3]
    const float* g;          // [Q] upstream gradient of this LOD's output (null: L2 mode)
    const float* target;     // L2 mode: [Q]
    float loss_scale;
    float* loss;             // L2 mode: += sum_q (d - target)^2
    long long Q;
    int D;
    float* gfeat[kMaxLods];
    float* gW1;
    float* gb1;
    float* gW2;
    float* gb2;
    int* err;
    long long polls;         // poll budget of each MMA wait
};

__device__ __forceinline__ void red_add_v4(float* addr, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&p);
}

// Butterfly reduce-scatter over the warp: returns, in lane l, the sum over
// all lanes of v[l] (31 shuffles for 32 values).
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            const float send = up ? v[i] : v[i + s];
            const float keep = up ? v[i + s] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

// Adds w_c * gz (this lane's 8 channels ga | gb) onto the 8 corners of
// every level 3..D of the slots of one round (8 slots, one per 4-lane
// group).  Groups whose slots lie in the same voxel at a level first sum
// their contributions pairwise over the groups (xor 4, 8, 16 in lanes) as
// long as the merged block of groups shares that voxel, so one atomic per
// corner serves the block.  Called by the whole warp.
__device__ __forceinline__ void scatter_round(const Tables& tb, float* const* gfeat, int D, int dd, int vox,
                                              uint32_t ijk, float q0, float q1, float q2, int lane, float4 ga,
                                              float4 gb) {
    const int l4 = lane & 3, g4 = lane >> 2, gbase = g4 << 2;
    int2 a = make_int2(-1, -1);
    if (dd >= kFirstFeatureDepth && 2 * l4 <= dd - kFirstFeatureDepth)
        a = __ldg(reinterpret_cast<const int2*>(tb.anc[dd] + (size_t)vox * 8) + l4);
#pragma unroll 1
    for (int dp = kFirstFeatureDepth; dp <= D; ++dp) {
        const int i = dp - kFirstFeatureDepth;
        const bool act = dp <= dd;
        const int v = __shfl_sync(0xffffffffu, (i & 1) ? a.y : a.x, gbase + (i >> 1));
        const int key = act ? v : -1 - g4;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const bool merge_any = __any_sync(0xffffffffu, __popc(peers) > 4);
        int2 cc = make_int2(0, 0);
        float w[8];
        if (act) {
            cc = __ldg(reinterpret_cast<const int2*>(tb.corners[dp] + (size_t)v * 8) + l4);
            const int sh = dd - dp;
            const float sc = pow2f(dp - 1);
            const float u0 = clamp01(__fsub_rn(__fmul_rn(q0, sc), (float)(unpack_i(ijk) >> sh)));
            const float u1 = clamp01(__fsub_rn(__fmul_rn(q1, sc), (float)(unpack_j(ijk) >> sh)));
            const float u2 = clamp01(__fsub_rn(__fmul_rn(q2, sc), (float)(unpack_k(ijk) >> sh)));
            trilinear_weights(u0, u1, u2, w);
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) w[c] = 0.0f;
        }
        // merge plan (the same for all 8 corners): which butterfly steps merge
        bool carry = act, uni = true;
        unsigned mstep = 0;                          // bit j: step o = 4 << j merges for this lane
        if (merge_any) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int o = 4 << j;
                const int pkey = __shfl_xor_sync(0xffffffffu, key, o);
                const int puni = __shfl_xor_sync(0xffffffffu, uni ? 1 : 0, o);
                if (uni && puni && key == pkey) {
                    // both halves now hold the block's sum; the lower half's carrier writes it
                    mstep |= 1u << j;
                    if (lane & o) carry = false;
                } else {
                    uni = false;
                }
            }
        }
        float* gf = act ? gfeat[i] : nullptr;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int cid = __shfl_sync(0xffffffffu, (c & 1) ? cc.y : cc.x, gbase + (c >> 1));
            float4 ra = make_float4(w[c] * ga.x, w[c] * ga.y, w[c] * ga.z, w[c] * ga.w);
            float4 rb = make_float4(w[c] * gb.x, w[c] * gb.y, w[c] * gb.z, w[c] * gb.w);
            if (merge_any) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int o = 4 << j;
                    float4 pa, pb;
                    pa.x = __shfl_xor_sync(0xffffffffu, ra.x, o); pa.y = __shfl_xor_sync(0xffffffffu, ra.y, o);
                    pa.z = __shfl_xor_sync(0xffffffffu, ra.z, o); pa.w = __shfl_xor_sync(0xffffffffu, ra.w, o);
                    pb.x = __shfl_xor_sync(0xffffffffu, rb.x, o); pb.y = __shfl_xor_sync(0xffffffffu, rb.y, o);
                    pb.z = __shfl_xor_sync(0xffffffffu, rb.z, o); pb.w = __shfl_xor_sync(0xffffffffu, rb.w, o);
                    if ((mstep >> j) & 1u) {
                        ra = make_float4(ra.x + pa.x, ra.y + pa.y, ra.z + pa.z, ra.w + pa.w);
                        rb = make_float4(rb.x + pb.x, rb.y + pb.y, rb.z + pb.z, rb.w + pb.w);
                    }
                }
            }
            if (carry) {
                float* p = gf + (size_t)cid * 32 + 8 * l4;
                red_add_v4(p, ra);
                red_add_v4(p + 4, rb);
            }
        }
    }
}

template <typename T, int IN>
__global__ void __launch_bounds__(kTQ, 2) k_backward_tc(const Tables tb, const TcArgs A) {
    constexpr int OFF = IN - kFeatDim;
    constexpr int KV = OFF ? 48 : 32;       // v columns: z (32) | x (3) | 0, a multiple of 16
    constexpr int KC = KV / 8;              // 16-byte chunks per A1 / W1 row
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem<KV>& S = *reinterpret_cast<TcSmem<KV>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;

    // stage W1 (z columns, bf16), the epilogue constants, and a zero A1
    for (int i = tid; i < kHidden * KV; i += kTQ) {
        const int h = i / KV, k = i - h * KV;
        const float w = k < kFeatDim ? A.W1[h * IN + OFF + k] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(S.W1 + tc::kmajor_offset(h, k, KC)) = __float2bfloat16_rn(w);
    }
    for (int h = tid; h < kHidden; h += kTQ) {
        S.epi[h] = make_float4(A.b1[h], A.W2[h], OFF ? A.W1[h * IN] : 0.f, OFF ? A.W1[h * IN + 1] : 0.f);
        S.wx2[h] = OFF ? A.W1[h * IN + 2] : 0.f;
    }
    for (int i = tid; i < (int)(sizeof(S.A1) / 16); i += kTQ)
        reinterpret_cast<uint4*>(S.A1)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) tc::mbar_init(&S.bar, 1);
    if (warp == 0) {
        tc::tmem_alloc(&S.taddr, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = S.taddr;
    const uint32_t lrow = taddr + ((uint32_t)(warp * 32) << 16);   // this warp's TMEM lane quarter
    uint32_t phase = 0;
    bool drained = true, any = false;
    float own_b1[4] = {0.f, 0.f, 0.f, 0.f}, own_w2[4] = {0.f, 0.f, 0.f, 0.f}, own_b2 = 0.f, own_loss = 0.f;
    float* gzs = reinterpret_cast<float*>(S.A2);
    const long long ntiles = (A.Q + kTQ - 1) / kTQ;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long qi = tile * kTQ + tid;
        const bool act = qi < A.Q;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, gq = 0.f, tgt = 0.f;
        if (act) {
            x0 = A.x[3 * qi];
            x1 = A.x[3 * qi + 1];
            x2 = A.x[3 * qi + 2];
            if (A.g) gq = A.g[qi];
            else tgt = A.target[qi];
        }
        int vox = -1;
        uint32_t ijk = 0;
        const int dd = act ? locate_descend(tb, A.D, x0, x1, x2, vox, ijk) : -1;
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
        // (A) z of the warp's 32 rows into A1 (lane l4 writes the 16-byte chunk of channels 8 l4..8 l4+7)
#pragma unroll 1
        for (int r = 0; r < 4; ++r) {
            const int s = r * 8 + g4;
            const int sdd = __shfl_sync(0xffffffffu, dd, s);
            const int svox = __shfl_sync(0xffffffffu, vox, s);
            const uint32_t sijk = __shfl_sync(0xffffffffu, ijk, s);
            const float s0 = __shfl_sync(0xffffffffu, q0, s);
            const float s1 = __shfl_sync(0xffffffffu, q1, s);
            const float s2 = __shfl_sync(0xffffffffu, q2, s);
            float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zb = za;
            if (sdd >= kFirstFeatureDepth) gather_slot4<T>(tb, sdd, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zb);
            *reinterpret_cast<uint4*>(S.A1 + tc::kmajor_offset(warp * 32 + s, 8 * l4, KC)) =
                make_uint4(pack_bf16(za.x, za.y), pack_bf16(za.z, za.w), pack_bf16(zb.x, zb.y), pack_bf16(zb.z, zb.w));
        }
        if constexpr (OFF != 0) {
            *reinterpret_cast<uint4*>(S.A1 + tc::kmajor_offset(tid, kFeatDim, KC)) =
                make_uint4(pack_bf16(x0, x1), pack_bf16(x2, 0.f), 0u, 0u);
        }
        // (B) MMA1: P = v W1^T (the x columns of W1 are zero here)
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a1 = tc::smem_u32(S.A1), w1 = tc::smem_u32(S.W1);
            const uint32_t idesc = tc::idesc_bf16_f32(kTQ, kHidden);
#pragma unroll
            for (int ks = 0; ks < KV / 16; ++ks)
                tc::mma_bf16(taddr + kColP, tc::smem_desc_kmajor(a1 + ks * 256, 128, 128 * KC),
                             tc::smem_desc_kmajor(w1 + ks * 256, 128, 128 * KC), idesc, ks > 0);
            tc::mma_commit(&S.bar);
        }
        bool ok = tc::mbar_wait(&S.bar, phase, A.polls);
        phase ^= 1u;
        tc::fence_after_sync();
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicExch(A.err, kStatusTimeout);
            drained = false;
            break;
        }
        // (C) epilogue: the prediction, then dpre (bf16 into A2) and the row sums of db1, dW2
        float dval = __ldg(A.b2);
#pragma unroll 1
        for (int c0 = 0; c0 < kHidden; c0 += 32) {
            float v[32];
            tc::tmem_ld32(lrow + kColP + (uint32_t)c0, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float4 e = S.epi[c0 + i];
                float pre = v[i] + e.x;
                if constexpr (OFF != 0) pre = fmaf(e.z, x0, fmaf(e.w, x1, fmaf(S.wx2[c0 + i], x2, pre)));
                dval = fmaf(e.y, fmaxf(pre, 0.0f), dval);
            }
        }
        if (!A.g) {
            const float err = act ? dval - tgt : 0.0f;
            gq = A.loss_scale * 2.0f * err;
            own_loss = fmaf(err, err, own_loss);
        }
        if (!act) gq = 0.0f;
        own_b2 += gq;
#pragma unroll 1
        for (int c0 = 0; c0 < kHidden; c0 += 32) {
            float v[32], rw[32];
            tc::tmem_ld32(lrow + kColP + (uint32_t)c0, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float4 e = S.epi[c0 + i];
                float pre = v[i] + e.x;
                if constexpr (OFF != 0) pre = fmaf(e.z, x0, fmaf(e.w, x1, fmaf(S.wx2[c0 + i], x2, pre)));
                rw[i] = gq * fmaxf(pre, 0.0f);
                v[i] = pre > 0.0f ? gq * e.y : 0.0f;                 // dpre
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                *reinterpret_cast<uint4*>(S.A2 + tc::kmajor_offset(tid, c0 + 8 * j, kHidden / 8)) =
                    make_uint4(pack_bf16(v[8 * j], v[8 * j + 1]), pack_bf16(v[8 * j + 2], v[8 * j + 3]),
                               pack_bf16(v[8 * j + 4], v[8 * j + 5]), pack_bf16(v[8 * j + 6], v[8 * j + 7]));
            own_w2[c0 >> 5] += reduce_scatter32(rw, lane);
            own_b1[c0 >> 5] += reduce_scatter32(v, lane);
        }
        // (D) MMA2: gv = dpre W1 (W1 MN-major); MMA3: dW1 += dpre^T v (A2, A1 MN-major)
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a1 = tc::smem_u32(S.A1), w1 = tc::smem_u32(S.W1), a2 = tc::smem_u32(S.A2);
            const uint32_t id2 = tc::idesc_bf16_f32(kTQ, KV) | (1u << 16);
            const uint32_t id3 = tc::idesc_bf16_f32(kHidden, KV) | (1u << 15) | (1u << 16);
            constexpr uint32_t kA2k = 128 * (kHidden / 8);   // A2: 8-row step (queries)
            constexpr uint32_t kVk = 128 * KC;               // A1 / W1: 8-row step
#pragma unroll
            for (int ks = 0; ks < kHidden / 16; ++ks)        // K = hidden units
                tc::mma_bf16(taddr + kColG, tc::smem_desc_kmajor(a2 + ks * 256, 128, kA2k),
                             tc::smem_desc_kmajor(w1 + ks * 2 * kVk, kVk, 128), id2, ks > 0);
#pragma unroll
            for (int ks = 0; ks < kTQ / 16; ++ks)            // K = queries
                tc::mma_bf16(taddr + kColW, tc::smem_desc_kmajor(a2 + ks * 2 * kA2k, kA2k, 128),
                             tc::smem_desc_kmajor(a1 + ks * 2 * kVk, kVk, 128), id3, any || ks > 0);
            tc::mma_commit(&S.bar);
        }
        any = true;
        ok = tc::mbar_wait(&S.bar, phase, A.polls);
        phase ^= 1u;
        tc::fence_after_sync();
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicExch(A.err, kStatusTimeout);
            drained = false;
            break;
        }
        // (E) gz rows (the z part of gv) staged over A2, then the corner scatter
        {
            float v[32];
            tc::tmem_ld32(lrow + kColG, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<float4*>(gzs + tid * kZStride + 4 * j) =
                    make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
        __syncwarp();
#pragma unroll 1
        for (int r = 0; r < 4; ++r) {
            const int s = r * 8 + g4;
            const int sdd = __shfl_sync(0xffffffffu, dd, s);
            const int svox = __shfl_sync(0xffffffffu, vox, s);
            const uint32_t sijk = __shfl_sync(0xffffffffu, ijk, s);
            const float s0 = __shfl_sync(0xffffffffu, q0, s);
            const float s1 = __shfl_sync(0xffffffffu, q1, s);
            const float s2 = __shfl_sync(0xffffffffu, q2, s);
            const float* gr = gzs + (warp * 32 + s) * kZStride + 8 * l4;
            scatter_round(tb, A.gfeat, A.D, sdd, svox, sijk, s0, s1, s2, lane,
                          *reinterpret_cast<const float4*>(gr), *reinterpret_cast<const float4*>(gr + 4));
        }
        __syncthreads();   // gz staging is A2: the next tile writes dpre there
    }
    // flush: per-lane unit sums, the loss and b2; dW1 from tensor memory (row = unit = thread)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        atomicAdd(&A.gb1[32 * i + lane], own_b1[i]);
        atomicAdd(&A.gW2[32 * i + lane], own_w2[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        own_b2 += __shfl_xor_sync(0xffffffffu, own_b2, o);
        own_loss += __shfl_xor_sync(0xffffffffu, own_loss, o);
    }
    if (lane == 0) {
        atomicAdd(A.gb2, own_b2);
        if (A.loss && !A.g) atomicAdd(A.loss, own_loss);
    }
    if (drained && any) {
#pragma unroll 1
        for (int c0 = 0; c0 < KV; c0 += 32) {
            float v[32];
            tc::tmem_ld32(lrow + kColW + (uint32_t)c0, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int k = c0 + i;
                if (k < kFeatDim) atomicAdd(&A.gW1[tid * IN + OFF + k], v[i]);
                else if (k < kFeatDim + OFF) atomicAdd(&A.gW1[tid * IN + (k - kFeatDim)], v[i]);
            }
        }
    }
    if (!drained) tc::mbar_wait(&S.bar, phase ^ 1u, kDefaultWaitPolls);   // let an expired MMA finish
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, kTmemCols);
}

template <typename T, int IN>
void launch_tc(const Tables& tb, const TcArgs& A, int grid, cudaStream_t st) {
    constexpr int KV = (IN - kFeatDim) ? 48 : 32;
    constexpr int smem = (int)((sizeof(TcSmem<KV>) + 1023) / 1024 * 1024);
    static std::atomic<unsigned long long> done{0};
    once_per_device(done, [] {
        cudaFuncSetAttribute(k_backward_tc<T, IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    k_backward_tc<T, IN><<<grid, kTQ, smem, st>>>(tb, A);
}

int run_backward_tc(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs, const float* x,
                    int64_t Q, uint32_t lod_mask, const float* grad_sdf, const float* target, float loss_scale,
                    float* loss, float* const* h_grad_feats, float* const* h_grad_W1, float* const* h_grad_b1,
                    float* const* h_grad_W2, float* grad_b2, cudaStream_t st, const char* who) {
    const std::string w(who);
    if (!svo || !feats || !decs) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL argument");
    if (Q < 0) return fail(NGLOD_ERR_INVALID_ARG, w + ": Q < 0");
    const int max_lod = svo->num_depths - kFirstFeatureDepth;
    if (lod_mask == 0u || (lod_mask >> max_lod) != 0u)
        return fail(NGLOD_ERR_INVALID_ARG, w + ": lod_mask must select LODs within 1..max LOD");
    if (feats->dtype != NGLOD_F32 && feats->dtype != NGLOD_F16)
        return fail(NGLOD_ERR_NOT_SUPPORTED, w + ": features must be F32 or F16");
    if (Q == 0) return NGLOD_OK;
    if (!x || (!grad_sdf && !target) || !h_grad_feats || !h_grad_W1 || !h_grad_b1 || !h_grad_W2 || !grad_b2)
        return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL input or gradient buffer");
    const int top = 31 - __builtin_clz(lod_mask) + 1;
    Tables tb;
    int rc = fill_tables(svo, feats, top, tb);
    if (rc) return rc;
    for (int l = 1; l <= top; ++l)
        if (!h_grad_feats[l - 1]) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL feature gradient");
    const bool f16 = feats->dtype == NGLOD_F16;
    int* err = svo->dstatus;
    NGLOD_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    const long long tiles = (Q + kTQ - 1) / kTQ;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)svo->num_sms * 2));
    int idx = 0;
    for (int lod = 1; lod <= max_lod; ++lod) {
        if (!((lod_mask >> (lod - 1)) & 1u)) continue;
        const nglod_decoder& dec = decs[lod - 1];
        if ((rc = check_decoder(&dec))) return rc;
        if (!h_grad_W1[lod - 1] || !h_grad_b1[lod - 1] || !h_grad_W2[lod - 1])
            return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL decoder gradient");
        TcArgs A;
        A.W1 = dec.W1;
        A.b1 = dec.b1;
        A.W2 = dec.W2;
        A.b2 = dec.b2;
        A.x = x;
        A.g = grad_sdf ? grad_sdf + (size_t)idx * (size_t)Q : nullptr;
        A.target = target;
        A.loss_scale = loss_scale;
        A.loss = loss ? loss + (lod - 1) : nullptr;
        A.Q = Q;
        A.D = lod + kFirstFeatureDepth - 1;
        for (int l = 0; l < kMaxLods; ++l) A.gfeat[l] = l < top ? h_grad_feats[l] : nullptr;
        A.gW1 = h_grad_W1[lod - 1];
        A.gb1 = h_grad_b1[lod - 1];
        A.gW2 = h_grad_W2[lod - 1];
        A.gb2 = grad_b2 + (lod - 1);
        A.err = err;
        A.polls = mma_wait_polls();
        if (dec.in_dim == 35) {
            if (f16) launch_tc<__half, 35>(tb, A, grid, st); else launch_tc<float, 35>(tb, A, grid, st);
        } else {
            if (f16) launch_tc<__half, 32>(tb, A, grid, st); else launch_tc<float, 32>(tb, A, grid, st);
        }
        NGLOD_CUDA(cudaGetLastError());
        ++idx;
    }
    int h = 0;
    NGLOD_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NGLOD_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(NGLOD_ERR_TIMEOUT, w + ": tensor-core wait expired");
    return NGLOD_OK;
}

}  // namespace
}  // namespace nglod

using namespace nglod;

extern "C" int sdf_backward_bf16(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs,
                                 const float* x, int64_t Q, uint32_t lod_mask, const float* grad_sdf,
                                 float* const* h_grad_feats, float* const* h_grad_W1, float* const* h_grad_b1,
                                 float* const* h_grad_W2, float* grad_b2, void* stream) {
    if (!grad_sdf) return fail(NGLOD_ERR_INVALID_ARG, "sdf_backward_bf16: NULL grad_sdf");
    return run_backward_tc(svo, feats, decs, x, Q, lod_mask, grad_sdf, nullptr, 0.f, nullptr, h_grad_feats, h_grad_W1,
                           h_grad_b1, h_grad_W2, grad_b2, (cudaStream_t)stream, "sdf_backward_bf16");
}

extern "C" int sdf_l2_backward_bf16(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs,
                                    const float* x, const float* target, int64_t Q, uint32_t lod_mask,
                                    float loss_scale, float* loss, float* const* h_grad_feats,
                                    float* const* h_grad_W1, float* const* h_grad_b1, float* const* h_grad_W2,
                                    float* grad_b2, void* stream) {
    if (!target) return fail(NGLOD_ERR_INVALID_ARG, "sdf_l2_backward_bf16: NULL target");
    return run_backward_tc(svo, feats, decs, x, Q, lod_mask, nullptr, target, loss_scale, loss, h_grad_feats,
                           h_grad_W1, h_grad_b1, h_grad_W2, grad_b2, (cudaStream_t)stream, "sdf_l2_backward_bf16");
}
