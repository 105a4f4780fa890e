// Tensor-core decodes for the sphere tracer and for sdf_query.
//
// The decoder's first layer over a batch of queries is a dense contraction:
// pre[q][h] = sum_k z[q][k] W1[h][k], N = 128 hidden units, K = 32 feature
// channels.
//
// Sphere tracing with the BF16 or the three-term FP32 decode, per image or
// batched (k_trace_warp_bf16, k_trace_batch_warp): each warp decodes its own
// 32 slots with warp-level MMAs (mma.sync m16n8k16, BF16 operands, FP32
// accumulation), the A operand built from the z the lane gathered itself, so
// no warp waits for another.
//
// tcgen05 (sdf_query, the FP8 tracer and batches, level blending): each CTA
// owns 128 query slots (thread i <-> A-tile row i <-> tensor-memory lane i):
//   1. gather: 4-lane groups interpolate each slot's z (FP32, 8 channels a
//      lane) and write it straight into the A tile, laid out as the MMA's
//      canonical K-major operand (8-row x 16-byte core matrices);
//   2. one thread issues the tcgen05.mma (A, B from shared memory, FP32
//      accumulator in 128 TMEM columns) and commits to an mbarrier;
//   3. epilogue: every thread loads its accumulator row with tcgen05.ld and
//      applies b1 (+ the FP32 x-term when in_dim = 35), ReLU and the W2 dot
//      product in FP32 on the CUDA cores.
// W1 (z part) is converted once per CTA and stays resident.  Several CTAs
// share an SM (4 x 128 TMEM columns), so one CTA's gathers overlap another's
// MMA and epilogue.  Every wait is bounded: on expiry the kernel raises an
// error flag, drains its MMA, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <type_traits>

#include "nglod_internal.cuh"
#include "query_common.cuh"
#include "tcgen05.cuh"
#include "trace_common.cuh"

namespace nglod {
namespace {

constexpr int kTM = 128;                 // queries per tile = threads per CTA
constexpr int kKc = kFeatDim / 8;        // 16-byte K chunks per operand row
constexpr uint32_t kLbo = 128;           // K-adjacent core matrices
constexpr uint32_t kSbo = 128 * kKc;     // M/N-adjacent 8-row groups
constexpr int kCtasPerSm = 4;           // 4 x 128 TMEM columns = the SM's 512

struct BfSmem {
    unsigned char A[kTM * kFeatDim * 2];      // z tile, bf16 or e4m3, K-major
    unsigned char B[kHidden * kFeatDim * 2];  // W1 (z columns), bf16 or e4m3, K-major
    float4 epi[kHidden];                      // (b1, W2, W1x_0, W1x_1)
    float4 bw[kHidden / 2];                   // (b1, W2) of units 2j and 2j + 1
    float wx2[kHidden];                       // W1x_2
    float amax[kTM / 32];                     // FP8: per-warp |W1z| maxima
    float acc_scale;                          // FP8: 1 / (W1 scale * z scale)
    uint64_t bar;
    uint32_t taddr;
};
constexpr float kE4M3Max = 448.0f;
// Shared memory is kept small so the rest of the SM's 256 KB serves as L1
// for the feature gathers; registers (>= 103 per thread) already keep
// residency at 4 CTAs per SM.  A fifth CTA on an SM would only wait in
// tcgen05.alloc until one of the four finished.
constexpr int kDynSmem = (int)((sizeof(BfSmem) + 1023) / 1024 * 1024);

// FP32-accurate decode on the tensor cores: z and W1 (z columns) each as a
// sum of three BF16 terms (x = x0 + x1 + x2, 24 significant bits), and the
// six products whose magnitude exceeds 2^-24 of the leading one accumulated
// in FP32 tensor memory.
struct BfSmem3 {
    unsigned char A[3][kTM * kFeatDim * 2];
    unsigned char B[3][kHidden * kFeatDim * 2];
    float4 epi[kHidden];
    float4 bw[kHidden / 2];
    float wx2[kHidden];
    float amax[kTM / 32];
    float acc_scale;
    uint64_t bar;
    uint32_t taddr;
};
constexpr int kDynSmem3 = (int)((sizeof(BfSmem3) + 1023) / 1024 * 1024);

// precision mode of the tensor-core decode: 0 BF16, 1 FP8-E4M3, 2 FP32 by
// three-term BF16 splits
template <int PM>
struct TcSmem {
    using type = BfSmem;
};
template <>
struct TcSmem<2> {
    using type = BfSmem3;
};

struct DecPtrsB {
    const float* W1;
    const float* b1;
    const float* W2;
    const float* b2;   // one float (device), read when the kernel starts
    float z_scale;     // FP8: z is multiplied by this before rounding to e4m3
    long long polls;   // poll budget of each tile's MMA wait
};

template <int IN, bool FP8>
__device__ __forceinline__ void stage_bf16_decoder(BfSmem& S, const DecPtrsB& dp) {
    constexpr int OFF = IN - kFeatDim;
    if constexpr (FP8) {
        // per-LOD weight scale: the largest |W1| of the z columns maps to 448
        float m = 0.0f;
        for (int i = threadIdx.x; i < kHidden * kFeatDim; i += blockDim.x)
            m = fmaxf(m, fabsf(dp.W1[(i / kFeatDim) * IN + OFF + i % kFeatDim]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) S.amax[threadIdx.x >> 5] = m;
        __syncthreads();
        float wmax = 0.0f;
#pragma unroll
        for (int w = 0; w < kTM / 32; ++w) wmax = fmaxf(wmax, S.amax[w]);
        const float ws = wmax > 0.0f ? kE4M3Max / wmax : 1.0f;
        if (threadIdx.x == 0) S.acc_scale = 1.0f / (ws * dp.z_scale);
        for (int i = threadIdx.x; i < kHidden * kFeatDim; i += blockDim.x) {
            const int h = i / kFeatDim, k = i - h * kFeatDim;
            const __nv_fp8_e4m3 q(dp.W1[h * IN + OFF + k] * ws);
            S.B[tc::kmajor_offset8(h, k, kFeatDim / 16)] = *reinterpret_cast<const unsigned char*>(&q);
        }
    } else {
        for (int i = threadIdx.x; i < kHidden * kFeatDim; i += blockDim.x) {
            const int h = i / kFeatDim, k = i - h * kFeatDim;
            *reinterpret_cast<__nv_bfloat16*>(S.B + tc::kmajor_offset(h, k, kKc)) =
                __float2bfloat16_rn(dp.W1[h * IN + OFF + k]);
        }
        if (threadIdx.x == 0) S.acc_scale = 1.0f;
    }
    for (int h = threadIdx.x; h < kHidden; h += blockDim.x) {
        const float x0 = OFF ? dp.W1[h * IN] : 0.f, x1 = OFF ? dp.W1[h * IN + 1] : 0.f;
        S.epi[h] = make_float4(dp.b1[h], dp.W2[h], x0, x1);
        S.wx2[h] = OFF ? dp.W1[h * IN + 2] : 0.f;
    }
    for (int j = threadIdx.x; j < kHidden / 2; j += blockDim.x)
        S.bw[j] = make_float4(dp.b1[2 * j], dp.W2[2 * j], dp.b1[2 * j + 1], dp.W2[2 * j + 1]);
}

// Writes this lane's four z channels of A-tile row `row` as bf16 or, scaled,
// as e4m3 (round to nearest, saturating at +-448).
template <bool FP8>
__device__ __forceinline__ void put_z(BfSmem& S, int row, int l, float4 z, float zs) {
    if constexpr (FP8) {
        const __nv_fp8x4_e4m3 q(make_float4(z.x * zs, z.y * zs, z.z * zs, z.w * zs));
        *reinterpret_cast<uint32_t*>(S.A + tc::kmajor_offset8(row, 4 * l, kFeatDim / 16)) =
            *reinterpret_cast<const uint32_t*>(&q);
    } else {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(z.x, z.y);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(z.z, z.w);
        uint2 v;
        v.x = *reinterpret_cast<const uint32_t*>(&lo);
        v.y = *reinterpret_cast<const uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(S.A + tc::kmajor_offset(row, 4 * l, kKc)) = v;
    }
}

// Makes the A-tile writes visible to the tensor core and meets the CTA's
// other threads (the barrier before an MMA); returns whether any thread's
// `act` is set.
__device__ __forceinline__ bool tile_barrier_or(bool act) {
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    return __syncthreads_or(act) != 0;
}

// Issues the tile's MMA (thread 0) and waits for it (all threads); returns
// false if the wait expired.  barrier = false: the caller has just passed
// tile_barrier_or.
template <bool FP8>
__device__ __forceinline__ bool mma_tile(BfSmem& S, uint32_t taddr, uint32_t& phase, long long polls,
                                         bool barrier = true) {
    if (barrier) {
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(S.A), b0 = tc::smem_u32(S.B);
        if constexpr (FP8) {
            // K = 32 e4m3 elements = 2 chunks of 16 B per row: one instruction
            constexpr uint32_t sbo8 = 128 * (kFeatDim / 16);
            tc::mma_e4m3(taddr, tc::smem_desc_kmajor(a0, kLbo, sbo8), tc::smem_desc_kmajor(b0, kLbo, sbo8),
                         tc::idesc_e4m3_f32(kTM, kHidden), false);
        } else {
            const uint32_t idesc = tc::idesc_bf16_f32(kTM, kHidden);
#pragma unroll
            for (int ks = 0; ks < kFeatDim / 16; ++ks)
                tc::mma_bf16(taddr, tc::smem_desc_kmajor(a0 + ks * 256, kLbo, kSbo),
                             tc::smem_desc_kmajor(b0 + ks * 256, kLbo, kSbo), idesc, ks > 0);
        }
        tc::mma_commit(&S.bar);
    }
    const bool ok = tc::mbar_wait(&S.bar, phase, polls);
    phase ^= 1u;
    tc::fence_after_sync();
    return ok;
}

// d = b2 + sum_h W2[h] relu(acc[h] + b1[h] (+ W1x[h] . x)) for this thread's
// row; with a mask pointer, also its ReLU mask (bit h: pre_h > 0).
template <int IN, class SM>
__device__ __forceinline__ float epilogue(const SM& S, uint32_t taddr, float b2, float x0, float x1, float x2,
                                          uint4* mask = nullptr) {
    const int warp = threadIdx.x >> 5;
    const float sc = S.acc_scale;
    float out = b2;
    uint32_t m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;
#pragma unroll 1
    for (int c0 = 0; c0 < kHidden; c0 += 32) {
        float v[32];
        tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        tc::tmem_wait_ld();
        uint32_t bits = 0u;
        if constexpr (IN == kFeatDim) {
            // (b1, W2) of two units per 16-byte shared load
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
                const float4 e = S.bw[(c0 + i) >> 1];
                const float p0 = fmaf(v[i], sc, e.x), p1 = fmaf(v[i + 1], sc, e.z);
                out = fmaf(e.y, fmaxf(p0, 0.0f), out);
                out = fmaf(e.w, fmaxf(p1, 0.0f), out);
                bits |= (p0 > 0.0f ? 1u : 0u) << i;
                bits |= (p1 > 0.0f ? 1u : 0u) << (i + 1);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float4 e = S.epi[c0 + i];
                float pre = fmaf(v[i], sc, e.x);
                pre = fmaf(e.z, x0, fmaf(e.w, x1, fmaf(S.wx2[c0 + i], x2, pre)));
                out = fmaf(e.y, fmaxf(pre, 0.0f), out);
                bits |= (pre > 0.0f ? 1u : 0u) << i;
            }
        }
        m0 = c0 == 0 ? bits : m0;
        m1 = c0 == 32 ? bits : m1;
        m2 = c0 == 64 ? bits : m2;
        m3 = c0 == 96 ? bits : m3;
    }
    if (mask) *mask = make_uint4(m0, m1, m2, m3);
    return out;
}

template <class SM>
__device__ __forceinline__ void setup_tmem(SM& S) {
    if (threadIdx.x == 0) tc::mbar_init(&S.bar, 1);
    if ((threadIdx.x >> 5) == 0) {
        tc::tmem_alloc(&S.taddr, kHidden);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

template <class SM>
__device__ __forceinline__ void teardown_tmem(SM& S, uint32_t taddr, bool drained, uint32_t phase) {
    if (!drained) tc::mbar_wait(&S.bar, phase ^ 1u, kDefaultWaitPolls);   // let an expired MMA finish
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(taddr, kHidden);
}

// Three BF16 terms of v: t0 = bf16(v), t1 = bf16(v - t0), t2 = bf16(v - t0 - t1)
// (each difference exact in FP32).
__device__ __forceinline__ void split3(float v, __nv_bfloat16& t0, __nv_bfloat16& t1, __nv_bfloat16& t2) {
    t0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(t0);
    t1 = __float2bfloat16_rn(r1);
    t2 = __float2bfloat16_rn(r1 - __bfloat162float(t1));
}

template <int IN>
__device__ __forceinline__ void stage_split_decoder(BfSmem3& S, const DecPtrsB& dp) {
    constexpr int OFF = IN - kFeatDim;
    for (int i = threadIdx.x; i < kHidden * kFeatDim; i += blockDim.x) {
        const int h = i / kFeatDim, k = i - h * kFeatDim;
        __nv_bfloat16 t[3];
        split3(dp.W1[h * IN + OFF + k], t[0], t[1], t[2]);
        const uint32_t o = tc::kmajor_offset(h, k, kKc);
#pragma unroll
        for (int p = 0; p < 3; ++p) *reinterpret_cast<__nv_bfloat16*>(S.B[p] + o) = t[p];
    }
    if (threadIdx.x == 0) S.acc_scale = 1.0f;
    for (int h = threadIdx.x; h < kHidden; h += blockDim.x) {
        const float x0 = OFF ? dp.W1[h * IN] : 0.f, x1 = OFF ? dp.W1[h * IN + 1] : 0.f;
        S.epi[h] = make_float4(dp.b1[h], dp.W2[h], x0, x1);
        S.wx2[h] = OFF ? dp.W1[h * IN + 2] : 0.f;
    }
    for (int j = threadIdx.x; j < kHidden / 2; j += blockDim.x)
        S.bw[j] = make_float4(dp.b1[2 * j], dp.W2[2 * j], dp.b1[2 * j + 1], dp.W2[2 * j + 1]);
}

// This lane's four z channels of A-tile row `row`, as three BF16 planes.
__device__ __forceinline__ void put_z_split(BfSmem3& S, int row, int l, float4 z) {
    const float zz[4] = {z.x, z.y, z.z, z.w};
    __nv_bfloat16 t[3][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) split3(zz[c], t[0][c], t[1][c], t[2][c]);
    const uint32_t o = tc::kmajor_offset(row, 4 * l, kKc);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const __nv_bfloat162 lo = __halves2bfloat162(t[p][0], t[p][1]);
        const __nv_bfloat162 hi = __halves2bfloat162(t[p][2], t[p][3]);
        uint2 v;
        v.x = *reinterpret_cast<const uint32_t*>(&lo);
        v.y = *reinterpret_cast<const uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(S.A[p] + o) = v;
    }
}

// The six products A_i B_j (i + j <= 2), smallest first, into one FP32
// accumulator; issued by thread 0, waited for by all (bounded).
__device__ __forceinline__ bool mma_tile_split(BfSmem3& S, uint32_t taddr, uint32_t& phase, long long polls,
                                               bool barrier = true) {
    if (barrier) {
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        constexpr int kPi[6] = {2, 1, 0, 1, 0, 0}, kPj[6] = {0, 1, 2, 0, 1, 0};
        const uint32_t idesc = tc::idesc_bf16_f32(kTM, kHidden);
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            const uint32_t a0 = tc::smem_u32(S.A[kPi[t]]), b0 = tc::smem_u32(S.B[kPj[t]]);
#pragma unroll
            for (int ks = 0; ks < kFeatDim / 16; ++ks)
                tc::mma_bf16(taddr, tc::smem_desc_kmajor(a0 + ks * 256, kLbo, kSbo),
                             tc::smem_desc_kmajor(b0 + ks * 256, kLbo, kSbo), idesc, t > 0 || ks > 0);
        }
        tc::mma_commit(&S.bar);
    }
    const bool ok = tc::mbar_wait(&S.bar, phase, polls);
    phase ^= 1u;
    tc::fence_after_sync();
    return ok;
}

template <int IN, int PM>
__device__ __forceinline__ void stage_any(typename TcSmem<PM>::type& S, const DecPtrsB& dp) {
    if constexpr (PM == 2) stage_split_decoder<IN>(S, dp);
    else stage_bf16_decoder<IN, PM == 1>(S, dp);
}

template <int PM>
__device__ __forceinline__ void put_any(typename TcSmem<PM>::type& S, int row, int l, float4 z, float zs) {
    if constexpr (PM == 2) put_z_split(S, row, l, z);
    else put_z<PM == 1>(S, row, l, z, zs);
}

template <int PM>
__device__ __forceinline__ bool mma_any(typename TcSmem<PM>::type& S, uint32_t taddr, uint32_t& phase,
                                        long long polls, bool barrier = true) {
    if constexpr (PM == 2) return mma_tile_split(S, taddr, phase, polls, barrier);
    else return mma_tile<PM == 1>(S, taddr, phase, polls, barrier);
}

// ---------------------------------------------------------------------------
// sphere tracing on tcgen05 (the FP8 decode, PM = 1, is the one launched)
// ---------------------------------------------------------------------------
template <typename T, int IN, int PM>
__global__ void __launch_bounds__(kTM, kCtasPerSm) k_trace_bf16(const DecPtrsB dp, const Tables tb, const TraceArgs A,
                                                      int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using SM = typename TcSmem<PM>::type;
    SM& S = *reinterpret_cast<SM*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    stage_any<IN, PM>(S, dp);
    for (int i = threadIdx.x; i < (int)(sizeof(S.A) / 16); i += blockDim.x)
        reinterpret_cast<uint4*>(S.A)[i] = make_uint4(0u, 0u, 0u, 0u);   // rows of idle warps stay finite
    setup_tmem(S);
    const uint32_t taddr = S.taddr;
    const float b2 = __ldg(dp.b2);
    uint32_t phase = 0;
    bool drained = true;
    RaySlot st;
    st.ray = -1;
    st.hit_ray = -1;
    RayQueue Qu;
    Qu.init();
    const int d0 = gather_first_depth(tb);
    for (;;) {
        refill(st, Qu, A, tb, lane);
        const bool act = st.ray >= 0;
        const float x0 = fmaf(st.t, st.dx, st.ox), x1 = fmaf(st.t, st.dy, st.oy), x2 = fmaf(st.t, st.dz, st.oz);
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
        // a warp without rays (the tail of the frame) leaves its 32 A-tile
        // rows as they are and skips its epilogue: its rows are never read
        const bool wact = __any_sync(0xffffffffu, act);
        if (wact) {
            const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
            const unsigned gm4 = 0xfu << gb4;
            // the warp's active slots, compacted: group g4 of round r takes
            // the (8 r + g4)-th, so a warp with na rays gathers in
            // ceil(na / 8) rounds (the rows of idle slots keep their last,
            // finite values; their results are not used)
            const unsigned am = __ballot_sync(0xffffffffu, act);
            // the first level's corner ids of the next round's slot are
            // fetched while this round's slot is gathered (ns = 32: no slot)
            // (every shuffle here runs on all 32 lanes: only the loads are conditional)
            int ns = g4 < __popc(am) ? kth_set_bit(am, g4) : 32;
            const int vox0 = __shfl_sync(0xffffffffu, st.vox, ns & 31);
            int2 nids = ns < 32 ? __ldg(corner_ids(tb, A.D, vox0, d0, l4)) : make_int2(0, 0);
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {
                if (8 * r >= __popc(am)) break;
                const int s = ns & 31;
                const bool sact = ns < 32;
                const int2 ids = nids;
                const int svox = __shfl_sync(0xffffffffu, st.vox, s);
                const uint32_t sijk = __shfl_sync(0xffffffffu, st.ijk, s);
                const float s0 = __shfl_sync(0xffffffffu, q0, s);
                const float s1 = __shfl_sync(0xffffffffu, q1, s);
                const float s2 = __shfl_sync(0xffffffffu, q2, s);
                if (r < 3) {
                    const int k = 8 * (r + 1) + g4;
                    ns = k < __popc(am) ? kth_set_bit(am, k) : 32;
                    const int nvox = __shfl_sync(0xffffffffu, st.vox, ns & 31);
                    if (ns < 32) nids = __ldg(corner_ids(tb, A.D, nvox, d0, l4));
                }
                if (sact) {
                    float4 za, zb;
                    gather_slot4_ids<T>(tb, A.D, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zb, ids);
                    put_any<PM>(S, warp * 32 + s, 2 * l4, za, dp.z_scale);
                    put_any<PM>(S, warp * 32 + s, 2 * l4 + 1, zb, dp.z_scale);
                }
            }
        }
        prefetch_next_ijk(st, A, tb);
        // one barrier both ends the loop (no ray left in the CTA) and
        // publishes the A tile to the MMA
        if (!tile_barrier_or(act)) break;
        const bool ok = mma_any<PM>(S, taddr, phase, dp.polls, false);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicExch(err, kStatusTimeout);
            drained = false;
            break;
        }
        uint4 mask = make_uint4(0u, 0u, 0u, 0u);
        const float dhat = wact ? epilogue<IN>(S, taddr, b2, x0, x1, x2, &mask) : 0.0f;
        if (act) step_update(st, dhat, A, tb);
        publish_hits(st, A, lane, mask);
    }
    teardown_tmem(S, taddr, drained, phase);
}

// ---------------------------------------------------------------------------
// sphere tracing, BF16 decode on warp-level MMAs (the three-term FP32
// decode, further below, shares the gather, stash and epilogue)
//
// The same contraction per step, but each warp decodes its own 32 slots:
// pre = z W1^T as 2 M tiles (16 slots each) x 16 N tiles (8 hidden units)
// x 2 K steps of mma.sync m16n8k16 (BF16 operands, FP32 accumulation), with
// A taken from the slots' gathered z and B (W1, BF16) from shared memory.
// No warp waits for another: a tcgen05 tile needs all 128 slots of the CTA
// gathered before its MMA, and that barrier waited for the slowest warp's
// gather at every step.  The K order of the tile is permuted so that every
// lane's fragment holds the channels it gathered: channel 8 l + 4 ks + c
// (lane l of a 4-lane group, c = 0..3) sits at K index 16 ks + 2 l + (c & 1)
// + 8 (c >> 1) of K step ks, and W1's columns follow the same order, which
// makes a lane's B fragment of an N tile one 16-byte load of its W1 row.
// ---------------------------------------------------------------------------
template <int IN>
struct WarpDec {
    uint4 w1[kHidden * kFeatDim / 8];   // W1 (z columns) as BF16: channels 8 j .. 8 j + 7 of unit h at [4 h + j]
    float4 bw[kHidden / 2];             // (b1, W2) of units 2 j and 2 j + 1
    float4 ex[IN == kFeatDim ? 1 : kHidden];   // in_dim 35: (W1x_0, W1x_1, W1x_2, 0) per unit
};
// Per warp, gather round and lane: the lane's BF16 z channels (lane-private:
// kept here between the gather and the MMAs, which need the registers).
struct WarpZ {
    uint4 zs[kTM / 32][4][32];
};
// in_dim 35: the x of the slot each lane gathered in each round.
template <int IN>
struct WarpX {
    float4 xs[kTM / 32][4][IN == kFeatDim ? 1 : 32];
};
template <int IN>
struct WarpSmem {
    WarpDec<IN> dec;
    WarpZ z;
    WarpX<IN> x;
};

__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Bits 2 q and 2 q + 1 of x (q = 0..3) moved to bits 8 q and 8 q + 1.
__device__ __forceinline__ uint32_t spread_pairs(uint32_t x) {
    return (x & 3u) | ((x & 0xcu) << 6) | ((x & 0x30u) << 12) | ((x & 0xc0u) << 18);
}

template <int IN>
__device__ __forceinline__ void stage_warp_decoder(WarpDec<IN>& S, const DecPtrsB& dp) {
    constexpr int OFF = IN - kFeatDim;
    for (int i = threadIdx.x; i < kHidden * kFeatDim / 8; i += blockDim.x) {
        const float* w = dp.W1 + (i >> 2) * IN + OFF + 8 * (i & 3);
        S.w1[i] = make_uint4(bf16x2_bits(w[0], w[1]), bf16x2_bits(w[2], w[3]), bf16x2_bits(w[4], w[5]),
                             bf16x2_bits(w[6], w[7]));
    }
    for (int j = threadIdx.x; j < kHidden / 2; j += blockDim.x)
        S.bw[j] = make_float4(dp.b1[2 * j], dp.W2[2 * j], dp.b1[2 * j + 1], dp.W2[2 * j + 1]);
    if constexpr (OFF != 0)
        for (int h = threadIdx.x; h < kHidden; h += blockDim.x)
            S.ex[h] = make_float4(dp.W1[h * IN], dp.W1[h * IN + 1], dp.W1[h * IN + 2], 0.f);
}

// Rows of idle slots stay finite.
template <int IN>
__device__ __forceinline__ void clear_warp_stash(WarpZ& Z, WarpX<IN>& X) {
    for (int i = threadIdx.x; i < (int)(sizeof(Z.zs) / 16); i += blockDim.x)
        (&Z.zs[0][0][0])[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = threadIdx.x; i < (int)(sizeof(X.xs) / 16); i += blockDim.x)
        (&X.xs[0][0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// The lane's 8 gathered channels as BF16 pairs (channels 8 l4 + 0..7).
__device__ __forceinline__ uint4 pack_bf16x8(float4 a, float4 b) {
    return make_uint4(bf16x2_bits(a.x, a.y), bf16x2_bits(a.z, a.w), bf16x2_bits(b.x, b.y), bf16x2_bits(b.z, b.w));
}

// One row's terms of units u and u + 1: pre = acc + b1 (+ W1x . x), the
// W2-weighted ReLU added to part, the ReLU bits set at sh and sh + 1.
template <int IN, class Dec>
__device__ __forceinline__ void warp_unit2(const Dec& S, int u, const float4& e, float c0, float c1,
                                           const float (&x)[3], float& part, uint32_t& bits, int sh) {
    float p0 = c0 + e.x, p1 = c1 + e.z;
    if constexpr (IN != kFeatDim) {
        const float4 w0 = S.ex[u], w1 = S.ex[u + 1];
        p0 = fmaf(w0.x, x[0], fmaf(w0.y, x[1], fmaf(w0.z, x[2], p0)));
        p1 = fmaf(w1.x, x[0], fmaf(w1.y, x[1], fmaf(w1.z, x[2], p1)));
    }
    part = fmaf(e.y, fmaxf(p0, 0.0f), part);
    part = fmaf(e.w, fmaxf(p1, 0.0f), part);
    bits |= (p0 > 0.0f ? 1u : 0u) << sh;
    bits |= (p1 > 0.0f ? 1u : 0u) << (sh + 1);
}

// Decodes the warp's gathered rows (Z.zs / X.xs of this warp; row h = 0..3
// of a lane is the slot its group gathered in round h, and the active slots
// were handed out in rank order, the (8 r + g)-th to group g of round r):
// returns sum_h W2_h relu(pre_h) (without b2) of this lane's slot, and in
// cm[h] the ReLU bits this lane holds of row h (bit 2 nt (+ 1) for unit
// 8 nt + 2 (lane % 4) (+ 1)).  Called by the whole warp, converged.
template <int IN>
__device__ __forceinline__ float warp_decode(const WarpDec<IN>& S, const WarpZ& Z, const WarpX<IN>& X, int warp,
                                             int lane, unsigned am, uint32_t (&cm)[4]) {
    const int g4 = lane >> 2, l4 = lane & 3;
    const bool two = __popc(am) > 16;
    // A fragments af[8 mt + 4 ks + e] (e as in mma_bf16_16816): rows g4 and
    // g4 + 8 of M tile mt are rows 2 mt and 2 mt + 1 of the lane
    uint32_t af[16];
    float rx[4][3];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const uint4 z = (h < 2 || two) ? Z.zs[warp][h][lane] : make_uint4(0u, 0u, 0u, 0u);
        const int b = 8 * (h >> 1) + (h & 1);
        af[b] = z.x;
        af[b + 2] = z.y;
        af[b + 4] = z.z;
        af[b + 6] = z.w;
        if constexpr (IN != kFeatDim) {
            const float4 xv = (h < 2 || two) ? X.xs[warp][h][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            rx[h][0] = xv.x;
            rx[h][1] = xv.y;
            rx[h][2] = xv.z;
        } else {
            rx[h][0] = rx[h][1] = rx[h][2] = 0.f;
        }
    }
    // 16 N tiles: lane (g4, l4) sums units 8 nt + 2 l4 (+ 1) of its rows
    float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 4; ++h) cm[h] = 0u;
#pragma unroll
    for (int nt = 0; nt < kHidden / 8; ++nt) {
        const uint4 bb = S.w1[(8 * nt + g4) * 4 + l4];
        const int u = 8 * nt + 2 * l4;
        const float4 e = S.bw[u >> 1];
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16_16816(c, af[0], af[1], af[2], af[3], make_uint2(bb.x, bb.y));
        mma_bf16_16816(c, af[4], af[5], af[6], af[7], make_uint2(bb.z, bb.w));
        warp_unit2<IN>(S, u, e, c[0], c[1], rx[0], part[0], cm[0], 2 * nt);
        warp_unit2<IN>(S, u, e, c[2], c[3], rx[1], part[1], cm[1], 2 * nt);
        if (two) {
            float c2[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16_16816(c2, af[8], af[9], af[10], af[11], make_uint2(bb.x, bb.y));
            mma_bf16_16816(c2, af[12], af[13], af[14], af[15], make_uint2(bb.z, bb.w));
            warp_unit2<IN>(S, u, e, c2[0], c2[1], rx[2], part[2], cm[2], 2 * nt);
            warp_unit2<IN>(S, u, e, c2[2], c2[3], rx[3], part[3], cm[3], 2 * nt);
        }
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        part[h] += __shfl_xor_sync(0xffffffffu, part[h], 1);
        part[h] += __shfl_xor_sync(0xffffffffu, part[h], 2);
    }
    // this lane's slot: round rank / 8 of group rank % 8
    const int rank = __popc(am & ((1u << lane) - 1u));
    const int src = 4 * (rank & 7), rsel = rank >> 3;
    float dsum = 0.f;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const float v = __shfl_sync(0xffffffffu, part[h], src);
        dsum = rsel == h ? v : dsum;
    }
    return dsum;
}

// The 128-bit ReLU mask (bit h: pre_h > 0) of this lane's slot from the
// warp_decode bits: word w of a row (units 32 w ..) has lane j of the group
// holding its bits 8 q + 2 j (+ 1) at bits 8 w + 2 q (+ 1) of cm; lane l4
// assembles word l4 of each row, then the slot's lane collects its row.
// Called by the whole warp, converged.
__device__ __forceinline__ uint4 warp_row_mask(const uint32_t (&cm)[4], int lane, unsigned am) {
    const int l4 = lane & 3, gb4 = (lane >> 2) << 2;
    uint32_t wd[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        uint32_t acc = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t o = __shfl_sync(0xffffffffu, cm[h], gb4 + j);
            acc |= spread_pairs((o >> (8 * l4)) & 0xffu) << (2 * j);
        }
        wd[h] = acc;
    }
    const int rank = __popc(am & ((1u << lane) - 1u));
    const int src = 4 * (rank & 7), rsel = rank >> 3;
    uint32_t m[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        uint32_t v = 0u;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint32_t o = __shfl_sync(0xffffffffu, wd[h], src + w);
            v = rsel == h ? o : v;
        }
        m[w] = v;
    }
    return make_uint4(m[0], m[1], m[2], m[3]);
}

// ---------------------------------------------------------------------------
// sphere tracing, FP32-accurate decode on warp-level MMAs: z and W1 (z
// columns) each as three BF16 terms (split3), the six products A_i B_j with
// i + j <= 2 accumulated smallest first in FP32, as in the tcgen05 form, per
// warp with mma.sync.  The gathered z waits in shared memory as FP32 and is
// split when its fragments are built.
// ---------------------------------------------------------------------------
template <int IN>
struct WarpDec3 {
    uint4 w1[3][kHidden * kFeatDim / 8];   // the three BF16 terms of W1, each laid out as WarpDec::w1
    float4 bw[kHidden / 2];
    float4 ex[IN == kFeatDim ? 1 : kHidden];
};
struct WarpZF {
    float4 zs[kTM / 32][4][32][2];         // per warp, round and lane: the lane's 8 FP32 z channels
};
template <int IN>
struct WarpSmem3 {
    WarpDec3<IN> dec;
    WarpZF z;
    WarpX<IN> x;
};

template <int IN>
__device__ __forceinline__ void stage_warp_decoder3(WarpDec3<IN>& S, const DecPtrsB& dp) {
    constexpr int OFF = IN - kFeatDim;
    for (int i = threadIdx.x; i < kHidden * kFeatDim / 8; i += blockDim.x) {
        const float* w = dp.W1 + (i >> 2) * IN + OFF + 8 * (i & 3);
        __nv_bfloat16 t[3][8];
#pragma unroll
        for (int c = 0; c < 8; ++c) split3(w[c], t[0][c], t[1][c], t[2][c]);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            uint32_t u[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const __nv_bfloat162 v = __halves2bfloat162(t[p][2 * c], t[p][2 * c + 1]);
                u[c] = *reinterpret_cast<const uint32_t*>(&v);
            }
            S.w1[p][i] = make_uint4(u[0], u[1], u[2], u[3]);
        }
    }
    for (int j = threadIdx.x; j < kHidden / 2; j += blockDim.x)
        S.bw[j] = make_float4(dp.b1[2 * j], dp.W2[2 * j], dp.b1[2 * j + 1], dp.W2[2 * j + 1]);
    if constexpr (OFF != 0)
        for (int h = threadIdx.x; h < kHidden; h += blockDim.x)
            S.ex[h] = make_float4(dp.W1[h * IN], dp.W1[h * IN + 1], dp.W1[h * IN + 2], 0.f);
}

// The three BF16 terms of a pair of FP32 values, as BF16 pairs.
__device__ __forceinline__ void split3_pair(float a, float b, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
    __nv_bfloat16 a0, a1, a2, b0, b1, b2;
    split3(a, a0, a1, a2);
    split3(b, b0, b1, b2);
    const __nv_bfloat162 v0 = __halves2bfloat162(a0, b0), v1 = __halves2bfloat162(a1, b1),
                         v2 = __halves2bfloat162(a2, b2);
    p0 = *reinterpret_cast<const uint32_t*>(&v0);
    p1 = *reinterpret_cast<const uint32_t*>(&v1);
    p2 = *reinterpret_cast<const uint32_t*>(&v2);
}

// warp_decode with the three-term products (same rows, results and bits).
template <int IN>
__device__ __forceinline__ float warp_decode3(const WarpDec3<IN>& S, const WarpZF& Z, const WarpX<IN>& X, int warp,
                                              int lane, unsigned am, uint32_t (&cm)[4]) {
    const int g4 = lane >> 2, l4 = lane & 3;
    const bool two = __popc(am) > 16;
    // af[p][8 mt + 4 ks + e]: term p of the A fragments
    uint32_t af[3][16];
    float rx[4][3];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zb = za;
        if (h < 2 || two) {
            za = Z.zs[warp][h][lane][0];
            zb = Z.zs[warp][h][lane][1];
        }
        const int b = 8 * (h >> 1) + (h & 1);
        split3_pair(za.x, za.y, af[0][b], af[1][b], af[2][b]);
        split3_pair(za.z, za.w, af[0][b + 2], af[1][b + 2], af[2][b + 2]);
        split3_pair(zb.x, zb.y, af[0][b + 4], af[1][b + 4], af[2][b + 4]);
        split3_pair(zb.z, zb.w, af[0][b + 6], af[1][b + 6], af[2][b + 6]);
        if constexpr (IN != kFeatDim) {
            const float4 xv = (h < 2 || two) ? X.xs[warp][h][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            rx[h][0] = xv.x;
            rx[h][1] = xv.y;
            rx[h][2] = xv.z;
        } else {
            rx[h][0] = rx[h][1] = rx[h][2] = 0.f;
        }
    }
    constexpr int kPi[6] = {2, 1, 0, 1, 0, 0}, kPj[6] = {0, 1, 2, 0, 1, 0};
    float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 4; ++h) cm[h] = 0u;
#pragma unroll
    for (int nt = 0; nt < kHidden / 8; ++nt) {
        const int wi = (8 * nt + g4) * 4 + l4;
        const uint4 bb[3] = {S.w1[0][wi], S.w1[1][wi], S.w1[2][wi]};
        const int u = 8 * nt + 2 * l4;
        const float4 e = S.bw[u >> 1];
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            const uint32_t* a = af[kPi[t]];
            const uint4& w = bb[kPj[t]];
            mma_bf16_16816(c, a[0], a[1], a[2], a[3], make_uint2(w.x, w.y));
            mma_bf16_16816(c, a[4], a[5], a[6], a[7], make_uint2(w.z, w.w));
        }
        warp_unit2<IN>(S, u, e, c[0], c[1], rx[0], part[0], cm[0], 2 * nt);
        warp_unit2<IN>(S, u, e, c[2], c[3], rx[1], part[1], cm[1], 2 * nt);
        if (two) {
            float c2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                const uint32_t* a = af[kPi[t]];
                const uint4& w = bb[kPj[t]];
                mma_bf16_16816(c2, a[8], a[9], a[10], a[11], make_uint2(w.x, w.y));
                mma_bf16_16816(c2, a[12], a[13], a[14], a[15], make_uint2(w.z, w.w));
            }
            warp_unit2<IN>(S, u, e, c2[0], c2[1], rx[2], part[2], cm[2], 2 * nt);
            warp_unit2<IN>(S, u, e, c2[2], c2[3], rx[3], part[3], cm[3], 2 * nt);
        }
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        part[h] += __shfl_xor_sync(0xffffffffu, part[h], 1);
        part[h] += __shfl_xor_sync(0xffffffffu, part[h], 2);
    }
    const int rank = __popc(am & ((1u << lane) - 1u));
    const int src = 4 * (rank & 7), rsel = rank >> 3;
    float dsum = 0.f;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const float v = __shfl_sync(0xffffffffu, part[h], src);
        dsum = rsel == h ? v : dsum;
    }
    return dsum;
}

template <int IN, bool SPLIT>
using WarpSmemT = std::conditional_t<SPLIT, WarpSmem3<IN>, WarpSmem<IN>>;

// SPLIT: the three-term FP32-accurate decode (warp_decode3), else BF16.
template <typename T, int IN, bool SPLIT>
__global__ void __launch_bounds__(kTM, kCtasPerSm) k_trace_warp_bf16(const DecPtrsB dp, const Tables tb,
                                                                     const TraceArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    WarpSmemT<IN, SPLIT>& S = *reinterpret_cast<WarpSmemT<IN, SPLIT>*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (SPLIT) {
        stage_warp_decoder3<IN>(S.dec, dp);
        for (int i = threadIdx.x; i < (int)(sizeof(S.z.zs) / 16); i += blockDim.x)
            (&S.z.zs[0][0][0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = threadIdx.x; i < (int)(sizeof(S.x.xs) / 16); i += blockDim.x)
            (&S.x.xs[0][0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        stage_warp_decoder<IN>(S.dec, dp);
        clear_warp_stash<IN>(S.z, S.x);
    }
    __syncthreads();
    const float b2 = __ldg(dp.b2);
    const bool want_mask = A.hit_mask != nullptr;
    RaySlot st;
    st.ray = -1;
    st.hit_ray = -1;
    RayQueue Qu;
    Qu.init();
    const int d0 = gather_first_depth(tb);
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;
    for (;;) {
        refill(st, Qu, A, tb, lane);
        const bool act = st.ray >= 0;
        const unsigned am = __ballot_sync(0xffffffffu, act);
        if (am == 0u) break;   // the queue is exhausted and the warp has no ray left
        const int na = __popc(am);
        const float x0 = fmaf(st.t, st.dx, st.ox), x1 = fmaf(st.t, st.dy, st.oy), x2 = fmaf(st.t, st.dz, st.oz);
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
        // gather, with the warp's active slots compacted: group g4 of round
        // r takes the (8 r + g4)-th, whose z becomes row g4 (r even) or
        // g4 + 8 (r odd) of M tile r / 2; the first level's corner ids of the
        // next round's slot load while this round's slot is gathered
        int ns = g4 < na ? kth_set_bit(am, g4) : 32;
        const int vox0 = __shfl_sync(0xffffffffu, st.vox, ns & 31);
        int2 nids = ns < 32 ? __ldg(corner_ids(tb, A.D, vox0, d0, l4)) : make_int2(0, 0);
#pragma unroll 1
        for (int r = 0; r < 4; ++r) {
            if (8 * r >= na) break;
            const int s = ns & 31;
            const bool sact = ns < 32;
            const int2 ids = nids;
            const int svox = __shfl_sync(0xffffffffu, st.vox, s);
            const uint32_t sijk = __shfl_sync(0xffffffffu, st.ijk, s);
            const float s0 = __shfl_sync(0xffffffffu, q0, s);
            const float s1 = __shfl_sync(0xffffffffu, q1, s);
            const float s2 = __shfl_sync(0xffffffffu, q2, s);
            float sx0 = 0.f, sx1 = 0.f, sx2 = 0.f;
            if constexpr (IN != kFeatDim) {
                sx0 = __shfl_sync(0xffffffffu, x0, s);
                sx1 = __shfl_sync(0xffffffffu, x1, s);
                sx2 = __shfl_sync(0xffffffffu, x2, s);
            }
            if (r < 3) {
                const int k = 8 * (r + 1) + g4;
                ns = k < na ? kth_set_bit(am, k) : 32;
                const int nvox = __shfl_sync(0xffffffffu, st.vox, ns & 31);
                if (ns < 32) nids = __ldg(corner_ids(tb, A.D, nvox, d0, l4));
            }
            if (sact) {
                float4 za, zb;
                gather_slot4_ids<T>(tb, A.D, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zb, ids);
                if constexpr (SPLIT) {
                    S.z.zs[warp][r][lane][0] = za;
                    S.z.zs[warp][r][lane][1] = zb;
                } else {
                    S.z.zs[warp][r][lane] = pack_bf16x8(za, zb);
                }
                if constexpr (IN != kFeatDim) S.x.xs[warp][r][lane] = make_float4(sx0, sx1, sx2, 0.f);
            }
        }
        prefetch_next_ijk(st, A, tb);
        uint32_t cm[4];
        float dsum;
        if constexpr (SPLIT) dsum = warp_decode3<IN>(S.dec, S.z, S.x, warp, lane, am, cm);
        else dsum = warp_decode<IN>(S.dec, S.z, S.x, warp, lane, am, cm);
        if (act) step_update(st, b2 + dsum, A, tb);
        const uint4 mask = want_mask && __any_sync(0xffffffffu, st.hit_ray >= 0) ? warp_row_mask(cm, lane, am)
                                                                                : make_uint4(0u, 0u, 0u, 0u);
        publish_hits(st, A, lane, mask);
    }
}

// Batched tracing with the BF16 warp-level decode (the decode of
// k_trace_warp_bf16, so every output is bit-identical to per-image calls):
// the groups one after another, each warp taking rays from the group's queue
// until it is empty; the CTA meets only to stage the next group's decoder.
template <typename T, int IN>
__global__ void __launch_bounds__(kTM, kCtasPerSm) k_trace_batch_warp(const TraceJob* __restrict__ jobs,
                                                                    const JobGroup* __restrict__ groups,
                                                                    int ngroups) {
    __shared__ __align__(16) WarpSmem<IN> S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;
    for (int gi = 0; gi < ngroups; ++gi) {
        // read in place (a register copy of the group spilled)
        const JobGroup& G = groups[gi];
        const DecPtrsB dp{G.W1, G.b1, G.W2, G.b2, G.z_scale, 0};
        __syncthreads();                      // every warp is done with the previous group's decoder
        stage_warp_decoder<IN>(S.dec, dp);
        clear_warp_stash<IN>(S.z, S.x);
        __syncthreads();
        const float b2 = __ldg(dp.b2);
        RaySlot st;
        st.ray = -1;
        st.hit_ray = -1;
        st.job = G.j0;
        RayQueue Qu;
        Qu.init();
        for (;;) {
            refill_batch(st, Qu, G, jobs, lane);
            const bool act = st.ray >= 0;
            const unsigned am = __ballot_sync(0xffffffffu, act);
            if (am == 0u) break;              // the group's queue is exhausted and the warp has no ray left
            const int na = __popc(am);
            const float x0 = fmaf(st.t, st.dx, st.ox), x1 = fmaf(st.t, st.dy, st.oy), x2 = fmaf(st.t, st.dz, st.oz);
            const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
            // the active slots in rank order, the (8 r + g4)-th to group g4 of round r
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {
                if (8 * r >= na) break;
                const int k = 8 * r + g4;
                const int ns = k < na ? kth_set_bit(am, k) : 32;
                const int s = ns & 31;
                const int sjob = __shfl_sync(0xffffffffu, st.job, s);
                const int svox = __shfl_sync(0xffffffffu, st.vox, s);
                const uint32_t sijk = __shfl_sync(0xffffffffu, st.ijk, s);
                const float s0 = __shfl_sync(0xffffffffu, q0, s);
                const float s1 = __shfl_sync(0xffffffffu, q1, s);
                const float s2 = __shfl_sync(0xffffffffu, q2, s);
                float sx0 = 0.f, sx1 = 0.f, sx2 = 0.f;
                if constexpr (IN != kFeatDim) {
                    sx0 = __shfl_sync(0xffffffffu, x0, s);
                    sx1 = __shfl_sync(0xffffffffu, x1, s);
                    sx2 = __shfl_sync(0xffffffffu, x2, s);
                }
                if (ns < 32) {
                    float4 za, zb;
                    gather_slot4<T>(jobs[sjob].tb, jobs[sjob].A.D, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zb);
                    S.z.zs[warp][r][lane] = pack_bf16x8(za, zb);
                    if constexpr (IN != kFeatDim) S.x.xs[warp][r][lane] = make_float4(sx0, sx1, sx2, 0.f);
                }
            }
            uint32_t cm[4];
            const float dsum = warp_decode<IN>(S.dec, S.z, S.x, warp, lane, am, cm);
            if (act) step_update(st, b2 + dsum, jobs[st.job].A, jobs[st.job].tb);
            const uint4 mask = __any_sync(0xffffffffu, st.hit_ray >= 0) ? warp_row_mask(cm, lane, am)
                                                                        : make_uint4(0u, 0u, 0u, 0u);
            publish_hits_batch(st, jobs, mask);
        }
    }
}

// ---------------------------------------------------------------------------
// sdf_query, BF16 decode: tiles of 128 points
// ---------------------------------------------------------------------------
template <typename T, int IN, int PM>
__global__ void __launch_bounds__(kTM, kCtasPerSm) k_query_bf16(const DecPtrsB dp, const Tables tb, const float* __restrict__ x,
                                                      long long Q, int D, float* __restrict__ sdf,
                                                      int8_t* __restrict__ deepest, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using SM = typename TcSmem<PM>::type;
    SM& S = *reinterpret_cast<SM*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;
    stage_any<IN, PM>(S, dp);
    setup_tmem(S);
    const uint32_t taddr = S.taddr;
    const float b2 = __ldg(dp.b2);
    uint32_t phase = 0;
    bool drained = true;
    const long long ntiles = (Q + kTM - 1) / kTM;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long qi = tile * kTM + threadIdx.x;
        const bool act = qi < Q;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        if (act) {
            x0 = x[3 * qi];
            x1 = x[3 * qi + 1];
            x2 = x[3 * qi + 2];
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
            float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zb = za;
            if (sdd >= kFirstFeatureDepth) gather_slot4<T>(tb, sdd, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zb);
            put_any<PM>(S, warp * 32 + s, 2 * l4, za, dp.z_scale);
            put_any<PM>(S, warp * 32 + s, 2 * l4 + 1, zb, dp.z_scale);
        }
        const bool ok = mma_any<PM>(S, taddr, phase, dp.polls);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicExch(err, kStatusTimeout);
            drained = false;
            break;
        }
        const float out = epilogue<IN>(S, taddr, b2, x0, x1, x2);
        if (act) {
            sdf[qi] = out;
            if (deepest) deepest[qi] = (int8_t)(dd >= kFirstFeatureDepth ? dd - kFirstFeatureDepth + 1 : 0);
        }
    }
    teardown_tmem(S, taddr, drained, phase);
}

template <typename K>
void prefer_l1(K kernel);

// ---------------------------------------------------------------------------
// batched sphere tracing (tensor-core decode): groups of jobs, one decoder
// per group, one persistent launch
// ---------------------------------------------------------------------------
template <typename T, int IN, bool FP8>
__global__ void __launch_bounds__(kTM, kCtasPerSm) k_trace_batch(const TraceJob* __restrict__ jobs,
                                                               const JobGroup* __restrict__ groups, int ngroups,
                                                               int* __restrict__ err, long long polls) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    BfSmem& S = *reinterpret_cast<BfSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (int)(sizeof(S.A) / 16); i += blockDim.x)
        reinterpret_cast<uint4*>(S.A)[i] = make_uint4(0u, 0u, 0u, 0u);   // rows of idle warps stay finite
    if (threadIdx.x == 0) tc::mbar_init(&S.bar, 1);
    if (warp == 0) {
        tc::tmem_alloc(&S.taddr, kHidden);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = S.taddr;
    uint32_t phase = 0;
    bool drained = true;
    for (int gi = 0; gi < ngroups && drained; ++gi) {
        const JobGroup G = groups[gi];
        const DecPtrsB dp{G.W1, G.b1, G.W2, G.b2, G.z_scale, polls};
        __syncthreads();                      // the previous group's epilogues are done
        stage_bf16_decoder<IN, FP8>(S, dp);
        tc::fence_proxy_async_smem();
        __syncthreads();
        const float b2 = __ldg(dp.b2);
        RaySlot st;
        st.ray = -1;
        st.hit_ray = -1;
        st.job = G.j0;
        RayQueue Qu;
        Qu.init();
        for (;;) {
            refill_batch(st, Qu, G, jobs, lane);
            const bool act = st.ray >= 0;
            if (!__syncthreads_or(act)) break;
            const float x0 = fmaf(st.t, st.dx, st.ox), x1 = fmaf(st.t, st.dy, st.oy), x2 = fmaf(st.t, st.dz, st.oz);
            const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
            const bool wact = __any_sync(0xffffffffu, act);   // idle warps: rows unread, no epilogue
            const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
            const unsigned gm4 = 0xfu << gb4;
#pragma unroll 1
            for (int r = 0; r < (wact ? 4 : 0); ++r) {
                const int s = r * 8 + g4;
                const int sact = __shfl_sync(0xffffffffu, act ? 1 : 0, s);
                const int sjob = __shfl_sync(0xffffffffu, st.job, s);
                const int svox = __shfl_sync(0xffffffffu, st.vox, s);
                const uint32_t sijk = __shfl_sync(0xffffffffu, st.ijk, s);
                const float s0 = __shfl_sync(0xffffffffu, q0, s);
                const float s1 = __shfl_sync(0xffffffffu, q1, s);
                const float s2 = __shfl_sync(0xffffffffu, q2, s);
                float4 za = make_float4(0.f, 0.f, 0.f, 0.f), zb = za;
                if (sact)
                    gather_slot4<T>(jobs[sjob].tb, jobs[sjob].A.D, svox, sijk, s0, s1, s2, gm4, gb4, l4, za, zb);
                put_z<FP8>(S, warp * 32 + s, 2 * l4, za, dp.z_scale);
                put_z<FP8>(S, warp * 32 + s, 2 * l4 + 1, zb, dp.z_scale);
            }
            const bool ok = mma_tile<FP8>(S, taddr, phase, polls);
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) atomicExch(err, kStatusTimeout);
                drained = false;
                break;
            }
            uint4 mask = make_uint4(0u, 0u, 0u, 0u);
            const float dhat = wact ? epilogue<IN>(S, taddr, b2, x0, x1, x2, &mask) : 0.0f;
            if (act) step_update(st, dhat, jobs[st.job].A, jobs[st.job].tb);
            publish_hits_batch(st, jobs, mask);
        }
    }
    teardown_tmem(S, taddr, drained, phase);
}

template <typename T, int IN, bool FP8>
void go_batch1(const TraceJob* jobs, const JobGroup* groups, int ngroups, int* err, int grid, cudaStream_t st) {
    static std::atomic<unsigned long long> done{0};
    if constexpr (FP8) {
        once_per_device(done, [] { prefer_l1(k_trace_batch<T, IN, true>); });
        k_trace_batch<T, IN, true><<<grid, kTM, kDynSmem, st>>>(jobs, groups, ngroups, err, mma_wait_polls());
    } else {
        // BF16: the warp-level decode, as in per-image tracing
        once_per_device(done, [] { prefer_l1(k_trace_batch_warp<T, IN>); });
        k_trace_batch_warp<T, IN><<<grid, kTM, 0, st>>>(jobs, groups, ngroups);
    }
}

DecPtrsB bptrs(const nglod_decoder* dec, float z_scale) {
    return DecPtrsB{dec->W1, dec->b1, dec->W2, dec->b2, z_scale, mma_wait_polls()};
}

template <typename K>
void prefer_l1(K kernel) {
    // shared-memory share of the unified L1/shared storage, in percent
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 40);
}

// the three-plane kernels need 52 KB of shared memory a CTA: their carveout
// keeps two CTAs per SM with the rest of the storage as L1
template <int PM, typename K>
void configure_tc(K kernel) {
    if constexpr (PM == 2) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem3);
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 50);
    } else {
        prefer_l1(kernel);
    }
}

// The warp-level tracers' shared memory: ~20 KB a CTA (BF16), leaving the
// rest of the storage to L1; the three-term form holds three W1 terms and
// FP32 z (~41 KB, 53 KB with in_dim 35): a carveout for 4 CTAs.
template <bool SPLIT, typename K>
void configure_warp(K kernel, int smem) {
    if constexpr (SPLIT) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             std::min(100, (4 * (smem + 1024) * 100 + 233471) / 233472));
    } else {
        prefer_l1(kernel);
    }
}

template <typename T, int IN, int PM>
void go_trace1(const DecPtrsB& P, const Tables& tb, const TraceArgs& A, int* err, int grid, cudaStream_t st) {
    static std::atomic<unsigned long long> done{0};
    if constexpr (PM != 1) {
        // BF16 and three-term FP32: the warp-level decode
        constexpr bool SPLIT = PM == 2;
        constexpr int smem = (int)sizeof(WarpSmemT<IN, SPLIT>);
        once_per_device(done, [] { configure_warp<SPLIT>(k_trace_warp_bf16<T, IN, SPLIT>, smem); });
        k_trace_warp_bf16<T, IN, SPLIT><<<grid, kTM, smem, st>>>(P, tb, A);
    } else {
        once_per_device(done, [] { configure_tc<PM>(k_trace_bf16<T, IN, PM>); });
        k_trace_bf16<T, IN, PM><<<grid, kTM, PM == 2 ? kDynSmem3 : kDynSmem, st>>>(P, tb, A, err);
    }
}

template <typename T, int IN>
void go_trace(const DecPtrsB& P, const Tables& tb, const TraceArgs& A, int* err, int grid, int pm, cudaStream_t st) {
    if (pm == 2) go_trace1<T, IN, 2>(P, tb, A, err, grid, st);
    else if (pm == 1) go_trace1<T, IN, 1>(P, tb, A, err, grid, st);
    else go_trace1<T, IN, 0>(P, tb, A, err, grid, st);
}

template <typename T, int IN, int PM>
void go_query1(const DecPtrsB& P, const Tables& tb, const float* x, long long Q, int D, float* sdf, int8_t* deep,
               int* err, int grid, cudaStream_t st) {
    static std::atomic<unsigned long long> done{0};
    once_per_device(done, [] { configure_tc<PM>(k_query_bf16<T, IN, PM>); });
    k_query_bf16<T, IN, PM><<<grid, kTM, PM == 2 ? kDynSmem3 : kDynSmem, st>>>(P, tb, x, Q, D, sdf, deep, err);
}

template <typename T, int IN>
void go_query(const DecPtrsB& P, const Tables& tb, const float* x, long long Q, int D, float* sdf, int8_t* deep,
              int* err, int grid, int pm, cudaStream_t st) {
    if (pm == 2) go_query1<T, IN, 2>(P, tb, x, Q, D, sdf, deep, err, grid, st);
    else if (pm == 1) go_query1<T, IN, 1>(P, tb, x, Q, D, sdf, deep, err, grid, st);
    else go_query1<T, IN, 0>(P, tb, x, Q, D, sdf, deep, err, grid, st);
}

}  // namespace

int launch_trace_bf16(const nglod_svo* svo, const nglod_decoder* dec, const Tables& tb, const TraceArgs& A,
                      bool f16, float fp8_z_absmax, cudaStream_t st, bool split) {
    const bool fp8 = fp8_z_absmax > 0.0f;
    const int pm = split ? 2 : fp8 ? 1 : 0;
    static_assert(sizeof(BfSmem) <= kDynSmem, "shared layout");
    // the error word shares the workspace header with the ray queue
    int* err = A.queue + 1;
    const int most = kCtasPerSm;
    const int grid = svo->num_sms * (A.ctas_per_sm > 0 ? std::min(A.ctas_per_sm, most) : most);
    const DecPtrsB P = bptrs(dec, fp8 ? kE4M3Max / fp8_z_absmax : 1.0f);
    if (dec->in_dim == 35) {
        if (f16) go_trace<__half, 35>(P, tb, A, err, grid, pm, st);
        else go_trace<float, 35>(P, tb, A, err, grid, pm, st);
    } else {
        if (f16) go_trace<__half, 32>(P, tb, A, err, grid, pm, st);
        else go_trace<float, 32>(P, tb, A, err, grid, pm, st);
    }
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

int launch_query_bf16(const nglod_svo* svo, const Tables& tb, const nglod_decoder* dec, const float* x,
                      long long Q, int D, float* sdf, int8_t* deepest, bool f16, float fp8_z_absmax,
                      cudaStream_t st, bool split) {
    const bool fp8 = fp8_z_absmax > 0.0f;
    const int pm = split ? 2 : fp8 ? 1 : 0;
    // the octree handle's device status word records an expired wait
    int* err = svo->dstatus;
    NGLOD_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    const long long tiles = (Q + kTM - 1) / kTM;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)svo->num_sms *
                                                                                   (split ? 2 : kCtasPerSm)));
    const DecPtrsB P = bptrs(dec, fp8 ? kE4M3Max / fp8_z_absmax : 1.0f);
    if (dec->in_dim == 35) {
        if (f16) go_query<__half, 35>(P, tb, x, Q, D, sdf, deepest, err, grid, pm, st);
        else go_query<float, 35>(P, tb, x, Q, D, sdf, deepest, err, grid, pm, st);
    } else {
        if (f16) go_query<__half, 32>(P, tb, x, Q, D, sdf, deepest, err, grid, pm, st);
        else go_query<float, 32>(P, tb, x, Q, D, sdf, deepest, err, grid, pm, st);
    }
    NGLOD_CUDA(cudaGetLastError());
    int h = 0;
    NGLOD_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NGLOD_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(NGLOD_ERR_TIMEOUT, "sdf_query: tensor-core wait expired");
    return NGLOD_OK;
}

}  // namespace nglod

namespace nglod {
int launch_trace_batch_tc(const TraceJob* jobs, const JobGroup* groups, int ngroups, int in_dim, bool f16, bool fp8,
                          int ctas_per_sm, int sms, int* err, cudaStream_t st) {
    const int grid = sms * std::max(1, std::min(ctas_per_sm > 0 ? ctas_per_sm : kCtasPerSm, kCtasPerSm));
#define NGLOD_GO(T, I, F) go_batch1<T, I, F>(jobs, groups, ngroups, err, grid, st)
    if (in_dim == 35) {
        if (f16) { if (fp8) NGLOD_GO(__half, 35, true); else NGLOD_GO(__half, 35, false); }
        else { if (fp8) NGLOD_GO(float, 35, true); else NGLOD_GO(float, 35, false); }
    } else {
        if (f16) { if (fp8) NGLOD_GO(__half, 32, true); else NGLOD_GO(__half, 32, false); }
        else { if (fp8) NGLOD_GO(float, 32, true); else NGLOD_GO(float, 32, false); }
    }
#undef NGLOD_GO
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}
}  // namespace nglod

// ---------------------------------------------------------------------------
// Level blending (Sec. 3.2, Eq. 3), BF16 decode: every slot decodes the
// feature sum up to depth D-1 with LOD L*'s decoder and the sum up to D with
// LOD L*+1's, and takes (1 - alpha) d_lo + alpha d_hi.  One gather pass fills
// both A tiles (the second only adds the deepest level); the two MMAs run
// one after the other through the same 128 TMEM columns, so residency stays
// at 4 CTAs per SM.
// ---------------------------------------------------------------------------
namespace nglod {
namespace {

struct BlendSmem {
    // each: its decoder's B tile and epilogue terms, its own A tile and mbarrier
    alignas(1024) BfSmem lo;
    alignas(1024) BfSmem hi;
};
constexpr int kBlendSmem = (int)((sizeof(BlendSmem) + 1023) / 1024 * 1024);

__device__ __forceinline__ void setup_blend(BlendSmem& S) {
    for (int i = threadIdx.x; i < (int)(sizeof(S.lo.A) / 16); i += blockDim.x) {
        reinterpret_cast<uint4*>(S.lo.A)[i] = make_uint4(0u, 0u, 0u, 0u);   // rows of idle warps stay finite
        reinterpret_cast<uint4*>(S.hi.A)[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(&S.lo.bar, 1);
        tc::mbar_init(&S.hi.bar, 1);
    }
    if ((threadIdx.x >> 5) == 0) {
        tc::tmem_alloc(&S.lo.taddr, kHidden);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Group-cooperative (4-lane groups): this lane's 8 channels of z_lo
// (depths 3..dd-1 of a depth-dd voxel) and z_hi = z_lo + psi_dd.
template <typename T>
__device__ __forceinline__ void gather_pair(const Tables& tb, int dd, int dlo, int vox, uint32_t ijk, float q0,
                                            float q1, float q2, unsigned gmask, int gbase, int l4, float4 (&zl)[2],
                                            float4 (&zh)[2]) {
    gather_slot4<T>(tb, dd, vox, ijk, q0, q1, q2, gmask, gbase, l4, zl[0], zl[1], min(dd, dlo));
    zh[0] = zl[0];
    zh[1] = zl[1];
    if (dd > dlo) {
        float4 p[2];
        gather_slot4<T>(tb, dd, vox, ijk, q0, q1, q2, gmask, gbase, l4, p[0], p[1], dd, dd);
#pragma unroll
        for (int h = 0; h < 2; ++h)
            zh[h] = make_float4(zl[h].x + p[h].x, zl[h].y + p[h].y, zl[h].z + p[h].z, zl[h].w + p[h].w);
    }
}

// Both MMAs and epilogues of a tile; returns 0 or which wait expired (1, 2).
template <int IN>
__device__ __forceinline__ int blend_decode(BlendSmem& S, uint32_t taddr, uint32_t& ph_lo, uint32_t& ph_hi,
                                            float b2lo, float b2hi, float alpha, float x0, float x1, float x2,
                                            bool wact, float& dhat, long long polls, uint4* mlo = nullptr,
                                            uint4* mhi = nullptr) {
    if (!__syncthreads_and(mma_tile<false>(S.lo, taddr, ph_lo, polls))) return 1;
    const float dlo = wact ? epilogue<IN>(S.lo, taddr, b2lo, x0, x1, x2, mlo) : 0.0f;
    if (!__syncthreads_and(mma_tile<false>(S.hi, taddr, ph_hi, polls))) return 2;
    const float dhi = wact ? epilogue<IN>(S.hi, taddr, b2hi, x0, x1, x2, mhi) : 0.0f;
    dhat = fmaf(alpha, dhi - dlo, dlo);
    return 0;
}

__device__ __forceinline__ void teardown_blend(BlendSmem& S, uint32_t taddr, int failed, uint32_t ph_lo,
                                               uint32_t ph_hi) {
    if (failed == 2) teardown_tmem(S.hi, taddr, false, ph_hi);
    else teardown_tmem(S.lo, taddr, failed == 0, ph_lo);
}

template <typename T, int IN>
__global__ void __launch_bounds__(kTM, kCtasPerSm) k_trace_blend_bf16(const DecPtrsB plo, const DecPtrsB phi,
                                                                     float alpha, const Tables tb, const TraceArgs A,
                                                                     int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    BlendSmem& S = *reinterpret_cast<BlendSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;
    stage_bf16_decoder<IN, false>(S.lo, plo);
    stage_bf16_decoder<IN, false>(S.hi, phi);
    setup_blend(S);
    const uint32_t taddr = S.lo.taddr;
    const float b2lo = __ldg(plo.b2), b2hi = __ldg(phi.b2);
    uint32_t ph_lo = 0, ph_hi = 0;
    int failed = 0;
    RaySlot st;
    st.ray = -1;
    st.hit_ray = -1;
    RayQueue Qu;
    Qu.init();
    for (;;) {
        refill(st, Qu, A, tb, lane);
        const bool act = st.ray >= 0;
        if (!__syncthreads_or(act)) break;
        const float x0 = fmaf(st.t, st.dx, st.ox), x1 = fmaf(st.t, st.dy, st.oy), x2 = fmaf(st.t, st.dz, st.oz);
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
        // the warp's active slots, compacted (as in k_trace_bf16); the rows
        // of idle slots keep finite values whose results are not used
        const unsigned am = __ballot_sync(0xffffffffu, act);
#pragma unroll 1
        for (int r = 0; r < 4; ++r) {
            if (8 * r >= __popc(am)) break;
            const bool sact = 8 * r + g4 < __popc(am);
            const int s = sact ? kth_set_bit(am, 8 * r + g4) : 0;
            const int svox = __shfl_sync(0xffffffffu, st.vox, s);
            const uint32_t sijk = __shfl_sync(0xffffffffu, st.ijk, s);
            const float s0 = __shfl_sync(0xffffffffu, q0, s);
            const float s1 = __shfl_sync(0xffffffffu, q1, s);
            const float s2 = __shfl_sync(0xffffffffu, q2, s);
            if (sact) {
                float4 zl[2], zh[2];
                gather_pair<T>(tb, A.D, A.D - 1, svox, sijk, s0, s1, s2, gm4, gb4, l4, zl, zh);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    put_z<false>(S.lo, warp * 32 + s, 2 * l4 + h, zl[h], 1.0f);
                    put_z<false>(S.hi, warp * 32 + s, 2 * l4 + h, zh[h], 1.0f);
                }
            }
        }
        prefetch_next_ijk(st, A, tb);
        float dhat = 0.0f;
        uint4 mlo = make_uint4(0u, 0u, 0u, 0u), mhi = mlo;
        failed = blend_decode<IN>(S, taddr, ph_lo, ph_hi, b2lo, b2hi, alpha, x0, x1, x2,
                                  __any_sync(0xffffffffu, act), dhat, plo.polls, &mlo, &mhi);
        if (failed) {
            if (threadIdx.x == 0) atomicExch(err, kStatusTimeout);
            break;
        }
        if (act) step_update(st, dhat, A, tb);
        publish_hits(st, A, lane, mlo, mhi);
    }
    teardown_blend(S, taddr, failed, ph_lo, ph_hi);
}

template <typename T, int IN>
__global__ void __launch_bounds__(kTM, kCtasPerSm) k_query_blend_bf16(const DecPtrsB plo, const DecPtrsB phi,
                                                                     float alpha, const Tables tb,
                                                                     const float* __restrict__ x, long long Q, int D,
                                                                     float* __restrict__ sdf, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    BlendSmem& S = *reinterpret_cast<BlendSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g4 = lane >> 2, l4 = lane & 3, gb4 = g4 << 2;
    const unsigned gm4 = 0xfu << gb4;
    stage_bf16_decoder<IN, false>(S.lo, plo);
    stage_bf16_decoder<IN, false>(S.hi, phi);
    setup_blend(S);
    const uint32_t taddr = S.lo.taddr;
    const float b2lo = __ldg(plo.b2), b2hi = __ldg(phi.b2);
    uint32_t ph_lo = 0, ph_hi = 0;
    int failed = 0;
    const long long ntiles = (Q + kTM - 1) / kTM;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long qi = tile * kTM + threadIdx.x;
        const bool act = qi < Q;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        if (act) {
            x0 = x[3 * qi];
            x1 = x[3 * qi + 1];
            x2 = x[3 * qi + 2];
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
            float4 zl[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)}, zh[2] = {zl[0], zl[1]};
            if (sdd >= kFirstFeatureDepth)
                gather_pair<T>(tb, sdd, D - 1, svox, sijk, s0, s1, s2, gm4, gb4, l4, zl, zh);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                put_z<false>(S.lo, warp * 32 + s, 2 * l4 + h, zl[h], 1.0f);
                put_z<false>(S.hi, warp * 32 + s, 2 * l4 + h, zh[h], 1.0f);
            }
        }
        float out = 0.0f;
        failed = blend_decode<IN>(S, taddr, ph_lo, ph_hi, b2lo, b2hi, alpha, x0, x1, x2,
                                  __any_sync(0xffffffffu, act), out, plo.polls);
        if (failed) {
            if (threadIdx.x == 0) atomicExch(err, kStatusTimeout);
            break;
        }
        if (act) sdf[qi] = out;
    }
    teardown_blend(S, taddr, failed, ph_lo, ph_hi);
}

template <typename T, int IN>
void go_blend(bool trace, const DecPtrsB& lo, const DecPtrsB& hi, float alpha, const Tables& tb, const TraceArgs* A,
              const float* x, long long Q, int D, float* sdf, int* err, int grid, cudaStream_t st) {
    static_assert(sizeof(BlendSmem) <= kBlendSmem && kBlendSmem <= 48 * 1024, "shared layout");
    if (trace) {
        static std::atomic<unsigned long long> done{0};
        once_per_device(done, [] { prefer_l1(k_trace_blend_bf16<T, IN>); });
        k_trace_blend_bf16<T, IN><<<grid, kTM, kBlendSmem, st>>>(lo, hi, alpha, tb, *A, err);
    } else {
        static std::atomic<unsigned long long> done{0};
        once_per_device(done, [] { prefer_l1(k_query_blend_bf16<T, IN>); });
        k_query_blend_bf16<T, IN><<<grid, kTM, kBlendSmem, st>>>(lo, hi, alpha, tb, x, Q, D, sdf, err);
    }
}

void go_blend_any(bool trace, int in_dim, bool f16, const DecPtrsB& lo, const DecPtrsB& hi, float alpha,
                  const Tables& tb, const TraceArgs* A, const float* x, long long Q, int D, float* sdf, int* err,
                  int grid, cudaStream_t st) {
    if (in_dim == 35) {
        if (f16) go_blend<__half, 35>(trace, lo, hi, alpha, tb, A, x, Q, D, sdf, err, grid, st);
        else go_blend<float, 35>(trace, lo, hi, alpha, tb, A, x, Q, D, sdf, err, grid, st);
    } else {
        if (f16) go_blend<__half, 32>(trace, lo, hi, alpha, tb, A, x, Q, D, sdf, err, grid, st);
        else go_blend<float, 32>(trace, lo, hi, alpha, tb, A, x, Q, D, sdf, err, grid, st);
    }
}

}  // namespace

int launch_trace_blend_bf16(const nglod_svo* svo, const nglod_decoder* lo, const nglod_decoder* hi, float alpha,
                            const Tables& tb, const TraceArgs& A, bool f16, cudaStream_t st) {
    int* err = A.queue + 1;      // the workspace header's status word
    go_blend_any(true, lo->in_dim, f16, bptrs(lo, 1.0f), bptrs(hi, 1.0f), alpha, tb, &A, nullptr, 0, A.D, nullptr,
                 err, svo->num_sms * (A.ctas_per_sm > 0 ? std::min(A.ctas_per_sm, kCtasPerSm) : kCtasPerSm), st);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}

int launch_query_blend_bf16(const nglod_svo* svo, const nglod_decoder* lo, const nglod_decoder* hi, float alpha,
                            const Tables& tb, const float* x, long long Q, int D, float* sdf, bool f16,
                            cudaStream_t st) {
    int* err = svo->dstatus;
    NGLOD_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    const long long tiles = (Q + kTM - 1) / kTM;
    const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)svo->num_sms * kCtasPerSm));
    go_blend_any(false, lo->in_dim, f16, bptrs(lo, 1.0f), bptrs(hi, 1.0f), alpha, tb, nullptr, x, Q, D, sdf, err,
                 grid, st);
    NGLOD_CUDA(cudaGetLastError());
    int h = 0;
    NGLOD_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NGLOD_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(NGLOD_ERR_TIMEOUT, "sdf_query_blend: tensor-core wait expired");
    return NGLOD_OK;
}
}  // namespace nglod
