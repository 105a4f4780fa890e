// sdf_backward: gradients of  sum_L sum_q g_L[q] * sdf_L(x_q)  -- the
// adjoint of the summed per-LOD loss of Eq. 4 -- with respect to the corner
// features of every level, each LOD decoder's parameters, and x.
//
// One launch per LOD L in the mask; a warp owns 32 queries at a time:
//   (A) 8-lane groups interpolate z (Sec. 3.2) into a shared row per query,
//       completed with x so the row is the decoder input v = [z, x];
//   (B) each lane runs its query's forward pass, forms dpre_h = g W2_h
//       [pre_h > 0], and accumulates db2, db1, dW2 (warp sums, one owner lane
//       per hidden unit) and gv = sum_h dpre_h W1[h] (reading each W1 row once
//       as broadcast 16-byte loads);
//   (C) dW1[h][k] = sum_q dpre_q[h] v_q[k]: the warp stages dpre for 32
//       hidden units at a time and each lane, now standing for one hidden
//       unit, sums over the 32 queries; the CTA accumulates in shared memory
//       and flushes with one atomic add per parameter at the end;
//   (D) feature gradients: every level's 8 corner rows of each query receive
//       w_c * gz (gz = the z part of gv), by 16-byte vector atomic adds from
//       the lanes that own those channels (shared corners add up);
//   (E) optional d/dx: W1x^T dpre + J^T gz (trilinear derivative weights),
//       added into grad_x (the launches of one call are stream-ordered).
// Interpolation weights are recomputed, never stored.
//
// Deterministic mode (the same kernel, DET = true): every contribution that
// the default mode adds with FP32 atomics -- the feature scatter of (D), the
// per-warp dW1 rows of (C) and the per-lane db1 / dW2 / db2 sums -- is
// converted exactly to a 128-bit two's-complement fixed-point number with
// quantum 2^-64 and added into a device accumulator with two 64-bit integer
// atomics (the low word's carry, read from the value the atomic returns,
// goes into the high word).  Integer addition is associative, so the sums
// do not depend on the order the atomics land in; a final pass rounds each
// sum once to FP32 and adds it into the caller's gradient.  Exact for
// contributions of magnitude >= 2^-41 (smaller ones lose the bits below
// 2^-64); sums must stay below 2^63 in magnitude.  A non-finite
// contribution raises a flag that turns every output of the call into NaN.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "nglod_internal.cuh"
#include "query_common.cuh"
#include "trace_common.cuh"

namespace nglod {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct BackArgs {
    const float* W1;
    const float* b1;
    const float* W2;
    const float* x;          // [Q, 3]
    const float* g;          // [Q] upstream gradient of this LOD's output (null: L2 mode)
    const float* target;     // L2 mode: [Q] target distances
    float loss_scale;        // L2 mode: g = loss_scale * 2 (d - target)
    const float* b2;         // decoder output bias, one float on the device (L2 mode forward)
    float* loss;             // L2 mode: += sum_q (d - target)^2 (device scalar)
    long long Q;
    int D;
    float* gfeat[kMaxLods];  // per LOD (index l - 1) [C_l, 32]
    float* gW1;              // [128, IN]
    float* gb1;              // [128]
    float* gW2;              // [128]
    float* gb2;              // [1]
    float* gx;               // [Q, 3] or null
    // deterministic mode: 128-bit fixed-point accumulators (2 words each)
    unsigned long long* fx_feat[kMaxLods];  // [C_l * 32]
    unsigned long long* fx_W1;               // [128 * IN]
    unsigned long long* fx_b1;               // [128]
    unsigned long long* fx_W2;               // [128]
    unsigned long long* fx_b2;               // [1]
    unsigned* fx_flag;                       // non-finite contribution seen
};

// v (FP32) as a 128-bit two's-complement fixed-point number, value * 2^64
// truncated toward zero, added into acc[0] (low word) and acc[1] (high).
__device__ __forceinline__ void fx_add(unsigned long long* acc, float v, unsigned* flag) {
    if (v == 0.0f) return;
    const uint32_t b = __float_as_uint(v);
    const int E = (int)((b >> 23) & 0xffu);
    // value = M * 2^(max(E,1) - 150), so value * 2^64 = M << (max(E,1) - 86)
    const int sh = (E ? E : 1) - 86;
    if (E == 0xff || sh > 103) {  // inf / nan, or |v| >= 2^63
        atomicOr(flag, 1u);
        return;
    }
    const unsigned long long M = (b & 0x7fffffu) | (E ? 0x800000u : 0u);
    unsigned long long lo, hi;
    if (sh >= 64) {
        lo = 0ull;
        hi = M << (sh - 64);
    } else if (sh > 0) {
        lo = M << sh;
        hi = M >> (64 - sh);
    } else {
        lo = (-sh) < 64 ? (M >> (-sh)) : 0ull;
        hi = 0ull;
    }
    if (b >> 31) {  // negate: ~x + 1 over the pair
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    if (lo) {
        const unsigned long long old = atomicAdd(acc, lo);
        hi += (old + lo < old) ? 1ull : 0ull;
    }
    if (hi) atomicAdd(acc + 1, hi);
}

struct BackSmem {
    SmemDecoder sd;
    float zb[kWarps][32 * kZStride];        // v rows: z (32) | x (3) | 0
    float dp[kWarps][32 * 33];              // dpre chunk [query][32 hidden units]
    float acc_w1[kHidden * kK4Max];         // dW1 in the reordered [z | x | 0] layout
    float acc_b1[kHidden], acc_w2[kHidden];
    float acc_b2;
};

__device__ __forceinline__ void red_add_v4(float* addr, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

template <typename T, int IN, bool DET>
__global__ void __launch_bounds__(kThreads) k_backward(const Tables tb, const BackArgs A) {
    constexpr int OFF = IN - kFeatDim;
    constexpr int K4 = OFF ? 36 : 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BackSmem& S = *reinterpret_cast<BackSmem*>(smem_raw);
    stage_decoder<IN>(S.sd, A.W1, A.b1, A.W2);
    for (int i = threadIdx.x; i < kHidden * kK4Max; i += blockDim.x) S.acc_w1[i] = 0.0f;
    for (int i = threadIdx.x; i < kHidden; i += blockDim.x) S.acc_b1[i] = S.acc_w2[i] = 0.0f;
    if (threadIdx.x == 0) S.acc_b2 = 0.0f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g8 = lane >> 3, l = lane & 7, gbase = g8 << 3;
    const unsigned gmask = 0xffu << gbase;
    float* zb = S.zb[warp];
    float* dpb = S.dp[warp];
    float own_b1[4] = {0.f, 0.f, 0.f, 0.f}, own_w2[4] = {0.f, 0.f, 0.f, 0.f}, own_b2 = 0.f;
    for (long long base = ((long long)blockIdx.x * kWarps + warp) * 32; base < A.Q;
         base += (long long)gridDim.x * kWarps * 32) {
        const long long qi = base + lane;
        const bool act = qi < A.Q;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, gq = 0.f;
        if (act) {
            x0 = A.x[3 * qi];
            x1 = A.x[3 * qi + 1];
            x2 = A.x[3 * qi + 2];
            if (A.g) gq = A.g[qi];
        }
        int vox;
        uint32_t ijk;
        const int dd = act ? locate_descend(tb, A.D, x0, x1, x2, vox, ijk) : -1;
        const float q0 = __fadd_rn(x0, 1.0f), q1 = __fadd_rn(x1, 1.0f), q2 = __fadd_rn(x2, 1.0f);
        // (A) z rows, completed with x
#pragma unroll 1
        for (int r = 0; r < 8; ++r) {
            const int s = r * 4 + g8;
            const int sdd = __shfl_sync(0xffffffffu, dd, s);
            const int svox = __shfl_sync(0xffffffffu, vox, s);
            const uint32_t sijk = __shfl_sync(0xffffffffu, ijk, s);
            const float s0 = __shfl_sync(0xffffffffu, q0, s);
            const float s1 = __shfl_sync(0xffffffffu, q1, s);
            const float s2 = __shfl_sync(0xffffffffu, q2, s);
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (sdd >= kFirstFeatureDepth) z = gather_slot<T>(tb, sdd, svox, sijk, s0, s1, s2, gmask, gbase, l);
            *reinterpret_cast<float4*>(zb + s * kZStride + 4 * l) = z;
        }
        *reinterpret_cast<float4*>(zb + lane * kZStride + 32) = OFF ? make_float4(x0, x1, x2, 0.f)
                                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        // (B) forward / backward through the decoder for this lane's query
        float v[K4], gv[K4];
#pragma unroll
        for (int j = 0; j < K4 / 4; ++j) {
            const float4 a = reinterpret_cast<const float4*>(zb + lane * kZStride)[j];
            v[4 * j] = a.x; v[4 * j + 1] = a.y; v[4 * j + 2] = a.z; v[4 * j + 3] = a.w;
            gv[4 * j] = gv[4 * j + 1] = gv[4 * j + 2] = gv[4 * j + 3] = 0.f;
        }
        if (!A.g) {
            // L2 mode: this LOD's prediction d, then g = scale * 2 (d - target)
            float dpred = __ldg(A.b2);
#pragma unroll 1
            for (int h = 0; h < kHidden; ++h) {
                const float4* w = reinterpret_cast<const float4*>(S.sd.W1 + h * K4);
                float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
                for (int j = 0; j < K4 / 4; ++j) {
                    const float4 ww = w[j];
                    a0 = fmaf(ww.x, v[4 * j], a0);
                    a1 = fmaf(ww.y, v[4 * j + 1], a1);
                    a0 = fmaf(ww.z, v[4 * j + 2], a0);
                    a1 = fmaf(ww.w, v[4 * j + 3], a1);
                }
                const float2 bw = S.sd.bw[h];
                dpred = fmaf(bw.y, fmaxf(a0 + a1 + bw.x, 0.0f), dpred);
            }
            const float err = act ? dpred - A.target[qi] : 0.0f;
            gq = A.loss_scale * 2.0f * err;
            float se = err * err;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
            if (lane == 0 && A.loss) atomicAdd(A.loss, se);
        }
        own_b2 += gq;
#pragma unroll 1
        for (int hc = 0; hc < kHidden; hc += 32) {
#pragma unroll 1
            for (int hh = 0; hh < 32; ++hh) {
                const int h = hc + hh;
                const float4* w = reinterpret_cast<const float4*>(S.sd.W1 + h * K4);
                float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
                for (int j = 0; j < K4 / 4; ++j) {
                    const float4 ww = w[j];
                    a0 = fmaf(ww.x, v[4 * j], a0);
                    a1 = fmaf(ww.y, v[4 * j + 1], a1);
                    a0 = fmaf(ww.z, v[4 * j + 2], a0);
                    a1 = fmaf(ww.w, v[4 * j + 3], a1);
                }
                const float2 bw = S.sd.bw[h];
                const float pre = a0 + a1 + bw.x;
                const float actv = pre > 0.0f ? pre : 0.0f;
                const float dpre = pre > 0.0f ? gq * bw.y : 0.0f;
#pragma unroll
                for (int j = 0; j < K4 / 4; ++j) {
                    const float4 ww = w[j];
                    gv[4 * j] = fmaf(dpre, ww.x, gv[4 * j]);
                    gv[4 * j + 1] = fmaf(dpre, ww.y, gv[4 * j + 1]);
                    gv[4 * j + 2] = fmaf(dpre, ww.z, gv[4 * j + 2]);
                    gv[4 * j + 3] = fmaf(dpre, ww.w, gv[4 * j + 3]);
                }
                dpb[lane * 33 + hh] = dpre;
                // db1 and dW2: warp sums, kept by the lane that owns unit h
                float s_b1 = dpre, s_w2 = gq * actv;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    s_b1 += __shfl_xor_sync(0xffffffffu, s_b1, o);
                    s_w2 += __shfl_xor_sync(0xffffffffu, s_w2, o);
                }
                if (lane == hh) {
                    own_b1[hc >> 5] += s_b1;
                    own_w2[hc >> 5] += s_w2;
                }
            }
            __syncwarp();
            // (C) dW1 rows of units hc..hc+31: lane = unit, sum over the 32 queries
            float accr[K4];
#pragma unroll
            for (int k = 0; k < K4; ++k) accr[k] = 0.f;
#pragma unroll 1
            for (int q = 0; q < 32; ++q) {
                const float dq = dpb[q * 33 + lane];
#pragma unroll
                for (int j = 0; j < K4 / 4; ++j) {
                    const float4 a = reinterpret_cast<const float4*>(zb + q * kZStride)[j];
                    accr[4 * j] = fmaf(dq, a.x, accr[4 * j]);
                    accr[4 * j + 1] = fmaf(dq, a.y, accr[4 * j + 1]);
                    accr[4 * j + 2] = fmaf(dq, a.z, accr[4 * j + 2]);
                    accr[4 * j + 3] = fmaf(dq, a.w, accr[4 * j + 3]);
                }
            }
            if constexpr (DET) {
#pragma unroll
                for (int k = 0; k < kFeatDim + OFF; ++k) {
                    const int col = k < kFeatDim ? OFF + k : k - kFeatDim;
                    fx_add(A.fx_W1 + 2 * ((size_t)(hc + lane) * IN + col), accr[k], A.fx_flag);
                }
            } else {
#pragma unroll
                for (int k = 0; k < K4; ++k) atomicAdd(&S.acc_w1[(hc + lane) * K4 + k], accr[k]);
            }
            __syncwarp();
        }
        // (D) feature gradients: w_c * gz onto every level's 8 corners
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 8; ++j)
            reinterpret_cast<float4*>(zb + lane * kZStride)[j] =
                make_float4(gv[4 * j], gv[4 * j + 1], gv[4 * j + 2], gv[4 * j + 3]);
        __syncwarp();
#pragma unroll 1
        for (int r = 0; r < 8; ++r) {
            const int s = r * 4 + g8;
            const int sdd = __shfl_sync(0xffffffffu, dd, s);
            const int svox = __shfl_sync(0xffffffffu, vox, s);
            const uint32_t sijk = __shfl_sync(0xffffffffu, ijk, s);
            const float sq[3] = {__shfl_sync(0xffffffffu, q0, s), __shfl_sync(0xffffffffu, q1, s),
                                 __shfl_sync(0xffffffffu, q2, s)};
            float part[3] = {0.f, 0.f, 0.f};
            if (sdd >= kFirstFeatureDepth) {
                const float4 gz = *reinterpret_cast<const float4*>(zb + s * kZStride + 4 * l);
                const int a = (l <= sdd - kFirstFeatureDepth) ? __ldg(tb.anc[sdd] + (size_t)svox * 8 + l) : -1;
                for (int dp2 = kFirstFeatureDepth; dp2 <= sdd; ++dp2) {
                    const int vv = __shfl_sync(gmask, a, gbase + dp2 - kFirstFeatureDepth);
                    const int cid = __ldg(tb.corners[dp2] + (size_t)vv * 8 + l);
                    const int sh = sdd - dp2;
                    const float sc = pow2f(dp2 - 1);
                    const uint32_t cc[3] = {unpack_i(sijk) >> sh, unpack_j(sijk) >> sh, unpack_k(sijk) >> sh};
                    float u[3];
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa) u[aa] = clamp01(__fsub_rn(__fmul_rn(sq[aa], sc), (float)cc[aa]));
                    float wts[8];
                    trilinear_weights(u[0], u[1], u[2], wts);
                    float* gf = A.gfeat[dp2 - kFirstFeatureDepth];
                    const void* fb = tb.feats[dp2 - kFirstFeatureDepth];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int id = __shfl_sync(gmask, cid, gbase + c);
                        if constexpr (DET) {
                            unsigned long long* fa = A.fx_feat[dp2 - kFirstFeatureDepth] + 2 * ((size_t)id * 32 + 4 * l);
                            fx_add(fa, wts[c] * gz.x, A.fx_flag);
                            fx_add(fa + 2, wts[c] * gz.y, A.fx_flag);
                            fx_add(fa + 4, wts[c] * gz.z, A.fx_flag);
                            fx_add(fa + 6, wts[c] * gz.w, A.fx_flag);
                        } else {
                            red_add_v4(gf + (size_t)id * 32 + 4 * l,
                                       make_float4(wts[c] * gz.x, wts[c] * gz.y, wts[c] * gz.z, wts[c] * gz.w));
                        }
                        if (A.gx) {
                            const float4 row = FeatLoad<T>::load(fb, id, l);
                            const float pc = row.x * gz.x + row.y * gz.y + row.z * gz.z + row.w * gz.w;
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
            }
            if (A.gx) {
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) {
                    part[aa] += __shfl_xor_sync(0xffffffffu, part[aa], 1);
                    part[aa] += __shfl_xor_sync(0xffffffffu, part[aa], 2);
                    part[aa] += __shfl_xor_sync(0xffffffffu, part[aa], 4);
                }
                if (l == 0) {
                    dpb[s * 4] = part[0];
                    dpb[s * 4 + 1] = part[1];
                    dpb[s * 4 + 2] = part[2];
                }
            }
        }
        // (E) d/dx
        __syncwarp();
        if (A.gx && act) {
            float gx[3] = {dpb[lane * 4], dpb[lane * 4 + 1], dpb[lane * 4 + 2]};
            if constexpr (OFF == 3) {
                gx[0] += gv[32];
                gx[1] += gv[33];
                gx[2] += gv[34];
            }
            A.gx[3 * qi] += gx[0];
            A.gx[3 * qi + 1] += gx[1];
            A.gx[3 * qi + 2] += gx[2];
        }
        __syncwarp();
    }
    if constexpr (DET) {
        // per-lane unit sums (a fixed order of queries per lane) straight to the accumulators
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            fx_add(A.fx_b1 + 2 * (32 * i + lane), own_b1[i], A.fx_flag);
            fx_add(A.fx_W2 + 2 * (32 * i + lane), own_w2[i], A.fx_flag);
        }
        float b2 = own_b2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b2 += __shfl_xor_sync(0xffffffffu, b2, o);
        if (lane == 0) fx_add(A.fx_b2, b2, A.fx_flag);
    } else {
        // flush: per-lane unit sums into shared, then the CTA adds once per parameter
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            atomicAdd(&S.acc_b1[32 * i + lane], own_b1[i]);
            atomicAdd(&S.acc_w2[32 * i + lane], own_w2[i]);
        }
        {
            float b2 = own_b2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b2 += __shfl_xor_sync(0xffffffffu, b2, o);
            if (lane == 0) atomicAdd(&S.acc_b2, b2);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kHidden * K4; i += blockDim.x) {
            const int h = i / K4, k = i - h * K4;
            int col;
            if (k < kFeatDim) col = OFF + k;
            else if (k < kFeatDim + OFF) col = k - kFeatDim;
            else continue;
            atomicAdd(&A.gW1[h * IN + col], S.acc_w1[i]);
        }
        for (int h = threadIdx.x; h < kHidden; h += blockDim.x) {
            atomicAdd(&A.gb1[h], S.acc_b1[h]);
            atomicAdd(&A.gW2[h], S.acc_w2[h]);
        }
        if (threadIdx.x == 0) atomicAdd(A.gb2, S.acc_b2);
    }
}

template <typename T, int IN, bool DET>
void launch_back(const Tables& tb, const BackArgs& A, int grid, cudaStream_t st) {
    static std::atomic<unsigned long long> done{0};
    once_per_device(done, [] {
        cudaFuncSetAttribute(k_backward<T, IN, DET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BackSmem));
    });
    k_backward<T, IN, DET><<<grid, kThreads, sizeof(BackSmem), st>>>(tb, A);
}

template <typename T, int IN>
void launch_back(const Tables& tb, const BackArgs& A, int grid, bool det, cudaStream_t st) {
    if (det) launch_back<T, IN, true>(tb, A, grid, st); else launch_back<T, IN, false>(tb, A, grid, st);
}

// out[i] += the FP32 rounding of the 128-bit fixed-point sum acc[i] * 2^-64
// (NaN for every element if a non-finite contribution was seen).
__global__ void k_fx_finalize(const unsigned long long* __restrict__ acc, float* __restrict__ out, long long n,
                              const unsigned* __restrict__ flag) {
    const bool bad = *flag != 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long lo = acc[2 * i], hi = acc[2 * i + 1];
        const bool neg = (hi >> 63) != 0ull;
        if (neg) {
            lo = ~lo + 1ull;
            hi = ~hi + (lo == 0ull ? 1ull : 0ull);
        }
        // |sum| = hi + lo * 2^-64; hi < 2^63 so both conversions are in range
        const double mag = __ull2double_rn(hi) + __ull2double_rn(lo) * 0x1p-64;
        const float v = bad ? __int_as_float(0x7fc00000) : (float)(neg ? -mag : mag);
        out[i] += v;
    }
}

}  // namespace
}  // namespace nglod

using namespace nglod;

namespace nglod {
namespace {

int run_backward(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs, const float* x,
                 int64_t Q, uint32_t lod_mask, const float* grad_sdf, const float* target, float loss_scale,
                 float* loss, float* const* h_grad_feats, float* const* h_grad_W1, float* const* h_grad_b1,
                 float* const* h_grad_W2, float* grad_b2, float* grad_x, bool det, cudaStream_t st,
                 const char* who) {
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
    const bool f16 = feats->dtype == NGLOD_F16;
    for (int l = 1; l <= top; ++l)
        if (!h_grad_feats[l - 1]) return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL feature gradient");
    const int grid = svo->num_sms * 2;
    // deterministic mode: one zeroed block of fixed-point accumulators --
    // the feature levels 1..top, then per selected LOD W1 | b1 | W2 | b2,
    // then the flag word
    unsigned long long* fx = nullptr;
    size_t fx_feat_off[kMaxLods] = {}, fx_dec_off[kMaxLods] = {};
    size_t fx_words = 0;
    if (det) {
        size_t n = 0;
        for (int l = 1; l <= top; ++l) {
            fx_feat_off[l - 1] = n;
            n += (size_t)svo->nc[l + kFirstFeatureDepth - 1] * kFeatDim;
        }
        for (int lod = 1; lod <= max_lod; ++lod) {
            if (!((lod_mask >> (lod - 1)) & 1u)) continue;
            fx_dec_off[lod - 1] = n;
            n += (size_t)kHidden * decs[lod - 1].in_dim + 2 * kHidden + 1;
        }
        fx_words = 2 * n + 2;
        NGLOD_CUDA(cudaMallocAsync((void**)&fx, fx_words * sizeof(unsigned long long), st));
        NGLOD_CUDA(cudaMemsetAsync(fx, 0, fx_words * sizeof(unsigned long long), st));
    }
    unsigned* fx_flag = det ? reinterpret_cast<unsigned*>(fx + fx_words - 2) : nullptr;
    int idx = 0;
    for (int lod = 1; lod <= max_lod; ++lod) {
        if (!((lod_mask >> (lod - 1)) & 1u)) continue;
        const nglod_decoder& dec = decs[lod - 1];
        rc = check_decoder(&dec);
        if (rc) return rc;
        if (!h_grad_W1[lod - 1] || !h_grad_b1[lod - 1] || !h_grad_W2[lod - 1])
            return fail(NGLOD_ERR_INVALID_ARG, w + ": NULL decoder gradient");
        BackArgs A;
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
        A.gx = grad_x;
        for (int l = 0; l < kMaxLods; ++l) A.fx_feat[l] = det && l < top ? fx + 2 * fx_feat_off[l] : nullptr;
        if (det) {
            A.fx_W1 = fx + 2 * fx_dec_off[lod - 1];
            A.fx_b1 = A.fx_W1 + 2 * (size_t)kHidden * dec.in_dim;
            A.fx_W2 = A.fx_b1 + 2 * kHidden;
            A.fx_b2 = A.fx_W2 + 2 * kHidden;
        } else {
            A.fx_W1 = A.fx_b1 = A.fx_W2 = A.fx_b2 = nullptr;
        }
        A.fx_flag = fx_flag;
        const long long need = (Q + kThreads - 1) / kThreads;
        const int g2 = (int)std::max<long long>(1, std::min<long long>(need, grid));
        if (dec.in_dim == 35) {
            if (f16) launch_back<__half, 35>(tb, A, g2, det, st); else launch_back<float, 35>(tb, A, g2, det, st);
        } else {
            if (f16) launch_back<__half, 32>(tb, A, g2, det, st); else launch_back<float, 32>(tb, A, g2, det, st);
        }
        NGLOD_CUDA(cudaGetLastError());
        ++idx;
    }
    if (det) {
        auto fin = [&](size_t off, float* out, long long n) {
            const int gr = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)grid * 8));
            k_fx_finalize<<<gr, 256, 0, st>>>(fx + 2 * off, out, n, fx_flag);
        };
        for (int l = 1; l <= top; ++l)
            fin(fx_feat_off[l - 1], h_grad_feats[l - 1], svo->nc[l + kFirstFeatureDepth - 1] * kFeatDim);
        for (int lod = 1; lod <= max_lod; ++lod) {
            if (!((lod_mask >> (lod - 1)) & 1u)) continue;
            const size_t o = fx_dec_off[lod - 1];
            const int in = decs[lod - 1].in_dim;
            fin(o, h_grad_W1[lod - 1], (long long)kHidden * in);
            fin(o + (size_t)kHidden * in, h_grad_b1[lod - 1], kHidden);
            fin(o + (size_t)kHidden * in + kHidden, h_grad_W2[lod - 1], kHidden);
            fin(o + (size_t)kHidden * in + 2 * kHidden, grad_b2 + (lod - 1), 1);
        }
        NGLOD_CUDA(cudaGetLastError());
        NGLOD_CUDA(cudaFreeAsync(fx, st));
    }
    return NGLOD_OK;
}

// Adam (the optimiser the paper trains with, supplementary Sec. A.3):
// m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr mhat / (sqrt(vhat) + eps)
// with bias-corrected mhat, vhat; the gradient is cleared for the next step.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        g[i] = 0.0f;
    }
}

}  // namespace
}  // namespace nglod

extern "C" int sdf_backward(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs,
                            const float* x, int64_t Q, uint32_t lod_mask, const float* grad_sdf,
                            float* const* h_grad_feats, float* const* h_grad_W1, float* const* h_grad_b1,
                            float* const* h_grad_W2, float* grad_b2, float* grad_x, int deterministic,
                            void* stream) {
    if (!grad_sdf) return fail(NGLOD_ERR_INVALID_ARG, "sdf_backward: NULL grad_sdf");
    return run_backward(svo, feats, decs, x, Q, lod_mask, grad_sdf, nullptr, 0.f, nullptr, h_grad_feats, h_grad_W1,
                        h_grad_b1, h_grad_W2, grad_b2, grad_x, deterministic != 0, (cudaStream_t)stream,
                        "sdf_backward");
}

extern "C" int sdf_l2_backward(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs,
                               const float* x, const float* target, int64_t Q, uint32_t lod_mask, float loss_scale,
                               float* loss, float* const* h_grad_feats, float* const* h_grad_W1,
                               float* const* h_grad_b1, float* const* h_grad_W2, float* grad_b2, void* stream) {
    if (!target) return fail(NGLOD_ERR_INVALID_ARG, "sdf_l2_backward: NULL target");
    return run_backward(svo, feats, decs, x, Q, lod_mask, nullptr, target, loss_scale, loss, h_grad_feats, h_grad_W1,
                        h_grad_b1, h_grad_W2, grad_b2, nullptr, false, (cudaStream_t)stream, "sdf_l2_backward");
}

extern "C" int nglod_adam_step(float* param, float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                               float beta2, float eps, int step, void* stream) {
    if (n < 0 || step < 1) return fail(NGLOD_ERR_INVALID_ARG, "nglod_adam_step: bad n or step");
    if (n == 0) return NGLOD_OK;
    if (!param || !grad || !m || !v) return fail(NGLOD_ERR_INVALID_ARG, "nglod_adam_step: NULL buffer");
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    const int grid = (int)std::min<long long>((n + 255) / 256, (long long)device_sms() * 16);
    k_adam<<<grid, 256, 0, (cudaStream_t)stream>>>(param, grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}
