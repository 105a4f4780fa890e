// nglod_sum_features: the summed corner table of one LOD (Sec. 3.2).
//
// Eq. 2 decodes z(x) = sum over LODs l = 1..L of psi_l(x), psi_l the
// trilinear interpolant of level l's corner features in the voxel of level l
// that holds x.  For x inside a voxel V of LOD L, every coarser voxel holding
// x also holds all of V, and its interpolant, a product of affine functions
// of the three coordinates, is trilinear on V as well; so z restricted to V
// is the trilinear interpolation of z's values at V's 8 corners.  This table
// stores those values once per corner of LOD L, which turns a render's 8 L
// row gathers per query into 8.
//
// One warp per (voxel of LOD L, corner) pair, lane = channel.  The corner's
// integer position P (at LOD L's resolution) gives, at each coarser depth,
// its local coordinates in the ancestor voxel: (P - base) / 2^s with
// s = L's depth - that depth <= 7, so u and 1 - u carry at most 8
// significant bits and every trilinear weight (a product of three) at most
// 24: the weights are exact in FP32 and the terms with weight 0 are skipped.
// The sum is carried as an unevaluated pair hi + lo of FP32 numbers: each
// product w r splits exactly into its rounded value and fmaf's remainder,
// each addition into its rounded value and the two-sum remainder (Knuth's
// TwoSum), and the remainders gather in lo, so the one final rounding of
// hi + lo dominates the error (FP64 arithmetic, the plain alternative, runs
// at a small fraction of the FP32 rate on GB300).  A corner shared by several
// voxels is computed by each of them with the same non-zero terms in the
// same order (where two of them have different ancestors, the corner lies on
// the ancestors' common face, edge or vertex, whose corners they share), so
// every write of a row carries the same value.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "nglod_internal.cuh"
#include "query_common.cuh"
#include "trace_common.cuh"

namespace nglod {
namespace {

template <typename T>
__device__ __forceinline__ float feat_at(const void* base, long long i);

template <>
__device__ __forceinline__ float feat_at<float>(const void* base, long long i) {
    return __ldg(static_cast<const float*>(base) + i);
}

template <>
__device__ __forceinline__ float feat_at<__half>(const void* base, long long i) {
    return __half2float(static_cast<const __half*>(base)[i]);
}

// hi + lo += w r, with the rounding errors of the product and of the sum
// kept in lo.
__device__ __forceinline__ void acc2(float& hi, float& lo, float w, float r) {
    const float p = __fmul_rn(w, r);
    const float ep = __fmaf_rn(w, r, -p);          // w r - p, exact
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float es = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));   // hi + p - s, exact
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(es, ep));
}

template <typename T>
__global__ void __launch_bounds__(256) k_sum_features(const Tables tb, int D, long long V, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long task = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < V * 8;
         task += nw) {
        const long long v = task >> 3;
        const int c = (int)(task & 7);
        const uint32_t ijk = tb.node[D][v].ijk;
        const uint32_t vc[3] = {unpack_i(ijk), unpack_j(ijk), unpack_k(ijk)};
        const uint32_t P[3] = {vc[0] + (c & 1), vc[1] + ((c >> 1) & 1), vc[2] + ((c >> 2) & 1)};
        float hi = 0.0f, lo = 0.0f;
#pragma unroll 1
        for (int dp = kFirstFeatureDepth; dp <= D; ++dp) {
            const int sh = D - dp;
            const int a = __ldg(tb.anc[D] + v * 8 + (dp - kFirstFeatureDepth));
            float u[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) u[ax] = (float)(P[ax] - ((vc[ax] >> sh) << sh)) * pow2f(-sh);
            const void* fb = tb.feats[dp - kFirstFeatureDepth];
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                float w = 1.0f;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) w *= ((cc >> ax) & 1) ? u[ax] : 1.0f - u[ax];
                if (w != 0.0f) {
                    const int row = __ldg(tb.corners[dp] + (size_t)a * 8 + cc);
                    acc2(hi, lo, w, feat_at<T>(fb, (long long)row * kFeatDim + lane));
                }
            }
        }
        const int row = __ldg(tb.corners[D] + v * 8 + c);
        out[(size_t)row * kFeatDim + lane] = __fadd_rn(hi, lo);
    }
}

}  // namespace
}  // namespace nglod

using namespace nglod;

extern "C" int nglod_sum_features(const nglod_svo* svo, const nglod_features* feats, int lod, float* out,
                                  void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!svo || !feats || !out) return fail(NGLOD_ERR_INVALID_ARG, "nglod_sum_features: NULL argument");
    const int D = lod + kFirstFeatureDepth - 1;
    if (lod < 1 || D >= svo->num_depths) return fail(NGLOD_ERR_INVALID_ARG, "nglod_sum_features: lod out of range");
    if (feats->summed_lod != 0)
        return fail(NGLOD_ERR_NOT_SUPPORTED, "nglod_sum_features: the input must be per-LOD tables");
    if ((reinterpret_cast<uintptr_t>(out) & 31u) != 0)
        return fail(NGLOD_ERR_INVALID_ARG, "nglod_sum_features: out must be 32-byte aligned");
    Tables tb;
    int rc = fill_tables(svo, feats, lod, tb);
    if (rc) return rc;
    const long long V = svo->n[D];
    if (V == 0) return NGLOD_OK;
    const int grid = (int)std::max<long long>(1, std::min<long long>((V * 8 + 7) / 8, (long long)svo->num_sms * 16));
    if (feats->dtype == NGLOD_F16) k_sum_features<__half><<<grid, 256, 0, st>>>(tb, D, V, out);
    else k_sum_features<float><<<grid, 256, 0, st>>>(tb, D, V, out);
    NGLOD_CUDA(cudaGetLastError());
    return NGLOD_OK;
}
