// Continuous level of detail (Sec. 3.2 "Level Blending", Eq. 3) and the LOD
// selection of Sec. 3.4: host entry points.  For a continuous LOD
// L~ >= 1, L* = floor(L~) and alpha = L~ - L*; the blended distance is
// (1 - alpha) d_{L*}(x) + alpha d_{L*+1}(x).  alpha = 0 is the plain query
// or trace at L*.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "nglod_internal.cuh"
#include "query_common.cuh"
#include "trace_common.cuh"

using namespace nglod;

namespace {

// Splits L~ into L* and alpha (exact: L~ - floor(L~) for L~ >= 1 is exact in
// FP32).  Returns an error code for L~ outside [1, num_lods].
int split_lod(const nglod_svo* svo, float lod_tilde, const char* who, int& lstar, float& alpha) {
    const int max_lod = svo->num_depths - kFirstFeatureDepth;
    if (!(lod_tilde >= 1.0f) || !(lod_tilde <= (float)max_lod))
        return fail(NGLOD_ERR_INVALID_ARG, std::string(who) + ": lod_tilde outside [1, max lod]");
    const float f = floorf(lod_tilde);
    lstar = (int)f;
    alpha = lod_tilde - f;
    return NGLOD_OK;
}

int check_pair(const nglod_decoder* lo, const nglod_decoder* hi, const char* who) {
    int rc = check_decoder(lo);
    if (!rc) rc = check_decoder(hi);
    if (rc) return rc;
    if (lo->in_dim != hi->in_dim)
        return fail(NGLOD_ERR_NOT_SUPPORTED, std::string(who) + ": the two decoders must share in_dim");
    return NGLOD_OK;
}

}  // namespace

extern "C" float nglod_lod_select(float distance, float d_near, float d_far, float lod_near, float lod_far) {
    if (!(d_far > d_near)) return distance <= d_near ? lod_near : lod_far;
    float s = (distance - d_near) / (d_far - d_near);
    s = fminf(fmaxf(s, 0.0f), 1.0f);
    return lod_near + s * (lod_far - lod_near);
}

extern "C" int sdf_query_blend(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* dec_lo,
                               const nglod_decoder* dec_hi, const float* x, int64_t Q, float lod_tilde,
                               int decode_dtype, float* sdf, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!svo) return fail(NGLOD_ERR_INVALID_ARG, "sdf_query_blend: NULL octree");
    int lstar;
    float alpha;
    int rc = split_lod(svo, lod_tilde, "sdf_query_blend", lstar, alpha);
    if (rc) return rc;
    if (alpha == 0.0f) return sdf_query(svo, feats, dec_lo, x, Q, lstar, decode_dtype, sdf, nullptr, nullptr, stream);
    if (Q < 0) return fail(NGLOD_ERR_INVALID_ARG, "sdf_query_blend: Q < 0");
    if (Q == 0) return NGLOD_OK;
    if (!x || !sdf) return fail(NGLOD_ERR_INVALID_ARG, "sdf_query_blend: NULL x or sdf");
    if ((rc = check_pair(dec_lo, dec_hi, "sdf_query_blend"))) return rc;
    Tables tb;
    if ((rc = fill_tables(svo, feats, lstar + 1, tb))) return rc;
    const bool f16 = feats->dtype == NGLOD_F16;
    const int D = lstar + kFirstFeatureDepth;      // depth of LOD L* + 1
    if (decode_dtype == NGLOD_F32)
        return launch_query_blend_f32(dec_lo, dec_hi, alpha, tb, x, Q, D, sdf, f16, svo->num_sms, st);
    if (decode_dtype == NGLOD_BF16) return launch_query_blend_bf16(svo, dec_lo, dec_hi, alpha, tb, x, Q, D, sdf, f16, st);
    return fail(NGLOD_ERR_NOT_SUPPORTED, "sdf_query_blend: decode_dtype must be F32 or BF16 when blending");
}

extern "C" int sphere_trace_blend(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* dec_lo,
                                  const nglod_decoder* dec_hi, const float* o, const float* d, int64_t R,
                                  float lod_tilde, const nglod_trace_params* params, const int32_t* ray_offsets,
                                  const int32_t* voxel_id, const float* t_range, void* work, size_t work_bytes,
                                  float* t_hit, uint8_t* hit, int32_t* steps, float* normal, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!svo || !params) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_blend: NULL octree or params");
    int lstar;
    float alpha;
    int rc = split_lod(svo, lod_tilde, "sphere_trace_blend", lstar, alpha);
    if (rc) return rc;
    if (alpha == 0.0f)
        return sphere_trace(svo, feats, dec_lo, o, d, R, lstar, params, ray_offsets, voxel_id, t_range, work,
                            work_bytes, t_hit, hit, steps, normal, stream);
    if (R < 0 || R >= (1ll << 31) - 64) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_blend: bad R");
    if (!(params->eps > 0.0f) || !(params->far_t > 0.0f) || params->max_steps < 1)
        return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_blend: eps, far_t and max_steps must be positive");
    if ((rc = check_normal_params(params, "sphere_trace_blend"))) return rc;
    if (params->ctas_per_sm < 0 || params->ctas_per_sm > 4)
        return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_blend: ctas_per_sm must lie in 0..4");
    if (R == 0) return NGLOD_OK;
    if (!o || !d || !ray_offsets || !t_hit || !hit || !work)
        return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_blend: NULL argument");
    if (work_bytes < sphere_trace_workspace(R))
        return fail(NGLOD_ERR_CAPACITY, "sphere_trace_blend: workspace too small");
    if (((uintptr_t)work & 255u) != 0)
        return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_blend: work must be 256-B aligned");
    if ((rc = check_pair(dec_lo, dec_hi, "sphere_trace_blend"))) return rc;
    Tables tb;
    if ((rc = fill_tables(svo, feats, lstar + 1, tb))) return rc;
    const bool f16 = feats->dtype == NGLOD_F16;
    TraceArgs A;
    A.o = o;
    A.d = d;
    A.R = R;
    A.D = lstar + kFirstFeatureDepth;              // lists at LOD L* + 1
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
    if ((rc = enqueue_ray_order(A, work, svo->node[A.D], st))) return rc;
    if ((rc = enable_hit_masks(A, work, st, true))) return rc;
    if (params->decode_dtype == NGLOD_F32)
        rc = launch_trace_blend_f32(dec_lo, dec_hi, alpha, tb, A, f16, svo->num_sms, st);
    else if (params->decode_dtype == NGLOD_BF16)
        rc = launch_trace_blend_bf16(svo, dec_lo, dec_hi, alpha, tb, A, f16, st);
    else
        return fail(NGLOD_ERR_NOT_SUPPORTED, "sphere_trace_blend: decode_dtype must be F32 or BF16 when blending");
    if (rc) return rc;
    if ((rc = enqueue_hit_order(A, work, st))) return rc;
    if (normal && params->want_normals)
        return params->normal_mode == NGLOD_NORMALS_FD
                   ? launch_normals_blend_fd(dec_lo, dec_hi, alpha, tb, A, params->fd_h, normal, f16, svo->num_sms, st)
                   : launch_normals_blend(dec_lo, dec_hi, alpha, tb, A, normal, f16, svo->num_sms, st);
    return NGLOD_OK;
}
