// sphere_trace_batch_*: many scenes and images of uneven size traced in one
// persistent launch.
//
// A batch fixes a set of jobs (octree, features, decoder, rays, their lists
// and outputs).  Jobs are grouped by decoder (same W1 pointer): inside a
// group one ray queue spans every job's rays, so CTAs move from image to
// image without a launch boundary and no slot idles while rays remain; the
// groups run back to back in the same launch, each staging its decoder once.
// sphere_trace_batch_run only enqueues device work (a reset kernel, the
// persistent trace launch and the per-job normal kernels), so a whole frame
// -- traversals plus this -- can be captured once in a CUDA graph and
// replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "nglod_internal.cuh"
#include "query_common.cuh"
#include "trace_common.cuh"

struct nglod_batch {
    int njobs = 0, ngroups = 0, decode = NGLOD_F32, in_dim = 32, ctas_per_sm = 0, want_normals = 0;
    int normal_mode = NGLOD_NORMALS_ANALYTIC;
    float fd_h = 0.f;
    bool f16 = false;
    float fp8_z = 0.f;
    nglod::TraceJob* d_jobs = nullptr;
    nglod::JobGroup* d_groups = nullptr;
    int* d_words = nullptr;            // [0, G) group queues, [G] status
    std::vector<nglod::TraceJob> h_jobs;
    std::vector<nglod_decoder> h_decs;
    std::vector<float*> normals;
    std::vector<bool> jobs_f16;
    int sms = 1;
};

namespace nglod {
namespace {

__global__ void k_batch_reset(TraceJob* __restrict__ jobs, int njobs, int* __restrict__ words, int nwords) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < njobs + nwords; i += gridDim.x * blockDim.x) {
        if (i < njobs) *jobs[i].A.hit_count = 0;
        else words[i - njobs] = 0;
    }
}

void destroy_batch(nglod_batch* b) {
    if (!b) return;
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_groups) cudaFree(b->d_groups);
    if (b->d_words) cudaFree(b->d_words);
    delete b;
}

}  // namespace
}  // namespace nglod

using namespace nglod;

extern "C" int sphere_trace_batch_create(const nglod_trace_job* jobs, int num_jobs, const nglod_trace_params* params,
                                         int ctas_per_sm, void* stream, nglod_batch** out) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!out) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_batch_create: out is NULL");
    *out = nullptr;
    if (!jobs || num_jobs < 1 || !params) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_batch_create: no jobs");
    if (!(params->eps > 0.0f) || !(params->far_t > 0.0f) || params->max_steps < 1)
        return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_batch_create: eps, far_t and max_steps must be positive");
    const int dec_t = params->decode_dtype;
    if (dec_t != NGLOD_F32 && dec_t != NGLOD_BF16 && dec_t != NGLOD_FP8E4M3)
        return fail(NGLOD_ERR_NOT_SUPPORTED, "sphere_trace_batch_create: decode_dtype");
    if (int e = check_normal_params(params, "sphere_trace_batch_create")) return e;
    nglod_batch* b = new (std::nothrow) nglod_batch();
    if (!b) return fail(NGLOD_ERR_OOM, "sphere_trace_batch_create: host allocation failed");
    b->decode = dec_t;
    b->ctas_per_sm = ctas_per_sm;
    b->want_normals = params->want_normals;
    b->normal_mode = params->normal_mode;
    b->fd_h = params->fd_h;
    b->sms = device_sms();
    // group jobs by decoder (W1 pointer), keeping first-seen order
    std::map<const float*, int> gid;
    std::vector<int> order_group;
    for (int j = 0; j < num_jobs; ++j) {
        if (!gid.count(jobs[j].dec.W1)) {
            const int g = (int)gid.size();
            gid[jobs[j].dec.W1] = g;
        }
    }
    const int G = (int)gid.size();
    std::vector<std::vector<int>> members(G);
    for (int j = 0; j < num_jobs; ++j) members[gid[jobs[j].dec.W1]].push_back(j);
    std::vector<JobGroup> groups(G);
    b->in_dim = jobs[0].dec.in_dim;
    b->f16 = jobs[0].feats.dtype == NGLOD_F16;
    int rc = NGLOD_OK;
    for (int g = 0; g < G && rc == NGLOD_OK; ++g) {
        JobGroup& gr = groups[g];
        gr.j0 = (int)b->h_jobs.size();
        long long base = 0;
        for (int j : members[g]) {
            const nglod_trace_job& J = jobs[j];
            if (!J.svo || J.R < 0 || J.R >= (1ll << 31) - 64 || (J.R > 0 && (!J.o || !J.d || !J.ray_offsets ||
                                                                            !J.t_hit || !J.hit || !J.work))) {
                rc = fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_batch_create: job " + std::to_string(j) + " is incomplete");
                break;
            }
            if (J.dec.in_dim != b->in_dim || (J.feats.dtype == NGLOD_F16) != b->f16) {
                rc = fail(NGLOD_ERR_NOT_SUPPORTED, "sphere_trace_batch_create: jobs must share in_dim and feature dtype");
                break;
            }
            if (J.work_bytes < sphere_trace_workspace(J.R) || ((uintptr_t)J.work & 255u)) {
                rc = fail(NGLOD_ERR_CAPACITY, "sphere_trace_batch_create: job workspace too small or unaligned");
                break;
            }
            TraceJob tj{};
            if ((rc = fill_tables(J.svo, &J.feats, J.lod, tj.tb))) break;
            if ((rc = check_decoder(&J.dec))) break;
            const int D = J.lod + kFirstFeatureDepth - 1;
            if (J.lod < 1 || D >= J.svo->num_depths) {
                rc = fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_batch_create: lod out of range");
                break;
            }
            TraceArgs& A = tj.A;
            A.o = J.o;
            A.d = J.d;
            A.R = J.R;
            A.D = D;
            A.eps = params->eps;
            A.far_t = params->far_t;
            A.max_steps = params->max_steps;
            A.osc = params->osc_check;
            A.offs = J.ray_offsets;
            A.vid = J.voxel_id;
            A.tr = (const float2*)J.t_range;
            A.t_hit = J.t_hit;
            A.hit = J.hit;
            A.steps = J.steps;
            A.queue = (int*)J.work;
            A.hit_count = (int*)J.work + 2;
            A.hit_vox = (int32_t*)((char*)J.work + trace_ws_hit_vox_offset());
            A.hit_list = (int32_t*)((char*)J.work + trace_ws_hit_list_offset(J.R));
            tj.ray_base = base;
            base += J.R;
            b->h_jobs.push_back(tj);
            b->h_decs.push_back(J.dec);
            b->normals.push_back(J.normal);
        }
        if (rc) break;
        // the group queue is a 32-bit counter that runs up to nrays + 32 per warp
        if (base > (1ll << 31) - (1ll << 24)) {
            rc = fail(NGLOD_ERR_NOT_SUPPORTED, "sphere_trace_batch_create: more than 2^31 - 2^24 rays per decoder group");
            break;
        }
        gr.j1 = (int)b->h_jobs.size();
        gr.nrays = base;
        const nglod_trace_job& J0 = jobs[members[g][0]];
        gr.W1 = J0.dec.W1;
        gr.b1 = J0.dec.b1;
        gr.W2 = J0.dec.W2;
        gr.b2 = J0.dec.b2;
        gr.z_scale = 1.0f;
        if (dec_t == NGLOD_FP8E4M3) {
            float zmax = 0.f;
            for (int j : members[g]) zmax = std::max(zmax, jobs[j].feats.fp8_z_absmax);
            if (!(zmax > 0.f)) {
                rc = fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_batch_create: FP8 decode needs feats.fp8_z_absmax");
                break;
            }
            gr.z_scale = 448.0f / zmax;
        }
    }
    if (rc) {
        destroy_batch(b);
        return rc;
    }
    b->njobs = (int)b->h_jobs.size();
    b->ngroups = G;
    cudaError_t e = cudaMalloc(&b->d_jobs, sizeof(TraceJob) * b->njobs);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_groups, sizeof(JobGroup) * G);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_words, sizeof(int) * (G + 1));
    if (e != cudaSuccess) {
        destroy_batch(b);
        return check_cuda(e, "sphere_trace_batch_create: cudaMalloc");
    }
    for (int g = 0; g < G; ++g) groups[g].queue = b->d_words + g;
    e = cudaMemcpyAsync(b->d_jobs, b->h_jobs.data(), sizeof(TraceJob) * b->njobs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_groups, groups.data(), sizeof(JobGroup) * G, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        destroy_batch(b);
        return check_cuda(e, "sphere_trace_batch_create: upload");
    }
    *out = b;
    return NGLOD_OK;
}

extern "C" int sphere_trace_batch_run(nglod_batch* b, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!b) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_batch_run: NULL batch");
    k_batch_reset<<<std::max(1, std::min((b->njobs + b->ngroups + 1 + 255) / 256, 64)), 256, 0, st>>>(
        b->d_jobs, b->njobs, b->d_words, b->ngroups + 1);
    NGLOD_CUDA(cudaGetLastError());
    int rc;
    if (b->decode == NGLOD_F32)
        rc = launch_trace_batch_f32(b->d_jobs, b->d_groups, b->ngroups, b->in_dim, b->f16, b->ctas_per_sm, b->sms, st);
    else
        rc = launch_trace_batch_tc(b->d_jobs, b->d_groups, b->ngroups, b->in_dim, b->f16, b->decode == NGLOD_FP8E4M3,
                                   b->ctas_per_sm, b->sms, b->d_words + b->ngroups, st);
    if (rc) return rc;
    if (b->want_normals) {
        for (int j = 0; j < b->njobs; ++j) {
            if (!b->normals[j] || b->h_jobs[j].A.R == 0) continue;
            rc = b->normal_mode == NGLOD_NORMALS_FD
                     ? launch_normals_fd(&b->h_decs[j], b->h_jobs[j].tb, b->h_jobs[j].A, b->fd_h, b->normals[j],
                                         b->f16, b->sms, st)
                     : launch_normals(&b->h_decs[j], b->h_jobs[j].tb, b->h_jobs[j].A, b->normals[j], b->f16,
                                      b->sms, st);
            if (rc) return rc;
        }
    }
    return NGLOD_OK;
}

extern "C" int sphere_trace_batch_status(nglod_batch* b, void* stream) {
    if (!b) return fail(NGLOD_ERR_INVALID_ARG, "sphere_trace_batch_status: NULL batch");
    int h = 0;
    NGLOD_CUDA(cudaMemcpyAsync(&h, b->d_words + b->ngroups, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    NGLOD_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (h == kStatusTimeout) return fail(NGLOD_ERR_TIMEOUT, "sphere_trace_batch: a tensor-core wait expired");
    return NGLOD_OK;
}

extern "C" void sphere_trace_batch_free(nglod_batch* b) { destroy_batch(b); }
