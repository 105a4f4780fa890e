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
#include "scan_common.cuh"
#include "trace_common.cuh"

struct nglod_batch {
    int njobs = 0, ngroups = 0, decode = NGLOD_F32, in_dim = 32, ctas_per_sm = 0, want_normals = 0;
    int normal_mode = NGLOD_NORMALS_ANALYTIC;
    float fd_h = 0.f;
    bool f16 = false;
    float fp8_z = 0.f;
    nglod::TraceJob* d_jobs = nullptr;
    nglod::JobGroup* d_groups = nullptr;
    int* d_words = nullptr;            // [0, G) group queues, [G] status, then G x kOrderBuckets counts
    int32_t* d_order = nullptr;        // per group: handout order of its 32-ray chunks
    uint8_t* d_keys = nullptr;         // per chunk: bucket of its longest list
    long long* d_gbase = nullptr;      // [G + 1] first chunk of each group (global chunk index)
    int* d_cursor = nullptr;           // G x kOrderBuckets
    long long nchunks = 0;
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
        if (i < njobs) {
            *jobs[i].A.hit_count = 0;
            // the batched tracers record the hits' masks (not for the FP8 decode)
            jobs[i].A.hit_count[kWsMaskFlagWord - 2] = jobs[i].A.hit_mask ? 1 : 0;
        }
        else words[i - njobs] = 0;
    }
}

void destroy_batch(nglod_batch* b) {
    if (!b) return;
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_groups) cudaFree(b->d_groups);
    if (b->d_words) cudaFree(b->d_words);
    if (b->d_order) cudaFree(b->d_order);
    if (b->d_keys) cudaFree(b->d_keys);
    if (b->d_gbase) cudaFree(b->d_gbase);
    if (b->d_cursor) cudaFree(b->d_cursor);
    delete b;
}

// Work-ordered handout inside each group (as in sphere_trace): every 32-ray
// chunk of a group's queue is keyed by its longest voxel list, and the
// chunks are counting-sorted longest first.  Chunk c of the batch lies in
// group g with gbase[g] <= c < gbase[g + 1]; its rays are those of the job
// whose (32-aligned) queue range holds it.
constexpr int kSmemGroups = 16;    // groups whose bucket counts a block keeps in shared memory

__device__ __forceinline__ int find_group(const long long* __restrict__ gbase, int G, long long c) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gbase[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_batch_keys(const TraceJob* __restrict__ jobs, const JobGroup* __restrict__ groups, int G,
                             const long long* __restrict__ gbase, long long nchunks, uint8_t* __restrict__ key,
                             int* __restrict__ hist) {
    __shared__ int h[kSmemGroups * kOrderBuckets];
    const int gs = min(G, kSmemGroups);
    for (int i = threadIdx.x; i < gs * kOrderBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += nw) {
        const int g = find_group(gbase, G, c);
        const long long gi = (c - gbase[g]) * 32;
        int lo = groups[g].j0, hi = groups[g].j1 - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].ray_base <= gi) lo = mid; else hi = mid - 1;
        }
        const TraceArgs& A = jobs[lo].A;
        const long long r = gi - jobs[lo].ray_base + lane;
        const int len = r < A.R ? (A.cnt ? A.cnt[r] : A.offs[r + 1] - A.offs[r]) : 0;
        const int m = __reduce_max_sync(0xffffffffu, len);
        if (lane == 0) {
            const int b = kOrderBuckets - 1 - min(max(m, 0), kOrderBuckets - 1);
            key[c] = (uint8_t)b;
            if (g < kSmemGroups) atomicAdd(&h[g * kOrderBuckets + b], 1);
            else atomicAdd(&hist[g * kOrderBuckets + b], 1);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < gs * kOrderBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One block per group: cursor = exclusive sum of its bucket counts.
__global__ void k_batch_order_scan(const int* __restrict__ hist, int* __restrict__ cursor) {
    __shared__ int ws[33];
    int total;
    const int i = blockIdx.x * kOrderBuckets + threadIdx.x;
    cursor[i] = block_exclusive_sum(hist[i], ws, total);
}

__global__ void k_batch_order_scatter(const long long* __restrict__ gbase, int G, long long nchunks,
                                      const uint8_t* __restrict__ key, int* __restrict__ cursor,
                                      int32_t* __restrict__ order) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < nchunks; c0 += stride) {
        const long long c = c0 + lane;
        const bool act = c < nchunks;
        const unsigned live = __ballot_sync(0xffffffffu, act);
        if (!act) continue;
        const int g = find_group(gbase, G, c);
        const int slot = g * kOrderBuckets + key[c];
        const unsigned peers = __match_any_sync(live, slot);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&cursor[slot], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        // the group's order array starts at its first chunk; entries are group-local chunks
        order[gbase[g] + base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)(c - gbase[g]);
    }
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
            // a summed corner table serves a trace with analytic normals (every
            // query inside a voxel of the job's LOD)
            if ((rc = fill_tables(J.svo, &J.feats, J.lod, tj.tb, b->normal_mode != NGLOD_NORMALS_FD))) break;
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
            A.cnt = J.ray_counts;
            A.vid = J.voxel_id;
            A.t_hit = J.t_hit;
            A.hit = J.hit;
            A.steps = J.steps;
            A.queue = (int*)J.work;
            A.hit_count = (int*)J.work + 2;
            A.hit_vox = (int32_t*)((char*)J.work + trace_ws_hit_vox_offset());
            A.hit_list = (int32_t*)((char*)J.work + trace_ws_hit_list_offset(J.R));
            A.wfrag = (uint2*)((char*)J.work + trace_ws_wfrag_offset(J.R));
            A.hit_mask = dec_t == NGLOD_FP8E4M3 ? nullptr : (uint4*)((char*)J.work + trace_ws_mask_offset(J.R));
            tj.ray_base = base;
            base += (J.R + 31) / 32 * 32;     // chunks of 32 never span two jobs
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
    std::vector<long long> gbase(G + 1, 0);
    for (int g = 0; g < G; ++g) gbase[g + 1] = gbase[g] + groups[g].nrays / 32;
    b->nchunks = gbase[G];
    cudaError_t e = cudaMalloc(&b->d_jobs, sizeof(TraceJob) * b->njobs);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_groups, sizeof(JobGroup) * G);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_words, sizeof(int) * (G + 1 + (size_t)G * kOrderBuckets));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_cursor, sizeof(int) * (size_t)G * kOrderBuckets);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_gbase, sizeof(long long) * (G + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int32_t) * std::max<long long>(1, b->nchunks));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_keys, std::max<long long>(1, b->nchunks));
    if (e != cudaSuccess) {
        destroy_batch(b);
        return check_cuda(e, "sphere_trace_batch_create: cudaMalloc");
    }
    for (int g = 0; g < G; ++g) {
        groups[g].queue = b->d_words + g;
        groups[g].order = b->d_order + gbase[g];
    }
    e = cudaMemcpyAsync(b->d_jobs, b->h_jobs.data(), sizeof(TraceJob) * b->njobs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_groups, groups.data(), sizeof(JobGroup) * G, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_gbase, gbase.data(), sizeof(long long) * (G + 1), cudaMemcpyHostToDevice, st);
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
    const int nwords = b->ngroups + 1 + b->ngroups * kOrderBuckets;
    k_batch_reset<<<std::max(1, std::min((b->njobs + nwords + 255) / 256, 64)), 256, 0, st>>>(
        b->d_jobs, b->njobs, b->d_words, nwords);
    NGLOD_CUDA(cudaGetLastError());
    if (b->nchunks > 0) {
        int* hist = b->d_words + b->ngroups + 1;
        const int gk = (int)std::max<long long>(1, std::min<long long>((b->nchunks + 7) / 8, (long long)b->sms * 4));
        k_batch_keys<<<gk, 256, 0, st>>>(b->d_jobs, b->d_groups, b->ngroups, b->d_gbase, b->nchunks, b->d_keys, hist);
        k_batch_order_scan<<<b->ngroups, kOrderBuckets, 0, st>>>(hist, b->d_cursor);
        const int gs = (int)std::max<long long>(1, std::min<long long>((b->nchunks + 255) / 256, (long long)b->sms * 4));
        k_batch_order_scatter<<<gs, 256, 0, st>>>(b->d_gbase, b->ngroups, b->nchunks, b->d_keys, b->d_cursor,
                                                   b->d_order);
        NGLOD_CUDA(cudaGetLastError());
    }
    int rc;
    if (b->decode == NGLOD_F32)
        rc = launch_trace_batch_f32(b->d_jobs, b->d_groups, b->ngroups, b->in_dim, b->f16, b->ctas_per_sm, b->sms, st);
    else
        rc = launch_trace_batch_tc(b->d_jobs, b->d_groups, b->ngroups, b->in_dim, b->f16, b->decode == NGLOD_FP8E4M3,
                                   b->ctas_per_sm, b->sms, b->d_words + b->ngroups, st);
    if (rc) return rc;
    // each job's hit list in ray order (A.queue is the start of the job's
    // trace workspace)
    for (int j = 0; j < b->njobs; ++j)
        if (b->h_jobs[j].A.R > 0 && (rc = enqueue_hit_order(b->h_jobs[j].A, b->h_jobs[j].A.queue, st))) return rc;
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
