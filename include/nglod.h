/*
 * libnglod -- C ABI of the Neural Geometric LOD rendering hot path on GB300.
 *
 * The method (Takikawa et al., "Neural Geometric Level of Detail", CVPR 2021)
 * stores a neural SDF as a sparse voxel octree (SVO) over [-1,1]^3 whose
 * voxels carry a feature vector at each of their 8 corners (shared between
 * neighbours), with one small MLP decoder per level of detail (Sec. 3.2).
 * Rendering intersects rays with the octree level by level (Sec. 3.4,
 * Algorithm 1; supplementary Sec. C) and then sphere-traces each ray through
 * its depth-ordered voxel list (Sec. 3.4, "Adaptive Ray Stepping").
 *
 * Conventions shared by every call:
 *  - Octree depth dp has resolution 2^dp; LOD l lives at depth l + 2
 *    (r_l = 4 * 2^l, supplementary Sec. A.1).  Depths 0..2 carry no features.
 *  - Voxel (i,j,k) at depth dp has the Morton key with bit b of i, j, k at
 *    bits 3b, 3b+1, 3b+2; a voxel id is the index of its key in the sorted key
 *    array of its depth.
 *  - Corner id: rank of the corner's Morton key (lattice (2^dp+1)^3) among the
 *    unique corner keys of that depth, ascending.  Features of LOD l are
 *    row-major [C_l, m] in corner-id order.
 *  - Pointers are DEVICE pointers unless their name starts with h_.  Every
 *    call is ordered on the given CUDA stream (a cudaStream_t passed as void*;
 *    NULL is the legacy default stream) and returns an int status; nothing
 *    throws across the ABI, nothing traps, and every device-side wait is
 *    bounded.  The text of the last error of the calling thread is returned
 *    by nglod_last_error().
 *  - Features and decoder weights are caller-owned.  The SVO handle owns its
 *    structure arrays.  Outputs are caller-owned with explicit capacities.
 */
#ifndef NGLOD_H
#define NGLOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    NGLOD_OK = 0,
    NGLOD_ERR_INVALID_ARG = 1,   /* bad pointer, size, LOD or octree         */
    NGLOD_ERR_CAPACITY = 2,      /* an output or workspace is too small      */
    NGLOD_ERR_CUDA = 3,          /* a CUDA runtime call failed               */
    NGLOD_ERR_OOM = 4,           /* device allocation failed                 */
    NGLOD_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired       */
    NGLOD_ERR_NOT_SUPPORTED = 6  /* shape or dtype outside what is built     */
};

/* Element types of features / decode arithmetic. */
enum { NGLOD_F32 = 0, NGLOD_F16 = 1, NGLOD_BF16 = 2, NGLOD_FP8E4M3 = 3, NGLOD_F32_SPLIT = 4 };

typedef struct nglod_svo nglod_svo;   /* opaque octree handle */

/* Corner features of LODs 1..num_lods (Sec. 3.2: z_V^(j) in R^m, shared). */
typedef struct {
    const void* feats[8];  /* feats[l-1]: [C_l, m] row-major, dtype below;
                              32-byte aligned (FP32) or 16-byte (FP16), else
                              NGLOD_ERR_INVALID_ARG                          */
    int dtype;             /* NGLOD_F32 or NGLOD_F16                         */
    int m;                 /* feature dimension; only 32 is built            */
    int num_lods;          /* number of valid entries in feats               */
    float fp8_z_absmax;    /* FP8 decode only: a bound on |z| (e.g. from
                              nglod_features_absmax); z is scaled so this
                              bound maps to 448, the largest e4m3 value     */
    int summed_lod;        /* 0: feats[l-1] are the per-LOD tables Z_l of
                              Eq. 2's sum.  L >= 1: feats[L-1] is the
                              summed corner table of LOD L written by
                              nglod_sum_features (dtype NGLOD_F32) and the
                              other entries are ignored; only sphere_trace
                              and sphere_trace_batch_create (analytic or no
                              normals), trace_normals and
                              nglod_features_absmax at lod = L accept it,
                              every other call returns
                              NGLOD_ERR_NOT_SUPPORTED                        */
} nglod_features;

/* One LOD's decoder (Eq. 2): d = W2 . relu(W1 v + b1) + b2 with
 * v = [x, z] (in_dim = m + 3) or v = z (in_dim = m).  FP32 master weights;
 * the BF16 decode rounds W1 and z to bf16 (round-to-nearest-even) and
 * accumulates in FP32.  Every parameter, b2 included, is read from device
 * memory by the kernels when they run, so an optimiser step that updates
 * them in place (nglod_adam_step) reaches the next call, or the next replay
 * of a captured CUDA graph, without any host copy.  NULL pointers are
 * NGLOD_ERR_INVALID_ARG. */
typedef struct {
    const float* W1;       /* [hidden, in_dim] row-major (device)             */
    const float* b1;       /* [hidden] (device)                               */
    const float* W2;       /* [hidden] (device)                               */
    const float* b2;       /* one float (device)                              */
    int in_dim;            /* 32 or 35                                        */
    int hidden;            /* only 128 is built                               */
} nglod_decoder;

/* Sphere-tracing parameters (supplementary Sec. A.4). */
typedef struct {
    float eps;             /* stop when d < eps (the paper uses 3e-4)         */
    float far_t;           /* miss when t > far_t (the paper uses 5)          */
    int max_steps;         /* miss after this many decodes (paper: 200)       */
    int osc_check;         /* 1: also stop when |d_k - d_(k-1)| < 6 eps; the
                              ray is then a hit iff |d_k| < 6 eps             */
    int decode_dtype;      /* NGLOD_F32 (CUDA cores), NGLOD_BF16,
                              NGLOD_FP8E4M3 or NGLOD_F32_SPLIT (tensor cores,
                              numerics as sdf_query; the tracers decode BF16
                              and F32_SPLIT per warp with mma.sync, FP8 and
                              blending on tcgen05)                          */
    int want_normals;      /* 1: write normals of hit rays                    */
    int normal_mode;       /* NGLOD_NORMALS_ANALYTIC (0): normalised analytic
                              gradient of the decoded SDF (FP32);
                              NGLOD_NORMALS_FD (1): central differences, the
                              form supplementary Sec. A.4 names -- the SDF
                              evaluated as sdf_query does (FP32 decode) at
                              x +- fd_h e_a and n = normalise of the three
                              differences                                  */
    float fd_h;            /* FD step in scene units, in (0, 1) (FD only)     */
    int ctas_per_sm;       /* persistent trace CTAs per SM (0: the most that
                              fit -- 4 for the tensor-core decodes, 2 for
                              FP32); fewer leave room on each SM for
                              concurrent kernels of other streams (0..4)    */
    const int32_t* ray_counts; /* NULL: the lists are CSR (ray_offsets has
                              R + 1 entries).  Else the lists as
                              svo_trace_rays_staged_async left them: ray i's
                              entries are voxel_id[ray_offsets[i] ..
                              ray_offsets[i] + ray_counts[i]) (device, R
                              int32 each; sphere_trace and
                              sphere_trace_blend; batches take theirs per
                              job, nglod_trace_job.ray_counts)             */
} nglod_trace_params;

#define NGLOD_NORMALS_ANALYTIC 0
#define NGLOD_NORMALS_FD 1

/* nglod_features_absmax -- the sum over LODs 1..lod of each feature table's
 * largest |value|, written to *h_out (synchronises).  The trilinear weights
 * are non-negative and sum to 1, so this bounds every |z_k(x; lod)|: the
 * natural fp8_z_absmax for decoding at that LOD.  For a summed table
 * (summed_lod = lod) it is that table's largest |value|. */
int nglod_features_absmax(const nglod_svo* svo, const nglod_features* feats, int lod, float* h_out,
                          void* stream);

/* nglod_sum_features -- the summed corner table of LOD `lod` (Sec. 3.2,
 * Eq. 2's z = sum over LODs 1..lod of the trilinear interpolants psi_l).
 * Inside one voxel V of LOD `lod` every coarser psi_l is trilinear too (V lies
 * in one voxel of each coarser level, whose interpolant is a product of
 * affine functions of x), so their sum equals the trilinear interpolation of
 * its own values at V's 8 corners.  out[c] = that sum at corner c of LOD
 * `lod` (the interpolants of the coarser levels are continuous across voxel
 * faces, so every voxel sharing the corner gives the same value): a render
 * then gathers 8 rows per query instead of 8 per level.  Only points inside
 * voxels of LOD `lod` may be queried through the table, which is what the
 * sphere tracer and its analytic normals do.
 *   feats   per-LOD tables (summed_lod = 0), F32 or F16
 *   out     device [C_lod, 32] FP32 (svo_info's corner count), 32-byte
 *           aligned; every row is written
 * The interpolation weights at the corners are exact dyadic numbers (exact
 * in FP32 up to LOD 8); each row is accumulated with the rounding errors of
 * every product and sum kept (an FP32 pair, levels in order 1..lod, corners
 * in index order) and rounded once, so the table is the same whichever
 * voxel a shared corner is computed from.
 * Stream-ordered, no synchronisation.
 * NGLOD_ERR_INVALID_ARG for NULL pointers, lod outside 1..svo's LODs or
 * features not covering lod; NGLOD_ERR_NOT_SUPPORTED for summed input. */
int nglod_sum_features(const nglod_svo* svo, const nglod_features* feats, int lod, float* out, void* stream);

/* Text of the calling thread's last error ("" if none). */
const char* nglod_last_error(void);

/* nglod_set_wait_polls -- the poll budget of the bounded wait each tcgen05
 * kernel (the BF16 / FP8 / FP32-split decodes of sdf_query, the FP8 decode
 * of sphere_trace and batches, sphere_trace_blend, sdf_query_blend, and the
 * tensor-core adjoint) takes on the completion of every tile's MMA.  The
 * BF16 and FP32-split decodes of sphere_trace and the BF16 batches run
 * warp-level MMAs, which complete in the issuing warp: no wait, no budget.
 * The paper has no counterpart: this is a testing hook for the expiry path.
 * polls >= 0 sets the budget of every launch that follows, process-wide
 * (0: every such wait expires at once, so the call reports
 * NGLOD_ERR_TIMEOUT without any GPU fault or hang); polls < 0 restores the
 * default (2^24 polls, tens of milliseconds).  After an expiry a kernel
 * raises its status word, waits for its MMA in flight with the default
 * budget, frees its tensor memory and returns; outputs of that call are
 * unspecified, and a later call with the default budget is unaffected.
 * Always returns NGLOD_OK. */
int nglod_set_wait_polls(int64_t polls);

/* svo_build -- Sec. 3.2 (SVO over [-1,1]^3, corner features shared between
 * neighbours) and Sec. 3.4 ("pointers ... precalculated in an initialization
 * step by iterating over all voxels").
 *   h_keys[dp]   host array of h_counts[dp] Morton keys of depth dp, strictly
 *                increasing; depth 0 must be exactly {0}; every key's parent
 *                (key >> 3) must exist at depth dp-1.
 *   num_depths   Dmax + 1, with 4 <= num_depths <= 11 (LOD 1..8).
 * Builds on the device: per-voxel packed coordinates, parent index, child
 * mask and first-child index, and for depths >= 3 the 8 corner ids per voxel
 * (deduplicated corners).  On success *out owns that memory (svo_free).
 * Errors: NGLOD_ERR_INVALID_ARG for a malformed octree (nothing allocated
 * survives), NGLOD_ERR_OOM / NGLOD_ERR_CUDA.  Synchronises the stream. */
int svo_build(const uint64_t* const* h_keys, const int64_t* h_counts,
              int num_depths, void* stream, nglod_svo** out);

/* Sizes of a built octree: h_voxels[dp] for dp < num_depths and
 * h_corners[l-1] for LOD l = 1..num_depths-3 (either array may be NULL). */
int svo_info(const nglod_svo* svo, int* h_num_depths, int64_t* h_voxels,
             int64_t* h_corners);

/* Device arrays owned by the handle, for inspection: per voxel of depth dp,
 * Node {uint32 ijk packed i | j<<10 | k<<20, int32 childbase, uint32
 * childmask, int32 parent} (16 B each) and, for dp >= 3, int32 corner ids
 * [V, 8] (corner c = cx | cy<<1 | cz<<2).  Pointers stay valid until
 * svo_free.  corners is set to NULL for dp < 3. */
int svo_device_arrays(const nglod_svo* svo, int dp, const void** node,
                      const int32_t** corners);

/* Copies depth dp's arrays to host memory (synchronous): h_node [V, 4] int32
 * Node records as above, h_corners [V, 8] and h_anc [V, 8] int32 (the voxel
 * ids at depths 3..dp containing each voxel, -1 beyond dp; dp >= 3 only).
 * Any output may be NULL. */
int svo_read_arrays(const nglod_svo* svo, int dp, void* h_node, int32_t* h_corners,
                    int32_t* h_anc);

/* Releases the handle and its device memory (NULL is allowed). */
void svo_free(nglod_svo* svo);

/* Workspace bytes svo_trace_rays needs for R rays and a staging list of
 * pair_capacity entries: a counter block, a 16-byte record per tile of 128
 * rays, one count per ray and 12 bytes per staged entry (the intermediate
 * per-level ray/voxel lists never leave on-chip memory). */
size_t svo_trace_rays_workspace(int64_t R, int64_t pair_capacity);

/* svo_trace_rays -- Algorithm 1 (RayTraceOctree) with Decide, ExclusiveSum,
 * Subdivide and Compactify of supplementary Sec. C, level by level from the
 * root down to depth target_lod + 2.  Front-to-back child order: rank
 * r = 0..7 visits child slot r XOR o, o = octant of the ray origin relative to
 * the voxel centre (bit a set iff origin_a >= centre_a).  Slab tests are FP32
 * round-to-nearest without contraction; a box is hit iff
 * max(t_near, 0) <= t_far (closed intervals).  A ray with a NaN/Inf component
 * or an all-zero direction hits nothing; a direction component below FLT_MIN
 * in magnitude makes that axis parallel.
 * The levels run per tile of 128 consecutive rays inside one persistent
 * kernel, each tile's frontier in shared memory (Decide, the block-wide
 * ExclusiveSum and Subdivide on chip; a tile whose frontier outgrows it
 * continues from its last level that fits in chunks of whole rays).  Tiles
 * stage their entries in any order;
 * a scan of the tile counts then places them in ray order, so the result
 * equals the global level-by-level sequence entry for entry.
 *   o, d          [R, 3] float32 origins / directions (device).
 *   work          device workspace of work_bytes >= svo_trace_rays_workspace(
 *                 R, pair_capacity); contents are scratch.
 *   pair_capacity staging-list capacity (entries); must be >= H.
 * Outputs (CSR over rays, grouped by ray, front to back within a ray):
 *   ray_offsets   [R + 1] int32; hits of ray i are [ray_offsets[i],
 *                 ray_offsets[i+1]).
 *   voxel_id      [hit_capacity] int32 voxel ids at the target depth.
 *   t_range       [hit_capacity, 2] float32 (t_enter, t_exit) per hit, or
 *                 NULL: not written (the tracers recompute each entry's
 *                 interval from its voxel with the same FP32 slab test).
 *   h_stats       host int64[2] (nullable): [0] = total hits H, [1] = largest
 *                 number of pairs Decide kept at any depth.
 * Errors: NGLOD_ERR_CAPACITY if H > hit_capacity or H > pair_capacity
 * (h_stats[0] then holds the H needed; outputs are unspecified);
 * NGLOD_ERR_INVALID_ARG.  No kernel waits on another.  Synchronises the
 * stream (to read H). */
int svo_trace_rays(const nglod_svo* svo, const float* o, const float* d, int64_t R,
                   int target_lod, void* work, size_t work_bytes, int64_t pair_capacity,
                   int32_t* ray_offsets, int32_t* voxel_id, float* t_range,
                   int64_t hit_capacity, int64_t* h_stats, void* stream);

/* svo_trace_rays_noalloc -- svo_trace_rays without a caller workspace and
 * without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they
 * render, such as a plugin inside an application that owns the GPU memory
 * budget, or a real-time loop that must not trigger the implicit
 * synchronisation of cudaMalloc/cudaFree mid-frame.
 * The workspace is a 32 MiB array built into the library, present on every
 * GPU that loads it until the process exits.  The first call on a device
 * (with that device current) looks up the array's device address; make it
 * before any stream capture.  Later calls outside a capture look it up again
 * (so a cudaDeviceReset, after which the array may move, is followed by a
 * fresh lookup); calls inside a capture reuse the last address found on that
 * device.  The staging capacity is whatever fits in
 * 32 MiB after the per-ray and per-tile records (about 2.1 M entries at
 * 2 M rays); R whose records alone exceed it is rejected with
 * NGLOD_ERR_CAPACITY before anything is read or launched, and more entries
 * than the staging capacity return NGLOD_ERR_CAPACITY like svo_trace_rays.
 * Every call reuses
 * the same array (counters and scan state are cleared at the start of each
 * call); calls that overlap on the GPU race on it.  Arguments, outputs,
 * results and the stream synchronisation are those of svo_trace_rays. */
int svo_trace_rays_noalloc(const nglod_svo* svo, const float* o, const float* d, int64_t R,
                           int target_lod, int32_t* ray_offsets, int32_t* voxel_id,
                           float* t_range, int64_t hit_capacity, int64_t* h_stats,
                           void* stream);

/* svo_trace_rays_async -- svo_trace_rays without the final host read-back,
 * so the whole traversal is enqueued on the stream and can be captured in a
 * CUDA graph.  The caller sizes pair_capacity and hit_capacity (e.g. from
 * an earlier svo_trace_rays of the same frame); overflow is
 * recorded in the workspace and reported by svo_trace_rays_check, and the
 * outputs are then unspecified.  Arguments as svo_trace_rays. */
int svo_trace_rays_async(const nglod_svo* svo, const float* o, const float* d, int64_t R,
                         int target_lod, void* work, size_t work_bytes, int64_t pair_capacity,
                         int32_t* ray_offsets, int32_t* voxel_id, float* t_range,
                         int64_t hit_capacity, void* stream);

/* svo_trace_rays_async_width -- svo_trace_rays_async with the persistent
 * traversal kernel launched at ctas_per_sm resident CTAs per SM (1..4; 0:
 * the most that fit, as svo_trace_rays_async).  A traversal CTA holds ~56 KB
 * of shared memory, so at the full width no tracer CTA of a concurrent
 * stream fits beside it; a narrower traversal leaves room on every SM for
 * another stream's sphere trace (the frame renderer tunes this).  Changes
 * only the schedule: the lists are identical.  NGLOD_ERR_INVALID_ARG for
 * ctas_per_sm outside 0..4; otherwise as svo_trace_rays_async. */
int svo_trace_rays_async_width(const nglod_svo* svo, const float* o, const float* d, int64_t R,
                               int target_lod, void* work, size_t work_bytes, int64_t pair_capacity,
                               int32_t* ray_offsets, int32_t* voxel_id, float* t_range,
                               int64_t hit_capacity, int ctas_per_sm, void* stream);

/* svo_trace_rays_staged_async -- svo_trace_rays_async without its placement
 * pass: the lists stay where the persistent traversal staged them in the
 * workspace (each ray's entries contiguous and front to back, the same
 * entries as the CSR lists; the rays' lists in no particular order), so the
 * traversal is one launch.  The paper's Compactify writes CSR; this form
 * exists for the renderers, whose tracers read a ray's list by its first
 * entry and count (nglod_trace_params.ray_counts, nglod_trace_job.ray_counts).
 * After a staging overflow a ray whose list did not fit whole gets count 0,
 * so a tracer reads only written entries.
 *   svo, o, d, R, target_lod, work, work_bytes, pair_capacity, ctas_per_sm
 *                 as svo_trace_rays_async_width.
 *   ray_first, ray_count, voxel_id  host pointers that receive device
 *                 addresses inside work: [R] int32 index of each ray's first
 *                 entry in voxel_id, [R] int32 its entry count, and the
 *                 [pair_capacity] int32 staged voxel ids.  Valid until the
 *                 workspace is reused.
 * Overflow of pair_capacity is reported by svo_trace_rays_check (outputs
 * then unspecified).  NGLOD_ERR_INVALID_ARG as svo_trace_rays_async_width.
 * Does not synchronise. */
int svo_trace_rays_staged_async(const nglod_svo* svo, const float* o, const float* d, int64_t R,
                                int target_lod, void* work, size_t work_bytes, int64_t pair_capacity,
                                int ctas_per_sm, const int32_t** ray_first, const int32_t** ray_count,
                                const int32_t** voxel_id, void* stream);

/* svo_trace_rays_check -- synchronises and reports the status of the last
 * traversal enqueued in this workspace (as svo_trace_rays would have): OK,
 * NGLOD_ERR_CAPACITY (h_stats = sizes needed) or NGLOD_ERR_TIMEOUT. */
int svo_trace_rays_check(const void* work, int target_lod, int64_t* h_stats, void* stream);

/* svo_trace_rays_sizes -- list sizes of the last svo_trace_rays that used this
 * workspace (synchronises the stream): h_sizes[dp] for dp = 0..n-1 is the
 * number of ray/voxel pairs at depth dp that Decide kept (dp = 0: rays whose
 * ray hits the root is not yet tested, i.e. R), the last entry being the
 * final hit count.  n <= 12. */
int svo_trace_rays_sizes(const void* work, int64_t* h_sizes, int n, void* stream);

/* sdf_query -- Sec. 3.2 and Eq. 2: for each point x, the voxels containing it
 * at depths 3..lod+2 (found from the root through the child masks using
 * q = fl32(x + 1), ijk = clamp(floor(q 2^(dp-1)), 0, 2^dp - 1)); per level the
 * trilinear interpolation psi of the 8 corner features with weights from
 * u = clamp(q 2^(dp-1) - ijk, 0, 1); z = sum of psi over levels; then the
 * decoder of that LOD.  A level whose voxel is absent (and every deeper one)
 * contributes 0; points outside [-1,1]^3 see z = 0.
 *   x         [Q, 3] float32.   sdf  [Q] float32 output.
 *   deepest   [Q] int8 (nullable): deepest LOD with a containing voxel (0 none).
 *   grad      [Q, 3] float32 (nullable): analytic d sdf / dx (FP32 decode).
 *   decode_dtype  NGLOD_F32 (CUDA cores) or NGLOD_BF16 (tensor cores: z and
 *                 W1's z columns rounded to bf16, FP32 accumulation; the
 *                 x columns, biases and W2 stay FP32) or NGLOD_FP8E4M3
 *                 (tensor cores: z scaled by 448 / feats->fp8_z_absmax and
 *                 W1's z columns by 448 / their largest |value| (a per-LOD
 *                 scale), both rounded to e4m3, FP32 accumulation, scales
 *                 undone before the bias) or NGLOD_F32_SPLIT (tensor cores
 *                 at FP32 accuracy: z and W1's z columns each split into
 *                 three BF16 terms, x = x0 + x1 + x2 exactly to 24 bits,
 *                 and the six products x_i w_j with i + j <= 2 accumulated
 *                 in FP32; not for level blending or batches).
 * Errors: NGLOD_ERR_INVALID_ARG (lod outside 1..num_depths-3, missing
 * features), NGLOD_ERR_NOT_SUPPORTED (m != 32, hidden != 128, in_dim not 32 or
 * 35, grad with BF16 decode), NGLOD_ERR_TIMEOUT (a bounded tensor-core wait
 * expired).  The FP32 decode does not synchronise; the BF16 decode
 * synchronises the stream to read its status. */
int sdf_query(const nglod_svo* svo, const nglod_features* feats,
              const nglod_decoder* dec, const float* x, int64_t Q, int lod,
              int decode_dtype, float* sdf, int8_t* deepest, float* grad,
              void* stream);

/* Workspace bytes sphere_trace needs for R rays. */
size_t sphere_trace_workspace(int64_t R);

/* sphere_trace -- Sec. 3.4 (Adaptive Ray Stepping) with the stopping rules
 * of supplementary Sec. A.4.  Per ray, with its list from svo_trace_rays at
 * the same LOD: t starts at the first entry; each iteration advances the
 * list cursor past entries with t_exit < t (the ray misses when the list runs
 * out), moves t up to the current entry's t_enter, queries the SDF at
 * x = o + t d from that voxel and its ancestors, and counts one step; d < eps
 * is a hit, otherwise t += d; t > far_t or max_steps reached is a miss.
 *   o, d, R, lod        as for svo_trace_rays (same rays, same LOD).
 *   ray_offsets, voxel_id   the CSR lists of svo_trace_rays, or with
 *                       params->ray_counts the staged lists of
 *                       svo_trace_rays_staged_async (ray_offsets = its
 *                       ray_first).
 *   t_range             not read (may be NULL): each entry's [t_enter,
 *                       t_exit] is recomputed from its voxel by the slab
 *                       test svo_trace_rays uses, which gives the same bits.
 *   work                device workspace >= sphere_trace_workspace(R).  After
 *                       the call, bytes [256, 256 + 4R) hold the int32 id (at
 *                       the target depth) of the voxel each hit ray stopped in,
 *                       -1 for misses, and int32 word 2 counts the hit rays,
 *                       whose ids follow (in increasing order, so that the
 *                       normals visit neighbouring hits together) from byte
 *                       256 + 4R rounded up to 256; trace_normals reads them.
 *                       The rest holds the order in which 32-ray groups are
 *                       handed to the persistent trace (by decreasing longest
 *                       list, so long rays start early; it changes only the
 *                       schedule, never a ray's outputs), per ray the ReLU
 *                       mask of a hit's last decode
 *                       (128 bits), which trace_normals reuses (not with the
 *                       FP8 decode, whose 4-bit z can zero or flip a
 *                       pre-activation: its normals recompute the forward
 *                       pass in FP32), and last the normals' scratch (their
 *                       masked-sum operand, 30 KB).
 * Outputs: t_hit [R] (+inf on miss), hit [R] uint8, steps [R] int32
 * (nullable: decodes taken), normal [R, 3] (nullable; normalised analytic
 * gradient of the decoded SDF at the hit point in FP32, or its central
 * differences with params->normal_mode = NGLOD_NORMALS_FD; zero on miss).
 * Errors: as sdf_query, plus NGLOD_ERR_INVALID_ARG for bad params.  Does not
 * synchronise. */
int sphere_trace(const nglod_svo* svo, const nglod_features* feats,
                 const nglod_decoder* dec, const float* o, const float* d, int64_t R,
                 int lod, const nglod_trace_params* params, const int32_t* ray_offsets,
                 const int32_t* voxel_id, const float* t_range, void* work,
                 size_t work_bytes, float* t_hit, uint8_t* hit, int32_t* steps,
                 float* normal, void* stream);

/* sdf_backward -- gradients of  sum_i sum_q grad_sdf[i][q] * sdf_(L_i)(x_q),
 * the adjoint of the per-LOD sum of Eq. 4 (Sec. 3.3: "summing them across
 * levels" trains every LOD's decoder and the shared features jointly), for
 * the LODs L_1 < L_2 < ... selected by lod_mask (bit L-1 selects LOD L).
 *   decs          host array of num_lods decoders (index L-1; only the
 *                 selected ones are read), FP32 weights on the device.
 *   x             [Q, 3] points; grad_sdf [popcount(lod_mask), Q] (row i for
 *                 the i-th selected LOD, increasing).
 *   h_grad_feats  host array of device pointers, [C_l, 32] FP32 per LOD
 *                 l = 1..highest selected LOD; ACCUMULATED (+=).
 *   h_grad_W1/_b1/_W2  host arrays (index L-1) of device pointers, shapes as
 *                 the decoder, accumulated; grad_b2 device [num_lods], acc.
 *   grad_x        [Q, 3] accumulated, nullable.
 *   deterministic 0: feature and weight gradients are summed with FP32
 *                 atomics, so their rounding order varies between runs.
 *                 1: every contribution is summed exactly in 128-bit fixed
 *                 point (quantum 2^-64; contributions below 2^-41 in
 *                 magnitude lose their bits under 2^-64; sums must stay
 *                 below 2^63) and each sum is rounded once to FP32, so
 *                 feature gradients are bit-identical between runs and
 *                 launch shapes, and decoder gradients between runs on one
 *                 device.  A non-finite contribution makes every gradient
 *                 output of the call NaN.  Allocates its accumulators
 *                 stream-ordered (16 B per gradient element) and frees
 *                 them before returning; NGLOD_ERR_CUDA if that fails.
 * Interpolation weights are recomputed from x, never stored.  Errors as
 * sdf_query.  Does not synchronise. */
int sdf_backward(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs,
                 const float* x, int64_t Q, uint32_t lod_mask, const float* grad_sdf,
                 float* const* h_grad_feats, float* const* h_grad_W1, float* const* h_grad_b1,
                 float* const* h_grad_W2, float* grad_b2, float* grad_x, int deterministic,
                 void* stream);

/* sdf_l2_backward -- one training step's gradients for the loss of Eq. 4,
 * J = loss_scale * sum_L sum_q (sdf_L(x_q) - target_q)^2 over the LODs in
 * lod_mask, computed in one pass per LOD (prediction, residual and adjoint
 * together; no separate forward launch).  loss (device [num_lods], nullable)
 * accumulates sum_q (sdf_L(x_q) - target_q)^2 per LOD.  Gradient buffers and
 * errors as sdf_backward (no x gradient).  Does not synchronise. */
int sdf_l2_backward(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs,
                    const float* x, const float* target, int64_t Q, uint32_t lod_mask,
                    float loss_scale, float* loss, float* const* h_grad_feats,
                    float* const* h_grad_W1, float* const* h_grad_b1, float* const* h_grad_W2,
                    float* grad_b2, void* stream);

/* sdf_backward_bf16 / sdf_l2_backward_bf16 -- the gradients of sdf_backward
 * and sdf_l2_backward (same arguments, same accumulation into the gradient
 * buffers) with the decoder's three contractions -- the pre-activations
 * v W1^T, gz = dpre W1 and dW1 = dpre^T v over 128-query tiles -- on the
 * tensor cores with BF16 operands and FP32 accumulation (mixed-precision
 * training; v = [z | x] and dpre rounded to BF16, W1's x columns, b1, W2,
 * the ReLU masks, the loss and every sum over queries other than dW1 in
 * FP32).  No x gradient and no deterministic mode (use sdf_backward).
 * Synchronises the stream to read its status: NGLOD_ERR_TIMEOUT if a
 * bounded tensor-core wait expired (the gradients are then incomplete). */
int sdf_backward_bf16(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs,
                      const float* x, int64_t Q, uint32_t lod_mask, const float* grad_sdf,
                      float* const* h_grad_feats, float* const* h_grad_W1, float* const* h_grad_b1,
                      float* const* h_grad_W2, float* grad_b2, void* stream);
int sdf_l2_backward_bf16(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* decs,
                         const float* x, const float* target, int64_t Q, uint32_t lod_mask,
                         float loss_scale, float* loss, float* const* h_grad_feats,
                         float* const* h_grad_W1, float* const* h_grad_b1, float* const* h_grad_W2,
                         float* grad_b2, void* stream);

/* nglod_sort_points -- reorders Q points by the Morton code of the depth-
 * `depth` octree cell (1 <= depth <= 7) containing them (a counting sort;
 * the order inside a cell is unspecified), so that neighbouring samples of
 * a training batch share voxels and corner rows.  x [Q, 3] -> x_out; extra
 * [Q] (nullable, e.g. the SDF targets) -> extra_out; perm [Q] (nullable)
 * receives the source index of each output point.  Outputs must not alias
 * inputs.  work: device buffer of nglod_sort_points_workspace(Q, depth)
 * bytes (4 Q + 2 x 4 x 8^depth bytes and change).  Eq. 4 sums over the
 * samples, so sorting a batch changes its gradients only by FP32 rounding
 * order.  Does not synchronise. */
size_t nglod_sort_points_workspace(int64_t Q, int depth);
int nglod_sort_points(const float* x, const float* extra, int64_t Q, int depth, float* x_out,
                      float* extra_out, int32_t* perm, void* work, size_t work_bytes, void* stream);

/* nglod_adam_step -- Adam (the optimiser of supplementary Sec. A.3) on n FP32
 * parameters: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps); grad is then
 * zeroed.  step counts from 1.  Does not synchronise. */
int nglod_adam_step(float* param, float* grad, float* m, float* v, int64_t n, float lr,
                    float beta1, float beta2, float eps, int step, void* stream);

/* sphere_trace_status -- synchronises the stream and reports whether the
 * last sphere_trace (or sphere_trace_blend) that used this workspace
 * completed: NGLOD_OK, or NGLOD_ERR_TIMEOUT if a bounded wait of a tcgen05
 * decode (FP8, blending) expired (its outputs are then invalid). */
int sphere_trace_status(const void* work, void* stream);

/* ---- Continuous LOD: level blending (Sec. 3.2, Eq. 3) ---------------------
 * For a continuous LOD L~ in [1, max lod], L* = floor(L~) and
 * alpha = L~ - L* (exact in FP32); the blended distance is
 *   d_L~(x) = (1 - alpha) d_L*(x) + alpha d_(L*+1)(x),
 * each term the query of sdf_query at that LOD (feature sum over the depths
 * 3..L+2 that contain x, absent levels contributing 0, then that LOD's
 * decoder).  dec_lo is LOD L*'s decoder, dec_hi LOD L*+1's (same in_dim;
 * dec_hi is not read when alpha = 0).  alpha = 0 is exactly the plain call
 * at L*.  Blending runs with decode_dtype NGLOD_F32 or NGLOD_BF16 (the
 * FP8 decode only at alpha = 0). */

/* sdf_query_blend -- d_L~ at Q points x [Q, 3] into sdf [Q].  Errors as
 * sdf_query, plus NGLOD_ERR_INVALID_ARG for L~ outside [1, max lod] and
 * NGLOD_ERR_NOT_SUPPORTED for decoders of different in_dim.  The FP32
 * decode does not synchronise; the BF16 decode synchronises to read its
 * status. */
int sdf_query_blend(const nglod_svo* svo, const nglod_features* feats,
                    const nglod_decoder* dec_lo, const nglod_decoder* dec_hi,
                    const float* x, int64_t Q, float lod_tilde, int decode_dtype,
                    float* sdf, void* stream);

/* sphere_trace_blend -- sphere_trace (Sec. 3.4 / A.4 stepping) of the
 * blended field d_L~.  The lists (ray_offsets, voxel_id; t_range is not
 * read and may be NULL) are those of svo_trace_rays at LOD ceil(L~): at L* + 1 when alpha > 0 (rays walk the
 * finer voxels, inside which both terms are defined; every step decodes
 * both LODs at the same point), at L* when alpha = 0 (the plain trace).
 * normal: the normalised blend (1 - alpha) grad d_L* + alpha grad d_(L*+1)
 * at the hit point.  Other arguments, outputs, workspace layout and errors
 * as sphere_trace.  Does not synchronise. */
int sphere_trace_blend(const nglod_svo* svo, const nglod_features* feats,
                       const nglod_decoder* dec_lo, const nglod_decoder* dec_hi,
                       const float* o, const float* d, int64_t R, float lod_tilde,
                       const nglod_trace_params* params, const int32_t* ray_offsets,
                       const int32_t* voxel_id, const float* t_range, void* work,
                       size_t work_bytes, float* t_hit, uint8_t* hit, int32_t* steps,
                       float* normal, void* stream);

/* nglod_lod_select -- the LOD selection of Sec. 3.4: L~ moves linearly
 * with the distance to the object, from lod_near at distance <= d_near to
 * lod_far at distance >= d_far (clamped outside; a step at d_near when
 * d_far <= d_near).  Host function, no device work. */
float nglod_lod_select(float distance, float d_near, float d_far, float lod_near, float lod_far);

/* One image of a batch: an octree with its features and the decoder of the
 * LOD it is traced at, its rays and their lists (svo_trace_rays at that LOD),
 * a trace workspace (>= sphere_trace_workspace(R)) and its outputs. */
typedef struct {
    const nglod_svo* svo;
    nglod_features feats;
    nglod_decoder dec;        /* jobs with the same dec.W1 pointer share one group */
    int lod;
    const float* o;
    const float* d;
    int64_t R;
    const int32_t* ray_offsets;
    const int32_t* voxel_id;
    const float* t_range;     /* not read (may be NULL), as for sphere_trace */
    void* work;
    size_t work_bytes;
    float* t_hit;
    uint8_t* hit;
    int32_t* steps;           /* nullable */
    float* normal;            /* nullable */
    const int32_t* ray_counts; /* NULL: CSR lists; else the staged lists of
                                  svo_trace_rays_staged_async (ray_offsets =
                                  its ray_first), as nglod_trace_params */
} nglod_trace_job;

typedef struct nglod_batch nglod_batch;   /* opaque */

/* sphere_trace_batch_create -- fixes a batch of jobs (their buffers must stay
 * valid) for tracing many scenes and images of uneven size in ONE persistent
 * launch (the same stepping rules as sphere_trace, Sec. 3.4 / A.4).  Jobs are
 * grouped by decoder; within a group one ray queue spans all jobs' rays.
 * All jobs share params, in_dim and the feature dtype.  ctas_per_sm: resident
 * CTAs per SM of the trace kernel (0 = default; 1..4 tensor-core, 1..3 FP32),
 * the knob the autotuner sets.  Uploads the job table (synchronises). */
int sphere_trace_batch_create(const nglod_trace_job* jobs, int num_jobs,
                              const nglod_trace_params* params, int ctas_per_sm, void* stream,
                              nglod_batch** out);

/* sphere_trace_batch_run -- enqueues one batched trace (reset, the persistent
 * trace kernel, then each job's normals if requested); no host
 * synchronisation, so it can be captured in a CUDA graph. */
int sphere_trace_batch_run(nglod_batch* batch, void* stream);

/* sphere_trace_batch_status -- synchronises; NGLOD_ERR_TIMEOUT if a bounded
 * tensor-core wait of the last run expired. */
int sphere_trace_batch_status(nglod_batch* batch, void* stream);

void sphere_trace_batch_free(nglod_batch* batch);

/* trace_normals -- surface normals of the rays a preceding sphere_trace call
 * (same work buffer, same stream, same decoder and LOD, want_normals = 0 or
 * 1) marked as hits:
 * the normalised analytic gradient of the decoded SDF (Eq. 2 chain rule
 * through the trilinear weights, Sec. 3.2) in FP32 at the hit point
 * x = o + t_hit d, using the hit voxel and the ReLU mask of the hit's last
 * decode recorded by sphere_trace (a blended trace records no masks for it:
 * the forward pass is then recomputed in FP32).  The masked sum
 * sum_h W2_h [mask_h] W1[h] runs as warp-level tensor-core products of the
 * 0/1 masks with W2 W1 split into three BF16 terms (exact products, FP32
 * sums); its operand is built in the workspace's last region, the only
 * bytes of work this call writes.  The paper
 * takes normals by finite differences (supplementary Sec. A.4); the analytic
 * gradient is their limit.  normal [R, 3]; zero for misses.  Does not
 * synchronise. */
int trace_normals(const nglod_svo* svo, const nglod_features* feats,
                  const nglod_decoder* dec, const float* o, const float* d, int64_t R,
                  int lod, const void* work, size_t work_bytes, const float* t_hit,
                  const uint8_t* hit, float* normal, void* stream);

/* trace_normals_fd -- as trace_normals, with the normals taken by central
 * differences of step fd_h in (0, 1) (NGLOD_NORMALS_FD of nglod_trace_params;
 * supplementary Sec. A.4): six sdf_query-style FP32 evaluations per hit. */
int trace_normals_fd(const nglod_svo* svo, const nglod_features* feats, const nglod_decoder* dec,
                     const float* o, const float* d, int64_t R, int lod, const void* work,
                     size_t work_bytes, const float* t_hit, const uint8_t* hit, float fd_h,
                     float* normal, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NGLOD_H */
