/*
 * Neural Geometric LOD -- plain CPU oracle (test infrastructure only).
 *
 * This file is the slow, obviously-correct reference that the CUDA path is
 * checked against.  Only the tests, the smoke entry point and the benchmark's
 * CPU-baseline leg may load it; the product path never does.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Arithmetic: FP64 everywhere except where the method itself decides an
 * integer in FP32 (the ray/voxel slab test and the voxel a point lies in);
 * there the same FP32 decision is written out here independently.  Build
 * with -ffp-contract=off so no multiply-add is fused.
 *
 * What each function follows:
 *   - octree, corner sharing, per-voxel corner pointers: Sec. 3.2, Sec. 3.4
 *     ("pointers ... precalculated in an initialization step");
 *   - ray/voxel lists: Sec. 3.4 and supplementary Sec. C (Decide, Subdivide,
 *     Compactify) -- computed here by brute force against every voxel of the
 *     target depth and ordered by the front-to-back child order of Sec. C;
 *   - feature query: Sec. 3.2 (trilinear psi per level, summed over levels);
 *   - decoder: Eq. 2 (one hidden layer, ReLU, linear output, Sec. A.1);
 *   - sphere tracing with adaptive stepping: Sec. 3.4 and Sec. A.4;
 *   - level blending of two consecutive LODs: Sec. 3.2, Eq. 3;
 *   - input gradient (normals) and parameter gradients of Eq. 4: chain rule.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (closed forms, brute-force DDA, affine-field exactness, O(h^2) convergence,
 * finite differences); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FIRST_FEATURE_DEPTH 3
#define MAX_DEPTH 12

/* ------------------------------------------------------------------------ */
/* Morton keys                                                              */
/* ------------------------------------------------------------------------ */
static uint64_t mk(int64_t i, int64_t j, int64_t k) {
    uint64_t key = 0;
    for (int b = 0; b < 21; ++b) {
        key |= (uint64_t)((i >> b) & 1) << (3 * b);
        key |= (uint64_t)((j >> b) & 1) << (3 * b + 1);
        key |= (uint64_t)((k >> b) & 1) << (3 * b + 2);
    }
    return key;
}

static void mk_decode(uint64_t key, int64_t *i, int64_t *j, int64_t *k) {
    *i = *j = *k = 0;
    for (int b = 0; b < 21; ++b) {
        *i |= (int64_t)((key >> (3 * b)) & 1) << b;
        *j |= (int64_t)((key >> (3 * b + 1)) & 1) << b;
        *k |= (int64_t)((key >> (3 * b + 2)) & 1) << b;
    }
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* index of key in sorted array, or -1 */
static int64_t find_key(const uint64_t *keys, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < n && keys[lo] == key) ? lo : -1;
}

static int64_t lower_bound_u64(const uint64_t *keys, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Octree                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int num_depths;                 /* Dmax + 1 */
    int64_t n[MAX_DEPTH + 1];
    uint64_t *keys[MAX_DEPTH + 1];
    /* per feature depth: sorted unique corner keys and 8 corner ids / voxel */
    int64_t nc[MAX_DEPTH + 1];
    uint64_t *ckeys[MAX_DEPTH + 1];
    int64_t *corner[MAX_DEPTH + 1];
} or_svo;

void or_svo_free(or_svo *s) {
    if (!s) return;
    for (int d = 0; d <= MAX_DEPTH; ++d) {
        free(s->keys[d]); free(s->ckeys[d]); free(s->corner[d]);
    }
    free(s);
}

/* Returns NULL if the keys are not a valid parent-closed octree. */
or_svo *or_svo_new(const uint64_t *const *keys, const int64_t *counts,
                   int num_depths) {
    if (num_depths < 1 || num_depths > MAX_DEPTH + 1) return NULL;
    or_svo *s = (or_svo *)calloc(1, sizeof(or_svo));
    s->num_depths = num_depths;
    for (int d = 0; d < num_depths; ++d) {
        s->n[d] = counts[d];
        s->keys[d] = (uint64_t *)malloc(sizeof(uint64_t) * (counts[d] > 0 ? counts[d] : 1));
        memcpy(s->keys[d], keys[d], sizeof(uint64_t) * counts[d]);
        for (int64_t v = 0; v < counts[d]; ++v) {
            if (d == 0 && s->keys[d][v] != 0) { or_svo_free(s); return NULL; }
            if (s->keys[d][v] >= ((uint64_t)1 << (3 * d)) && d > 0) { or_svo_free(s); return NULL; }
            if (v > 0 && s->keys[d][v] <= s->keys[d][v - 1]) { or_svo_free(s); return NULL; }
            if (d > 0 && find_key(s->keys[d - 1], s->n[d - 1], s->keys[d][v] >> 3) < 0) {
                or_svo_free(s); return NULL;
            }
        }
    }
    if (s->n[0] != 1) { or_svo_free(s); return NULL; }
    for (int d = FIRST_FEATURE_DEPTH; d < num_depths; ++d) {
        int64_t V = s->n[d];
        uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t) * (8 * V + 1));
        for (int64_t v = 0; v < V; ++v) {
            int64_t i, j, k;
            mk_decode(s->keys[d][v], &i, &j, &k);
            for (int c = 0; c < 8; ++c)
                all[8 * v + c] = mk(i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1));
        }
        qsort(all, (size_t)(8 * V), sizeof(uint64_t), cmp_u64);
        int64_t u = 0;
        for (int64_t t = 0; t < 8 * V; ++t)
            if (u == 0 || all[t] != all[u - 1]) all[u++] = all[t];
        s->nc[d] = u;
        s->ckeys[d] = all;
        s->corner[d] = (int64_t *)malloc(sizeof(int64_t) * (8 * V + 1));
        for (int64_t v = 0; v < V; ++v) {
            int64_t i, j, k;
            mk_decode(s->keys[d][v], &i, &j, &k);
            for (int c = 0; c < 8; ++c)
                s->corner[d][8 * v + c] = find_key(
                    all, u, mk(i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1)));
        }
    }
    return s;
}

int64_t or_corner_count(const or_svo *s, int lod) {
    int d = lod + FIRST_FEATURE_DEPTH - 1;
    return (d >= FIRST_FEATURE_DEPTH && d < s->num_depths) ? s->nc[d] : -1;
}

/* Per-voxel structure at depth d, for build parity.  corner ids only for
 * feature depths (else left untouched). */
void or_svo_arrays(const or_svo *s, int d, int32_t *parent, uint8_t *childmask,
                   int32_t *childbase, int32_t *corners) {
    for (int64_t v = 0; v < s->n[d]; ++v) {
        uint64_t key = s->keys[d][v];
        parent[v] = d == 0 ? -1 : (int32_t)find_key(s->keys[d - 1], s->n[d - 1], key >> 3);
        uint8_t m = 0;
        int32_t base = 0;
        if (d + 1 < s->num_depths) {
            base = (int32_t)lower_bound_u64(s->keys[d + 1], s->n[d + 1], key << 3);
            for (int c = 0; c < 8; ++c)
                if (find_key(s->keys[d + 1], s->n[d + 1], (key << 3) | (uint64_t)c) >= 0)
                    m |= (uint8_t)(1u << c);
        }
        childmask[v] = m;
        childbase[v] = base;
        if (d >= FIRST_FEATURE_DEPTH && corners)
            for (int c = 0; c < 8; ++c) corners[8 * v + c] = (int32_t)s->corner[d][8 * v + c];
    }
}

/* ------------------------------------------------------------------------ */
/* Ray / voxel intersection (FP32 slab test, written independently)         */
/* ------------------------------------------------------------------------ */
/* Voxel bounds at depth d: lo = -1 + i * 2^(1-d), exact in FP32 for d <= 23.
 * Per axis with |d_a| >= FLT_MIN: inv = 1/d_a (IEEE), t0 = (lo-o)*inv,
 * t1 = (hi-o)*inv, tmin = smaller, tmax = larger.  An axis with |d_a| <
 * FLT_MIN is parallel: it constrains nothing if lo <= o <= hi, else misses.
 * t_near = max over axes of tmin, t_far = min of tmax; hit iff
 * max(t_near, 0) <= t_far; the stored interval is [max(t_near,0), t_far]. */
static int slab32(const float o[3], const float inv[3], const int par[3],
                  int64_t ijk[3], int d, float *tin, float *tout) {
    const float s = ldexpf(1.0f, 1 - d);
    float tn = -INFINITY, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        volatile float lo = (float)ijk[a] * s - 1.0f;
        volatile float hi = (float)(ijk[a] + 1) * s - 1.0f;
        if (par[a]) {
            if (!(lo <= o[a] && o[a] <= hi)) return 0;
            continue;
        }
        volatile float dl = lo - o[a];
        volatile float dh = hi - o[a];
        volatile float t0 = dl * inv[a];
        volatile float t1 = dh * inv[a];
        float mn = t0 < t1 ? t0 : t1;
        float mx = t0 < t1 ? t1 : t0;
        if (mn > tn) tn = mn;
        if (mx < tf) tf = mx;
    }
    float te = tn > 0.0f ? tn : 0.0f;
    if (!(te <= tf)) return 0;
    *tin = te;
    *tout = tf;
    return 1;
}

static int ray_setup(const float *o, const float *d, float inv[3], int par[3]) {
    int zero = 0;
    for (int a = 0; a < 3; ++a) {
        if (isnan(o[a]) || isnan(d[a]) || isinf(o[a]) || isinf(d[a])) return 0;
        par[a] = fabsf(d[a]) < 1.17549435e-38f;
        zero += par[a];
        volatile float one = 1.0f;
        inv[a] = par[a] ? 0.0f : one / d[a];
    }
    return zero < 3;
}

typedef struct { int64_t vid; uint64_t order; float tin, tout; } hit_t;

static int cmp_hit(const void *a, const void *b) {
    uint64_t x = ((const hit_t *)a)->order, y = ((const hit_t *)b)->order;
    return (x > y) - (x < y);
}

/* Front-to-back key (Sec. C, "OrderedChildren"): for each depth 1..D, the
 * child slot of the ancestor XOR the octant of the ray origin relative to
 * the centre of that ancestor's parent (bit a set iff o_a >= centre_a). */
static uint64_t order_key(uint64_t key, int D, const float o[3]) {
    int64_t i, j, k;
    mk_decode(key, &i, &j, &k);
    uint64_t ord = 0;
    for (int d = 1; d <= D; ++d) {
        int sh = D - d;
        int slot = (int)((key >> (3 * sh)) & 7);
        int64_t pc[3] = {i >> (sh + 1), j >> (sh + 1), k >> (sh + 1)};
        int oct = 0;
        for (int a = 0; a < 3; ++a) {
            volatile float c = (float)(2 * pc[a] + 1) * ldexpf(1.0f, -(d - 1)) - 1.0f;
            if (o[a] >= c) oct |= 1 << a;
        }
        ord = (ord << 3) | (uint64_t)(slot ^ oct);
    }
    return ord;
}

/* All voxels of depth D hit by one ray, front to back.  Returns count; *out
 * is malloc'ed (caller frees). */
static int64_t ray_hits(const or_svo *s, int D, const float *o, const float *d,
                        hit_t **out) {
    float inv[3];
    int par[3];
    *out = NULL;
    if (!ray_setup(o, d, inv, par)) return 0;
    int64_t cap = 64, n = 0;
    hit_t *h = (hit_t *)malloc(sizeof(hit_t) * cap);
    for (int64_t v = 0; v < s->n[D]; ++v) {
        int64_t ijk[3];
        mk_decode(s->keys[D][v], &ijk[0], &ijk[1], &ijk[2]);
        float tin, tout;
        if (slab32(o, inv, par, ijk, D, &tin, &tout)) {
            if (n == cap) { cap *= 2; h = (hit_t *)realloc(h, sizeof(hit_t) * cap); }
            h[n].vid = v;
            h[n].order = order_key(s->keys[D][v], D, o);
            h[n].tin = tin;
            h[n].tout = tout;
            ++n;
        }
    }
    qsort(h, (size_t)n, sizeof(hit_t), cmp_hit);
    *out = h;
    return n;
}

/* Ray/voxel lists at target LOD as CSR.  Pass voxel_id == NULL to only count
 * (ray_offsets is still filled).  Returns the total number of hits. */
int64_t or_trace_rays(const or_svo *s, const float *o, const float *d, int64_t R,
                      int lod, int64_t *ray_offsets, int32_t *voxel_id,
                      float *t_range, int nthreads) {
    int D = lod + FIRST_FEATURE_DEPTH - 1;
    if (D < 0 || D >= s->num_depths) return -1;
    int64_t *cnt = (int64_t *)calloc((size_t)(R + 1), sizeof(int64_t));
    hit_t **lists = (hit_t **)calloc((size_t)(R + 1), sizeof(hit_t *));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
#endif
    for (int64_t r = 0; r < R; ++r) cnt[r] = ray_hits(s, D, o + 3 * r, d + 3 * r, &lists[r]);
    int64_t total = 0;
    for (int64_t r = 0; r < R; ++r) {
        ray_offsets[r] = total;
        if (voxel_id)
            for (int64_t t = 0; t < cnt[r]; ++t) {
                voxel_id[total + t] = (int32_t)lists[r][t].vid;
                t_range[2 * (total + t)] = lists[r][t].tin;
                t_range[2 * (total + t) + 1] = lists[r][t].tout;
            }
        total += cnt[r];
        free(lists[r]);
    }
    ray_offsets[R] = total;
    free(cnt);
    free(lists);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Feature query and decoder (Sec. 3.2, Eq. 2)                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *W1;   /* [hidden, in_dim] row-major */
    const double *b1;   /* [hidden] */
    const double *W2;   /* [hidden] */
    double b2;
    int in_dim, hidden;
} or_dec;

/* Trilinear weights of corner c (bit a = upper side along axis a) and, if
 * dw != NULL, their derivatives w.r.t. u_a. */
static void tri_weights(const double u[3], double w[8], double dw[8][3]) {
    for (int c = 0; c < 8; ++c) {
        double f[3], df[3];
        for (int a = 0; a < 3; ++a) {
            int up = (c >> a) & 1;
            f[a] = up ? u[a] : 1.0 - u[a];
            df[a] = up ? 1.0 : -1.0;
        }
        w[c] = f[0] * f[1] * f[2];
        if (dw) {
            dw[c][0] = df[0] * f[1] * f[2];
            dw[c][1] = f[0] * df[1] * f[2];
            dw[c][2] = f[0] * f[1] * df[2];
        }
    }
}

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/* Voxel ids containing x at each depth 0..D via integer coordinates:
 * q = fl32(x + 1); ijk = clamp(floor(q * 2^(d-1)), 0, 2^d - 1).  A point
 * outside [-1,1]^3 (or NaN) is in no voxel.  vids[d] = -1 if absent.
 * Returns the deepest depth with a voxel (or -1). */
static int locate32(const or_svo *s, const float x[3], int D, int64_t vids[],
                    int64_t ijks[][3]) {
    int deepest = -1;
    for (int a = 0; a < 3; ++a)
        if (!(x[a] >= -1.0f && x[a] <= 1.0f)) {
            for (int d = 0; d <= D; ++d) vids[d] = -1;
            return -1;
        }
    volatile float q[3];
    for (int a = 0; a < 3; ++a) q[a] = x[a] + 1.0f;
    int alive = 1;
    for (int d = 0; d <= D; ++d) {
        int64_t ijk[3];
        for (int a = 0; a < 3; ++a) {
            volatile float g = q[a] * ldexpf(1.0f, d - 1);
            int64_t c = (int64_t)floorf(g);
            int64_t hi = ((int64_t)1 << d) - 1;
            ijk[a] = c < 0 ? 0 : (c > hi ? hi : c);
            ijks[d][a] = ijk[a];
        }
        vids[d] = alive ? find_key(s->keys[d], s->n[d], mk(ijk[0], ijk[1], ijk[2])) : -1;
        if (vids[d] < 0) alive = 0; else deepest = d;
    }
    return deepest;
}

/* z(x; L) and its Jacobian dz/dx (jz may be NULL), given the voxel id at
 * each feature depth (-1 = absent, contributes 0). */
static void feature_sum(const or_svo *s, const double *const *feats, int m,
                        int D, const int64_t vids[], const int64_t ijks[][3],
                        const double x[3], double *z, double *jz /* [m][3] */) {
    for (int k = 0; k < m; ++k) z[k] = 0.0;
    if (jz) for (int k = 0; k < 3 * m; ++k) jz[k] = 0.0;
    for (int d = FIRST_FEATURE_DEPTH; d <= D; ++d) {
        int64_t v = vids[d];
        if (v < 0) continue;
        const double *Z = feats[d - FIRST_FEATURE_DEPTH];
        double scale = ldexp(1.0, d - 1);
        double u[3], w[8], dw[8][3];
        for (int a = 0; a < 3; ++a) u[a] = clamp01((x[a] + 1.0) * scale - (double)ijks[d][a]);
        tri_weights(u, w, dw);
        for (int c = 0; c < 8; ++c) {
            const double *row = Z + (size_t)s->corner[d][8 * v + c] * (size_t)m;
            for (int k = 0; k < m; ++k) {
                z[k] += w[c] * row[k];
                if (jz)
                    for (int a = 0; a < 3; ++a) jz[3 * k + a] += dw[c][a] * scale * row[k];
            }
        }
    }
}

/* Decoder of Eq. 2: v = [x, z] (in_dim = m + 3) or v = z (in_dim = m). */
static double decode(const or_dec *dec, const double x[3], const double *z, int m,
                     double *pre_out) {
    int off = dec->in_dim - m;
    double out = dec->b2;
    for (int h = 0; h < dec->hidden; ++h) {
        const double *w = dec->W1 + (size_t)h * dec->in_dim;
        double acc = dec->b1[h];
        for (int a = 0; a < off; ++a) acc += w[a] * x[a];
        for (int k = 0; k < m; ++k) acc += w[off + k] * z[k];
        if (pre_out) pre_out[h] = acc;
        out += dec->W2[h] * (acc > 0.0 ? acc : 0.0);
    }
    return out;
}

/* d(decode)/dx given z and its Jacobian. */
static void decode_grad_x(const or_dec *dec, const double x[3], const double *z,
                          const double *jz, int m, double g[3]) {
    int off = dec->in_dim - m;
    double *gz = (double *)calloc((size_t)m, sizeof(double));
    g[0] = g[1] = g[2] = 0.0;
    for (int h = 0; h < dec->hidden; ++h) {
        const double *w = dec->W1 + (size_t)h * dec->in_dim;
        double acc = dec->b1[h];
        for (int a = 0; a < off; ++a) acc += w[a] * x[a];
        for (int k = 0; k < m; ++k) acc += w[off + k] * z[k];
        if (acc > 0.0) {
            for (int a = 0; a < off; ++a) g[a] += dec->W2[h] * w[a];
            for (int k = 0; k < m; ++k) gz[k] += dec->W2[h] * w[off + k];
        }
    }
    for (int k = 0; k < m; ++k)
        for (int a = 0; a < 3; ++a) g[a] += gz[k] * jz[3 * k + a];
    free(gz);
}

static or_dec mkdec(const double *W1, const double *b1, const double *W2, double b2,
                    int in_dim, int hidden) {
    or_dec d = {W1, b1, W2, b2, in_dim, hidden};
    return d;
}

/* SDF at LOD `lod` for Q points (FP32 input, FP64 arithmetic).
 * feats[l-1] = features of LOD l as double [C_l, m]; decoder of that LOD.
 * deepest (nullable) = deepest feature LOD containing the point (0 = none).
 * grad (nullable) = d sdf / dx, [Q,3]. */
void or_sdf_query(const or_svo *s, const double *const *feats, int m,
                  const double *W1, const double *b1, const double *W2, double b2,
                  int in_dim, int hidden, const float *x, int64_t Q, int lod,
                  double *sdf, int32_t *deepest, double *grad, int nthreads) {
    int D = lod + FIRST_FEATURE_DEPTH - 1;
    or_dec dec = mkdec(W1, b1, W2, b2, in_dim, hidden);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t q = 0; q < Q; ++q) {
        int64_t vids[MAX_DEPTH + 1], ijks[MAX_DEPTH + 1][3];
        int dd = locate32(s, x + 3 * q, D, vids, ijks);
        double xd[3] = {x[3 * q], x[3 * q + 1], x[3 * q + 2]};
        double *z = (double *)malloc(sizeof(double) * (size_t)m * 4);
        double *jz = z + m;
        feature_sum(s, feats, m, D, vids, ijks, xd, z, grad ? jz : NULL);
        sdf[q] = decode(&dec, xd, z, m, NULL);
        if (deepest) deepest[q] = dd >= FIRST_FEATURE_DEPTH ? dd - FIRST_FEATURE_DEPTH + 1 : 0;
        if (grad) decode_grad_x(&dec, xd, z, jz, m, grad + 3 * q);
        free(z);
    }
}

/* ------------------------------------------------------------------------ */
/* Sphere tracing with adaptive stepping (Sec. 3.4, Sec. A.4)                */
/* ------------------------------------------------------------------------ */
/* Per ray, with its front-to-back list of target-depth voxels:
 *   t starts at the first entry; each iteration skips list entries whose
 *   exit lies before t (discarding the ray when the list runs out), jumps t
 *   to the entry point of the current voxel if t is before it, queries the
 *   SDF at x = o + t d using that voxel and its ancestors, and counts one
 *   step.  d < eps is a hit; otherwise t += d; t > far or steps == max_steps
 *   is a miss.  With osc != 0 the oscillation test |d_k - d_(k-1)| < 6 eps
 *   also stops the ray, as a hit iff |d_k| < 6 eps.
 * Outputs: t_hit (+inf on miss), hit, steps, x_hit (last query point),
 * normal = normalised analytic gradient at x_hit (0 on miss). */
/* The tracer of or_sphere_trace and or_sphere_trace_blend.  With lo == NULL
 * the distance is the decoder `hi` at LOD `lod`; otherwise it is Eq. 3's
 * blend (1 - alpha) d_lo + alpha d_hi, where d_lo decodes the feature sum
 * over depths 3..D-1 with `lo` and d_hi the sum over 3..D with `hi`, both at
 * the same point, and the normal is the normalised blend of their
 * gradients. */
static void trace_impl(const or_svo *s, const double *const *feats, int m, const or_dec *hi,
                       const or_dec *lo, double alpha, const float *o, const float *dir,
                       int64_t R, int lod, double eps, double far_, int max_steps, int osc,
                       double *t_hit, uint8_t *hit, int32_t *steps, double *x_hit,
                       double *normal, int nthreads) {
    int D = lod + FIRST_FEATURE_DEPTH - 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t r = 0; r < R; ++r) {
        hit_t *lst;
        int64_t n = ray_hits(s, D, o + 3 * r, dir + 3 * r, &lst);
        double oo[3] = {o[3 * r], o[3 * r + 1], o[3 * r + 2]};
        double dd[3] = {dir[3 * r], dir[3 * r + 1], dir[3 * r + 2]};
        double *z = (double *)malloc(sizeof(double) * (size_t)m * 8);
        double *jz = z + m;
        double *zl = z + 4 * m;
        double *jzl = zl + m;
        int64_t vids[MAX_DEPTH + 1], ijks[MAX_DEPTH + 1][3];
        int k = 0, is_hit = 0;
        double t = n > 0 ? (double)lst[0].tin : INFINITY;
        double x[3] = {0, 0, 0}, dprev = NAN;
        int64_t cur = 0;
        while (n > 0) {
            while (cur < n && t > (double)lst[cur].tout) ++cur;
            if (cur == n) break;
            if (t < (double)lst[cur].tin) t = (double)lst[cur].tin;
            if (t > far_) break;
            for (int a = 0; a < 3; ++a) x[a] = oo[a] + t * dd[a];
            /* the containing voxel and its ancestors (parents always exist) */
            uint64_t key = s->keys[D][lst[cur].vid];
            int64_t i, j, kk;
            mk_decode(key, &i, &j, &kk);
            for (int d = 0; d <= D; ++d) {
                int sh = D - d;
                vids[d] = find_key(s->keys[d], s->n[d], key >> (3 * sh));
                ijks[d][0] = i >> sh; ijks[d][1] = j >> sh; ijks[d][2] = kk >> sh;
            }
            feature_sum(s, feats, m, D, vids, ijks, x, z, NULL);
            double dk = decode(hi, x, z, m, NULL);
            if (lo) {
                feature_sum(s, feats, m, D - 1, vids, ijks, x, zl, NULL);
                dk = (1.0 - alpha) * decode(lo, x, zl, m, NULL) + alpha * dk;
            }
            ++k;
            if (dk < eps) { is_hit = 1; break; }
            if (osc && k > 1 && fabs(dk - dprev) < 6.0 * eps) {
                is_hit = fabs(dk) < 6.0 * eps;
                break;
            }
            dprev = dk;
            t += dk;
            if (t > far_) break;
            if (k >= max_steps) break;
        }
        hit[r] = (uint8_t)is_hit;
        steps[r] = k;
        t_hit[r] = is_hit ? t : INFINITY;
        for (int a = 0; a < 3; ++a) {
            x_hit[3 * r + a] = is_hit ? x[a] : 0.0;
            normal[3 * r + a] = 0.0;
        }
        if (is_hit) {
            feature_sum(s, feats, m, D, vids, ijks, x, z, jz);
            double g[3];
            decode_grad_x(hi, x, z, jz, m, g);
            if (lo) {
                double gl[3];
                feature_sum(s, feats, m, D - 1, vids, ijks, x, zl, jzl);
                decode_grad_x(lo, x, zl, jzl, m, gl);
                for (int a = 0; a < 3; ++a) g[a] = (1.0 - alpha) * gl[a] + alpha * g[a];
            }
            double nn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            if (nn > 0.0)
                for (int a = 0; a < 3; ++a) normal[3 * r + a] = g[a] / nn;
        }
        free(z);
        free(lst);
    }
}

void or_sphere_trace(const or_svo *s, const double *const *feats, int m,
                     const double *W1, const double *b1, const double *W2, double b2,
                     int in_dim, int hidden, const float *o, const float *dir,
                     int64_t R, int lod, double eps, double far_, int max_steps, int osc,
                     double *t_hit, uint8_t *hit, int32_t *steps, double *x_hit,
                     double *normal, int nthreads) {
    or_dec dec = mkdec(W1, b1, W2, b2, in_dim, hidden);
    trace_impl(s, feats, m, &dec, NULL, 0.0, o, dir, R, lod, eps, far_, max_steps, osc, t_hit, hit,
               steps, x_hit, normal, nthreads);
}

/* Level blending (Sec. 3.2, Eq. 3) while sphere tracing: rays walk their
 * lists at LOD lod_hi = L* + 1 and every step decodes
 * (1 - alpha) d_{L*}(x) + alpha d_{L*+1}(x), alpha in [0, 1]; decoder "lo"
 * is LOD L*'s, "hi" is LOD L*+1's.  Outputs as or_sphere_trace. */
void or_sphere_trace_blend(const or_svo *s, const double *const *feats, int m,
                           const double *W1lo, const double *b1lo, const double *W2lo, double b2lo,
                           const double *W1hi, const double *b1hi, const double *W2hi, double b2hi,
                           int in_dim, int hidden, const float *o, const float *dir, int64_t R,
                           int lod_hi, double alpha, double eps, double far_, int max_steps, int osc,
                           double *t_hit, uint8_t *hit, int32_t *steps, double *x_hit,
                           double *normal, int nthreads) {
    or_dec lo = mkdec(W1lo, b1lo, W2lo, b2lo, in_dim, hidden);
    or_dec hi = mkdec(W1hi, b1hi, W2hi, b2hi, in_dim, hidden);
    trace_impl(s, feats, m, &hi, &lo, alpha, o, dir, R, lod_hi, eps, far_, max_steps, osc, t_hit, hit,
               steps, x_hit, normal, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Gradients of  sum_L g_L(q) * sdf_L(x_q)  (the adjoint of Eq. 4's terms)   */
/* ------------------------------------------------------------------------ */
/* lods[0..nl-1] are the LODs whose outputs carry gradient grad_sdf[i][q];
 * decoders are given per LOD (index lod-1) through arrays of pointers.
 * All gradient outputs accumulate (+=).  Serial on purpose. */
void or_sdf_backward(const or_svo *s, const double *const *feats, int m,
                     const double *const *W1, const double *const *b1,
                     const double *const *W2, const double *b2, int in_dim, int hidden,
                     const float *x, int64_t Q, const int32_t *lods, int nl,
                     const double *grad_sdf, double *const *g_feats,
                     double *const *g_W1, double *const *g_b1, double *const *g_W2,
                     double *g_b2, double *g_x) {
    double *z = (double *)malloc(sizeof(double) * (size_t)m * 4);
    double *jz = z + m;
    double *pre = (double *)malloc(sizeof(double) * (size_t)hidden);
    double *gz = (double *)malloc(sizeof(double) * (size_t)m);
    for (int li = 0; li < nl; ++li) {
        int lod = lods[li];
        int D = lod + FIRST_FEATURE_DEPTH - 1;
        or_dec dec = mkdec(W1[lod - 1], b1[lod - 1], W2[lod - 1], b2[lod - 1], in_dim, hidden);
        int off = in_dim - m;
        for (int64_t q = 0; q < Q; ++q) {
            double g = grad_sdf[(size_t)li * (size_t)Q + (size_t)q];
            int64_t vids[MAX_DEPTH + 1], ijks[MAX_DEPTH + 1][3];
            locate32(s, x + 3 * q, D, vids, ijks);
            double xd[3] = {x[3 * q], x[3 * q + 1], x[3 * q + 2]};
            feature_sum(s, feats, m, D, vids, ijks, xd, z, jz);
            decode(&dec, xd, z, m, pre);
            g_b2[lod - 1] += g;
            for (int k = 0; k < m; ++k) gz[k] = 0.0;
            double gx[3] = {0, 0, 0};
            for (int h = 0; h < hidden; ++h) {
                double act = pre[h] > 0.0 ? pre[h] : 0.0;
                g_W2[lod - 1][h] += g * act;
                if (pre[h] <= 0.0) continue;
                double gp = g * dec.W2[h];
                g_b1[lod - 1][h] += gp;
                const double *w = dec.W1 + (size_t)h * in_dim;
                double *gw = g_W1[lod - 1] + (size_t)h * in_dim;
                for (int a = 0; a < off; ++a) { gw[a] += gp * xd[a]; gx[a] += gp * w[a]; }
                for (int k = 0; k < m; ++k) { gw[off + k] += gp * z[k]; gz[k] += gp * w[off + k]; }
            }
            for (int k = 0; k < m; ++k)
                for (int a = 0; a < 3; ++a) gx[a] += gz[k] * jz[3 * k + a];
            if (g_x) for (int a = 0; a < 3; ++a) g_x[3 * q + a] += gx[a];
            /* scatter into the corner features of every level <= lod */
            for (int d = FIRST_FEATURE_DEPTH; d <= D; ++d) {
                int64_t v = vids[d];
                if (v < 0) continue;
                double scale = ldexp(1.0, d - 1), u[3], w8[8];
                for (int a = 0; a < 3; ++a) u[a] = clamp01((xd[a] + 1.0) * scale - (double)ijks[d][a]);
                tri_weights(u, w8, NULL);
                double *GZ = g_feats[d - FIRST_FEATURE_DEPTH];
                for (int c = 0; c < 8; ++c) {
                    double *row = GZ + (size_t)s->corner[d][8 * v + c] * (size_t)m;
                    for (int k = 0; k < m; ++k) row[k] += w8[c] * gz[k];
                }
            }
        }
    }
    free(z); free(pre); free(gz);
}

/* z(x; L) = sum over levels of the trilinear feature interpolation (Sec. 3.2)
 * for Q points, [Q, m] FP64 -- the decoder input, exposed so tests can bound
 * the effect of rounding z (e.g. to bf16) on the decoded distance. */
void or_feature_sum(const or_svo *s, const double *const *feats, int m, const float *x, int64_t Q,
                    int lod, double *z) {
    int D = lod + FIRST_FEATURE_DEPTH - 1;
    for (int64_t q = 0; q < Q; ++q) {
        int64_t vids[MAX_DEPTH + 1], ijks[MAX_DEPTH + 1][3];
        locate32(s, x + 3 * q, D, vids, ijks);
        double xd[3] = {x[3 * q], x[3 * q + 1], x[3 * q + 2]};
        feature_sum(s, feats, m, D, vids, ijks, xd, z + (size_t)q * (size_t)m, NULL);
    }
}
