"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module defines *inputs only*: analytic CSG scenes and their exact signed
distance, the sparse-voxel-octree occupancy (which voxels exist), pinhole
camera rays, Gaussian-initialised corner features and per-LOD decoder weights.
It holds none of the rendering method's arithmetic (no ray/box test, no
trilinear interpolation, no decoder evaluation, no sphere tracing).

Conventions fixed here and used by every consumer:

* Bounding volume [-1, 1]^3 (Sec. 3.2).  Octree depth ``dp`` has resolution
  ``2**dp``; LOD ``l`` lives at depth ``l + 2`` (r_l = r_0 * 2**l with r_0 = 4,
  supplementary Sec. A.1); depths 0..2 are structural only.
* Voxel ``(i, j, k)`` at depth ``dp`` has Morton key
  ``sum_b bit_b(i) << 3b | bit_b(j) << 3b+1 | bit_b(k) << 3b+2``; the child in
  slot ``c = cx | cy << 1 | cz << 2`` of a parent with key ``p`` has key
  ``8 p + c``.  Each depth is given as a sorted array of unique keys; the voxel
  id used everywhere is the index into that array.
* The corners of depth-``dp`` voxels are points of the ``(2**dp + 1)**3``
  lattice.  The corner id is the rank of the corner's Morton key among the
  unique corner keys of that depth, sorted ascending; the feature table of LOD
  ``l`` is ``[C_l, m]`` in that order (shared corners, Sec. 3.2).
* Occupancy follows the sparsity rule "a voxel is allocated only if it
  contains surface" (Sec. 3.2), made concrete as: keep a voxel iff
  ``|sdf(center)| < half-diagonal``, evaluated top-down so only children of
  kept voxels are considered (parents always exist, Sec. 3.4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FIRST_FEATURE_DEPTH = 3      # LOD 1 = resolution 8 (r_0 * 2)
PRIM_SPHERE, PRIM_BOX, PRIM_CAPSULE = 0, 1, 2


# ----------------------------------------------------------------------------
# Morton keys
# ----------------------------------------------------------------------------
def morton_encode(i, j, k) -> np.ndarray:
    """Interleave up to 21-bit integer coordinates into uint64 Morton keys."""
    i = np.asarray(i, dtype=np.uint64)
    j = np.asarray(j, dtype=np.uint64)
    k = np.asarray(k, dtype=np.uint64)
    key = np.zeros(np.broadcast(i, j, k).shape, dtype=np.uint64)
    one = np.uint64(1)
    for b in range(21):
        bb = np.uint64(b)
        key |= ((i >> bb) & one) << np.uint64(3 * b)
        key |= ((j >> bb) & one) << np.uint64(3 * b + 1)
        key |= ((k >> bb) & one) << np.uint64(3 * b + 2)
    return key


def morton_decode(key) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    key = np.asarray(key, dtype=np.uint64)
    i = np.zeros(key.shape, dtype=np.int64)
    j = np.zeros(key.shape, dtype=np.int64)
    k = np.zeros(key.shape, dtype=np.int64)
    one = np.uint64(1)
    for b in range(21):
        i |= ((key >> np.uint64(3 * b)) & one).astype(np.int64) << b
        j |= ((key >> np.uint64(3 * b + 1)) & one).astype(np.int64) << b
        k |= ((key >> np.uint64(3 * b + 2)) & one).astype(np.int64) << b
    return i, j, k


# ----------------------------------------------------------------------------
# Analytic CSG scenes (ground-truth SDF, not the neural method)
# ----------------------------------------------------------------------------
@dataclass
class Scene:
    """Union of primitives; ``params`` meaning depends on the primitive type.

    sphere:  params[0] = radius
    box:     params[0:3] = half extents (axis aligned)
    capsule: params[0:3] = half-segment vector, params[3] = radius
    """
    types: np.ndarray                     # int32 [n]
    centers: np.ndarray                   # float64 [n, 3]
    params: np.ndarray                    # float64 [n, 4]
    name: str = "scene"

    @property
    def n(self) -> int:
        return int(self.types.shape[0])


def sphere_scene(radius: float = 0.5) -> Scene:
    """The analytic sphere of radius ``radius`` centred at the origin."""
    return Scene(types=np.array([PRIM_SPHERE], np.int32),
                 centers=np.zeros((1, 3)),
                 params=np.array([[radius, 0.0, 0.0, 0.0]]),
                 name=f"sphere_r{radius}")


def csg_scene(n: int, seed: int = 0) -> Scene:
    """Union of ``n`` seeded random spheres, boxes and capsules.

    Per primitive, in this draw order: type = integers(3); centre ~
    U[-0.65, 0.65]^3; sphere radius ~ U[0.05, 0.3]; box half extents ~
    U[0.05, 0.3]^3; capsule half-segment = unit normal direction x
    U[0.05, 0.3] and radius 0.5 x U[0.05, 0.3].
    """
    rng = np.random.default_rng(seed)
    types = np.zeros(n, np.int32)
    centers = np.zeros((n, 3))
    params = np.zeros((n, 4))
    for p in range(n):
        t = int(rng.integers(3))
        types[p] = t
        centers[p] = rng.uniform(-0.65, 0.65, 3)
        if t == PRIM_SPHERE:
            params[p, 0] = rng.uniform(0.05, 0.3)
        elif t == PRIM_BOX:
            params[p, 0:3] = rng.uniform(0.05, 0.3, 3)
        else:
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            params[p, 0:3] = v * rng.uniform(0.05, 0.3)
            params[p, 3] = 0.5 * rng.uniform(0.05, 0.3)
    return Scene(types, centers, params, name=f"csg{n}_s{seed}")


def _bound_radius(scene: Scene) -> np.ndarray:
    """Radius of a sphere about each primitive's centre that contains it."""
    rb = np.empty(scene.n)
    for p, (t, q) in enumerate(zip(scene.types, scene.params)):
        if t == PRIM_SPHERE:
            rb[p] = q[0]
        elif t == PRIM_BOX:
            rb[p] = math.sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2])
        else:
            rb[p] = math.sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) + q[3]
    return rb


def _primitive_sdf(t: int, c: np.ndarray, q: np.ndarray, p: np.ndarray) -> np.ndarray:
    """SDF of one primitive type at points p [n, 3]; c and q are one
    primitive's centre and params ([3], [4]) or one row per point ([n, 3],
    [n, 4])."""
    d = p - c
    if t == PRIM_SPHERE:
        return np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]) - q[..., 0]
    if t == PRIM_BOX:
        a = np.abs(d) - q[..., 0:3]
        e = np.maximum(a, 0.0)
        return (np.sqrt(e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1] + e[:, 2] * e[:, 2])
                + np.minimum(np.maximum(np.maximum(a[:, 0], a[:, 1]), a[:, 2]), 0.0))
    h = q[..., 0:3]
    pa = d + h                      # segment from c - h to c + h
    ba = 2.0 * h
    tt = np.clip((pa[:, 0] * ba[..., 0] + pa[:, 1] * ba[..., 1] + pa[:, 2] * ba[..., 2])
                 / (ba[..., 0] * ba[..., 0] + ba[..., 1] * ba[..., 1] + ba[..., 2] * ba[..., 2]), 0.0, 1.0)
    e = pa - tt[:, None] * ba
    return np.sqrt(e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1] + e[:, 2] * e[:, 2]) - q[..., 3]


def _pair_sdf(scene: Scene, prim: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """SDF of primitive prim[i] at pts[i], for every pair i."""
    out = np.empty(prim.shape[0])
    ty = scene.types[prim]
    for t in (PRIM_SPHERE, PRIM_BOX, PRIM_CAPSULE):
        sel = np.flatnonzero(ty == t)
        if sel.size:
            pr = prim[sel]
            out[sel] = _primitive_sdf(t, scene.centers[pr], scene.params[pr], pts[sel])
    return out


def scene_sdf(scene: Scene, pts: np.ndarray, cap=None, chunk: int = 1 << 13) -> np.ndarray:
    """Exact CSG signed distance (min over primitive SDFs), float64 [N].

    Every primitive SDF here is 1-Lipschitz and <= 0 at the primitive's
    centre, so |x - c_p| bounds it from above, and |x - c_p| - rb_p (rb_p =
    bounding radius) from below.  A primitive whose lower bound exceeds the
    smallest upper bound (plus 1e-9 for rounding) cannot be the minimum and
    is skipped; the result is the same min.  With ``cap`` (scalar or [N]),
    values >= cap are only guaranteed to stay >= cap (primitives whose lower
    bound exceeds cap are skipped too; such points may return +inf).
    """
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.empty(pts.shape[0])
    rb = _bound_radius(scene)
    cen = scene.centers
    for s in range(0, pts.shape[0], chunk):
        p = pts[s:s + chunk]
        dv = p[:, None, :] - cen[None, :, :]
        dist = np.sqrt(dv[..., 0] * dv[..., 0] + dv[..., 1] * dv[..., 1] + dv[..., 2] * dv[..., 2])
        lim = dist.min(axis=1)
        if cap is not None:
            cp = np.broadcast_to(np.asarray(cap, np.float64), (pts.shape[0],))[s:s + chunk]
            lim = np.minimum(lim, cp)
        live = (dist - rb[None, :]) <= (lim + 1e-9)[:, None]
        best = np.full(p.shape[0], np.inf)
        for k in range(scene.n):
            rows = np.flatnonzero(live[:, k])
            if rows.size:
                best[rows] = np.minimum(best[rows], _primitive_sdf(int(scene.types[k]), cen[k],
                                                                   scene.params[k], p[rows]))
        out[s:s + chunk] = best
    return out


# ----------------------------------------------------------------------------
# Octree occupancy
# ----------------------------------------------------------------------------
@dataclass
class Octree:
    """Occupied voxels per depth 0..max_depth as sorted unique Morton keys."""
    keys: list                                   # list[np.ndarray uint64]
    scene: Scene | None = None
    corner_keys: list = field(default_factory=list)   # per feature depth
    prim_pairs: list | None = None               # per depth (voxel index, primitive) candidates

    @property
    def max_depth(self) -> int:
        return len(self.keys) - 1

    @property
    def max_lod(self) -> int:
        return self.max_depth - (FIRST_FEATURE_DEPTH - 1)

    def counts(self) -> list[int]:
        return [int(k.shape[0]) for k in self.keys]

    def corner_counts(self) -> list[int]:
        return [int(c.shape[0]) for c in self.corner_keys]


def voxel_centers(keys: np.ndarray, dp: int) -> np.ndarray:
    i, j, k = morton_decode(keys)
    s = 2.0 / (1 << dp)
    return np.stack([-1.0 + (i + 0.5) * s, -1.0 + (j + 0.5) * s,
                     -1.0 + (k + 0.5) * s], axis=1)


def unique_corner_keys(keys: np.ndarray) -> np.ndarray:
    """Sorted unique Morton keys of the lattice corners of the given voxels."""
    i, j, k = morton_decode(keys)
    parts = []
    for c in range(8):
        parts.append(morton_encode(i + (c & 1), j + ((c >> 1) & 1),
                                   k + ((c >> 2) & 1)))
    return np.unique(np.concatenate(parts)) if parts else np.zeros(0, np.uint64)


def build_octree(scene: Scene, max_depth: int) -> Octree:
    """Top-down occupancy: keep a voxel iff |sdf(centre)| < half diagonal.

    The min over primitives is taken over each voxel's candidate set
    rel(v) = {p : |centre(v) - c_p| - rb_p <= 3 hd_v} (hd_v = half diagonal,
    rb_p = bounding radius).  A child's set is inside its parent's (child
    centres lie hd_child from the parent's, and hd_parent = 2 hd_child), so
    the sets are built top-down from pairs.  The minimising primitive of any
    point within 2 hd_v of the centre with |sdf| < 2 hd_v lies in rel(v)
    (its lower bound is at most its value), so the keep decision and the
    corner distances of kept voxels are the exact min; the sets are kept on
    the octree (``prim_pairs``) for the corner distances.
    """
    rb = _bound_radius(scene)
    keys = [np.zeros(1, np.uint64)]
    pv = np.zeros(scene.n, np.int64)                 # pair -> voxel index at this depth
    pp = np.arange(scene.n, dtype=np.int64)          # pair -> primitive
    pairs = [(pv, pp)]
    for dp in range(1, max_depth + 1):
        parents = keys[-1]
        cand = (parents[:, None] * np.uint64(8)
                + np.arange(8, dtype=np.uint64)[None, :]).reshape(-1)
        half_diag = math.sqrt(3.0) * (2.0 / (1 << dp)) * 0.5
        cc = voxel_centers(cand, dp)
        ci = (pv[:, None] * 8 + np.arange(8)[None, :]).reshape(-1)
        cp = np.repeat(pp, 8)
        dv = cc[ci] - scene.centers[cp]
        lb = np.sqrt(dv[:, 0] * dv[:, 0] + dv[:, 1] * dv[:, 1] + dv[:, 2] * dv[:, 2]) - rb[cp]
        live = lb <= 3.0 * half_diag + 1e-9
        ci, cp = ci[live], cp[live]
        best = np.full(cand.shape[0], np.inf)
        np.minimum.at(best, ci, _pair_sdf(scene, cp, cc[ci]))
        keep = np.abs(best) < half_diag
        newidx = np.cumsum(keep) - 1
        sel = keep[ci]
        pv, pp = newidx[ci[sel]], cp[sel]
        keys.append(cand[keep])                      # parents sorted => candidates sorted
        pairs.append((pv, pp))
    oct_ = Octree(keys=keys, scene=scene)
    oct_.prim_pairs = pairs
    oct_.corner_keys = [unique_corner_keys(keys[dp])
                        for dp in range(FIRST_FEATURE_DEPTH, max_depth + 1)]
    return oct_


def corner_sdf(octree: Octree, scene: Scene, li: int) -> np.ndarray:
    """Exact scene SDF at the corners of feature level li (depth 3 + li),
    from the candidate sets of build_octree (min over a voxel's set)."""
    dp = FIRST_FEATURE_DEPTH + li
    ck = octree.corner_keys[li]
    pairs = getattr(octree, "prim_pairs", None)
    if pairs is None or octree.scene is not scene:
        return scene_sdf(scene, corner_positions(ck, dp))
    pv, pp = pairs[dp]
    keys = octree.keys[dp]
    i, j, k = morton_decode(keys)
    owner = np.empty(ck.shape[0], np.int64)
    for c in range(8):
        ckey = morton_encode(i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1))
        owner[np.searchsorted(ck, ckey)] = np.arange(keys.shape[0])
    order = np.argsort(pv, kind="stable")
    pv, pp = pv[order], pp[order]
    start = np.searchsorted(pv, np.arange(keys.shape[0]))
    cnt = np.searchsorted(pv, np.arange(keys.shape[0]), side="right") - start
    n = cnt[owner]
    corner = np.repeat(np.arange(ck.shape[0]), n)
    first = np.repeat(start[owner], n)
    within = np.arange(corner.shape[0]) - np.repeat(np.cumsum(n) - n, n)
    prim = pp[first + within]
    pos = corner_positions(ck, dp)
    out = np.full(ck.shape[0], np.inf)
    np.minimum.at(out, corner, _pair_sdf(scene, prim, pos[corner]))
    return out


def full_octree(max_depth: int) -> Octree:
    """Every voxel occupied at every depth (a dense grid), for tests."""
    keys = [np.arange(8 ** dp, dtype=np.uint64) for dp in range(max_depth + 1)]
    oct_ = Octree(keys=keys)
    oct_.corner_keys = [unique_corner_keys(keys[dp])
                        for dp in range(FIRST_FEATURE_DEPTH, max_depth + 1)]
    return oct_


def corner_positions(corner_keys: np.ndarray, dp: int) -> np.ndarray:
    """World positions (float64 [C, 3]) of lattice corners at depth ``dp``."""
    i, j, k = morton_decode(corner_keys)
    s = 2.0 / (1 << dp)
    return np.stack([-1.0 + i * s, -1.0 + j * s, -1.0 + k * s], axis=1)


# ----------------------------------------------------------------------------
# Learned-parameter stand-ins
# ----------------------------------------------------------------------------
def init_features(octree: Octree, m: int = 32, seed: int = 0,
                  sigma: float = 0.01) -> list[np.ndarray]:
    """Corner features ~ N(0, sigma^2) per LOD (float32 [C_l, m]), Sec. 4."""
    rng = np.random.default_rng(seed)
    return [rng.normal(0.0, sigma, (c.shape[0], m)).astype(np.float32)
            for c in octree.corner_keys]


def readout_features(octree: Octree, scene: Scene, m: int = 32, seed: int = 0,
                     sigma: float = 0.01) -> list[np.ndarray]:
    """Features whose channel ``l - 1`` at LOD ``l`` holds sdf(corner).

    Channels ``0..L_max-1`` are zero except that one; the remaining channels
    are N(0, sigma^2).  Paired with ``readout_decoder(l)``, LOD ``l`` then
    decodes exactly the level-``l`` trilinear interpolant of the corner-sampled
    analytic SDF (a closed form the tests use).
    """
    rng = np.random.default_rng(seed)
    L = len(octree.corner_keys)
    assert L <= m
    feats = []
    for li, ck in enumerate(octree.corner_keys):
        dp = FIRST_FEATURE_DEPTH + li
        f = rng.normal(0.0, sigma, (ck.shape[0], m))
        f[:, :L] = 0.0
        f[:, li] = corner_sdf(octree, scene, li)
        feats.append(f.astype(np.float32))
    return feats


@dataclass
class Decoder:
    """One LOD's MLP: d = W2 . relu(W1 v + b1) + b2, v = [x, z] or z."""
    W1: np.ndarray      # float32 [hidden, in_dim]
    b1: np.ndarray      # float32 [hidden]
    W2: np.ndarray      # float32 [hidden]
    b2: float
    in_dim: int

    @property
    def hidden(self) -> int:
        return int(self.W1.shape[0])

    def n_params(self) -> int:
        return int(self.W1.size + self.b1.size + self.W2.size + 1)


def init_decoder(lod: int, in_dim: int = 32, hidden: int = 128) -> Decoder:
    """W ~ N(0, 1/fan_in), zero biases; seed 1 + lod."""
    rng = np.random.default_rng(1 + lod)
    W1 = rng.normal(0.0, 1.0 / math.sqrt(in_dim), (hidden, in_dim))
    W2 = rng.normal(0.0, 1.0 / math.sqrt(hidden), hidden)
    return Decoder(W1.astype(np.float32), np.zeros(hidden, np.float32),
                   W2.astype(np.float32), 0.0, in_dim)


def readout_decoder(lod: int, in_dim: int = 32, hidden: int = 128) -> Decoder:
    """Random W1 except rows 0/1 = +/- e_(channel lod-1); W2 = (1, -1, 0, ...).

    The output is relu(z_c) - relu(-z_c) = z_c with c = lod - 1, yet every
    hidden unit is still computed (dense cost, realistic step counts).
    """
    dec = init_decoder(lod, in_dim, hidden)
    off = in_dim - 32 if in_dim > 32 else 0
    dec.W1[0, :] = 0.0
    dec.W1[1, :] = 0.0
    dec.W1[0, off + lod - 1] = 1.0
    dec.W1[1, off + lod - 1] = -1.0
    dec.W2[:] = 0.0
    dec.W2[0] = 1.0
    dec.W2[1] = -1.0
    return dec


# ----------------------------------------------------------------------------
# Camera rays
# ----------------------------------------------------------------------------
def default_eye(dist: float = 2.5) -> np.ndarray:
    v = np.array([1.0, 0.8, 1.2])
    return dist * v / np.linalg.norm(v)


def camera_rays(width: int, height: int, eye=None, target=(0.0, 0.0, 0.0),
                up=(0.0, 1.0, 0.0), vfov_deg: float = 50.0, tile: int = 0):
    """Pinhole rays through pixel centres, float32 origins/directions [R, 3].

    ``tile > 0`` emits the rays in tile-major order (``tile x tile`` pixel
    blocks, row-major inside and across blocks) so neighbouring ray indices
    are neighbouring pixels; ``pixel`` gives each ray's row-major pixel index.
    """
    eye = default_eye() if eye is None else np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    upv = np.asarray(up, np.float64)
    if abs(np.dot(fwd, upv)) > 0.999:
        upv = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    right = np.cross(fwd, upv)
    right /= np.linalg.norm(right)
    up2 = np.cross(right, fwd)
    th = math.tan(math.radians(vfov_deg) * 0.5)
    aspect = width / height
    py, px = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    pixel = (py * width + px).reshape(-1)
    if tile > 0:
        ty, tx = py // tile, px // tile
        order = np.lexsort(((px % tile).reshape(-1), (py % tile).reshape(-1),
                            tx.reshape(-1), ty.reshape(-1)))
        pixel = pixel[order]
    pyf = (pixel // width).astype(np.float64)
    pxf = (pixel % width).astype(np.float64)
    sx = ((pxf + 0.5) / width * 2.0 - 1.0) * th * aspect
    sy = (1.0 - (pyf + 0.5) / height * 2.0) * th
    d = fwd[None, :] + sx[:, None] * right[None, :] + sy[:, None] * up2[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(eye, d.shape)
    return (np.ascontiguousarray(o, dtype=np.float32),
            np.ascontiguousarray(d, dtype=np.float32), pixel.astype(np.int64))


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------
def plain_sphere(max_lod: int = 3):
    """Unit-sphere scene (r = 0.5) with an octree to ``max_lod``."""
    sc = sphere_scene(0.5)
    return sc, build_octree(sc, max_lod + FIRST_FEATURE_DEPTH - 1)


def csg_workload(n: int = 64, seed: int = 0, max_lod: int = 5):
    sc = csg_scene(n, seed)
    return sc, build_octree(sc, max_lod + FIRST_FEATURE_DEPTH - 1)


def uniform_points(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)


def points_in_voxels(octree: Octree, dp: int, n: int, seed: int,
                     margin: float = 1e-3) -> np.ndarray:
    """Uniform points inside random occupied voxels of depth ``dp``.

    ``margin`` (in voxel units) keeps points off the faces so the containing
    voxel is unambiguous under any rounding.
    """
    rng = np.random.default_rng(seed)
    keys = octree.keys[dp]
    pick = keys[rng.integers(0, keys.shape[0], n)]
    i, j, k = morton_decode(pick)
    s = 2.0 / (1 << dp)
    u = rng.uniform(margin, 1.0 - margin, (n, 3))
    p = np.stack([-1.0 + (i + u[:, 0]) * s, -1.0 + (j + u[:, 1]) * s,
                  -1.0 + (k + u[:, 2]) * s], axis=1)
    return p.astype(np.float32)


# ----------------------------------------------------------------------------
# Training samples (inputs of the summed per-LOD L2 loss)
# ----------------------------------------------------------------------------
def _primitive_surface(scene: Scene, p: int, n: int, rng) -> np.ndarray:
    """n points uniformly distributed on primitive p's surface."""
    t, c, q = scene.types[p], scene.centers[p], scene.params[p]
    if t == PRIM_SPHERE:
        v = rng.normal(size=(n, 3))
        return c + q[0] * v / np.linalg.norm(v, axis=1, keepdims=True)
    if t == PRIM_BOX:
        h = q[0:3]
        areas = np.array([h[1] * h[2], h[0] * h[2], h[0] * h[1]] * 2)
        face = rng.choice(6, n, p=areas / areas.sum())
        u = rng.uniform(-1.0, 1.0, (n, 3)) * h
        axis = face % 3
        sign = np.where(face < 3, 1.0, -1.0)
        u[np.arange(n), axis] = sign * h[axis]
        return c + u
    h, r = q[0:3], q[3]
    L = 2.0 * np.linalg.norm(h)
    axis = h / np.linalg.norm(h)
    side = rng.uniform(size=n) < (2 * np.pi * r * L) / (2 * np.pi * r * L + 4 * np.pi * r * r)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    perp = v - (v @ axis)[:, None] * axis
    perp /= np.maximum(np.linalg.norm(perp, axis=1, keepdims=True), 1e-12)
    s = rng.uniform(-0.5 * L, 0.5 * L, n)
    cyl = c + s[:, None] * axis + r * perp
    cap = c + np.where((v @ axis)[:, None] >= 0, h, -h) + r * v
    return np.where(side[:, None], cyl, cap)


def surface_samples(scene: Scene, n: int, seed: int) -> np.ndarray:
    """Points on the union's surface: primitives chosen in proportion to their
    area, points on them drawn uniformly, and points inside another primitive
    (union SDF < -1e-7) rejected."""
    rng = np.random.default_rng(seed)
    areas = []
    for t, q in zip(scene.types, scene.params):
        if t == PRIM_SPHERE:
            areas.append(4 * np.pi * q[0] ** 2)
        elif t == PRIM_BOX:
            areas.append(8 * (q[0] * q[1] + q[1] * q[2] + q[0] * q[2]))
        else:
            L = 2.0 * np.linalg.norm(q[0:3])
            areas.append(2 * np.pi * q[3] * L + 4 * np.pi * q[3] ** 2)
    areas = np.array(areas)
    out = []
    have = 0
    while have < n:
        m = int((n - have) * 1.5) + 64
        which = rng.choice(scene.n, m, p=areas / areas.sum())
        pts = np.empty((m, 3))
        for p in np.unique(which):
            sel = which == p
            pts[sel] = _primitive_surface(scene, int(p), int(sel.sum()), rng)
        keep = scene_sdf(scene, pts) >= -1e-7
        keep &= np.all(np.abs(pts) <= 1.0, axis=1)
        out.append(pts[keep])
        have += int(keep.sum())
    return np.concatenate(out)[:n]


def training_batch(scene: Scene, n: int, seed: int, sigma: float = 0.01, mix: str = "half"):
    """SDF samples with float32 targets from the exact scene SDF (Sec. 3.3
    sampling).  mix "half": half near-surface (surface + N(0, sigma^2)), half
    uniform in [-1,1]^3; mix "paper": surface, near-surface and uniform points
    in the ratio 2:2:1."""
    rng = np.random.default_rng(seed + 7919)
    if mix == "paper":
        n_surf, n_near = 2 * n // 5, 2 * n // 5
        surf = surface_samples(scene, n_surf, seed)
        near = surface_samples(scene, n_near, seed + 1) + rng.normal(0.0, sigma, (n_near, 3))
        parts = [surf, near]
    elif mix == "half":
        n_near = n // 2
        parts = [surface_samples(scene, n_near, seed) + rng.normal(0.0, sigma, (n_near, 3))]
    else:
        raise ValueError(f"training_batch: unknown mix {mix!r}")
    n_uni = n - sum(len(p) for p in parts)
    parts.append(rng.uniform(-1.0, 1.0, (n_uni, 3)))
    x = np.clip(np.concatenate(parts), -1.0, 1.0).astype(np.float32)
    return x, scene_sdf(scene, x.astype(np.float64)).astype(np.float32)


def _batch_item(args):
    s, n, lod, w, h, readout = args
    sc = csg_scene(n, s)
    oc = build_octree(sc, lod + FIRST_FEATURE_DEPTH - 1)
    feats = readout_features(oc, sc) if readout else None
    oc.prim_pairs = None                         # not needed past the build; keeps the pickle small
    return sc, oc, lod, w, h, feats


def batching_workload(n_scenes: int = 32, seed: int = 0, min_prims: int = 8, max_prims: int = 256,
                      min_lod: int = 3, max_lod: int = 6, min_side: int = 128, max_side: int = 1024,
                      readout: bool = True, workers: int = 1):
    """Seeded multi-scene workload: scene s = CSG(U{min_prims..max_prims},
    seed s), octree to LOD U{min_lod..max_lod}, image U{min_side..max_side}
    wide and high (one draw each per scene, in that order, from
    default_rng(seed)).  Returns (scene, octree, lod, width, height, readout
    features or None) per scene; ``workers`` > 1 builds them in a spawned
    process pool."""
    rng = np.random.default_rng(seed)
    items = []
    for s in range(n_scenes):
        n = int(rng.integers(min_prims, max_prims + 1))
        lod = int(rng.integers(min_lod, max_lod + 1))
        w = int(rng.integers(min_side, max_side + 1))
        h = int(rng.integers(min_side, max_side + 1))
        items.append((s, n, lod, w, h, readout))
    if workers <= 1:
        return [_batch_item(a) for a in items]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batch_item, items))
