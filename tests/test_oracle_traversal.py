"""Pins for the oracle's ray/voxel lists (Sec. 3.4; supplementary Sec. C).

The oracle computes each ray's list by brute force over every voxel of the
target depth, ordered by the front-to-back child order.  These tests pin it
to things other than itself:

* hand-derived lists for axis-aligned rays (closed-form entry/exit times);
* the tie rule for a ray lying in a centre plane (origin octant with >=);
* an independent float64 3D-DDA (Amanatides & Woo grid walk) on dense
  octrees -- same voxels, same order, same entry/exit times;
* on a sparse octree, the DDA walk filtered to occupied voxels (the
  hierarchical culling loses nothing);
* degenerate inputs: R = 0, NaN rays, zero directions, parallel axes.
"""
import math

import numpy as np
import pytest

from paper_2101_10994_gb300 import scenes as S


def dda_walk(o, d, res):
    """Ordered grid cells crossed by the ray (t > 0) in [-1,1]^3, float64."""
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    t0, t1 = 0.0, math.inf
    for a in range(3):
        if d[a] == 0.0:
            if not (-1.0 <= o[a] <= 1.0):
                return []
            continue
        ta, tb = (-1.0 - o[a]) / d[a], (1.0 - o[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    if t0 > t1:
        return []
    h = 2.0 / res
    p = o + t0 * d
    cell = [min(res - 1, max(0, int(math.floor((p[a] + 1.0) / h)))) for a in range(3)]
    step = [1 if d[a] > 0 else -1 for a in range(3)]
    tnext, tdelta = [], []
    for a in range(3):
        if d[a] == 0.0:
            tnext.append(math.inf)
            tdelta.append(math.inf)
        else:
            edge = (cell[a] + (1 if d[a] > 0 else 0)) * h - 1.0
            tnext.append((edge - o[a]) / d[a])
            tdelta.append(h / abs(d[a]))
    out, t = [], t0
    while True:
        a = int(np.argmin(tnext))
        out.append((tuple(cell), t, min(tnext[a], t1)))
        t = tnext[a]
        cell[a] += step[a]
        tnext[a] += tdelta[a]
        if not (0 <= cell[a] < res) or t > t1:
            break
    return out


def ray_list(ora, o, d, lod):
    offs, vid, tr = ora.trace_rays(np.asarray(o, np.float32)[None], np.asarray(d, np.float32)[None], lod)
    return vid[offs[0]:offs[1]], tr[offs[0]:offs[1]]


@pytest.fixture(scope="module")
def dense4(oracle_mod):
    return oracle_mod.OracleSVO(S.full_octree(4).keys)


def test_axis_ray_closed_form(dense4):
    # res 16 (LOD 2): ray along +x at y, z inside cell (9, 3): x cells 0..15,
    # t_enter = 2 + i/8, t_exit = 2 + (i+1)/8, all exact in FP32.
    y0, z0 = -1.0 + 9.5 / 8, -1.0 + 3.25 / 8
    vid, tr = ray_list(dense4, (-3.0, y0, z0), (1.0, 0.0, 0.0), 2)
    exp = S.morton_encode(np.arange(16), 9, 3).astype(np.int64)
    assert vid.tolist() == exp.tolist()
    np.testing.assert_array_equal(tr[:, 0], 2.0 + np.arange(16) / 8.0)
    np.testing.assert_array_equal(tr[:, 1], 2.0 + (np.arange(16) + 1) / 8.0)
    # reversed direction visits the cells in reverse order
    vid2, tr2 = ray_list(dense4, (3.0, y0, z0), (-1.0, 0.0, 0.0), 2)
    assert vid2.tolist() == exp[::-1].tolist()
    np.testing.assert_array_equal(tr2[:, 0], 2.0 + np.arange(16) / 8.0)


def test_center_plane_tie_rule(dense4):
    # Ray lying in the plane y = 0 (a centre plane at every depth): closed
    # intervals make both rows j = 7 and j = 8 hit.  The origin octant uses
    # o_y >= c_y, so the upper row comes first at the root and within it the
    # cells run along +x; then the lower row.
    z0 = -1.0 + 5.5 / 8
    vid, tr = ray_list(dense4, (-3.0, 0.0, z0), (1.0, 0.0, 0.0), 2)
    exp = np.concatenate([S.morton_encode(np.arange(8), 8, 5), S.morton_encode(np.arange(8, 16), 8, 5),
                          S.morton_encode(np.arange(8), 7, 5), S.morton_encode(np.arange(8, 16), 7, 5)])
    # at the root the x order splits into halves: (x lo, y hi), (x hi, y hi),
    # (x lo, y lo), (x hi, y lo)
    assert vid.tolist() == exp.astype(np.int64).tolist()
    assert len(vid) == 32


@pytest.mark.parametrize("lod", [1, 2])
def test_dense_matches_dda(dense4, lod):
    rng = np.random.default_rng(7)
    res = 4 << lod
    n_rays = 300
    dirs = rng.normal(size=(n_rays, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    origins = -3.0 * dirs + rng.uniform(-0.9, 0.9, (n_rays, 3))
    o32 = origins.astype(np.float32)
    d32 = dirs.astype(np.float32)
    offs, vid, tr = dense4.trace_rays(o32, d32, lod)
    checked = 0
    for r in range(n_rays):
        walk = dda_walk(o32[r], d32[r], res)
        exp = [int(S.morton_encode(*c)) for c, _, _ in walk]
        got = vid[offs[r]:offs[r + 1]].tolist()
        assert got == exp, f"ray {r}"
        if walk:
            tin = np.array([w[1] for w in walk])
            tout = np.array([w[2] for w in walk])
            np.testing.assert_allclose(tr[offs[r]:offs[r + 1], 0], tin, rtol=0, atol=2e-6)
            np.testing.assert_allclose(tr[offs[r]:offs[r + 1], 1], tout, rtol=0, atol=2e-6)
            # generic rays: entry times non-decreasing along the list
            assert np.all(np.diff(tr[offs[r]:offs[r + 1], 0]) >= 0)
            checked += 1
    assert checked > 250


def test_sparse_is_filtered_dda(oracle_mod):
    sc, oc = S.csg_workload(16, seed=3, max_lod=3)
    ora = oracle_mod.OracleSVO(oc.keys)
    occupied = set(int(k) for k in oc.keys[5])
    index = {int(k): i for i, k in enumerate(oc.keys[5])}
    o, d, _ = S.camera_rays(24, 24)
    offs, vid, tr = ora.trace_rays(o, d, 3)
    for r in range(o.shape[0]):
        exp = [index[k] for k in (int(S.morton_encode(*c)) for c, _, _ in dda_walk(o[r], d[r], 32))
               if k in occupied]
        assert vid[offs[r]:offs[r + 1]].tolist() == exp


def test_degenerate_rays(dense4):
    # R = 0
    offs, vid, tr = dense4.trace_rays(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), 1)
    assert offs.tolist() == [0] and vid.size == 0
    o = np.array([[np.nan, 0, 0], [-3, 0.1, 0.1], [-3, 0.1, 0.1], [-3, 5.0, 0.1],
                  [0.05, 0.05, 0.05]], np.float32)
    d = np.array([[1, 0, 0], [0, 0, 0], [np.nan, 0, 0], [1, 0, 0], [0, 0, 1]], np.float32)
    offs, vid, tr = dense4.trace_rays(o, d, 1)
    n = np.diff(offs)
    assert n[0] == 0          # NaN origin
    assert n[1] == 0          # zero direction
    assert n[2] == 0          # NaN direction
    assert n[3] == 0          # parallel to x, outside the y slab
    # origin inside the cube: first voxel contains it, entered at t = 0
    assert n[4] == 4 and tr[offs[4], 0] == 0.0
    assert vid[offs[4]] == int(S.morton_encode(4, 4, 4))


def test_subset_lemma_on_hierarchy(oracle_mod):
    # Every hit voxel's parent is hit by the same ray (FP32 monotone rounding),
    # so coarse culling never drops a fine hit.
    sc, oc = S.csg_workload(16, seed=5, max_lod=2)
    ora = oracle_mod.OracleSVO(oc.keys)
    o, d, _ = S.camera_rays(20, 20)
    fine = ora.trace_rays(o, d, 2)
    coarse = ora.trace_rays(o, d, 1)
    for r in range(o.shape[0]):
        f = set((oc.keys[4][v] >> np.uint64(3)).item() for v in fine[1][fine[0][r]:fine[0][r + 1]])
        c = set(oc.keys[3][v].item() for v in coarse[1][coarse[0][r]:coarse[0][r + 1]])
        assert f <= c
