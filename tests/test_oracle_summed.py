"""Pins for the identity behind summed corner tables, on the oracle alone.

Inside one voxel V of LOD L, Eq. 2's z = sum over LODs 1..L of the trilinear
interpolants psi_l is trilinear: every coarser voxel holding a point of V
holds all of V, and its interpolant is a product of affine functions of the
coordinates.  So z is fixed by 8 values on V, and those values at a corner
shared by two voxels of LOD L agree (the coarser interpolants are continuous
across faces).  Checked here in FP64 with the oracle's multi-level z:

* the trilinear function through z at u in {1/4, 3/4}^3 of a voxel gives z at
  random points of that voxel to rounding;
* its corner values agree between face neighbours at their 4 shared corners;
* a sum that stopped at LOD L - 1 (a dropped level) is not the sum.
"""
import numpy as np
import pytest

from paper_2101_10994_gb300 import scenes as S


def basis(u):
    """Trilinear basis b_c(u), c = cx | cy<<1 | cz<<2, for u [n, 3] -> [n, 8]."""
    out = np.ones((u.shape[0], 8))
    for c in range(8):
        for a in range(3):
            out[:, c] *= u[:, a] if (c >> a) & 1 else 1.0 - u[:, a]
    return out


def points(ijk, u, D):
    s = 2.0 / (1 << D)
    return -1.0 + (ijk[:, None, :] + u[None, :, :]) * s      # [V, n, 3]


@pytest.fixture(scope="module")
def setup(oracle_mod):
    sc, oc = S.csg_workload(16, seed=5, max_lod=3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.init_features(oc, seed=2, sigma=0.1)
    return oc, ora, feats


def corner_values(ora, feats, ijk, lod):
    """Per voxel, the 8 corner values of the trilinear function through z at
    u in {1/4, 3/4}^3 (a dyadic design: exact sample positions)."""
    D = lod + S.FIRST_FEATURE_DEPTH - 1
    u8 = np.array([[(c & 1) * 0.5 + 0.25, ((c >> 1) & 1) * 0.5 + 0.25, ((c >> 2) & 1) * 0.5 + 0.25]
                   for c in range(8)])
    x = points(ijk, u8, D).reshape(-1, 3)
    z = ora.feature_sum(feats, x, lod).reshape(ijk.shape[0], 8, -1)
    Binv = np.linalg.inv(basis(u8))
    return np.einsum("cs,vsm->vcm", Binv, z)                    # [V, 8, m]


def test_multilevel_z_is_trilinear_in_each_voxel(setup, oracle_mod):
    oc, ora, feats = setup
    lod = 3
    D = lod + S.FIRST_FEATURE_DEPTH - 1
    rng = np.random.default_rng(0)
    keys = oc.keys[D][rng.choice(oc.keys[D].shape[0], 60, replace=False)]
    ijk = np.stack(S.morton_decode(keys), axis=1).astype(np.float64)
    Zc = corner_values(ora, feats, ijk, lod)
    u = rng.uniform(0.01, 0.99, (12, 3))
    z = ora.feature_sum(feats, points(ijk, u, D).reshape(-1, 3), lod).reshape(ijk.shape[0], 12, -1)
    pred = np.einsum("nc,vcm->vnm", basis(u), Zc)
    # the sample points are FP32 on the oracle's side: compare at the FP32
    # positions' rounding (|grad z| ~ sigma 2^D per unit, positions to 2^-24)
    assert np.abs(pred - z).max() <= 1e-6, np.abs(pred - z).max()
    # non-trivial: the field varies inside the voxels
    assert np.abs(z - z.mean(axis=1, keepdims=True)).max() > 1e-3


def test_corner_values_shared_between_neighbours(setup):
    oc, ora, feats = setup
    lod = 3
    D = lod + S.FIRST_FEATURE_DEPTH - 1
    keys = oc.keys[D]
    i, j, k = S.morton_decode(keys)
    have = set(keys.tolist())
    pairs = []
    for a in range(3):
        step = [0, 0, 0]
        step[a] = 1
        nb = S.morton_encode(i + step[0], j + step[1], k + step[2])
        for v, key in enumerate(nb.tolist()):
            if key in have:
                pairs.append((v, int(np.searchsorted(keys, key)), a))
    assert len(pairs) > 50
    pairs = pairs[:: max(1, len(pairs) // 80)]
    ijk = np.stack([i, j, k], axis=1).astype(np.float64)
    va = np.array([p[0] for p in pairs])
    vb = np.array([p[1] for p in pairs])
    Za = corner_values(ora, feats, ijk[va], lod)
    Zb = corner_values(ora, feats, ijk[vb], lod)
    for n, (_, _, a) in enumerate(pairs):
        for c in range(8):
            if (c >> a) & 1:                       # corner on a's high face = the neighbour's low face
                assert np.abs(Za[n, c] - Zb[n, c & ~(1 << a)]).max() <= 1e-6


def test_dropped_level_is_detected(setup):
    # a table built from LODs 1..L-1 only differs from the sum by the finest
    # level's interpolant: O(sigma), far above the tolerances above
    oc, ora, feats = setup
    lod = 3
    D = lod + S.FIRST_FEATURE_DEPTH - 1
    ijk = np.stack(S.morton_decode(oc.keys[D][:40]), axis=1).astype(np.float64)
    x = points(ijk, np.array([[0.3, 0.6, 0.2]]), D).reshape(-1, 3)
    full = ora.feature_sum(feats, x, lod)
    partial = full - ora.feature_sum(feats[:lod - 1] + [np.zeros_like(feats[lod - 1])], x, lod)
    assert np.abs(partial).max() > 1e-2
