"""Pins for the oracle's feature query and decoder (Sec. 3.2, Eq. 2).

* Trilinear interpolation reproduces affine corner fields exactly and the
  multi-level sum is the sum of the per-level affines.
* The decoder matches a numpy float64 forward of the same weights, and a
  readout decoder returns one input coordinate exactly (x first in [x, z]).
* Shared corners make the field continuous across voxel faces.
* Corner-sampled analytic SDF converges to the sphere at O(h^2).
* Points outside every voxel see z = 0; the analytic input gradient matches
  the affine closed form and central finite differences.
"""
import json
import os

import numpy as np
import pytest

from paper_2101_10994_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def readout_on(channel, in_dim=32, hidden=128, sign_seed=0):
    dec = S.init_decoder(1, in_dim, hidden)
    dec.W1[0, :] = 0.0
    dec.W1[1, :] = 0.0
    dec.W1[0, channel] = 1.0
    dec.W1[1, channel] = -1.0
    dec.W2[:] = 0.0
    dec.W2[0], dec.W2[1] = 1.0, -1.0
    return dec


def affine_features(oc, m, seed):
    rng = np.random.default_rng(seed)
    A, b, feats = [], [], []
    for li, ck in enumerate(oc.corner_keys):
        Al = rng.normal(size=(m, 3))
        bl = rng.normal(size=m)
        p = S.corner_positions(ck, S.FIRST_FEATURE_DEPTH + li)
        feats.append(p @ Al.T + bl)
        A.append(Al)
        b.append(bl)
    return feats, A, b


@pytest.fixture(scope="module")
def sphere5(oracle_mod):
    sc, oc = S.plain_sphere(3)
    return sc, oc, oracle_mod.OracleSVO(oc.keys)


def test_paper_constants():
    g = json.load(open(GOLDEN))
    dec = S.init_decoder(1, in_dim=g["feature_dim_m"]["value"] + 3, hidden=g["hidden_dim_h"]["value"])
    assert dec.n_params() == g["inference_params_per_query"]["value"]
    kb = g["decoder_storage_kb_approx"]
    total_kb = kb["lods"] * dec.n_params() * kb["bytes_per_param"] / 1024
    assert abs(total_kb - kb["value"]) < 3.0
    # LOD l has resolution r_0 * 2^l and lives at depth l + 2
    r0 = g["initial_resolution_r0"]["value"]
    for lod in range(1, 7):
        assert 2 ** (lod + S.FIRST_FEATURE_DEPTH - 1) == r0 * 2 ** lod


@pytest.mark.parametrize("lod", [1, 2, 3])
def test_affine_field_exact(sphere5, lod):
    sc, oc, ora = sphere5
    feats, A, b = affine_features(oc, 32, seed=lod)
    x = S.points_in_voxels(oc, 5, 400, seed=11)
    for c in (0, 7, 31):
        sdf, deep = ora.sdf_query(feats, readout_on(c), x, lod)
        exp = sum(x.astype(np.float64) @ A[l][c] + b[l][c] for l in range(lod))
        np.testing.assert_allclose(sdf, exp, rtol=0, atol=1e-12)
        assert np.all(deep == lod)


def test_decoder_matches_numpy(sphere5):
    sc, oc, ora = sphere5
    feats, A, b = affine_features(oc, 32, seed=5)
    x = S.points_in_voxels(oc, 5, 300, seed=12)
    xd = x.astype(np.float64)
    z = sum(xd @ A[l].T + b[l] for l in range(3))
    for in_dim in (32, 35):
        dec = S.init_decoder(3, in_dim)
        dec.b1 = np.random.default_rng(3).normal(size=128).astype(np.float32)
        dec.b2 = 0.25
        v = np.concatenate([xd, z], axis=1) if in_dim == 35 else z
        W1 = dec.W1.astype(np.float64)
        ref = np.maximum(v @ W1.T + dec.b1.astype(np.float64), 0.0) @ dec.W2.astype(np.float64) + dec.b2
        sdf, _ = ora.sdf_query(feats, dec, x, 3)
        np.testing.assert_allclose(sdf, ref, rtol=1e-12, atol=1e-12)


def test_x_comes_first(sphere5):
    sc, oc, ora = sphere5
    feats = S.init_features(oc)
    x = S.points_in_voxels(oc, 5, 50, seed=13)
    for a in range(3):
        sdf, _ = ora.sdf_query(feats, readout_on(a, in_dim=35), x, 3)
        np.testing.assert_allclose(sdf, x[:, a].astype(np.float64), atol=1e-15)


def test_continuity_across_faces(sphere5):
    sc, oc, ora = sphere5
    feats = S.init_features(oc, seed=4)
    dec = S.init_decoder(3)
    keys = oc.keys[5]
    kset = set(int(k) for k in keys)
    i, j, k = S.morton_decode(keys)
    pts = []
    rng = np.random.default_rng(2)
    for n in range(len(keys)):
        if int(S.morton_encode(i[n] + 1, j[n], k[n])) in kset and len(pts) < 200:
            face = -1.0 + (i[n] + 1) * (2.0 / 32)
            y = -1.0 + (j[n] + rng.uniform(0.1, 0.9)) * (2.0 / 32)
            z = -1.0 + (k[n] + rng.uniform(0.1, 0.9)) * (2.0 / 32)
            pts.append((face, y, z))
    pts = np.array(pts)
    lo = pts.copy()
    lo[:, 0] = np.nextafter(pts[:, 0].astype(np.float32), np.float32(-2))
    hi = pts.copy()
    hi[:, 0] = np.nextafter(pts[:, 0].astype(np.float32), np.float32(2))
    a, _ = ora.sdf_query(feats, dec, lo.astype(np.float32), 3)
    b, _ = ora.sdf_query(feats, dec, hi.astype(np.float32), 3)
    assert len(pts) > 50
    np.testing.assert_allclose(a, b, atol=1e-5)


def test_sphere_converges_h2(oracle_mod):
    sc, oc = S.plain_sphere(5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc)
    x = S.points_in_voxels(oc, 7, 4000, seed=21)
    exact = np.linalg.norm(x.astype(np.float64), axis=1) - 0.5
    errs = []
    for lod in range(1, 6):
        sdf, _ = ora.sdf_query(feats, S.readout_decoder(lod), x, lod)
        errs.append(np.abs(sdf - exact).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    # trilinear interpolation of a smooth field: error ~ h^2, ratio ~ 4
    assert np.all(ratios > 3.5) and np.all(ratios < 4.5), (errs, ratios)
    # bound (h^2 / 8) * sum_a max|f_aa| with |f_aa| <= 1/|x|; the corners of
    # a kept voxel lie within 1.75 h of the surface, so |x| >= 0.5 - 1.75 h
    for lod, e in zip(range(2, 6), errs[1:]):
        h = 2.0 / (4 << lod)
        assert e <= h * h / 8.0 * 3.0 / (0.5 - 1.75 * h)


def test_outside_points_see_zero_features(sphere5):
    sc, oc, ora = sphere5
    feats = S.init_features(oc)
    dec = S.init_decoder(2, 35)
    dec.b1 = np.linspace(-1, 1, 128).astype(np.float32)
    dec.b2 = 0.5
    x = np.array([[1.5, 0, 0], [0, -1.01, 0], [0.0, 0.0, 0.0], [np.nan, 0, 0]], np.float32)
    sdf, deep = ora.sdf_query(feats, dec, x, 2)
    W1 = dec.W1.astype(np.float64)
    for q in (0, 1):
        v = np.concatenate([x[q].astype(np.float64), np.zeros(32)])
        ref = np.maximum(W1 @ v + dec.b1, 0) @ dec.W2.astype(np.float64) + dec.b2
        assert abs(sdf[q] - ref) < 1e-12 and deep[q] == 0
    assert deep[2] == 0          # the sphere octree has no voxel at the centre
    assert deep[3] == 0


def test_gradient_affine_and_fd(sphere5):
    sc, oc, ora = sphere5
    feats, A, b = affine_features(oc, 32, seed=9)
    x = S.points_in_voxels(oc, 5, 100, seed=31, margin=0.2)
    sdf, deep, g = ora.sdf_query(feats, readout_on(4), x, 3, grad=True)
    np.testing.assert_allclose(g, np.tile(sum(A[l][4] for l in range(3)), (100, 1)), atol=1e-11)
    # random field: central differences, h = 1e-3 (the difference of the
    # actual float32 abscissae is the denominator).  Biases of +/-5 keep every
    # hidden unit firmly on (even) or off (odd) near the samples, so no ReLU
    # kink lies between x - h and x + h; the gradient must use only the even
    # units.
    feats = S.init_features(oc, seed=3)
    dec = S.init_decoder(3, 35)
    dec.b1 = np.where(np.arange(128) % 2 == 0, 5.0, -5.0).astype(np.float32)
    _, _, g = ora.sdf_query(feats, dec, x, 3, grad=True)
    for a in range(3):
        xp, xm = x.copy(), x.copy()
        xp[:, a] += np.float32(1e-3)
        xm[:, a] -= np.float32(1e-3)
        fp, _ = ora.sdf_query(feats, dec, xp, 3)
        fm, _ = ora.sdf_query(feats, dec, xm, 3)
        fd = (fp - fm) / (xp[:, a].astype(np.float64) - xm[:, a].astype(np.float64))
        np.testing.assert_allclose(fd, g[:, a], rtol=1e-5, atol=1e-6 * np.abs(g).max())
    # all units off: the gradient vanishes
    dec.b1[:] = -5.0
    _, _, g0 = ora.sdf_query(feats, dec, x, 3, grad=True)
    assert np.all(g0 == 0.0)
