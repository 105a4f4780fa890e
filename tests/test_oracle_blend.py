"""Pins of the oracle's continuous LOD (Sec. 3.2 "Level Blending", Eq. 3)
and of the LOD selection of Sec. 3.4.

The readout scene gives a closed form independent of the oracle's feature
machinery: with readout features and decoders, LOD L decodes exactly I_L,
the trilinear interpolant of the (FP32-stored) analytic SDF at the corners
of the depth-(L+2) cell containing x.  So Eq. 3 must give
(1 - alpha) I_L* + alpha I_(L*+1), computed here from scene_sdf at the 8
corners of each cell -- a dropped weight, a swapped alpha or a wrong level
fails it.
"""
import numpy as np
import pytest

from paper_2101_10994_gb300 import scenes as S


def interp_readout(scene, lod, x):
    """I_L(x) from scene_sdf at the corners of x's depth-(lod+2) cell."""
    D = lod + S.FIRST_FEATURE_DEPTH - 1
    sc = float(1 << (D - 1))
    x64 = np.asarray(x, np.float64)
    x32 = x64.astype(np.float32)
    # the cell by the FP32 rule of Sec. 3.2's point location, the weights in FP64
    ijk = np.clip(np.floor((x32 + np.float32(1.0)).astype(np.float64) * sc), 0, (1 << D) - 1)
    u = np.clip((x64 + 1.0) * sc - ijk, 0.0, 1.0)
    h = 2.0 / (1 << D)
    out = np.zeros(len(x))
    for c in range(8):
        off = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], np.float64)
        corner = -1.0 + (ijk + off) * h
        f = S.scene_sdf(scene, corner).astype(np.float32).astype(np.float64)
        w = np.prod(np.where(off[None, :] > 0, u, 1.0 - u), axis=1)
        out += w * f
    return out


def blended_closed_form(scene, lod_tilde, x):
    lstar = int(np.floor(lod_tilde))
    a = lod_tilde - lstar
    lo = interp_readout(scene, lstar, x)
    return lo if a == 0 else (1 - a) * lo + a * interp_readout(scene, lstar + 1, x)


@pytest.fixture(scope="module")
def csg():
    sc, oc = S.csg_workload(16, seed=5, max_lod=4)
    return sc, oc, S.readout_features(oc, sc)


@pytest.mark.parametrize("lod_tilde", [1.0, 1.5, 2.25, 3.75, 4.0])
def test_query_blend_readout_closed_form(oracle_mod, csg, lod_tilde):
    sc, oc, feats = csg
    ora = oracle_mod.OracleSVO(oc.keys)
    lstar = int(np.floor(lod_tilde))
    hi = min(lstar + 1, 4)
    # points inside voxels of the finer LOD, where both terms are defined
    x = S.points_in_voxels(oc, hi + S.FIRST_FEATURE_DEPTH - 1, 3000, 11)
    got = ora.sdf_query_blend(feats, S.readout_decoder(lstar), S.readout_decoder(hi), x, lod_tilde)
    ref = blended_closed_form(sc, lod_tilde, x)
    assert np.abs(got - ref).max() < 1e-9, np.abs(got - ref).max()


def test_query_blend_is_linear_in_alpha(oracle_mod, csg):
    # d(L* + a) is affine in a between the two integer LODs (Eq. 3)
    sc, oc, feats = csg
    ora = oracle_mod.OracleSVO(oc.keys)
    dec2, dec3 = S.init_decoder(2), S.init_decoder(3)
    x = S.uniform_points(2000, 3)
    d2, _ = ora.sdf_query(feats, dec2, x, 2)
    d3, _ = ora.sdf_query(feats, dec3, x, 3)
    for a in (0.125, 0.5, 0.875):
        got = ora.sdf_query_blend(feats, dec2, dec3, x, 2 + a)
        assert np.allclose(got, d2 + a * (d3 - d2), rtol=0, atol=1e-12)


def test_trace_blend_alpha_limits(oracle_mod):
    sc, oc = S.plain_sphere(3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc)
    o, d, _ = S.camera_rays(48, 48)
    plain3 = ora.sphere_trace(feats, S.readout_decoder(3), o, d, 3, eps=1e-3, max_steps=64)
    # alpha = 1 on lists at L* + 1 is the plain trace at L* + 1, bit for bit
    b1 = ora.sphere_trace_blend(feats, S.readout_decoder(2), S.readout_decoder(3), o, d, 2.0, eps=1e-3,
                                max_steps=64, alpha=1.0)
    for k in ("t", "hit", "steps", "normal"):
        assert np.array_equal(b1[k], plain3[k]), k
    # an integer L~ is the plain trace at L~
    plain2 = ora.sphere_trace(feats, S.readout_decoder(2), o, d, 2, eps=1e-3, max_steps=64)
    b0 = ora.sphere_trace_blend(feats, S.readout_decoder(2), S.readout_decoder(3), o, d, 2.0, eps=1e-3,
                                max_steps=64)
    for k in ("t", "hit", "steps", "normal"):
        assert np.array_equal(b0[k], plain2[k]), k


def test_trace_blend_stops_on_the_blended_field(oracle_mod):
    sc, oc = S.plain_sphere(3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc)
    o, d, _ = S.camera_rays(64, 64)
    eps, lt = 1e-3, 2.25      # alpha = 0.25: a swapped alpha changes the field
    out = ora.sphere_trace_blend(feats, S.readout_decoder(2), S.readout_decoder(3), o, d, lt, eps=eps,
                                 max_steps=64)
    h = out["hit"].astype(bool)
    assert h.sum() > 500
    xh = out["x"][h]
    # the stop rule of Sec. A.4 on Eq. 3's field, evaluated independently
    F = blended_closed_form(sc, lt, xh)
    assert np.all(F < eps + 1e-12)
    # the first crossing: still positive a few eps before the hit
    back = xh - 3 * eps * d[h].astype(np.float64)
    assert np.all(blended_closed_form(sc, lt, back) > 0)
    # both interpolants approximate |x| - 0.5 (to ~h^2 / 8 * |curvature| at
    # the coarser level), so the blended hits lie on the sphere to that
    # order, and away from the silhouette at the analytic root
    r = np.linalg.norm(xh, axis=1)
    assert np.abs(r - 0.5).max() < 0.012, np.abs(r - 0.5).max()
    oo = o[h].astype(np.float64)
    dd = d[h].astype(np.float64)
    b = -(oo * dd).sum(1)
    c = (oo * oo).sum(1) - 0.25
    facing = b * b - c > 0.05
    t_true = b - np.sqrt(np.maximum(b * b - c, 0.0))
    assert np.abs(out["t"][h] - t_true)[facing].max() < 0.02
    # normal: the normalised gradient of the blended field (central
    # differences of the closed form, away from cell faces of both levels)
    hs = 1e-6
    g = np.zeros_like(xh)
    for a in range(3):
        e = np.zeros(3)
        e[a] = hs
        g[:, a] = (blended_closed_form(sc, lt, xh + e) - blended_closed_form(sc, lt, xh - e)) / (2 * hs)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    far_from_faces = np.ones(len(xh), bool)
    for lod in (2, 3):
        D = lod + S.FIRST_FEATURE_DEPTH - 1
        f = (xh + 1.0) * (1 << (D - 1))
        far_from_faces &= np.all(np.abs(f - np.round(f)) > 1e-3, axis=1)
    ang = np.degrees(np.arccos(np.clip((out["normal"][h] * g).sum(1), -1, 1)))[far_from_faces]
    assert far_from_faces.sum() > 300
    assert ang.max() < 0.01, ang.max()


def test_lod_select(oracle_mod):
    sel = oracle_mod.lod_select
    assert sel(0.5, 1.0, 3.0, 5.0, 2.0) == 5.0
    assert sel(1.0, 1.0, 3.0, 5.0, 2.0) == 5.0
    assert sel(2.0, 1.0, 3.0, 5.0, 2.0) == 3.5
    assert sel(3.0, 1.0, 3.0, 5.0, 2.0) == 2.0
    assert sel(9.0, 1.0, 3.0, 5.0, 2.0) == 2.0
    dist = np.linspace(0, 5, 101)
    v = sel(dist, 1.0, 3.0, 5.0, 2.0)
    assert np.all(np.diff(v) <= 0)


def test_library_lod_select_matches(oracle_mod):
    # a host function of the library (no device work)
    from paper_2101_10994_gb300 import nglod as ng
    for dist in np.linspace(0, 5, 41):
        for (dn, df, ln, lf) in ((1.0, 3.0, 5.0, 2.0), (0.5, 4.0, 1.0, 6.0)):
            assert abs(ng.lod_select(dist, dn, df, ln, lf) - oracle_mod.lod_select(dist, dn, df, ln, lf)) < 1e-6
