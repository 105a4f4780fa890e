"""Pins for the oracle's sphere tracing with adaptive stepping (Sec. 3.4, A.4).

* A plane SDF stored as affine corner features is decoded exactly, so the
  sphere-tracing residual follows f_(k+1) = f_k (1 + n.d): the step count,
  the hit depth, the max-step cut-off, the far-plane clip and the optional
  oscillation rule all have closed forms.
* Corner-sampled analytic sphere: hits converge to the analytic root
  b - sqrt(b^2 - c) within the interpolation bound, and normals to x/|x|
  at O(h).
* Rays with an empty voxel list miss with zero steps.
"""
import math

import numpy as np
import pytest

from paper_2101_10994_gb300 import scenes as S


def plane_setup(cos_nd=-0.3, offset=0.1):
    n = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
    tvec = np.cross(n, [0.0, 0.0, 1.0])
    tvec /= np.linalg.norm(tvec)
    d = cos_nd * n + math.sqrt(1 - cos_nd ** 2) * tvec
    p_star = offset * n
    o = p_star - 3.5 * d
    oc = S.full_octree(3)
    ck = oc.corner_keys[0]
    p = S.corner_positions(ck, 3)
    f = np.zeros((ck.shape[0], 32))
    f[:, 0] = p @ n - offset
    dec = S.readout_decoder(1)
    return oc, [f], dec, n, offset, o.astype(np.float32)[None], d.astype(np.float32)[None]


def plane_sequence(ora, oc, o, d, n, offset, eps, max_steps, far=5.0, osc=False):
    """Closed-form step count / hit depth for the plane (float64)."""
    offs, vid, tr = ora.trace_rays(o, d, 1)
    t = float(tr[0, 0])
    od, dd = o[0].astype(np.float64), d[0].astype(np.float64)
    ratio = 1.0 + float(n @ dd)
    f = float(n @ (od + t * dd)) - offset
    prev = None
    for k in range(1, max_steps + 1):
        if f < eps:
            return True, t, k
        if osc and prev is not None and abs(f - prev) < 6 * eps:
            return abs(f) < 6 * eps, (t if abs(f) < 6 * eps else math.inf), k
        prev = f
        t += f
        if t > far:
            return False, math.inf, k
        f *= ratio
    return False, math.inf, max_steps


@pytest.fixture(scope="module")
def plane(oracle_mod):
    oc, feats, dec, n, off, o, d = plane_setup()
    return oracle_mod.OracleSVO(oc.keys), oc, feats, dec, n, off, o, d


@pytest.mark.parametrize("eps,max_steps", [(1e-3, 200), (3e-4, 200), (1e-3, 10)])
def test_plane_closed_form(plane, eps, max_steps):
    ora, oc, feats, dec, n, off, o, d = plane
    hit, t, k = plane_sequence(ora, oc, o, d, n, off, eps, max_steps)
    out = ora.sphere_trace(feats, dec, o, d, 1, eps=eps, max_steps=max_steps)
    assert out["steps"][0] == k
    assert bool(out["hit"][0]) == hit
    if hit:
        assert abs(out["t"][0] - t) < 1e-12
        # converged to the true plane crossing at t = 3.5 within eps / |n.d|
        assert abs(out["t"][0] - 3.5) < eps / 0.3 + 1e-9
        np.testing.assert_allclose(out["normal"][0], n, atol=1e-12)
    else:
        assert math.isinf(out["t"][0])
    if max_steps == 200:
        assert hit and k > 15          # residual ratio 0.7: many steps


def test_plane_far_and_oscillation(plane):
    ora, oc, feats, dec, n, off, o, d = plane
    out = ora.sphere_trace(feats, dec, o, d, 1, eps=1e-3, max_steps=200, far=3.0)
    hit, t, k = plane_sequence(ora, oc, o, d, n, off, 1e-3, 200, far=3.0)
    assert not hit and not out["hit"][0] and out["steps"][0] == k
    for eps in (1e-3, 1e-2):
        out = ora.sphere_trace(feats, dec, o, d, 1, eps=eps, max_steps=200, osc=True)
        hit, t, k = plane_sequence(ora, oc, o, d, n, off, eps, 200, osc=True)
        assert out["steps"][0] == k and bool(out["hit"][0]) == hit
        if hit:
            assert abs(out["t"][0] - t) < 1e-12


def test_sphere_hits_analytic_root(oracle_mod):
    sc, oc = S.plain_sphere(3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc)
    o, d, _ = S.camera_rays(96, 96)
    out = ora.sphere_trace(feats, S.readout_decoder(3), o, d, 3, eps=1e-3, max_steps=32)
    od, dd = o.astype(np.float64), d.astype(np.float64)
    b = -(od * dd).sum(1)
    c = (od * od).sum(1) - 0.25
    disc = b * b - c
    miss_dist = np.sqrt(np.maximum((od * od).sum(1) - b * b, 0))
    clear = miss_dist < 0.45                       # analytic ray hits well inside
    assert np.all(out["hit"][clear] == 1)
    assert np.all(out["hit"][miss_dist > 0.55] == 0)
    h = out["hit"].astype(bool) & clear
    t_an = b[h] - np.sqrt(disc[h])
    x = od[h] + t_an[:, None] * dd[h]
    cos = np.abs((x / np.linalg.norm(x, axis=1, keepdims=True) * dd[h]).sum(1))
    sel = cos > 0.5
    hh = 2.0 / 32
    bound = (hh * hh / 8.0 * 3.0 / (0.5 - 1.75 * hh) + 1e-3) / cos[sel]
    assert np.all(np.abs(out["t"][h][sel] - t_an[sel]) <= bound)
    assert sel.sum() > 500


def test_sphere_normals_converge(oracle_mod):
    sc, oc = S.plain_sphere(5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc)
    o, d, _ = S.camera_rays(40, 40)
    worst = []
    for lod in (3, 4, 5):
        out = ora.sphere_trace(feats, S.readout_decoder(lod), o, d, lod, eps=1e-4, max_steps=64)
        h = out["hit"].astype(bool)
        x = out["x"][h]
        nrm = x / np.linalg.norm(x, axis=1, keepdims=True)
        cosang = np.clip((out["normal"][h] * nrm).sum(1), -1, 1)
        worst.append(np.degrees(np.arccos(cosang)).mean())
    # trilinear gradients converge at O(h): the mean angle roughly halves
    assert worst[0] > worst[1] > worst[2]
    assert worst[2] < 0.6 * worst[1] and worst[1] < 0.6 * worst[0]
    assert worst[2] < 1.0


def test_empty_list_misses(oracle_mod):
    sc, oc = S.plain_sphere(3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc)
    o = np.array([[3, 3, 3], [0, 3, 0]], np.float32)
    d = np.array([[1, 0, 0], [0, 1, 0]], np.float32)
    out = ora.sphere_trace(feats, S.readout_decoder(3), o, d, 3)
    assert np.all(out["hit"] == 0) and np.all(out["steps"] == 0)
    assert np.all(np.isinf(out["t"])) and np.all(out["normal"] == 0)
