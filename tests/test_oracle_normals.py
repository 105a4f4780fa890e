"""Pins of the oracle's finite-difference normals (supplementary Sec. A.4):
closed forms on affine fields, where central differences are exact, and
agreement with the independently pinned analytic gradient on a smooth
(kink-free) random field, where they converge to it as O(h^2)."""
import numpy as np
import pytest

from paper_2101_10994_gb300 import scenes as S

from test_oracle_query import affine_features, readout_on


@pytest.fixture(scope="module")
def sphere5(oracle_mod):
    sc, oc = S.plain_sphere(3)
    return sc, oc, oracle_mod.OracleSVO(oc.keys)


def angle_deg(a, b):
    a = a / np.linalg.norm(a, axis=1, keepdims=True)
    b = b / np.linalg.norm(b, axis=1, keepdims=True)
    return np.degrees(np.arccos(np.clip((a * b).sum(1), -1.0, 1.0)))


@pytest.mark.parametrize("lod", [1, 3])
def test_fd_normal_affine_closed_form(sphere5, lod):
    # z_c(x) = sum_l A_l[c] . x + b_l[c] inside the octree: the FD normal is
    # A[c] / |A[c]| up to the FP32 rounding of x +- h (relative ~1e-4 of h)
    sc, oc, ora = sphere5
    feats, A, b = affine_features(oc, 32, seed=20 + lod)
    x = S.points_in_voxels(oc, 5, 300, seed=12, margin=0.2)
    for c in (0, 13):
        n = ora.fd_normals(feats, readout_on(c), x, lod, h=1e-3)
        exp = np.tile(sum(A[l][c] for l in range(lod)), (len(x), 1))
        assert np.abs(np.linalg.norm(n, axis=1) - 1.0).max() < 1e-12
        assert angle_deg(n, exp).max() < 0.01, angle_deg(n, exp).max()
        # a flipped sign or a swapped axis is far off
        assert angle_deg(n, -exp).min() > 170.0


def test_fd_normal_blend_affine_closed_form(sphere5):
    # Eq. 3 on affine fields: (1 - alpha) sum_(l<=L*) A_l + alpha sum_(l<=L*+1) A_l
    sc, oc, ora = sphere5
    feats, A, b = affine_features(oc, 32, seed=7)
    x = S.points_in_voxels(oc, 5, 300, seed=13, margin=0.2)
    c = 5
    n = ora.fd_normals(feats, readout_on(c), x, None, h=1e-3, dec_hi=readout_on(c), lod_tilde=2.25)
    g = 0.75 * (A[0][c] + A[1][c]) + 0.25 * (A[0][c] + A[1][c] + A[2][c])
    assert angle_deg(n, np.tile(g, (len(x), 1))).max() < 0.01


def test_fd_normal_equals_gradient_inside_voxels(sphere5):
    # hidden units firmly on (even) or off (odd): no ReLU kink near the
    # samples, so the decoder is affine in [x, z]; z is trilinear, i.e. affine
    # in each coordinate with the others fixed.  Within one voxel the SDF is
    # then exactly linear along each axis and the central difference equals
    # the analytic gradient (independently pinned) for every step h that
    # stays inside the voxel, up to the FP32 rounding of x +- h.
    sc, oc, ora = sphere5
    feats = S.init_features(oc, seed=3, sigma=0.1)
    dec = S.init_decoder(3, 35)
    dec.b1 = np.where(np.arange(128) % 2 == 0, 5.0, -5.0).astype(np.float32)
    x = S.points_in_voxels(oc, 5, 300, seed=31, margin=0.4)   # >= 0.025 from every face
    _, _, g = ora.sdf_query(feats, dec, x, 3, grad=True)
    for h in (2e-2, 4e-3, 1e-3):
        e = angle_deg(ora.fd_normals(feats, dec, x, 3, h=h), g)
        assert e.max() < 0.005, (h, e.max())
