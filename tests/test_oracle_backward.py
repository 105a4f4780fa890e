"""Pins for the oracle's parameter gradients of the summed per-LOD loss (Eq. 4).

The oracle's ``sdf_backward`` returns the gradient of
sum_i sum_q g[i, q] * sdf_(lod_i)(x_q) w.r.t. the corner features of every
level, each LOD's decoder weights, and x.  It is checked against central
finite differences of the oracle's forward query in float64 (h = 1e-6 on
parameters) and, for the features, against the closed form of a readout
decoder (gradient = g * trilinear weight, only on the read channel).
"""
import numpy as np
import pytest

from paper_2101_10994_gb300 import scenes as S


@pytest.fixture(scope="module")
def setup(oracle_mod):
    sc, oc = S.plain_sphere(3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = [f.astype(np.float64) for f in S.init_features(oc, seed=1, sigma=0.3)]
    decs = [S.init_decoder(lod, 35) for lod in (1, 2, 3)]
    for dd in decs:
        dd.b1 = np.random.default_rng(5).normal(0, 0.5, 128).astype(np.float32)
        dd.b2 = 0.1
    x = S.points_in_voxels(oc, 5, 24, seed=3, margin=0.05)
    lods = [1, 2, 3]
    g = np.random.default_rng(9).normal(size=(3, 24))
    return ora, oc, feats, decs, x, lods, g


def loss(ora, feats, decs, x, lods, g):
    tot = 0.0
    for i, lod in enumerate(lods):
        sdf, _ = ora.sdf_query(feats, decs[lod - 1], x, lod)
        tot += float(g[i] @ sdf)
    return tot


def fd(ora, feats, decs, x, lods, g, arr, idx, h=1e-6):
    old = arr[idx]
    arr[idx] = old + h
    lp = loss(ora, feats, decs, x, lods, g)
    arr[idx] = old - h
    lm = loss(ora, feats, decs, x, lods, g)
    arr[idx] = old
    return (lp - lm) / (2 * h)


def as64(dec):
    dec.W1 = dec.W1.astype(np.float64)
    dec.b1 = dec.b1.astype(np.float64)
    dec.W2 = dec.W2.astype(np.float64)
    return dec


def test_backward_matches_fd(setup):
    ora, oc, feats, decs, x, lods, g = setup
    decs = [as64(d) for d in decs]
    gr = ora.sdf_backward(feats, decs, x, lods, g)
    rng = np.random.default_rng(0)
    # features: pick corners with non-zero gradient at every level
    for li in range(3):
        nz = np.argwhere(np.abs(gr["feats"][li]) > 1e-8)
        for r in nz[rng.choice(len(nz), 6, replace=False)]:
            num = fd(ora, feats, decs, x, lods, g, feats[li], tuple(r))
            assert abs(num - gr["feats"][li][tuple(r)]) < 1e-6 * max(1, abs(num))
    for li in range(3):
        d = decs[li]
        for _ in range(6):
            idx = (rng.integers(128), rng.integers(35))
            num = fd(ora, feats, decs, x, lods, g, d.W1, idx)
            assert abs(num - gr["W1"][li][idx]) < 1e-6 * max(1, abs(num))
        for _ in range(4):
            h = int(rng.integers(128))
            assert abs(fd(ora, feats, decs, x, lods, g, d.b1, h) - gr["b1"][li][h]) < 1e-6
            assert abs(fd(ora, feats, decs, x, lods, g, d.W2, h) - gr["W2"][li][h]) < 1e-6
        assert abs(gr["b2"][li] - g[li].sum()) < 1e-12


def test_feature_grad_readout_closed_form(oracle_mod):
    # Readout decoder on channel c = lod - 1: d sdf / d z = e_c, and z sums
    # psi over every level <= lod, so at each level l the 8 corner rows of
    # the voxel containing x get the trilinear weights w_c(x) on channel c
    # (summing to 1) and every other entry is zero.
    sc, oc = S.plain_sphere(3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc)
    x = S.points_in_voxels(oc, 5, 1, seed=8, margin=0.1)
    decs = [S.readout_decoder(l) for l in (1, 2, 3)]
    gr = ora.sdf_backward(feats, decs, x, [3], np.ones((1, 1)))
    xd = x[0].astype(np.float64)
    for li in range(3):
        G = gr["feats"][li].copy()
        dp = S.FIRST_FEATURE_DEPTH + li
        gl = (xd + 1.0) * 2.0 ** (dp - 1)
        ijk = np.floor(gl).astype(np.int64)
        u = gl - ijk
        ck = oc.corner_keys[li]
        total = 0.0
        for c in range(8):
            bits = [(c >> a) & 1 for a in range(3)]
            w = np.prod([u[a] if bits[a] else 1 - u[a] for a in range(3)])
            key = S.morton_encode(ijk[0] + bits[0], ijk[1] + bits[1], ijk[2] + bits[2])
            row = int(np.searchsorted(ck, key))
            assert ck[row] == key
            assert abs(G[row, 2] - w) < 1e-12
            total += G[row, 2]
            G[row, 2] = 0.0
        assert abs(total - 1.0) < 1e-12
        assert np.abs(G).max() < 1e-12
