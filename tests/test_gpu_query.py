"""sdf_query on the GPU vs the FP64 oracle: |dSDF| <= 1e-5 for the FP32
decode (the tolerance the method is held to), identical deepest LOD, and the
analytic input gradient; FP16 features compare against the oracle fed the
same FP16 values (promoted exactly)."""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu
TOL = 1e-5


def query_points(oc, n, seed):
    D = oc.max_depth
    pts = [S.points_in_voxels(oc, D, n, seed), S.uniform_points(n // 2, seed + 1),
           np.array([[1.0, 1.0, 1.0], [-1.0, -1.0, -1.0], [1.2, 0, 0], [0, 0, -1.5], [np.nan, 0, 0]],
                    np.float32)]
    # voxel faces at the finest depth: shared corners keep the field continuous there
    f = S.points_in_voxels(oc, D, 64, seed + 2)
    f[:, 0] = np.round((f[:, 0] + 1) * 2 ** (D - 1)) / 2 ** (D - 1) - 1
    pts.append(f.astype(np.float32))
    return np.ascontiguousarray(np.concatenate(pts), np.float32)


@pytest.mark.parametrize("scene", ["sphere", "csg"])
@pytest.mark.parametrize("in_dim", [32, 35])
@pytest.mark.parametrize("fdt", ["f32", "f16"])
def test_query_vs_oracle(ng, oracle_mod, scene, in_dim, fdt):
    if scene == "sphere":
        sc, oc = S.plain_sphere(3)
    else:
        sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    feats = S.init_features(oc, seed=0, sigma=0.1)
    if fdt == "f16":
        feats = [f.astype(np.float16) for f in feats]
    svo = ng.svo_build(oc.keys)
    ora = oracle_mod.OracleSVO(oc.keys)
    F = ng.Features(feats, fdt)
    x = query_points(oc, 3000, seed=5)
    xt = torch.from_numpy(x).cuda()
    for lod in range(1, oc.max_lod + 1):
        dec = S.init_decoder(lod, in_dim)
        dec.b1 = np.random.default_rng(lod).normal(0, 0.1, 128).astype(np.float32)
        dec.b2 = -0.05
        sdf, deep = ng.sdf_query(svo, F, ng.DecoderDev.from_decoder(dec), xt, lod, deepest=True)
        ref, rdeep = ora.sdf_query(feats, dec, x, lod)
        err = np.abs(sdf.cpu().numpy().astype(np.float64) - ref)
        assert np.nanmax(err) <= TOL, (lod, np.nanmax(err))
        np.testing.assert_array_equal(deep.cpu().numpy(), rdeep)


def test_query_gradient_vs_oracle(ng, oracle_mod):
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    feats = S.init_features(oc, seed=3, sigma=0.1)
    svo = ng.svo_build(oc.keys)
    ora = oracle_mod.OracleSVO(oc.keys)
    F = ng.Features(feats)
    x = S.points_in_voxels(oc, 7, 4000, seed=9)
    for lod, in_dim in ((5, 35), (3, 32)):
        dec = S.init_decoder(lod, in_dim)
        # biases +/-5 keep every hidden unit away from its ReLU kink, so FP32
        # and FP64 take the same branch everywhere
        dec.b1 = np.where(np.arange(128) % 2 == 0, 5.0, -5.0).astype(np.float32)
        _, g = ng.sdf_query(svo, F, ng.DecoderDev.from_decoder(dec), torch.from_numpy(x).cuda(), lod, grad=True)
        _, _, rg = ora.sdf_query(feats, dec, x, lod, grad=True)
        g = g.cpu().numpy().astype(np.float64)
        # FP32 sums of ~35 x 128 products of size |g| carry a relative error of
        # a few 1e-6 per term; 5e-5 of the largest component bounds it
        scale = np.abs(rg).max(axis=1, keepdims=True)
        assert np.all(np.abs(g - rg) <= 5e-5 * np.maximum(scale, 1.0)), np.abs(g - rg).max()
        cosang = (g * rg).sum(1) / np.linalg.norm(g, axis=1) / np.linalg.norm(rg, axis=1)
        assert np.degrees(np.arccos(np.clip(cosang, -1, 1))).max() < 0.01


def test_query_rejects_bad_args(ng):
    sc, oc = S.plain_sphere(3)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(S.init_features(oc))
    dec = ng.DecoderDev.from_decoder(S.init_decoder(1))
    x = torch.zeros((4, 3), device="cuda")
    for lod in (0, 4):
        with pytest.raises(ng.NglodError) as e:
            ng.sdf_query(svo, F, dec, x, lod)
        assert e.value.code == ng.ERR_INVALID_ARG
    bad = ng.DecoderDev(np.zeros((64, 32), np.float32), np.zeros(64, np.float32), np.zeros(64, np.float32), 0.0)
    with pytest.raises(ng.NglodError) as e:
        ng.sdf_query(svo, F, bad, x, 1)
    assert e.value.code == ng.ERR_NOT_SUPPORTED
    assert ng.sdf_query(svo, F, dec, torch.zeros((0, 3), device="cuda"), 1).numel() == 0


def test_query_full_size_sampled(ng, oracle_mod):
    # the benchmark's standalone configuration: 2^22 points uniform inside the
    # LOD-5 voxels of CSG-64, readout decoder, one call; 6000 sampled outputs
    # against the oracle (FP32 within 1e-5, BF16 within its rounding bound
    # 2^-8 |z_c| for the readout channel c)
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    feats, dec = S.readout_features(oc, sc), S.readout_decoder(5)
    svo = ng.svo_build(oc.keys)
    ora = oracle_mod.OracleSVO(oc.keys)
    x = S.points_in_voxels(oc, 7, 1 << 22, 21)
    F, D = ng.Features(feats), ng.DecoderDev.from_decoder(dec)
    xt = torch.from_numpy(x).cuda()
    sel = np.random.default_rng(0).choice(len(x), 6000, replace=False)
    ref, _ = ora.sdf_query(feats, dec, x[sel], 5)
    z = ora.feature_sum(feats, x[sel], 5)[:, 4]
    got = ng.sdf_query(svo, F, D, xt, 5).cpu().numpy()[sel].astype(np.float64)
    assert np.abs(got - ref).max() <= TOL
    got = ng.sdf_query(svo, F, D, xt, 5, decode="bf16").cpu().numpy()[sel].astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(z) + TOL)
    svo.free()


@pytest.mark.parametrize("in_dim,fdt", [(32, "f32"), (35, "f16")])
def test_query_f32tc_vs_oracle(ng, oracle_mod, in_dim, fdt):
    # the FP32-accurate tensor-core decode (three-term BF16 splits, six
    # products): the FP32 tolerance 1e-5 against the FP64 oracle
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    feats = S.init_features(oc, seed=0, sigma=0.1)
    if fdt == "f16":
        feats = [f.astype(np.float16) for f in feats]
    svo = ng.svo_build(oc.keys)
    ora = oracle_mod.OracleSVO(oc.keys)
    F = ng.Features(feats, fdt)
    x = query_points(oc, 3000, seed=7)
    xt = torch.from_numpy(x).cuda()
    for lod in (1, 3, 5):
        dec = S.init_decoder(lod, in_dim)
        dec.b1 = np.random.default_rng(lod).normal(0, 0.1, 128).astype(np.float32)
        dec.b2 = -0.05
        sdf, deep = ng.sdf_query(svo, F, ng.DecoderDev.from_decoder(dec), xt, lod, decode="f32tc", deepest=True)
        ref, rdeep = ora.sdf_query(feats, dec, x, lod)
        err = np.abs(sdf.cpu().numpy().astype(np.float64) - ref)
        assert np.nanmax(err) <= TOL, (lod, np.nanmax(err))
        np.testing.assert_array_equal(deep.cpu().numpy(), rdeep)
    svo.free()
