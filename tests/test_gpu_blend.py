"""Continuous LOD (Sec. 3.2 "Level Blending", Eq. 3) on the GPU vs the FP64
oracle: sdf_query_blend and sphere_trace_blend, FP32 and BF16 decode.

Tolerances are those of the plain calls: FP32 |d| within 1e-5, hit depth
within 1e-3 on rays both sides hit, normals within 0.5 degrees of the
oracle's blended gradient at the GPU's own hit point (in the voxel the GPU
stopped in).  BF16: the oracle runs with both decoders' W1 z-columns
rounded to bf16, and the query error is bounded by the blend of the two
decoders' z-rounding bounds.  An integer L~ must reproduce the plain call
bit for bit.
"""
import numpy as np
import pytest
import torch

import parity_util as P
from paper_2101_10994_gb300 import scenes as S
from test_gpu_trace import decode_bound, oracle_decoder_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    return sc, oc


def decoders(kind, in_dim=32):
    if kind == "readout":
        return {l: S.readout_decoder(l, in_dim=in_dim) for l in range(1, 6)}
    out = {}
    for l in range(1, 6):
        dd = S.init_decoder(l, in_dim)
        dd.b1 = np.random.default_rng(10 + l).normal(0, 0.1, 128).astype(np.float32)
        out[l] = dd
    return out


@pytest.mark.parametrize("kind,in_dim,fdt", [("readout", 32, "f32"), ("random", 35, "f32"), ("random", 32, "f16")])
def test_query_blend_f32(ng, oracle_mod, scene, kind, in_dim, fdt):
    sc, oc = scene
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc) if kind == "readout" else S.init_features(oc, seed=0, sigma=0.1)
    if fdt == "f16":
        feats = [f.astype(np.float16) for f in feats]
    decs = decoders(kind, in_dim)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats, fdt)
    D = {l: ng.DecoderDev.from_decoder(decs[l]) for l in decs}
    x = np.concatenate([S.points_in_voxels(oc, 7, 5000, 3), S.points_in_voxels(oc, 5, 2000, 4),
                        S.uniform_points(1000, 5)])
    tx = torch.from_numpy(x).cuda()
    for lt in (1.5, 2.25, 3.0, 4.75):
        ls = int(np.floor(lt))
        got = ng.sdf_query_blend(svo, F, D[ls], D[min(ls + 1, 5)], tx, lt).cpu().numpy().astype(np.float64)
        ref = ora.sdf_query_blend(feats, decs[ls], decs[min(ls + 1, 5)], x, lt)
        scale = max(1.0, float(np.abs(ref).max()))
        assert np.abs(got - ref).max() <= 1e-5 * scale, (lt, np.abs(got - ref).max())
        if lt == 3.0:
            plain = ng.sdf_query(svo, F, D[3], tx, 3).cpu()
            assert torch.equal(plain, torch.from_numpy(got.astype(np.float32)))
    svo.free()


def test_query_blend_bf16_within_rounding_bound(ng, oracle_mod, scene):
    sc, oc = scene
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.init_features(oc, seed=0, sigma=0.1)
    decs = decoders("random", 32)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats)
    D = {l: ng.DecoderDev.from_decoder(decs[l]) for l in decs}
    x = np.concatenate([S.points_in_voxels(oc, 7, 6000, 3), S.uniform_points(1000, 4)])
    tx = torch.from_numpy(x).cuda()
    for lt in (2.5, 4.25):
        ls = int(np.floor(lt))
        a = lt - ls
        got = ng.sdf_query_blend(svo, F, D[ls], D[ls + 1], tx, lt, decode="bf16").cpu().numpy().astype(np.float64)
        lo, hi = oracle_decoder_for(decs[ls], "bf16"), oracle_decoder_for(decs[ls + 1], "bf16")
        ref = ora.sdf_query_blend(feats, lo, hi, x, lt)

        def bound(dec, lod):
            z = ora.feature_sum(feats, x, lod)
            return 2.0 ** -8 * (np.abs(dec.W2.astype(np.float64))[None, :] *
                                (np.abs(z) @ np.abs(dec.W1.astype(np.float64)).T)).sum(1)
        b = (1 - a) * bound(lo, ls) + a * bound(hi, ls + 1)
        assert np.all(np.abs(got - ref) <= b + 1e-5), (np.abs(got - ref) - b).max()
    svo.free()


def blended_unit_normal(ora, oc, feats, dlo, dhi, lt, vox):
    """x -> the oracle's unit gradient of the blend, evaluated with x clamped
    into the GPU's hit voxels (depth of LOD ceil(L~))."""
    ls = int(np.floor(lt))
    a = lt - ls
    lo, s = P.voxel_lo(oc, ls + S.FIRST_FEATURE_DEPTH, vox)

    def unit(xx):
        xc = np.clip(xx, lo + 1e-4 * s, lo + s - 1e-4 * s).astype(np.float32)
        _, _, g0 = ora.sdf_query(feats, dlo, xc, ls, grad=True)
        _, _, g1 = ora.sdf_query(feats, dhi, xc, ls + 1, grad=True)
        g = (1 - a) * g0 + a * g1
        return g / np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-300)
    return unit


@pytest.mark.parametrize("decode", ["f32", "bf16"])
def test_trace_blend_vs_oracle(ng, oracle_mod, scene, decode):
    # hit masks, hit depth (eps straddles counted, parity_util) and every hit
    # normal (one-sided at ReLU kinks) against the oracle's blended trace
    sc, oc = scene
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc)
    decs = decoders("readout")
    lt = 4.25
    ls = 4
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats)
    dlo, dhi = ng.DecoderDev.from_decoder(decs[ls]), ng.DecoderDev.from_decoder(decs[ls + 1])
    o, d, _ = S.camera_rays(384, 384, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, ng.blend_lists_lod(lt))
    out = ng.sphere_trace_blend(svo, F, dlo, dhi, to, td, lists, lt, max_steps=128, decode=decode)
    ng.sphere_trace_status(out)
    g = {k: v.cpu().numpy() for k, v in out.items() if k != "work"}
    sel = np.random.default_rng(4).choice(len(o), 2500, replace=False)
    olo, ohi = oracle_decoder_for(decs[ls], decode), oracle_decoder_for(decs[ls + 1], decode)
    ref = ora.sphere_trace_blend(feats, olo, ohi, o[sel], d[sel], lt, eps=1e-3, max_steps=128)
    gh, rh = g["hit"][sel].astype(bool), ref["hit"].astype(bool)
    both = gh & rh
    assert both.sum() > 500
    xg = P.hit_points(o[sel], d[sel], g["t"][sel], gh)
    xo = P.hit_points(o[sel], d[sel], ref["t"], rh)
    # the blend of the two decoders' bounds on |GPU decode - oracle decode|
    a = lt - ls
    bound = np.maximum(*[(1 - a) * decode_bound(ora, feats, olo, ls, x, decode) +
                         a * decode_bound(ora, feats, ohi, ls + 1, x, decode) for x in (xg, xo)])
    strad = P.straddles(lambda x: ora.sdf_query_blend(feats, olo, ohi, x, lt), 1e-3, bound, xo, xg)
    assert int((gh != rh).sum()) <= 2 and np.all(strad[gh != rh])
    dt = np.abs(g["t"][sel].astype(np.float64) - ref["t"])
    far = both & (dt > 1e-3)
    assert np.all(strad[far]) and far.sum() <= max(2, int(0.005 * both.sum())), far.sum()
    if decode == "f32":
        assert (g["steps"][sel] == ref["steps"]).mean() >= 0.999
    unit = blended_unit_normal(ora, oc, feats, olo, ohi, lt, g["hit_voxel"][sel][gh])
    a0, amin = P.min_normal_angle(unit, xg[gh], g["normal"][sel][gh].astype(np.float64))
    print(f"\nBLEND PARITY {decode}: {int(both.sum())} hits, {int((gh != rh).sum())} mismatches, {int(far.sum())} "
          f"straddles beyond 1e-3, normals max {amin.max():.3f} deg ({int((a0 > 0.5).sum())} at a kink)")
    assert amin.max() <= 0.5, amin.max()
    svo.free()


@pytest.mark.parametrize("decode", ["f32", "bf16"])
def test_trace_blend_integer_lod_is_plain(ng, scene, decode):
    sc, oc = scene
    feats = S.readout_features(oc, sc)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats)
    D3, D4 = ng.DecoderDev.from_decoder(S.readout_decoder(3)), ng.DecoderDev.from_decoder(S.readout_decoder(4))
    o, d, _ = S.camera_rays(200, 120, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, 3)
    a = ng.sphere_trace_blend(svo, F, D3, D4, to, td, lists, 3.0, decode=decode)
    b = ng.sphere_trace(svo, F, D3, to, td, lists, decode=decode)
    for k in ("t", "hit", "steps", "normal"):
        assert torch.equal(a[k], b[k]), k
    svo.free()


def test_blend_rejects_bad_input(ng, scene):
    sc, oc = scene
    feats = S.readout_features(oc, sc)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats)
    D2 = ng.DecoderDev.from_decoder(S.readout_decoder(2))
    D3b = ng.DecoderDev.from_decoder(S.readout_decoder(3, in_dim=35))
    x = torch.from_numpy(S.uniform_points(100, 1)).cuda()
    for lt in (0.5, 5.5, float("nan")):
        with pytest.raises(ng.NglodError):
            ng.sdf_query_blend(svo, F, D2, D2, x, lt)
    with pytest.raises(ng.NglodError):
        ng.sdf_query_blend(svo, F, D2, D3b, x, 2.5)
    with pytest.raises(ng.NglodError):
        ng.sdf_query_blend(svo, F, D2, D2, x, 2.5, decode="fp8")
    o, d, _ = S.camera_rays(32, 32)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, 2)
    with pytest.raises(ValueError):
        ng.sphere_trace_blend(svo, F, D2, D2, to, td, lists, 2.5)
    svo.free()
