"""Central-difference normals (normal_mode "fd", supplementary Sec. A.4) on
the GPU vs the oracle's FD normals at the GPU's own hit points.

Both sides evaluate the SDF at the same FP32 points x +- h e_a (x = the
FP32 fma o + t d of the GPU's hit depth); the GPU in FP32, the oracle in
FP64.  With the FP32 query within delta = 1e-5 of the oracle, each
difference is off by at most 2 delta, so the normal's angle is off by at
most asin(2 sqrt(3) delta / |g|) for the oracle's difference vector g --
the per-ray bound the tests check.
"""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu

DELTA = 1e-5


def hit_points(o, d, t):
    x = (t.astype(np.float64)[:, None] * d.astype(np.float64) + o.astype(np.float64)).astype(np.float32)
    return x


def check(ora_normals, got, g_norm, what):
    cosang = np.clip((got * ora_normals).sum(1), -1.0, 1.0)
    ang = np.arccos(cosang)
    bound = np.arcsin(np.minimum(1.0, 2.0 * np.sqrt(3.0) * DELTA / np.maximum(g_norm, 1e-30)))
    ok = ang <= bound + 1e-6
    assert ok.all(), (what, np.degrees(ang[~ok]).max(), np.degrees(bound[~ok]).min(), int((~ok).sum()))
    assert np.abs(np.linalg.norm(got, axis=1) - 1.0).max() < 1e-5


def oracle_fd(ora, feats, dec, x, lod, h, dec_hi=None, lod_tilde=None):
    n = ora.fd_normals(feats, dec, x, lod, h=h, dec_hi=dec_hi, lod_tilde=lod_tilde)
    # |g|: the oracle's difference vector, for the per-ray bound
    pts = np.repeat(x[:, None, :], 6, axis=1)
    for a in range(3):
        pts[:, 2 * a, a] = (x[:, a] + np.float32(h)).astype(np.float32)
        pts[:, 2 * a + 1, a] = (x[:, a] - np.float32(h)).astype(np.float32)
    if lod_tilde is None:
        f, _ = ora.sdf_query(feats, dec, pts.reshape(-1, 3), lod)
    else:
        f = ora.sdf_query_blend(feats, dec, dec_hi, pts.reshape(-1, 3), lod_tilde)
    f = f.reshape(-1, 6)
    return n, np.linalg.norm(f[:, 0::2] - f[:, 1::2], axis=1)


@pytest.mark.parametrize("decoder,decode,fdt", [("readout", "f32", "f32"), ("random35", "f32", "f16"),
                                                 ("readout", "bf16", "f32")])
def test_fd_normals_vs_oracle(ng, oracle_mod, decoder, decode, fdt):
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    if decoder == "readout":
        feats, dec = S.readout_features(oc, sc), S.readout_decoder(5)
    else:
        feats, dec = S.readout_features(oc, sc), S.init_decoder(5, 35)
        dec.b1 = np.random.default_rng(0).normal(0, 0.05, 128).astype(np.float32)
    if fdt == "f16":
        feats = [f.astype(np.float16).astype(np.float32) for f in feats]
    o, d, _ = S.camera_rays(512, 512, tile=8)
    svo = ng.svo_build(oc.keys)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    L = ng.svo_trace_rays(svo, to, td, 5)
    F = ng.Features(feats, fdt)
    D = ng.DecoderDev.from_decoder(dec)
    h = 1e-3
    out = ng.sphere_trace(svo, F, D, to, td, L, eps=1e-3, max_steps=128, decode=decode, normal_mode="fd", fd_h=h)
    ng.sphere_trace_status(out)
    hit = out["hit"].cpu().numpy().astype(bool)
    n = out["normal"].cpu().numpy()
    assert np.all(n[~hit] == 0.0)
    idx = np.flatnonzero(hit)
    idx = idx[np.random.default_rng(1).choice(len(idx), min(3000, len(idx)), replace=False)]
    x = hit_points(o[idx], d[idx], out["t"].cpu().numpy()[idx])
    ref, gn = oracle_fd(ora, feats, dec, x, 5, h)
    check(ref, n[idx], gn, (decoder, decode, fdt))
    # trace_normals_fd after the same trace writes the same normals
    n2 = ng.trace_normals(svo, F, D, to, td, L, dict(out, normal=None), normal_mode="fd", fd_h=h)["normal"]
    assert torch.equal(n2, out["normal"])
    if decoder == "readout":
        # on the true SDF's interpolant the FD normal approaches the analytic
        # one (same trace, analytic mode); a random decoder's hits often sit on
        # the octree's boundary, where x +- h leaves the finest voxels and the
        # features of the missing levels drop out of the difference
        an = ng.trace_normals(svo, F, D, to, td, L, dict(out, normal=None))["normal"].cpu().numpy()
        ang = np.degrees(np.arccos(np.clip((an[hit] * n[hit]).sum(1), -1, 1)))
        assert np.median(ang) < 0.5, np.median(ang)
    svo.free()


def test_fd_normals_blend_vs_oracle(ng, oracle_mod):
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.readout_features(oc, sc)
    dlo, dhi = S.readout_decoder(3), S.readout_decoder(4)
    o, d, _ = S.camera_rays(256, 256, tile=8)
    svo = ng.svo_build(oc.keys)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lt = 3.4
    L = ng.svo_trace_rays(svo, to, td, ng.blend_lists_lod(lt))
    F = ng.Features(feats)
    h = 2e-3
    out = ng.sphere_trace_blend(svo, F, ng.DecoderDev.from_decoder(dlo), ng.DecoderDev.from_decoder(dhi), to, td, L,
                                lt, eps=1e-3, max_steps=128, normal_mode="fd", fd_h=h)
    ng.sphere_trace_status(out)
    hit = out["hit"].cpu().numpy().astype(bool)
    assert hit.sum() > 1000
    n = out["normal"].cpu().numpy()
    x = hit_points(o[hit], d[hit], out["t"].cpu().numpy()[hit])
    ref, gn = oracle_fd(ora, feats, dlo, x, None, h, dec_hi=dhi, lod_tilde=float(np.float32(lt)))
    check(ref, n[hit], gn, "blend")
    svo.free()


def test_fd_normals_reject_bad_step(ng):
    sc, oc = S.plain_sphere(3)
    feats, dec = S.readout_features(oc, sc), S.readout_decoder(3)
    svo = ng.svo_build(oc.keys)
    o, d, _ = S.camera_rays(64, 64)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    L = ng.svo_trace_rays(svo, to, td, 3)
    for h in (0.0, -1e-3, 1.5, float("nan")):
        with pytest.raises(ng.NglodError) as e:
            ng.sphere_trace(svo, ng.Features(feats), ng.DecoderDev.from_decoder(dec), to, td, L, normal_mode="fd",
                            fd_h=h)
        assert e.value.code == ng.ERR_INVALID_ARG
    svo.free()
