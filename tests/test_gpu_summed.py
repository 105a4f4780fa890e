"""Summed corner tables (nglod_sum_features) against the FP64 oracle.

Inside a voxel of LOD L, Eq. 2's z = sum over LODs 1..L of the trilinear
interpolants is itself trilinear (every coarser voxel holding the point holds
the whole voxel), so z equals the trilinear interpolation of its values at
the voxel's corners.  Checked here: the table interpolated at points inside
voxels reproduces the oracle's multi-level z; the tracers reading the table
(FP32, BF16 and FP32-accurate tensor-core decodes, analytic normals) meet the
per-level path's tolerances against the oracle; the chunked frame renderer
gives the single-pass output; calls that may query points outside voxels of
LOD L refuse the table.
"""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

from test_gpu_trace import compare, oracle_decoder_for

pytestmark = pytest.mark.gpu


def interp_table(svo, table, lod, n, seed, margin=1e-3):
    """Points inside random voxels of LOD ``lod`` and the trilinear
    interpolation (FP64) of the summed table at them."""
    D = lod + S.FIRST_FEATURE_DEPTH - 1
    node, corners, _ = svo.read_arrays(D)
    rng = np.random.default_rng(seed)
    v = rng.integers(0, node.shape[0], n)
    ijk = node[v, 0].astype(np.int64)
    c = np.stack([ijk & 1023, (ijk >> 10) & 1023, (ijk >> 20) & 1023], axis=1).astype(np.float64)
    s = 2.0 / (1 << D)
    x = (-1.0 + (c + rng.uniform(margin, 1.0 - margin, (n, 3))) * s).astype(np.float32)
    u = (x.astype(np.float64) + 1.0) / s - c
    z = np.zeros((n, table.shape[1]))
    for k in range(8):
        w = np.ones(n)
        for a in range(3):
            w *= u[:, a] if (k >> a) & 1 else 1.0 - u[:, a]
        z += w[:, None] * table[corners[v, k]].astype(np.float64)
    return x, z


@pytest.mark.parametrize("lod,fdt", [(3, "f32"), (5, "f32"), (5, "f16")])
def test_summed_table_reproduces_multilevel_z(ng, oracle_mod, lod, fdt):
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.init_features(oc, seed=3, sigma=0.1)
    if fdt == "f16":
        feats = [f.astype(np.float16) for f in feats]
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats, fdt)
    Fs = F.summed(svo, lod)
    assert Fs.summed_lod == lod and Fs.tables[lod - 1].shape == (svo.corners[lod - 1], 32)
    table = Fs.tables[lod - 1].cpu().numpy()
    assert np.all(np.isfinite(table))
    x, z = interp_table(svo, table, lod, 4000, seed=lod)
    ref = ora.feature_sum(feats, x, lod)
    # the table rows are FP32 roundings of FP64 sums: interpolation error
    # within a few FP32 ulps of the rows' magnitude
    err = np.abs(z - ref)
    assert err.max() <= 1e-6 * (1.0 + np.abs(ref).max()), err.max()
    # the finest level alone contributes its own corner row exactly (weight 1
    # at the corner); a table that dropped a level would be off by O(sigma)
    assert np.abs(ref).max() > 0.05
    svo.free()


def trace_summed(ng, svo, F, dec, lod, o, d, decode, sel):
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, lod)
    out = ng.sphere_trace(svo, F, ng.DecoderDev.from_decoder(dec), to, td, lists, eps=1e-3, max_steps=128,
                          decode=decode, normals=True)
    ng.sphere_trace_status(out)
    return {k: v.cpu().numpy()[sel] for k, v in out.items() if k != "work"}


@pytest.mark.parametrize("decode", ["f32", "bf16", "f32tc"])
def test_csg64_lod5_summed_trace_vs_oracle(ng, oracle_mod, decode):
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats, dec = S.readout_features(oc, sc), S.readout_decoder(5)
    svo = ng.svo_build(oc.keys)
    Fs = ng.Features(feats).summed(svo, 5)
    o, d, _ = S.camera_rays(512, 512, tile=8)
    sel = np.random.default_rng(4).choice(len(o), 3000, replace=False)
    gs = trace_summed(ng, svo, Fs, dec, 5, o, d, decode, sel)
    ref = ora.sphere_trace(feats, oracle_decoder_for(dec, decode), o[sel], d[sel], 5, eps=1e-3, max_steps=128)
    c = compare(ora, feats, dec, 5, o, d, gs, ref, 1e-3, sel=sel, oc=oc)
    assert c["both"] > 500
    if decode == "bf16":
        assert c["mismatch"] <= 3, c["mismatch"]
        assert np.mean(c["dt"] <= 1e-3) >= 0.995, np.sort(c["dt"])[-10:]
        assert c["dt"].max() <= 1e-3 + 2e-4, c["dt"].max()
    else:
        assert c["mismatch"] <= 1, c["mismatch"]
        assert c["dt"].max() <= 1e-3, c["dt"].max()
    assert c["ang"].max() <= 0.5, c["ang"].max()
    svo.free()


def test_plain_sphere_summed_x_concat(ng, oracle_mod):
    # in_dim 35 (x concatenated to z) with a random decoder: the table
    # replaces only z
    sc, oc = S.plain_sphere(3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats, dec = S.init_features(oc, sigma=0.1), S.init_decoder(3, 35)
    dec.b1 = np.random.default_rng(0).normal(0, 0.05, 128).astype(np.float32)
    svo = ng.svo_build(oc.keys)
    Fs = ng.Features(feats).summed(svo, 3)
    o, d, _ = S.camera_rays(128, 128)
    sel = np.arange(len(o))
    gs = trace_summed(ng, svo, Fs, dec, 3, o, d, "f32", sel)
    ref = ora.sphere_trace(feats, dec, o, d, 3, eps=1e-3, max_steps=128)
    c = compare(ora, feats, dec, 3, o, d, gs, ref, 1e-3, oc=oc)
    assert c["mismatch"] <= 2 and c["both"] > 1500, (c["mismatch"], c["both"])
    assert np.mean(c["dt"] <= 1e-3) >= 0.999 and c["dt"].max() <= 1.5e-3, c["dt"].max()
    assert c["ang"].max() <= 0.5, c["ang"].max()
    svo.free()


def test_summed_frame_renderer_equals_single_pass(ng):
    from paper_2101_10994_gb300.frame import FrameRenderer
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    svo = ng.svo_build(oc.keys)
    Fs = ng.Features(S.readout_features(oc, sc)).summed(svo, 5)
    D = ng.DecoderDev.from_decoder(S.readout_decoder(5))
    o, d, _ = S.camera_rays(640, 360, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, 5)
    ref = ng.sphere_trace(svo, Fs, D, to, td, lists, decode="bf16", normals=True)
    fr = FrameRenderer(svo, Fs, D, to, td, 5, chunks=3, decode="bf16")
    fr.frame()
    fr.check()
    for k in ("t", "hit", "steps", "normal"):
        assert torch.equal(fr.out[k], ref[k]), k
    # trace_normals on the recorded hits gives the tracer's normals
    n2 = ref["normal"].clone().zero_()
    out2 = dict(ref)
    out2["normal"] = n2
    ng.trace_normals(svo, Fs, D, to, td, lists, out2)
    torch.cuda.synchronize()
    assert torch.equal(n2[ref["hit"].bool()], ref["normal"][ref["hit"].bool()])
    svo.free()


def test_summed_table_refused_off_voxel(ng):
    sc, oc = S.csg_workload(16, seed=5, max_lod=3)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(S.readout_features(oc, sc))
    Fs = F.summed(svo, 3)
    D = ng.DecoderDev.from_decoder(S.readout_decoder(3))
    x = torch.zeros((64, 3), device="cuda")
    with pytest.raises(ng.NglodError, match="summed"):
        ng.sdf_query(svo, Fs, D, x, 3)                        # points anywhere
    o, d, _ = S.camera_rays(64, 64, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, 3)
    with pytest.raises(ng.NglodError, match="summed"):
        ng.sphere_trace(svo, Fs, D, to, td, lists, normal_mode="fd")   # FD leaves the voxel
    lists2 = ng.svo_trace_rays(svo, to, td, 2)
    with pytest.raises(ng.NglodError, match="own LOD"):
        ng.sphere_trace(svo, Fs, ng.DecoderDev.from_decoder(S.readout_decoder(2)), to, td, lists2)
    with pytest.raises(ValueError):
        Fs.summed(svo, 3)                                     # already summed
    fc = Fs.c()                                               # the C call refuses it too
    rc = ng.lib().nglod_sum_features(svo.h, ng.C.byref(fc), 3, Fs.tables[2].data_ptr(), None)
    assert rc == ng.ERR_NOT_SUPPORTED and "per-LOD" in ng.lib().nglod_last_error().decode()
    # the FP8 bound of a summed table is that table's largest |value|
    b = Fs.set_fp8_bound(svo, 3)
    assert b == pytest.approx(float(Fs.tables[2].abs().max()), rel=0, abs=0)
    assert b <= F.set_fp8_bound(svo, 3) * (1 + 1e-6)
    svo.free()
