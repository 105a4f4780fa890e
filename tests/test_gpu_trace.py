"""sphere_trace on the GPU vs the FP64 oracle (Sec. 3.4, A.4).

FP32 decode: identical hit masks, hit depth within 1e-3 scene units, and
normals within 0.5 degrees of the oracle's gradient at the GPU's own hit
point, taken in the voxel the GPU's ray stopped in (the trilinear field's
gradient jumps across voxel faces, so "the same x" includes the voxel).  BF16 decode (tensor cores): the oracle runs with the same
bf16-rounded W1 z-columns; rounding z to bf16 changes the decoded distance by
at most 2^-8 sum_h |W2_h| sum_k |W1_hk z_k|, which can move the stop test
d < eps by one step of size ~eps on rays whose distance lands within that
bound of eps -- those are the only allowed hit-depth outliers.
"""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).bfloat16().float().numpy()


def oracle_decoder_for(dec, decode):
    if decode != "bf16":
        return dec
    d2 = S.Decoder(dec.W1.copy(), dec.b1.copy(), dec.W2.copy(), dec.b2, dec.in_dim)
    off = dec.in_dim - 32
    d2.W1[:, off:] = bf16_round(dec.W1[:, off:])
    return d2


def trace_both(ng, ora, oc, feats, fdt, dec, lod, o, d, eps, max_steps, decode, sample=None, osc=False):
    svo = ng.svo_build(oc.keys)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    L = ng.svo_trace_rays(svo, to, td, lod)
    F = ng.Features(feats, fdt)
    out = ng.sphere_trace(svo, F, ng.DecoderDev.from_decoder(dec), to, td, L, eps=eps, max_steps=max_steps,
                          decode=decode, osc=osc, normals=True)
    ng.sphere_trace_status(out)
    g = {k: v.cpu().numpy() for k, v in out.items() if k != "work"}
    sel = np.arange(len(o)) if sample is None else sample
    ref = ora.sphere_trace(feats, oracle_decoder_for(dec, decode), o[sel], d[sel], lod, eps=eps,
                           max_steps=max_steps, osc=osc)
    gs = {k: v[sel] for k, v in g.items()}
    svo.free()
    return gs, ref


def oracle_normal_in_voxel(ora, oc, feats, dec, lod, x, vox):
    """Oracle gradient direction at x, inside the given target-depth voxel
    (x is clamped into the voxel by 1e-4 of its size, so a hit on a face is
    evaluated in the voxel the tracer stopped in)."""
    D = lod + S.FIRST_FEATURE_DEPTH - 1
    i, j, k = S.morton_decode(oc.keys[D][vox])
    s = 2.0 / (1 << D)
    lo = np.stack([-1 + i * s, -1 + j * s, -1 + k * s], axis=1)
    def unit(xx):
        _, _, g = ora.sdf_query(feats, dec, np.clip(xx, lo + 1e-4 * s, lo + s - 1e-4 * s).astype(np.float32),
                                lod, grad=True)
        return g / np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-300)
    n0 = unit(x)
    # a ReLU kink within 5e-5 of x makes the gradient ill-defined there; a
    # point whose oracle direction moves by more than 0.2 degrees (under half
    # the 0.5-degree tolerance) within that radius is reported as not stable
    # instead of compared
    stable = np.ones(len(x), bool)
    for a in range(3):
        for sgn in (-1.0, 1.0):
            xs = x.copy()
            xs[:, a] += sgn * 5e-5
            stable &= np.degrees(np.arccos(np.clip((unit(xs) * n0).sum(1), -1, 1))) <= 0.2
    return n0, stable


def compare(ora, feats, dec, lod, o, d, gs, ref, eps, decode="f32", sel=None, oc=None):
    o = o if sel is None else o[sel]
    d = d if sel is None else d[sel]
    gh, rh = gs["hit"].astype(bool), ref["hit"].astype(bool)
    mismatch = int((gh != rh).sum())
    both = gh & rh
    dt = np.abs(gs["t"][both].astype(np.float64) - ref["t"][both])
    # normals at the same x: the GPU's FP32 normal vs the oracle's gradient
    # at the GPU's own hit point, in the voxel the GPU's ray stopped in
    x = o[gh].astype(np.float64) + gs["t"][gh].astype(np.float64)[:, None] * d[gh].astype(np.float64)
    nref, stable = oracle_normal_in_voxel(ora, oc, feats, dec, lod, x, gs["hit_voxel"][gh])
    ang = np.degrees(np.arccos(np.clip((gs["normal"][gh][stable] * nref[stable]).sum(1), -1, 1)))
    return dict(mismatch=mismatch, both=int(both.sum()), dt=dt, ang=ang,
                stable=float(stable.mean()) if stable.size else 1.0,
                steps_eq=float((gs["steps"] == ref["steps"]).mean()))


@pytest.mark.parametrize("decoder", ["readout", "random35"])
def test_plain_sphere_f32(ng, oracle_mod, decoder):
    sc, oc = S.plain_sphere(3)
    ora = oracle_mod.OracleSVO(oc.keys)
    if decoder == "readout":
        feats, dec = S.readout_features(oc, sc), S.readout_decoder(3)
    else:
        feats, dec = S.init_features(oc, sigma=0.1), S.init_decoder(3, 35)
        dec.b1 = np.random.default_rng(0).normal(0, 0.05, 128).astype(np.float32)
    o, d, _ = S.camera_rays(128, 128)
    gs, ref = trace_both(ng, ora, oc, feats, "f32", dec, 3, o, d, 1e-3, 32, "f32")
    c = compare(ora, feats, dec, 3, o, d, gs, ref, 1e-3, oc=oc)
    assert c["mismatch"] <= 2 and c["both"] > 1500, (c["mismatch"], c["both"])
    assert np.mean(c["dt"] <= 1e-3) >= 0.999 and c["dt"].max() <= 1.5e-3, c["dt"].max()
    assert c["ang"].max() <= 0.5, c["ang"].max()
    assert c["stable"] >= (0.99 if decoder == "readout" else 0.8), c["stable"]
    assert c["steps_eq"] >= 0.999


@pytest.mark.parametrize("decode", ["f32", "f32tc"])
def test_csg64_lod5_1080p_sampled_f32(ng, oracle_mod, decode):
    # the benchmark's frame, in the benchmark's configuration; "f32tc" is the
    # FP32-accurate tensor-core decode, held to the same tolerances
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats, dec = S.readout_features(oc, sc), S.readout_decoder(5)
    o, d, _ = S.camera_rays(1920, 1080, tile=8)
    rng = np.random.default_rng(1)
    sel = rng.choice(len(o), 1500, replace=False)
    gs, ref = trace_both(ng, ora, oc, feats, "f32", dec, 5, o, d, 1e-3, 128, decode, sample=sel)
    c = compare(ora, feats, dec, 5, o, d, gs, ref, 1e-3, sel=sel, oc=oc)
    assert c["mismatch"] <= 1 and c["both"] > 300
    assert c["dt"].max() <= 1e-3, c["dt"].max()
    assert c["ang"].max() <= 0.5


def test_trace_options_f32(ng, oracle_mod):
    sc, oc = S.csg_workload(16, seed=5, max_lod=3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = [f.astype(np.float16) for f in S.readout_features(oc, sc)]
    dec = S.readout_decoder(3, in_dim=35)
    o, d, _ = S.camera_rays(96, 96, tile=8)
    for eps, ms, osc in ((1e-3, 1, False), (3e-4, 200, False), (1e-2, 64, True)):
        gs, ref = trace_both(ng, ora, oc, feats, "f16", dec, 3, o, d, eps, ms, "f32", osc=osc)
        c = compare(ora, feats, dec, 3, o, d, gs, ref, eps, oc=oc)
        assert c["mismatch"] <= 2, (eps, ms, osc)
        if c["both"]:
            assert np.mean(c["dt"] <= 1e-3) >= 0.999
            assert c["ang"].max() <= 0.5
        assert c["steps_eq"] >= 0.995
        if ms == 1:
            assert np.all(gs["steps"] <= 1)


@pytest.mark.parametrize("fdt", ["f32", "f16"])
def test_csg64_lod5_bf16(ng, oracle_mod, fdt):
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats, dec = S.readout_features(oc, sc), S.readout_decoder(5)
    if fdt == "f16":
        feats = [f.astype(np.float16) for f in feats]
    o, d, _ = S.camera_rays(512, 512, tile=8)
    rng = np.random.default_rng(2)
    sel = rng.choice(len(o), 3000, replace=False)
    gs, ref = trace_both(ng, ora, oc, feats, fdt, dec, 5, o, d, 1e-3, 128, "bf16", sample=sel)
    c = compare(ora, feats, dec, 5, o, d, gs, ref, 1e-3, sel=sel, oc=oc)
    assert c["both"] > 500
    assert c["mismatch"] <= 3, c["mismatch"]
    assert np.mean(c["dt"] <= 1e-3) >= 0.995, np.sort(c["dt"])[-10:]
    assert c["dt"].max() <= 1e-3 + 2e-4, c["dt"].max()
    assert c["ang"].max() <= 0.5, c["ang"].max()


def test_bf16_query_within_rounding_bound(ng, oracle_mod):
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.init_features(oc, seed=0, sigma=0.1)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats)
    x = np.concatenate([S.points_in_voxels(oc, 7, 6000, 3), S.uniform_points(1000, 4)])
    for in_dim in (32, 35):
        dec = S.init_decoder(5, in_dim)
        dec.b1 = np.random.default_rng(7).normal(0, 0.1, 128).astype(np.float32)
        got = ng.sdf_query(svo, F, ng.DecoderDev.from_decoder(dec), torch.from_numpy(x).cuda(), 5,
                           decode="bf16").cpu().numpy().astype(np.float64)
        od = oracle_decoder_for(dec, "bf16")
        ref, _ = ora.sdf_query(feats, od, x, 5)
        z = ora.feature_sum(feats, x, 5)
        off = in_dim - 32
        bound = 2.0 ** -8 * (np.abs(od.W2.astype(np.float64))[None, :] *
                             (np.abs(z) @ np.abs(od.W1[:, off:].astype(np.float64)).T)).sum(1)
        err = np.abs(got - ref)
        assert np.all(err <= bound + 1e-5), (err - bound).max()
        assert bound.max() < 0.05
    svo.free()
