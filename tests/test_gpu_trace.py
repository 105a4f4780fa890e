"""sphere_trace on the GPU vs the FP64 oracle (Sec. 3.4, A.4).

FP32 decode (CUDA cores, and the FP32-accurate tensor-core decode): hit masks
agree, hit depth within 1e-3 scene units on every ray both sides hit except
counted eps straddles, and every hit's normal within 0.5 degrees of the
oracle's gradient at the GPU's own hit point, taken in the voxel the GPU's
ray stopped in (the trilinear field's gradient jumps across voxel faces, so
"the same x" includes the voxel), or, at a ReLU kink, of the gradient of the
piece on the other side (parity_util).  BF16 decode (tensor cores): the
oracle runs with the same bf16-rounded W1 z-columns; rounding z to bf16
changes the decoded distance by at most 2^-8 sum_h |W2_h| sum_k |W1_hk z_k|,
which can move the stop test d < eps by one step on rays whose distance
lands within that bound of eps -- the straddles, the only rays allowed past
the hit-depth tolerance, each checked to be one and their number bounded.
"""
import numpy as np
import pytest
import torch

import parity_util as P
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


def trace_both(ng, ora, oc, feats, fdt, dec, lod, o, d, eps, max_steps, decode, sample=None, osc=False,
               chunks=0, ctas_per_sm=0):
    """GPU trace (single call, or with ``chunks`` the frame renderer the
    benchmark times) and the oracle's trace of the same rays (or a sample)."""
    svo = ng.svo_build(oc.keys)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    F = ng.Features(feats, fdt)
    D = ng.DecoderDev.from_decoder(dec)
    if chunks:
        from paper_2101_10994_gb300.frame import FrameRenderer
        fr = FrameRenderer(svo, F, D, to, td, lod, chunks=chunks, eps=eps, max_steps=max_steps, decode=decode,
                           ctas_per_sm=ctas_per_sm)
        fr.frame()
        fr.check()
        out = dict(fr.out)
        # the hit voxel of each ray, from each chunk's trace workspace
        out["hit_voxel"] = torch.cat([c["swork"][256:256 + 4 * c["n"]].view(torch.int32) for c in fr.chunks])
    else:
        L = ng.svo_trace_rays(svo, to, td, lod)
        out = ng.sphere_trace(svo, F, D, to, td, L, eps=eps, max_steps=max_steps, decode=decode, osc=osc,
                              normals=True, ctas_per_sm=ctas_per_sm)
        ng.sphere_trace_status(out)
    g = {k: v.cpu().numpy() for k, v in out.items() if k != "work"}
    sel = np.arange(len(o)) if sample is None else sample
    ref = ora.sphere_trace(feats, oracle_decoder_for(dec, decode), o[sel], d[sel], lod, eps=eps,
                           max_steps=max_steps, osc=osc)
    gs = {k: v[sel] for k, v in g.items()}
    svo.free()
    return gs, ref


def decode_bound(ora, feats, dec_o, lod, x, decode):
    """Bound on |GPU decode - oracle decode| at the points x (NaN rows: 0).
    FP32 decodes: the FP32 query tolerance 1e-5.  BF16: rounding z to bf16
    moves the distance by at most 2^-8 sum_h |W2_h| sum_k |W1_hk z_k|."""
    b = np.full(len(x), 1e-5)
    if decode != "bf16":
        return b
    ok = np.all(np.isfinite(x), axis=1)
    if ok.any():
        z = ora.feature_sum(feats, x[ok], lod)
        off = dec_o.in_dim - 32
        b[ok] += 2.0 ** -8 * (np.abs(dec_o.W2.astype(np.float64))[None, :] *
                              (np.abs(z) @ np.abs(dec_o.W1[:, off:].astype(np.float64)).T)).sum(1)
    return b


def compare(ora, feats, dec, lod, o, d, gs, ref, eps, decode="f32", sel=None, oc=None):
    """Hit masks, hit depths (straddles accounted) and normals at the GPU's
    own hit points in the GPU's voxels, as in parity_util."""
    o = o if sel is None else o[sel]
    d = d if sel is None else d[sel]
    dec_o = oracle_decoder_for(dec, decode)
    gh, rh = gs["hit"].astype(bool), ref["hit"].astype(bool)
    xg = P.hit_points(o, d, gs["t"], gh)
    xo = P.hit_points(o, d, ref["t"], rh)
    bound = np.maximum(decode_bound(ora, feats, dec_o, lod, xg, decode),
                       decode_bound(ora, feats, dec_o, lod, xo, decode))
    strad = P.straddles(P.oracle_distance(ora, feats, dec_o, lod), eps, bound, xo, xg)
    both = gh & rh
    dt = np.zeros(len(o))
    dt[both] = np.abs(gs["t"][both].astype(np.float64) - ref["t"][both])
    # normals: the GPU's FP32 normal vs the oracle's gradient at the GPU's
    # own hit point, in the voxel the GPU's ray stopped in
    D = lod + S.FIRST_FEATURE_DEPTH - 1
    lo, s = P.voxel_lo(oc, D, gs["hit_voxel"][gh])

    def unit(xx):
        _, _, g = ora.sdf_query(feats, dec_o, np.clip(xx, lo + 1e-4 * s, lo + s - 1e-4 * s).astype(np.float32),
                                lod, grad=True)
        return g / np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-300)
    a0, amin = P.min_normal_angle(unit, xg[gh], gs["normal"][gh].astype(np.float64))
    far = both & (dt > 1e-3)
    c = dict(mismatch=int((gh != rh).sum()), mismatch_straddle=bool(np.all(strad[gh != rh])),
             both=int(both.sum()), dt=dt[both], dt_plain=dt[both & ~strad], n_straddle_far=int(far.sum()),
             far_all_straddle=bool(np.all(strad[far])), dt_straddle_max=float(dt[far].max()) if far.any() else 0.0,
             ang=amin, n_kink=int((a0 > 0.5).sum()), ang_at_x=a0,
             steps_eq=float((gs["steps"] == ref["steps"]).mean()))
    print(f"\nTRACE PARITY lod={lod} decode={decode}: {c['both']} hits both sides, {c['mismatch']} hit-mask "
          f"mismatches; hit depth max {c['dt_plain'].max() if c['dt_plain'].size else 0:.2e} outside straddles, "
          f"{c['n_straddle_far']} straddle rays beyond 1e-3 (max {c['dt_straddle_max']:.2e}); normals max "
          f"{amin.max() if amin.size else 0:.3f} deg, {c['n_kink']} at a ReLU kink")
    return c


def assert_parity(c, max_mismatch, min_both, max_straddle_frac=0.005):
    """Every ray within the hit-depth tolerance except counted straddles; every
    mismatch a straddle; every hit normal within 0.5 degrees."""
    assert c["both"] >= min_both, c["both"]
    assert c["mismatch"] <= max_mismatch and c["mismatch_straddle"], (c["mismatch"], c["mismatch_straddle"])
    assert np.all(c["dt_plain"] <= 1e-3), c["dt_plain"].max()
    assert c["far_all_straddle"], "a ray beyond the 1e-3 hit-depth tolerance is not an eps straddle"
    assert c["n_straddle_far"] <= max(2, int(max_straddle_frac * c["both"])), c["n_straddle_far"]
    assert c["dt_straddle_max"] <= 0.05, c["dt_straddle_max"]
    assert np.all(c["ang"] <= 0.5), c["ang"].max()


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
    assert_parity(c, max_mismatch=2, min_both=1500)
    assert c["steps_eq"] >= 0.999


@pytest.mark.parametrize("decode,fdt", [("bf16", "f32"), ("bf16", "f16"), ("f32tc", "f32")])
def test_plain_sphere_in35_tensor_decodes(ng, oracle_mod, decode, fdt):
    # the warp-level tracers with the x-concatenated decoder (in_dim 35: the
    # x term added in FP32 to each unit's accumulator) against the oracle.
    # FP32-accurate: a random decoder.  BF16: the read-out decoder (a
    # distance-like field: on a random decoder, which is none, BF16 rounding
    # sends sphere-tracing trajectories elsewhere) with two more units that
    # read x, adding 0.05 w.x to the field, so the x term reaches the output
    sc, oc = S.plain_sphere(3)
    ora = oracle_mod.OracleSVO(oc.keys)
    if decode == "bf16":
        feats, dec = S.readout_features(oc, sc), S.readout_decoder(3, in_dim=35)
        w = np.array([0.3, -0.2, 0.1], np.float32)
        for u, sgn in ((2, 1.0), (3, -1.0)):
            dec.W1[u, :] = 0.0
            dec.W1[u, 0:3] = sgn * w
            dec.b1[u] = 0.0
            dec.W2[u] = sgn * 0.05
    else:
        feats, dec = S.init_features(oc, sigma=0.1), S.init_decoder(3, 35)
        dec.b1 = np.random.default_rng(0).normal(0, 0.05, 128).astype(np.float32)
    if fdt == "f16":
        feats = [f.astype(np.float16) for f in feats]
    o, d, _ = S.camera_rays(128, 128)
    gs, ref = trace_both(ng, ora, oc, feats, fdt, dec, 3, o, d, 1e-3, 32, decode)
    c = compare(ora, feats, dec, 3, o, d, gs, ref, 1e-3, decode=decode, oc=oc)
    assert_parity(c, max_mismatch=2, min_both=1500)


@pytest.mark.parametrize("decode,chunks,ctas", [("f32", 0, 0), ("f32tc", 0, 0), ("bf16", 4, 2), ("bf16", 0, 0)])
def test_csg64_lod5_1080p_sampled(ng, oracle_mod, decode, chunks, ctas):
    # the benchmark's frame: CSG-64 seed 0, LOD 5, 1920x1080 tile-ordered
    # rays, per-level FP32 feature tables, 128 steps, eps 1e-3; "f32tc" is the
    # FP32-accurate tensor-core decode (held to the FP32 tolerances), "bf16"
    # the headline decode, once through the frame renderer in the launch
    # configuration the benchmark's autotuner picks (4 chunks on 4 streams, 2
    # trace CTAs per SM) and once as a single call; 3000 sampled rays
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats, dec = S.readout_features(oc, sc), S.readout_decoder(5)
    o, d, _ = S.camera_rays(1920, 1080, tile=8)
    rng = np.random.default_rng(1)
    sel = rng.choice(len(o), 3000, replace=False)
    gs, ref = trace_both(ng, ora, oc, feats, "f32", dec, 5, o, d, 1e-3, 128, decode, sample=sel, chunks=chunks,
                         ctas_per_sm=ctas)
    c = compare(ora, feats, dec, 5, o, d, gs, ref, 1e-3, decode=decode, sel=sel, oc=oc)
    assert_parity(c, max_mismatch=2, min_both=600)


def test_trace_options_f32(ng, oracle_mod):
    sc, oc = S.csg_workload(16, seed=5, max_lod=3)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = [f.astype(np.float16) for f in S.readout_features(oc, sc)]
    dec = S.readout_decoder(3, in_dim=35)
    o, d, _ = S.camera_rays(96, 96, tile=8)
    for eps, ms, osc in ((1e-3, 1, False), (3e-4, 200, False), (1e-2, 64, True)):
        gs, ref = trace_both(ng, ora, oc, feats, "f16", dec, 3, o, d, eps, ms, "f32", osc=osc)
        c = compare(ora, feats, dec, 3, o, d, gs, ref, eps, oc=oc)
        if osc:
            # the oscillation rule stops on |d_k - d_(k-1)| < 6 eps, a second
            # comparison that can straddle; hit masks and normals as above
            assert c["mismatch"] <= 2 and c["ang"].max() <= 0.5
            assert np.mean(c["dt"] <= 1e-3) >= 0.995
        else:
            # one decode per ray: only rays starting within eps of the surface hit
            assert_parity(c, max_mismatch=2, min_both=0 if ms == 1 else 100)
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
    c = compare(ora, feats, dec, 5, o, d, gs, ref, 1e-3, decode="bf16", sel=sel, oc=oc)
    assert_parity(c, max_mismatch=3, min_both=500)


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


@pytest.mark.parametrize("decode", ["f32", "bf16", "f32tc"])
def test_entry_intervals_recomputed_bit_exact(ng, decode):
    # The tracers do not read the lists' t ranges: each entry's [t_enter,
    # t_exit] is recomputed from its voxel with the traversal's FP32 slab
    # test.  With eps above every distance a ray stops at its first decode,
    # i.e. at t = its first entry's t_enter (Sec. 3.4: t starts at the first
    # voxel), so t_hit must equal the traversal's t_range bit for bit; rays
    # starting inside occupied voxels (t_enter = 0) are included.
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(S.readout_features(oc, sc))
    dec = ng.DecoderDev.from_decoder(S.readout_decoder(5))
    o, d, _ = S.camera_rays(256, 256, tile=8)
    rng = np.random.default_rng(4)
    inside = S.points_in_voxels(oc, 7, 4000, 5).astype(np.float32)
    dirs = rng.normal(size=(4000, 3))
    dirs = (dirs / np.linalg.norm(dirs, axis=1, keepdims=True)).astype(np.float32)
    o = np.concatenate([o, inside])
    d = np.concatenate([d, dirs])
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, 5)
    out = ng.sphere_trace(svo, F, dec, to, td, lists, eps=1e9, far=1e9, max_steps=1, decode=decode, normals=False)
    ng.sphere_trace_status(out)
    offs = lists.ray_offsets.cpu().numpy()
    tr = lists.t_range.cpu().numpy()
    nonempty = offs[1:] > offs[:-1]
    assert nonempty.sum() > 20000 and nonempty[-4000:].sum() > 3000
    hit = out["hit"].cpu().numpy().astype(bool)
    assert np.array_equal(hit, nonempty)
    t = out["t"].cpu().numpy()
    first = tr[offs[:-1][nonempty], 0]
    assert np.array_equal(t[nonempty].view(np.uint32), first.view(np.uint32))
    assert np.sum(first == 0) > 3000           # the rays starting inside occupied voxels
    svo.free()


@pytest.mark.parametrize("decode", ["f32", "bf16", "fp8"])
def test_hit_list_in_ray_order(ng, decode):
    # after a trace the workspace holds the hit rays' ids in increasing order
    # (int32 word 2 = their count; the list starts at 256 + 4R rounded up to
    # 256), and the normals computed from it equal the ones of a second
    # trace_normals call over the same workspace
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(S.readout_features(oc, sc))
    if decode == "fp8":
        F.set_fp8_bound(svo, 5)
    dec = ng.DecoderDev.from_decoder(S.readout_decoder(5))
    o, d, _ = S.camera_rays(300, 200, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    lists = ng.svo_trace_rays(svo, to, td, 5, t_range=False)
    out = ng.sphere_trace(svo, F, dec, to, td, lists, decode=decode, normals=True)
    ng.sphere_trace_status(out)
    R = len(o)
    w = out["work"].cpu().numpy().view(np.int32)
    n = int(w[2])
    start = (256 + 4 * R + 255) // 256 * 256 // 4
    hit = out["hit"].cpu().numpy().astype(bool)
    assert n == hit.sum() > 1000
    np.testing.assert_array_equal(w[start:start + n], np.flatnonzero(hit))
    again = dict(out, normal=torch.empty_like(out["normal"]))
    ng.trace_normals(svo, F, dec, to, td, lists, again)
    assert torch.equal(again["normal"], out["normal"])
    svo.free()
