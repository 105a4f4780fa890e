"""FP8 (E4M3) decode on the tensor cores vs the FP64 oracle.

z is scaled by 448 / B (B = sum over levels of each feature table's largest
|value|, which bounds |z|) and W1's z columns by 448 / max|W1z| (a per-LOD
scale), both rounded to e4m3 (3 mantissa bits: relative error <= 2^-4 for
normal values, absolute <= 2^-10 in scaled units below 2^-6), accumulated in
FP32.  The decoded distance then differs from the exact one by at most
sum_h |W2_h| sum_k (|W1_hk| e_z,k + e_w,hk |z_k| + e_w,hk e_z,k) -- checked
per query.  The sphere tracer's FP8 errors are reported against the oracle.
"""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def e4m3_err(v, scale):
    return 2.0 ** -4 * np.abs(v) + 2.0 ** -10 / scale


def test_fp8_query_within_rounding_bound(ng, oracle_mod):
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats = S.init_features(oc, seed=0, sigma=0.1)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats)
    B = F.set_fp8_bound(svo, 5)
    assert abs(B - sum(np.abs(f).max() for f in feats)) < 1e-6 * B
    x = np.concatenate([S.points_in_voxels(oc, 7, 6000, 3), S.uniform_points(1000, 4)])
    for in_dim in (32, 35):
        dec = S.init_decoder(5, in_dim)
        dec.b1 = np.random.default_rng(7).normal(0, 0.1, 128).astype(np.float32)
        got = ng.sdf_query(svo, F, ng.DecoderDev.from_decoder(dec), torch.from_numpy(x).cuda(), 5,
                           decode="fp8").cpu().numpy().astype(np.float64)
        ref, _ = ora.sdf_query(feats, dec, x, 5)
        z = ora.feature_sum(feats, x, 5)
        off = in_dim - 32
        W1 = dec.W1[:, off:].astype(np.float64)
        sz, sw = 448.0 / B, 448.0 / np.abs(W1).max()
        ez, ew = e4m3_err(z, sz), e4m3_err(W1, sw)
        dpre = ez @ np.abs(W1).T + np.abs(z) @ ew.T + ez @ ew.T
        bound = dpre @ np.abs(dec.W2.astype(np.float64))
        err = np.abs(got - ref)
        assert np.all(err <= bound + 1e-5), (err - bound).max()
        assert np.median(err) < 0.25 * np.median(bound)
    svo.free()


def test_fp8_trace_errors_vs_oracle(ng, oracle_mod):
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    ora = oracle_mod.OracleSVO(oc.keys)
    feats, dec = S.readout_features(oc, sc), S.readout_decoder(5)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats)
    F.set_fp8_bound(svo, 5)
    o, d, _ = S.camera_rays(512, 512, tile=8)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    L = ng.svo_trace_rays(svo, to, td, 5)
    out = ng.sphere_trace(svo, F, ng.DecoderDev.from_decoder(dec), to, td, L, eps=1e-3, max_steps=128,
                          decode="fp8")
    ng.sphere_trace_status(out)
    sel = np.random.default_rng(2).choice(len(o), 3000, replace=False)
    ref = ora.sphere_trace(feats, dec, o[sel], d[sel], 5, eps=1e-3, max_steps=128)
    gh = out["hit"].cpu().numpy()[sel].astype(bool)
    rh = ref["hit"].astype(bool)
    both = gh & rh
    dt = np.abs(out["t"].cpu().numpy()[sel][both] - ref["t"][both])
    print(f"FP8 trace: hit mismatch {int((gh != rh).sum())}/{len(sel)}, both {int(both.sum())}, "
          f"|dt| median {np.median(dt):.2e} p99 {np.percentile(dt, 99):.2e} max {dt.max():.2e}")
    assert (gh != rh).mean() < 0.02
    assert np.median(dt) < 1e-3
    svo.free()
