"""sdf_backward on the GPU vs the FP64 oracle adjoint (itself pinned by
finite differences and closed forms): feature, decoder-weight and x gradients
of the summed per-LOD objective (Eq. 4), plus a direct finite-difference
check of the GPU gradient through the GPU forward pass."""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


# FP32 gradients summed by atomics: an element's error is a few FP32
# roundings of its own terms, which may cancel (sums over thousands of
# points of both signs), so besides 2e-5 of its own value each element is
# allowed 4e-6 of the tensor's largest element -- five times less than a
# single max-error / max-value ratio of 2e-5 would allow it, which would let
# the small gradients of corners touched by few points go unchecked.
RTOL, ATOL_FRAC = 2e-5, 4e-6


def elem_err(a, b):
    """max_i |a_i - b_i| / (RTOL |b_i| + ATOL_FRAC max|b|): <= 1 iff every
    element is within its tolerance."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(np.abs(b).max(), 1e-30)
    return float((np.abs(a - b) / (RTOL * np.abs(b) + ATOL_FRAC * scale)).max())


def kink_x_check(ora, feats, decs, x, lods, g, gx, ref_x, step=5e-5):
    """x gradients: every point within 1e-4 (relative to its largest
    component) of the oracle's, except points at a ReLU kink of one of the
    decoders, where the FP32 mask may take the other side: those must match
    the oracle's gradient a step away on one side (x +- step e_a) within the
    drift of the trilinear gradient over that step (5e-3).  Returns the
    number of kink points."""
    e = np.abs(gx - ref_x).max(axis=1) / np.maximum(np.abs(ref_x).max(axis=1), 1e-6)
    bad = np.flatnonzero(e >= 1e-4)
    if bad.size == 0:
        return 0
    best = np.full(bad.size, np.inf)
    for a in range(3):
        for sgn in (-1.0, 1.0):
            xs = x[bad].copy()
            xs[:, a] = (xs[:, a] + np.float32(sgn * step)).astype(np.float32)
            rx = ora.sdf_backward(feats, decs, xs, lods, g[:, bad])["x"]
            best = np.minimum(best, np.abs(gx[bad] - rx).max(axis=1) / np.maximum(np.abs(rx).max(axis=1), 1e-6))
    assert np.all(best < 5e-3), (bad[best >= 5e-3], best.max())
    return int(bad.size)


@pytest.mark.parametrize("scene,in_dim", [("sphere", 32), ("sphere", 35), ("csg", 32)])
def test_backward_vs_oracle(ng, oracle_mod, scene, in_dim):
    if scene == "sphere":
        sc, oc = S.plain_sphere(3)
    else:
        sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    L = oc.max_lod
    feats = S.init_features(oc, seed=2, sigma=0.1)
    decs = []
    for lod in range(1, L + 1):
        d = S.init_decoder(lod, in_dim)
        d.b1 = np.random.default_rng(lod).normal(0, 0.1, 128).astype(np.float32)
        d.b2 = 0.01 * lod
        decs.append(d)
    rng = np.random.default_rng(4)
    x = np.concatenate([S.points_in_voxels(oc, oc.max_depth, 3000, 5), S.uniform_points(1000, 6)])
    lods = list(range(1, L + 1)) if L <= 3 else [2, 4, 5]
    g = rng.normal(size=(len(lods), len(x))).astype(np.float32)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats)
    D = [ng.DecoderDev.from_decoder(d) for d in decs]
    gx = torch.zeros((len(x), 3), device="cuda")
    gr = ng.sdf_backward(svo, F, D, torch.from_numpy(x).cuda(), lods, torch.from_numpy(g).cuda(), grad_x=gx)
    ref = ora = oracle_mod.OracleSVO(oc.keys).sdf_backward(feats, decs, x, lods, g)
    for li in range(L):
        assert elem_err(gr["feats"][li].cpu().numpy(), ref["feats"][li]) <= 1, li
    for lod in lods:
        i = lod - 1
        assert elem_err(gr["W1"][i].cpu().numpy(), ref["W1"][i]) <= 1, lod
        assert elem_err(gr["b1"][i].cpu().numpy(), ref["b1"][i]) <= 1, lod
        assert elem_err(gr["W2"][i].cpu().numpy(), ref["W2"][i]) <= 1, lod
        assert abs(gr["b2"][i].item() - ref["b2"][i]) < 1e-3 * max(1.0, abs(ref["b2"][i]))
    for lod in range(1, L + 1):
        if lod not in lods:
            assert gr["W1"][lod - 1].abs().max().item() == 0.0
    # x gradient: every point, one-sided at ReLU kinks
    nk = kink_x_check(oracle_mod.OracleSVO(oc.keys), feats, decs, x, lods, g, gx.cpu().numpy().astype(np.float64),
                      ref["x"])
    assert nk <= 0.01 * len(x), nk
    svo.free()


def test_backward_fd_on_gpu(ng):
    # central differences of the GPU forward pass (h = 1e-3 on features and
    # weights) against the GPU adjoint, for the objective sum_q g_q sdf_L(x_q)
    sc, oc = S.plain_sphere(3)
    feats = S.init_features(oc, seed=2, sigma=0.1)
    dec = S.init_decoder(3, 32)
    dec.b1 = np.random.default_rng(1).normal(0, 0.1, 128).astype(np.float32)
    decs = [S.init_decoder(1, 32), S.init_decoder(2, 32), dec]
    x = S.points_in_voxels(oc, 5, 64, 7, margin=0.05)
    g = np.random.default_rng(3).normal(size=(1, len(x))).astype(np.float32)
    svo = ng.svo_build(oc.keys)
    xt = torch.from_numpy(x).cuda()
    gt = torch.from_numpy(g).cuda()
    D = [ng.DecoderDev.from_decoder(d) for d in decs]
    gr = ng.sdf_backward(svo, ng.Features(feats), D, xt, [3], gt)

    def objective(fs, dd):
        out = ng.sdf_query(svo, ng.Features(fs), ng.DecoderDev.from_decoder(dd), xt, 3).double()
        return float((out * gt[0].double()).sum())

    rng = np.random.default_rng(0)
    gf = gr["feats"][2].cpu().numpy()
    nz = np.argwhere(np.abs(gf) > 1e-3 * np.abs(gf).max())
    for r in nz[rng.choice(len(nz), 5, replace=False)]:
        fp = [f.copy() for f in feats]
        fm = [f.copy() for f in feats]
        fp[2][tuple(r)] += 1e-3
        fm[2][tuple(r)] -= 1e-3
        num = (objective(fp, dec) - objective(fm, dec)) / 2e-3
        assert abs(num - gf[tuple(r)]) < 2e-3 * max(1.0, abs(num)), (num, gf[tuple(r)])
    gw = gr["W1"][2].cpu().numpy()
    for _ in range(5):
        idx = (int(rng.integers(128)), int(rng.integers(32)))
        dp_, dm_ = S.init_decoder(3, 32), S.init_decoder(3, 32)
        for dd in (dp_, dm_):
            dd.b1 = dec.b1.copy()
        dp_.W1[idx] += 1e-3
        dm_.W1[idx] -= 1e-3
        num = (objective(feats, dp_) - objective(feats, dm_)) / 2e-3
        assert abs(num - gw[idx]) < 2e-3 * max(1.0, abs(num)), (num, gw[idx])
    svo.free()


def test_l2_backward_vs_oracle(ng, oracle_mod):
    # fused prediction + residual + adjoint == oracle adjoint of
    # scale * sum_L sum_q (sdf_L - d)^2, with g computed from oracle predictions
    sc, oc = S.csg_workload(16, seed=1, max_lod=4)
    feats = S.init_features(oc, seed=3, sigma=0.1)
    decs = [S.init_decoder(l, 32) for l in range(1, 5)]
    for i, d in enumerate(decs):
        d.b1 = np.random.default_rng(i).normal(0, 0.1, 128).astype(np.float32)
        d.b2 = 0.02
    x, tgt = S.training_batch(sc, 4096, 11)
    lods = [1, 3, 4]
    scale = 1.0 / len(x)
    svo = ng.svo_build(oc.keys)
    D = [ng.DecoderDev.from_decoder(d) for d in decs]
    grads = ng.new_grads(svo, D)
    loss = torch.zeros(4, device="cuda")
    ng.sdf_l2_backward(svo, ng.Features(feats), D, torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda(),
                       lods, scale, grads, loss)
    ora = oracle_mod.OracleSVO(oc.keys)
    g = []
    for i, lod in enumerate(lods):
        pred, _ = ora.sdf_query(feats, decs[lod - 1], x, lod)
        g.append(scale * 2.0 * (pred - tgt))
        assert abs(loss[lod - 1].item() - ((pred - tgt) ** 2).sum()) < 1e-4 * ((pred - tgt) ** 2).sum()
    ref = ora.sdf_backward(feats, decs, x, lods, np.array(g))
    for li in range(4):
        assert elem_err(grads["feats"][li].cpu().numpy(), ref["feats"][li]) <= 1, li
    for lod in lods:
        assert elem_err(grads["W1"][lod - 1].cpu().numpy(), ref["W1"][lod - 1]) <= 1
        assert elem_err(grads["W2"][lod - 1].cpu().numpy(), ref["W2"][lod - 1]) <= 1
    assert loss[1].item() == 0.0
    svo.free()


def test_adam_step_formula(ng):
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=5000).astype(np.float32)
    m0 = rng.normal(0, 0.1, 5000).astype(np.float32)
    v0 = rng.uniform(0, 0.1, 5000).astype(np.float32)
    g0 = rng.normal(size=5000).astype(np.float32)
    p, m, v, g = (torch.from_numpy(a.copy()).cuda() for a in (p0, m0, v0, g0))
    lr, b1, b2, eps, t = 1e-3, 0.9, 0.999, 1e-8, 7
    ng.adam_step(p, g, m, v, lr, t, b1, b2, eps)
    me = b1 * m0.astype(np.float64) + (1 - b1) * g0
    ve = b2 * v0.astype(np.float64) + (1 - b2) * g0.astype(np.float64) ** 2
    pe = p0 - lr * (me / (1 - b1 ** t)) / (np.sqrt(ve / (1 - b2 ** t)) + eps)
    # FP32 kernel vs FP64 formula: 1 - 0.999 rounded to FP32 is off by 5e-5
    # relative, which bounds the error of v (and of the step through sqrt(v))
    np.testing.assert_allclose(m.cpu().numpy(), me, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(v.cpu().numpy(), ve, rtol=1e-4, atol=1e-9)
    np.testing.assert_allclose(p.cpu().numpy(), pe, rtol=1e-5, atol=1e-6)
    assert g.abs().max().item() == 0.0


@pytest.mark.parametrize("fdtype,in_dim", [("f32", 32), ("f16", 35)])
def test_deterministic_backward(ng, oracle_mod, fdtype, in_dim):
    # deterministic=1: two runs give bit-identical gradients, the feature
    # gradients are also identical when the points come in another order,
    # and the values agree with the FP64 oracle adjoint and the atomic path.
    # Hidden units sit firmly on or off (biases +-1 against pre-activations
    # of spread ~0.1), so no FP32-vs-FP64 ReLU flip among the 72k
    # (query, LOD) pairs moves a coarse corner's summed gradient.
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    feats = S.init_features(oc, seed=2, sigma=0.1)
    decs = []
    for lod in range(1, 6):
        d = S.init_decoder(lod, in_dim)
        d.b1 = np.where(np.random.default_rng(lod).random(128) < 0.5, 1.0, -1.0).astype(np.float32)
        decs.append(d)
    x = np.concatenate([S.points_in_voxels(oc, 7, 20000, 5), S.uniform_points(4000, 6)])
    lods = [2, 4, 5]
    g = np.random.default_rng(4).normal(size=(len(lods), len(x))).astype(np.float32)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats, dtype=fdtype)
    D = [ng.DecoderDev.from_decoder(d) for d in decs]
    xt, gt = torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()

    def run(det, perm=None):
        xx, gg = (xt, gt) if perm is None else (xt[perm].contiguous(), gt[:, perm].contiguous())
        gx = torch.zeros((len(x), 3), device="cuda")
        gr = ng.sdf_backward(svo, F, D, xx, lods, gg, grad_x=gx, deterministic=det)
        torch.cuda.synchronize()
        return gr, gx
    a, ax = run(True)
    b, bx = run(True)
    for k in ("W1", "b1", "W2"):
        for i in range(5):
            assert torch.equal(a[k][i], b[k][i]), (k, i)
    assert torch.equal(a["b2"], b["b2"])
    for li in range(5):
        assert torch.equal(a["feats"][li], b["feats"][li]), li
    assert torch.equal(ax, bx)
    perm = torch.randperm(len(x), generator=torch.Generator().manual_seed(0)).cuda()
    p, _ = run(True, perm)
    for li in range(5):
        assert torch.equal(a["feats"][li], p["feats"][li]), li
    f, _ = run(False)
    ffeats = [t.astype(np.float16).astype(np.float32) for t in feats] if fdtype == "f16" else feats
    ref = oracle_mod.OracleSVO(oc.keys).sdf_backward(ffeats, decs, x, lods, g)
    for li in range(5):
        assert elem_err(a["feats"][li].cpu().numpy(), ref["feats"][li]) <= 1, li
        assert elem_err(a["feats"][li].cpu().numpy(), f["feats"][li].cpu().numpy()) <= 1, li
    for lod in lods:
        i = lod - 1
        for k in ("W1", "b1", "W2"):
            assert elem_err(a[k][i].cpu().numpy(), ref[k][i]) <= 1, (k, lod)
        assert abs(a["b2"][i].item() - ref["b2"][i]) < 1e-3 * max(1.0, abs(ref["b2"][i]))
    svo.free()


def test_deterministic_backward_nonfinite(ng):
    # a non-finite upstream gradient turns every output of the call into NaN
    sc, oc = S.plain_sphere(3)
    feats = S.init_features(oc, seed=2, sigma=0.1)
    decs = [S.init_decoder(l, 32) for l in (1, 2, 3)]
    x = S.points_in_voxels(oc, 5, 256, 7)
    g = np.ones((1, len(x)), np.float32)
    g[0, 17] = np.inf
    svo = ng.svo_build(oc.keys)
    gr = ng.sdf_backward(svo, ng.Features(feats), [ng.DecoderDev.from_decoder(d) for d in decs],
                         torch.from_numpy(x).cuda(), [3], torch.from_numpy(g).cuda(), deterministic=True)
    torch.cuda.synchronize()
    assert torch.isnan(gr["W1"][2]).all() and torch.isnan(gr["feats"][0]).all()
    svo.free()
