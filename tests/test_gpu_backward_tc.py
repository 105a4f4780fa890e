"""The tensor-core adjoint (BF16 operands, FP32 accumulation) against the
FP32 adjoint of the same objective (itself checked against the FP64 oracle).

The decoders' hidden units sit firmly on or off (biases +-1 against
pre-activations of spread ~0.1), so rounding v = [z | x] to BF16 (relative
2^-9) flips no ReLU mask; every remaining difference is BF16 rounding of
dpre, v and W1 inside the three contractions, a relative error of at most
2^-8 per product.  The checks: per tensor, the largest difference within
2^-6 of the tensor's largest value and the relative Frobenius error below
2^-7; the L2 loss (its prediction reads the BF16 pre-activations) within
2^-7; and training with the tensor-core adjoint lowers the loss as the FP32
one does."""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def firm_decoders(L, in_dim):
    decs = []
    for lod in range(1, L + 1):
        d = S.init_decoder(lod, in_dim)
        d.b1 = np.where(np.random.default_rng(lod).random(128) < 0.5, 1.0, -1.0).astype(np.float32)
        d.b2 = 0.01 * lod
        decs.append(d)
    return decs


def close(a, b, what):
    a = a.detach().cpu().numpy().astype(np.float64)
    b = b.detach().cpu().numpy().astype(np.float64)
    m = np.abs(b).max()
    if m == 0.0:
        assert np.abs(a).max() == 0.0, what
        return
    assert np.abs(a - b).max() <= 2.0 ** -6 * m, (what, np.abs(a - b).max() / m)
    assert np.linalg.norm(a - b) <= 2.0 ** -7 * np.linalg.norm(b), (what, np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("in_dim,fdt,order", [(32, "f32", "given"), (35, "f16", "given"), (32, "f32", "sorted"),
                                               (35, "f32", "sorted")])
def test_tc_backward_matches_fp32(ng, in_dim, fdt, order):
    # "sorted": the points reordered by their depth-7 cells, so the warps'
    # corner updates merge (one atomic per block of samples in a voxel)
    sc, oc = S.csg_workload(64, seed=0, max_lod=5)
    feats = S.init_features(oc, seed=2, sigma=0.1)
    decs = firm_decoders(5, in_dim)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats, fdt)
    D = [ng.DecoderDev.from_decoder(d) for d in decs]
    x = np.concatenate([S.points_in_voxels(oc, 7, 30000, 5), S.uniform_points(3000, 6)])   # ragged last tile
    lods = [2, 4, 5]
    g = np.random.default_rng(4).normal(size=(len(lods), len(x))).astype(np.float32)
    xt, gt = torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()
    if order == "sorted":
        xt, _, perm = ng.sort_points(xt, None, 7)
        gt = gt[:, perm.long()].contiguous()
    ref = ng.sdf_backward(svo, F, D, xt, lods, gt)
    got = ng.sdf_backward(svo, F, D, xt, lods, gt, mma="bf16")
    for li in range(5):
        close(got["feats"][li], ref["feats"][li], f"feats{li}")
    for lod in lods:
        for k in ("W1", "b1", "W2"):
            close(got[k][lod - 1], ref[k][lod - 1], f"{k}{lod}")
    close(got["b2"], ref["b2"], "b2")
    for lod in (1, 3):
        assert float(got["W1"][lod - 1].abs().max()) == 0.0
    svo.free()


def test_tc_l2_backward_and_loss(ng):
    sc, oc = S.csg_workload(16, seed=1, max_lod=4)
    feats = S.init_features(oc, seed=3, sigma=0.1)
    decs = firm_decoders(4, 32)
    x, tgt = S.training_batch(sc, 5000, 11)
    svo = ng.svo_build(oc.keys)
    F = ng.Features(feats)
    D = [ng.DecoderDev.from_decoder(d) for d in decs]
    xt, tt = torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda()
    lods = [1, 3, 4]
    out = {}
    for mma in ("f32", "bf16"):
        grads = ng.new_grads(svo, D)
        loss = torch.zeros(4, device="cuda")
        ng.sdf_l2_backward(svo, F, D, xt, tt, lods, 1.0 / len(x), grads, loss, mma=mma)
        out[mma] = (grads, loss)
    (gr, lr), (gb, lb) = out["f32"], out["bf16"]
    for lod in lods:
        assert abs(lb[lod - 1].item() - lr[lod - 1].item()) <= 2.0 ** -7 * lr[lod - 1].item()
    assert lb[1].item() == 0.0
    for li in range(4):
        close(gb["feats"][li], gr["feats"][li], f"feats{li}")
    for lod in lods:
        for k in ("W1", "b1", "W2"):
            close(gb[k][lod - 1], gr[k][lod - 1], f"{k}{lod}")
    svo.free()


def test_tc_training_lowers_loss(ng):
    from paper_2101_10994_gb300.train import Trainer
    sc, oc = S.csg_workload(16, seed=1, max_lod=3)
    svo = ng.svo_build(oc.keys)
    x, tgt = S.training_batch(sc, 1 << 14, 5)
    xt, tt = torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda()
    final = {}
    for mma in ("f32", "bf16"):
        tr = Trainer(svo, S.init_features(oc, seed=0, sigma=0.01), [S.init_decoder(l, 32) for l in (1, 2, 3)],
                     lr=1e-2, mma=mma)
        first = tr.step(xt, tt).cpu().numpy()
        for _ in range(40):
            last = tr.step(xt, tt).cpu().numpy()
        assert np.all(last < 0.5 * first), (mma, first, last)
        final[mma] = last
    assert np.all(final["bf16"] < 1.5 * final["f32"]), final
    svo.free()
