"""sdf_query / sdf_backward as a torch.autograd.Function: PyTorch losses
differentiate through the library's kernels.  Checked against the oracle's
gradients (FP64) of the same loss."""
import numpy as np
import pytest
import torch

from paper_2101_10994_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def test_autograd_matches_oracle(ng, oracle_mod):
    from paper_2101_10994_gb300.autograd import NeuralSDF
    sc, oc = S.csg_workload(16, seed=5, max_lod=3)
    svo = ng.svo_build(oc.keys)
    feats = S.init_features(oc, seed=0, sigma=0.1)
    decs = [S.init_decoder(l, 32) for l in (1, 2, 3)]
    for l, d in enumerate(decs):
        d.b1 = np.random.default_rng(3 + l).normal(0, 0.1, 128).astype(np.float32)
    field = NeuralSDF(svo, feats, decs)
    x_np = np.concatenate([S.points_in_voxels(oc, 5, 3000, 1), S.uniform_points(500, 2)])
    x = torch.from_numpy(x_np).cuda().requires_grad_()
    target = torch.from_numpy(S.scene_sdf(sc, x_np).astype(np.float32)).cuda()
    lod = 3
    pred = field(x, lod)
    loss = ((pred - target) ** 2).sum()
    loss.backward()
    # the oracle's adjoint (FP64) for the cotangent PyTorch hands the function: 2 (pred - target)
    ora = oracle_mod.OracleSVO(oc.keys)
    pred_o, _ = ora.sdf_query(feats, decs[lod - 1], x_np, lod)
    assert np.abs(pred.detach().cpu().numpy() - pred_o).max() < 1e-5
    g = 2.0 * (pred.detach() - target).cpu().numpy()
    ref = ora.sdf_backward(feats, decs, x_np, [lod], g[None, :])

    def close(a, b, name):
        a = a.detach().cpu().numpy().astype(np.float64)
        scale = max(1.0, np.abs(b).max())
        assert np.abs(a - b).max() <= 5e-5 * scale, (name, np.abs(a - b).max(), scale)
    for l in range(lod):
        close(field.feats[l].grad, ref["feats"][l], f"feats{l}")
    close(field.W1[lod - 1].grad, ref["W1"][lod - 1], "W1")
    close(field.b1[lod - 1].grad, ref["b1"][lod - 1], "b1")
    close(field.W2[lod - 1].grad, ref["W2"][lod - 1], "W2")
    assert abs(field.b2.grad[lod - 1].item() - ref["b2"][lod - 1]) < 1e-3 * max(1.0, abs(ref["b2"][lod - 1]))
    # x gradient: ReLU kinks can sit within rounding of a point; compare the bulk
    e = np.abs(x.grad.cpu().numpy() - ref["x"]).max(axis=1) / np.maximum(np.abs(ref["x"]).max(axis=1), 1e-6)
    assert np.mean(e < 1e-4) > 0.99, np.sort(e)[-5:]
    # decoders of other LODs receive no gradient
    assert float(field.W1[0].grad.abs().max()) == 0.0
    svo.free()


def test_autograd_trains(ng):
    # a few steps of torch.optim.Adam on the Eq. 4 objective at two LODs through
    # the autograd function lower the loss
    from paper_2101_10994_gb300.autograd import NeuralSDF
    sc, oc = S.csg_workload(16, seed=1, max_lod=3)
    svo = ng.svo_build(oc.keys)
    field = NeuralSDF(svo, S.init_features(oc, seed=0, sigma=0.01),
                      [S.init_decoder(l, 32) for l in (1, 2, 3)])
    x_np = np.concatenate([S.points_in_voxels(oc, 5, 4000, 1), S.uniform_points(1000, 2)])
    x = torch.from_numpy(x_np).cuda()
    target = torch.from_numpy(S.scene_sdf(sc, x_np).astype(np.float32)).cuda()
    opt = torch.optim.Adam(field.parameters(), lr=1e-2)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        loss = sum(((field(x, l) - target) ** 2).mean() for l in (2, 3))
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert losses[-1] < 0.5 * losses[0], losses[::5]
    svo.free()
