"""The SDF of Eq. 2 as a differentiable PyTorch function.

The forward pass is the library's FP32 sdf_query; the backward pass is its
adjoint, sdf_backward (gradients of the features of every level, of the
LOD's decoder and of x, interpolation weights recomputed, never stored).
PyTorch only holds the leaf tensors and chains the gradients; every step of
the SDF and of its gradient runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import nglod as ng


class NeuralSDF:
    """Corner features of LODs 1..L and the per-LOD decoders as leaf tensors
    that require gradients."""

    def __init__(self, svo: ng.SVO, feats, decoders, device="cuda"):
        import torch
        self.svo = svo
        self.feats = [torch.as_tensor(np.asarray(f), dtype=torch.float32).to(device).requires_grad_()
                      for f in feats]
        self.W1 = [torch.as_tensor(np.asarray(d.W1), dtype=torch.float32).to(device).requires_grad_() for d in decoders]
        self.b1 = [torch.as_tensor(np.asarray(d.b1), dtype=torch.float32).to(device).requires_grad_() for d in decoders]
        self.W2 = [torch.as_tensor(np.asarray(d.W2), dtype=torch.float32).to(device).requires_grad_() for d in decoders]
        self.b2 = torch.tensor([float(d.b2) for d in decoders], dtype=torch.float32, device=device,
                               requires_grad=True)

    def parameters(self):
        return self.feats + self.W1 + self.b1 + self.W2 + [self.b2]

    def __call__(self, x, lod: int):
        return _SDF.apply(x, int(lod), self, *self.parameters())


def _views(field):
    F = ng.Features.from_tensors([f.detach() for f in field.feats])
    b2 = field.b2.detach()
    decs = [ng.DecoderDev.from_tensors(w1.detach(), b1.detach(), w2.detach(), b2[i:i + 1])
            for i, (w1, b1, w2) in enumerate(zip(field.W1, field.b1, field.W2))]
    return F, decs


def _make_sdf():
    import torch

    class SDF(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, lod, field, *params):
            F, decs = _views(field)
            ctx.save_for_backward(x)
            ctx.lod, ctx.field = lod, field
            return ng.sdf_query(field.svo, F, decs[lod - 1], x.detach().contiguous(), lod)

        @staticmethod
        def backward(ctx, g):
            (x,) = ctx.saved_tensors
            field, lod = ctx.field, ctx.lod
            F, decs = _views(field)
            grads = ng.new_grads(field.svo, decs, x.device)
            gx = torch.zeros_like(x) if ctx.needs_input_grad[0] else None
            ng.sdf_backward(field.svo, F, decs, x.detach().contiguous(), [lod],
                            g.detach().reshape(1, -1).contiguous().float(), grads, gx)
            out = [gx, None, None]
            out += grads["feats"][:len(field.feats)]
            out += grads["W1"] + grads["b1"] + grads["W2"] + [grads["b2"]]
            return tuple(out)

    return SDF


class _Lazy:
    _fn = None

    def apply(self, *a):
        if _Lazy._fn is None:
            _Lazy._fn = _make_sdf()
        return _Lazy._fn.apply(*a)


_SDF = _Lazy()
