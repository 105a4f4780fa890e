"""Training of the octree features and per-LOD decoders on the GPU (Eq. 4).

Each step runs, per LOD, the fused prediction + L2 residual + adjoint kernel
(sdf_l2_backward) over one batch, then the Adam kernel over every parameter
tensor (features of every level, each decoder's W1, b1, W2, b2).  Only the
library's kernels touch the parameters; PyTorch holds the buffers.
"""
from __future__ import annotations

import numpy as np

from . import nglod as ng


class Trainer:
    def __init__(self, svo: ng.SVO, feats, decoders, lr: float = 1e-3, device="cuda", mma: str = "f32",
                 sort_depth: int | None = 7):
        """mma = "bf16": the adjoint's decoder contractions on the tensor cores.
        sort_depth: each batch is first reordered by the Morton code of its
        points' cells at that depth (nglod_sort_points; None: as given)."""
        import torch
        self.torch = torch
        self.svo = svo
        self.F = ng.Features(feats, "f32", device)
        D0 = [ng.DecoderDev.from_decoder(d, device) for d in decoders]
        # one device vector of the LODs' b2; each decoder points at its entry,
        # so Adam updates it in place and the kernels read it from there
        self.b2 = torch.tensor([float(d.b2) for d in decoders], dtype=torch.float32, device=device)
        self.D = [ng.DecoderDev.from_tensors(d.W1, d.b1, d.W2, self.b2[i:i + 1]) for i, d in enumerate(D0)]
        self.grads = ng.new_grads(svo, self.D, device)
        self.params = (list(self.F.tables) + [d.W1 for d in self.D] + [d.b1 for d in self.D] +
                       [d.W2 for d in self.D] + [self.b2])
        self.gparams = (list(self.grads["feats"]) + self.grads["W1"] + self.grads["b1"] + self.grads["W2"] +
                        [self.grads["b2"]])
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.lr = lr
        self.mma = mma
        self.sort_depth = None if sort_depth is None else min(int(sort_depth), 7)
        self.sort_buf = {}
        self.t = 0
        self.L = len(self.D)

    def step(self, x, target, lods=None):
        """One Adam step on a batch; returns the per-LOD mean squared error."""
        torch = self.torch
        lods = lods or list(range(1, self.L + 1))
        loss = torch.zeros(self.L, dtype=torch.float32, device=x.device)
        Q = int(x.shape[0])
        if self.sort_depth:
            x, target, _ = ng.sort_points(x, target, self.sort_depth, out=self.sort_buf)
        ng.sdf_l2_backward(self.svo, self.F, self.D, x, target, lods, 1.0 / Q, self.grads, loss, mma=self.mma)
        self.t += 1
        for p, g, m, v in zip(self.params, self.gparams, self.m, self.v):
            ng.adam_step(p, g, m, v, self.lr, self.t)
        return loss / Q

    def export(self):
        """Current parameters as numpy (features per LOD, scenes.Decoder list)."""
        from .scenes import Decoder
        feats = [t.cpu().numpy() for t in self.F.tables]
        b2 = self.b2.cpu().numpy()
        decs = [Decoder(d.W1.cpu().numpy(), d.b1.cpu().numpy(), d.W2.cpu().numpy(), float(b2[i]), d.in_dim)
                for i, d in enumerate(self.D)]
        return feats, decs
