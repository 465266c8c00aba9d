"""torch.autograd.Function over the differentiable stage of libquark (FP32 form): the last Update
& Fuse step and the final render, as a function of the volume entering the step, the step's
pyramid level and the step's weights.  Forward and backward both run in the library's CUDA
kernels (quark_stage_forward / quark_stage_backward); this module only marshals tensors.
"""
from __future__ import annotations

from typing import Dict, List

import numpy as np
import torch

from . import quark

# names of the stage weights in a make_weights-style dict; {j} is the last step
STAGE_WEIGHT_NAMES = {"attn_g": "attn_g_{j}", "Wq": "Wq_{j}", "Wo": "Wo_{j}", "W_beta": "W_beta",
                      "conv_g": "conv_g_{j}", "conv1_w": "conv1_w_{j}", "conv1_b": "conv1_b_{j}",
                      "conv2_w": "conv2_w_{j}", "conv2_b": "conv2_b_{j}", "w_d": "w_d", "b_d": "b_d",
                      "w_sigma": "w_sigma", "b_sigma": "b_sigma"}


class Stage:
    """The context, pyramid and LDM a differentiable stage runs on, plus the full weight set
    (the stage's own weights are refreshed from the tensors given to the Function)."""

    def __init__(self, ctx: quark.Context, pyr: quark.Pyramid, ldm: quark.LDM, weights: Dict[str, np.ndarray],
                 target):
        self.ctx, self.pyr, self.ldm, self.target = ctx, pyr, ldm, target
        self.weights = {k: np.array(v, np.float32, copy=True) for k, v in weights.items()}
        j = len(ctx.cfg.scales) - 1
        self.names = {f: n.format(j=j) for f, n in STAGE_WEIGHT_NAMES.items()}
        self._loaded = None

    def load(self, tensors: List[torch.Tensor]):
        key = tuple(int(t._version) for t in tensors) + tuple(t.data_ptr() for t in tensors)
        if key == self._loaded:
            return
        for f, t in zip(quark.STAGE_GRAD_FIELDS, tensors):
            self.weights[self.names[f]] = t.detach().cpu().numpy().astype(np.float32).reshape(
                self.weights[self.names[f]].shape)
        self.ctx.load_weights(self.weights)
        self._loaded = key

    def weight_tensors(self, device="cuda") -> List[torch.Tensor]:
        return [torch.tensor(self.weights[self.names[f]], device=device) for f in quark.STAGE_GRAD_FIELDS]


class QuarkStageFn(torch.autograd.Function):
    """rgba = stage(v_in, feat, *weights); weights in quark.STAGE_GRAD_FIELDS order.  The loss may
    depend on the RGB channels only (the render's adjoint covers RGB)."""

    @staticmethod
    def forward(fctx, stage: Stage, v_in: torch.Tensor, feat: torch.Tensor, *weights: torch.Tensor):
        stage.load(list(weights))
        tgt = stage.ldm  # output size from the context's target
        cam = stage.target
        rgba = torch.empty(cam.height, cam.width, 4, device=v_in.device)
        stage.ctx.stage_forward(stage.pyr, feat.contiguous(), v_in.contiguous(), tgt, rgba)
        fctx.stage = stage
        fctx.shapes = [w.shape for w in weights]
        fctx.save_for_backward(v_in, feat)
        return rgba

    @staticmethod
    def backward(fctx, g_rgba: torch.Tensor):
        v_in, feat = fctx.saved_tensors
        stage: Stage = fctx.stage
        if g_rgba[..., 3].abs().max().item() != 0.0:
            raise RuntimeError("the differentiable stage propagates gradients of the RGB channels only")
        dl = g_rgba[..., :3].contiguous().float()
        dv_in = torch.empty_like(v_in)
        dfeat = torch.empty_like(feat)
        grads = {f: torch.empty(int(np.prod(s)) if len(s) else 1, device=v_in.device)
                 for f, s in zip(quark.STAGE_GRAD_FIELDS, fctx.shapes)}
        stage.ctx.stage_backward(stage.pyr, feat.contiguous(), v_in.contiguous(), stage.ldm, dl, dv_in, dfeat, grads)
        return (None, dv_in, dfeat) + tuple(grads[f].reshape(s) for f, s in zip(quark.STAGE_GRAD_FIELDS, fctx.shapes))
