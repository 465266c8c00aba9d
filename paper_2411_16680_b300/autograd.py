"""torch.autograd.Functions over libquark's differentiation form (FP32).  Forward and backward run
in the library's CUDA kernels; this module only marshals tensors.

  QuarkNetworkFn  the whole novel-view render -- encoder, every Update & Fuse step with its
                  transitions, the final render -- as a function of every weight tensor it
                  depends on (quark_encode_pyramid / quark_update_fuse / quark_render_ldm forward,
                  their *_bwd calls in reverse order backward); the paper trains the whole network
                  end to end through its differentiable render (Sec. 3.1, Sec. 3.4).
  QuarkStageFn    the last Update & Fuse step and the final render, as a function of the volume
                  entering the step, the step's pyramid level and the step's weights
                  (quark_stage_forward / quark_stage_backward).
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


# ---------------------------------------------------------------------------------------------
# The whole network
# ---------------------------------------------------------------------------------------------

# weights the novel-view render depends on (W_a / b_a, the appearance decoder, do not reach it:
# the render blends the input images' colours with beta)
NETWORK_SHARED = ("enc_w", "enc_b", "v0", "w_d", "b_d", "w_sigma", "b_sigma", "W_beta")
NETWORK_STEP = ("attn_g", "Wq", "Wo", "conv_g", "conv1_w", "conv1_b", "conv2_w", "conv2_b")
NETWORK_COLLAPSE = ("col_w1", "col_b1", "col_w2", "col_b2")


def network_weight_names(cfg) -> List[str]:
    """make_weights names of every tensor QuarkNetworkFn differentiates, in its argument order."""
    names = list(NETWORK_SHARED)
    for j, (k, L) in enumerate(cfg.scales):
        names += [f"{n}_{j}" for n in NETWORK_STEP]
        if j > 0 and cfg.scales[j - 1][1] == 2 * L:
            names += [f"{n}_{j}" for n in NETWORK_COLLAPSE]
    return names


class Network:
    """One scene rendered by a context in the FP32 form: the input images (a device tensor
    [V, H, W, 3]), their cameras, the target camera and the full weight set (the differentiated
    tensors are refreshed from the Function's arguments)."""

    def __init__(self, ctx: quark.Context, images: torch.Tensor, cams, target, weights: Dict[str, np.ndarray]):
        self.ctx, self.images, self.cams, self.target = ctx, images.contiguous(), cams, target
        self.weights = {k: np.array(v, np.float32, copy=True) for k, v in weights.items()}
        self.names = network_weight_names(ctx.cfg)
        self.pyr = None
        self._loaded = None

    def load(self, tensors: List[torch.Tensor]):
        key = tuple(int(t._version) for t in tensors) + tuple(t.data_ptr() for t in tensors)
        if key == self._loaded:
            return
        for n, t in zip(self.names, tensors):
            self.weights[n] = t.detach().cpu().numpy().astype(np.float32).reshape(self.weights[n].shape)
        self.ctx.load_weights(self.weights)
        self._loaded = key

    def weight_tensors(self, device="cuda") -> List[torch.Tensor]:
        return [torch.tensor(self.weights[n], device=device) for n in self.names]

    def forward(self):
        """Encode, every step (keeping the volumes for the backward), render: (rgba, ldm)."""
        self.pyr = self.ctx.encode_pyramid(self.images, self.cams, into=self.pyr)
        ldm = self.ctx.ldm_create(self.target)
        ldm.keep_steps(True)
        for j in range(len(self.ctx.cfg.scales)):
            self.ctx.update_fuse(self.pyr, j, ldm)
        rgba = torch.empty(self.target.height, self.target.width, 4, device=self.images.device)
        self.ctx.render_ldm(ldm, self.pyr, rgba)
        return rgba, ldm

    def backward(self, ldm: quark.LDM, dl_drgb: torch.Tensor) -> Dict[str, torch.Tensor]:
        """Every differentiated weight's gradient of the loss whose RGB gradient is dl_drgb."""
        cfg, ctx, dev = self.ctx.cfg, self.ctx, self.images.device
        grads = {n: torch.zeros(self.weights[n].shape, device=dev) for n in self.names}
        V = len(self.cams)
        Hi, Wi = self.images.shape[1], self.images.shape[2]
        n = len(cfg.scales) - 1
        k, L = cfg.scales[n]
        H, W = self.target.height // k, self.target.width // k
        dv = torch.empty(L, H, W, cfg.C, device=dev)
        dbeta = torch.empty(H, W, L, V, device=dev)
        ctx.render_ldm_bwd(ldm, self.pyr, dl_drgb.contiguous().float(), dv, dbeta, grads)
        dfeat = {kk: torch.zeros(V, Hi // kk, Wi // kk, cfg.C, device=dev) for kk in {s[0] for s in cfg.scales}}
        for j in range(n, -1, -1):
            kj = cfg.scales[j][0]
            dv_prev = None
            if j > 0:
                kp, Lp = cfg.scales[j - 1]
                dv_prev = torch.empty(Lp, self.target.height // kp, self.target.width // kp, cfg.C, device=dev)
            ctx.update_fuse_bwd(self.pyr, j, ldm, dv, dbeta if j == n else None, dv_prev, dfeat[kj], grads)
            dv = dv_prev
        ctx.encode_pyramid_bwd(self.pyr, dfeat, grads)
        return grads


class QuarkNetworkFn(torch.autograd.Function):
    """rgba = network(*weights); weights in network_weight_names(cfg) order.  The loss may depend
    on the RGB channels only (the render's adjoint covers RGB)."""

    @staticmethod
    def forward(fctx, net: Network, *weights: torch.Tensor):
        net.load(list(weights))
        rgba, ldm = net.forward()
        fctx.net, fctx.ldm = net, ldm
        fctx.shapes = [w.shape for w in weights]
        return rgba

    @staticmethod
    def backward(fctx, g_rgba: torch.Tensor):
        net: Network = fctx.net
        if g_rgba[..., 3].abs().max().item() != 0.0:
            raise RuntimeError("the network's backward propagates gradients of the RGB channels only")
        grads = net.backward(fctx.ldm, g_rgba[..., :3])
        fctx.ldm.release()
        return (None,) + tuple(grads[n].reshape(s) for n, s in zip(net.names, fctx.shapes))
