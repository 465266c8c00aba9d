"""FP64 reference gradients of the network, by torch autograd of a float64 formulation.

TEST INFRASTRUCTURE ONLY (see quark_oracle.py); the CUDA path never imports it.

Two functions of the weights are differentiated:
  stage     the last Update & Fuse step and the final render, as a function of the volume
            entering the step, the step's pyramid level and its weights;
  network   the whole novel-view render from the input images: the encoder (3x3 conv and the
            2x2 mean-pool chain, Sec. 3.2.1), every Update & Fuse step with its transition
            (initialisation with v0 at the depth anchors, layer collapse, x2 upsample; Sec.
            3.2.2, Sec. 3.3) and the final render (Sec. 3.1 Eq. 1, Sec. 3.2.3), as a function of
            every weight tensor -- the paper trains the whole network end to end through its
            differentiable render (Sec. 3.1, Sec. 3.4).
Both are written with plain torch float64 CPU ops, following the same passages as
quark_oracle.py.  Bilinear sampling is written out as index gathers with differentiable weights,
so the gradient reaches both the sampled maps and the sample coordinates (through the decoded
depth).  The forwards equal quark_oracle.forward; the gradients are pinned to central finite
differences in tests/test_oracle_grad_pins.py.
"""
from __future__ import annotations

import math
from typing import Dict

import numpy as np
import torch

Z_MIN = 1e-6

# weight tensors of the stage, by their synth.make_weights names (j = the last step)
STAGE_WEIGHTS = ("attn_g_{j}", "Wq_{j}", "Wo_{j}", "conv_g_{j}", "conv1_w_{j}", "conv1_b_{j}", "conv2_w_{j}",
                 "conv2_b_{j}", "w_d", "b_d", "w_sigma", "b_sigma", "W_beta")


def _K(cam, k):
    return torch.tensor(np.diag([1.0 / k, 1.0 / k, 1.0]) @ cam.K, dtype=torch.float64)


def _depth(t, L, near, far):
    ell = torch.arange(1, L + 1, dtype=torch.float64).reshape((L,) + (1,) * (t.dim() - 1))
    return 1.0 / (((ell - 0.5) / L + 0.5 / L * torch.tanh(t)) * (1 / near - 1 / far) + 1 / far)


def _project(d, H, W, k, cam_t, cam_m):
    """Pixel coords in view m of target pixels (grid H x W at factor k) at depth d [L, H, W]."""
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64) + 0.5,
                            torch.arange(W, dtype=torch.float64) + 0.5, indexing="ij")
    p = torch.stack([xs, ys, torch.ones_like(xs)], -1)
    ray = p @ torch.linalg.inv(_K(cam_t, k)).T
    Xc = ray[None] * d[..., None]
    Rt = torch.tensor(cam_t.R)
    tt = torch.tensor(cam_t.t)
    Xw = (Xc - tt) @ Rt
    Xm = Xw @ torch.tensor(cam_m.R).T + torch.tensor(cam_m.t)
    z = Xm[..., 2]
    valid = z > Z_MIN
    zs = torch.where(valid, z, torch.ones_like(z))
    uvw = Xm @ _K(cam_m, k).T
    return uvw[..., 0] / zs, uvw[..., 1] / zs, valid


def _bilinear(F, u, v, valid):
    """F [h, w, C]; zero padding; differentiable in F and in (u, v)."""
    h, w, C = F.shape
    x = u - 0.5
    y = v - 0.5
    x0 = torch.floor(x).detach()
    y0 = torch.floor(y).detach()
    fx = (x - x0)[..., None]
    fy = (y - y0)[..., None]
    x0 = x0.long()
    y0 = y0.long()
    flat = F.reshape(h * w, C)
    out = 0.0
    for dy, dx, wt in ((0, 0, (1 - fy) * (1 - fx)), (0, 1, (1 - fy) * fx), (1, 0, fy * (1 - fx)), (1, 1, fy * fx)):
        iy, ix = y0 + dy, x0 + dx
        inside = (iy >= 0) & (iy < h) & (ix >= 0) & (ix < w)
        idx = (iy.clamp(0, h - 1) * w + ix.clamp(0, w - 1)).reshape(-1)
        vals = flat[idx].reshape(iy.shape + (C,))
        out = out + wt * torch.where(inside[..., None], vals, torch.zeros_like(vals))
    return torch.where(valid[..., None], out, torch.zeros_like(out))


def _rmsnorm(v, g):
    return g * v / torch.sqrt((v * v).mean(-1, keepdim=True) + 1e-6)


def _conv(x, w, b):
    """k x k per layer plane (k = 3, or 1 for the conv_kernel option), zero pad: x [L, H, W, C],
    w [k, k, Cin, Cout]."""
    y = torch.nn.functional.conv2d(x.permute(0, 3, 1, 2), w.permute(3, 2, 0, 1), b, padding=w.shape[0] // 2)
    return y.permute(0, 2, 3, 1)


def _resize(a, s):
    """Edge-clamped bilinear resize by integer s of a [L, H, W, D] (pixel centres aligned)."""
    if s == 1:
        return a
    L, H, W, D = a.shape

    def taps(n_out, n_in):
        src = (torch.arange(n_out, dtype=torch.float64) + 0.5) / s - 0.5
        i0 = torch.floor(src)
        w1 = src - i0
        i0 = i0.long()
        return i0.clamp(0, n_in - 1), (i0 + 1).clamp(0, n_in - 1), w1

    y0, y1, wy = taps(H * s, H)
    x0, x1, wx = taps(W * s, W)
    wy = wy[:, None, None]
    wx = wx[None, :, None]
    r0, r1 = a[:, y0], a[:, y1]
    top = r0[:, :, x0] * (1 - wx) + r0[:, :, x1] * wx
    bot = r1[:, :, x0] * (1 - wx) + r1[:, :, x1] * wx
    return top * (1 - wy) + bot * wy


def stage_forward(cfg, scene, V_in: torch.Tensor, F: torch.Tensor, Wt: Dict[str, torch.Tensor]) -> torch.Tensor:
    """RGBA of the novel view from the volume entering the last step (V_in [L, H, W, C]) and the
    step's pyramid level F ([V, h, w, C]); Wt maps make_weights names to float64 tensors."""
    j = cfg.n_scales - 1
    k, L = cfg.scales[j]
    C, heads = cfg.C, cfg.heads
    H, W = cfg.out_h // k, cfg.out_w // k
    w = lambda n: Wt[n.format(j=j)]
    # back-projection at the depths decoded from V_in
    d = _depth(V_in @ w("w_d") + w("b_d")[0], L, cfg.near, cfg.far)
    Delta = []
    for m, cam in enumerate(scene.cams):
        u, v, valid = _project(d, H, W, k, scene.target, cam)
        Delta.append(_bilinear(F[m], u, v, valid))
    Delta = torch.stack(Delta, -2)  # [L, H, W, V, C]
    # one-to-many attention block and the blend logits of the last step
    x = _rmsnorm(V_in, w("attn_g_{j}"))
    heads_out = []
    for i in range(heads):
        q = x @ w("Wq_{j}")[:, i * C:(i + 1) * C]
        p = torch.softmax(torch.einsum("lyxc,lyxmc->lyxm", q, Delta) / math.sqrt(C), -1)
        heads_out.append(torch.einsum("lyxm,lyxmc->lyxc", p, Delta))
    V_attn = V_in + torch.cat(heads_out, -1) @ w("Wo_{j}")
    beta = torch.einsum("lyxc,lyxmc->lyxm", x @ w("W_beta"), Delta) / math.sqrt(C)
    # residual conv block
    n = _rmsnorm(V_attn, w("conv_g_{j}"))
    h1 = _conv(n, w("conv1_w_{j}"), w("conv1_b_{j}"))
    V_out = V_attn + _conv(torch.nn.functional.gelu(h1), w("conv2_w_{j}"), w("conv2_b_{j}"))
    # render
    s = k
    t_up = _resize((V_out @ w("w_d") + w("b_d")[0])[..., None], s)[..., 0]
    s_up = _resize((V_out @ w("w_sigma") + w("b_sigma")[0])[..., None], s)[..., 0]
    b_up = _resize(beta, s)
    dr = _depth(t_up, L, cfg.near, cfg.far)
    alpha = torch.sigmoid(s_up)
    bw = torch.softmax(b_up, -1)
    col = 0.0
    for m, cam in enumerate(scene.cams):
        u, v, valid = _project(dr, cfg.out_h, cfg.out_w, 1, scene.target, cam)
        img = torch.tensor(scene.images[m], dtype=torch.float64)
        col = col + bw[..., m:m + 1] * _bilinear(img, u, v, valid)
    rgb = torch.zeros(cfg.out_h, cfg.out_w, 3, dtype=torch.float64)
    T = torch.ones(cfg.out_h, cfg.out_w, dtype=torch.float64)
    for li in range(L - 1, -1, -1):
        rgb = rgb + (T * alpha[li])[..., None] * col[li]
        T = T * (1 - alpha[li])
    return torch.cat([rgb, (1 - T)[..., None]], -1)


def stage_loss_and_grads(cfg, scene, V_in: np.ndarray, F: np.ndarray, W: Dict[str, np.ndarray],
                         wl: np.ndarray):
    """Loss sum(wl * rgb) and its gradients w.r.t. V_in, F and the stage weights (float64)."""
    j = cfg.n_scales - 1
    Vt = torch.tensor(np.asarray(V_in, np.float64), requires_grad=True)
    Ft = torch.tensor(np.asarray(F, np.float64), requires_grad=True)
    names = [n.format(j=j) for n in STAGE_WEIGHTS]
    Wt = {n: torch.tensor(np.asarray(W[n], np.float64), requires_grad=True) for n in names}
    rgba = stage_forward(cfg, scene, Vt, Ft, Wt)
    loss = (torch.tensor(np.asarray(wl, np.float64)) * rgba[..., :3]).sum()
    grads = torch.autograd.grad(loss, [Vt, Ft] + [Wt[n] for n in names])
    out = {"V_in": grads[0].numpy(), "F": grads[1].numpy()}
    out.update({n: g.numpy() for n, g in zip(names, grads[2:])})
    return float(loss.detach()), out


# ---------------------------------------------------------------------------------------------
# The whole network (uniform schedule, one-to-many attention)
# ---------------------------------------------------------------------------------------------

# weights every step shares (the decoders, the blend query, the encoder and the initial feature)
NETWORK_SHARED = ("enc_w", "enc_b", "v0", "w_d", "b_d", "w_sigma", "b_sigma", "W_a", "b_a", "W_beta")
NETWORK_STEP = ("attn_g_{j}", "Wq_{j}", "Wo_{j}", "conv_g_{j}", "conv1_w_{j}", "conv1_b_{j}", "conv2_w_{j}",
                "conv2_b_{j}")
NETWORK_COLLAPSE = ("col_w1_{j}", "col_b1_{j}", "col_w2_{j}", "col_b2_{j}")


def network_weight_names(cfg):
    """Every weight tensor the novel-view render depends on (the layer-collapse MLP of step j only
    where the layer count halves into step j)."""
    names = list(NETWORK_SHARED)
    for j in range(cfg.n_scales):
        names += [n.format(j=j) for n in NETWORK_STEP]
        if j > 0 and cfg.scales[j - 1][1] == 2 * cfg.scales[j][1]:
            names += [n.format(j=j) for n in NETWORK_COLLAPSE]
    return names


def _encode(images: torch.Tensor, enc_w, enc_b, levels):
    """Sec. 3.2.1 (reading: one 3x3 conv at full resolution, zero pad, bias, then 2x2 mean pools):
    {k: F_k [V, H/k, W/k, C]} for the levels asked for."""
    F = torch.nn.functional.conv2d(images.permute(0, 3, 1, 2), enc_w.permute(3, 2, 0, 1), enc_b, padding=1)
    out, k = {}, 1
    while k <= max(levels):
        if k in levels:
            out[k] = F.permute(0, 2, 3, 1)
        F = torch.nn.functional.avg_pool2d(F, 2)
        k *= 2
    return out


def _collapse(V, w1, b1, w2, b2):
    """Layer Collapse (Sec. 3.2.2): pairs of adjacent layers -> their mean plus MLP(concat)."""
    a, b = V[0::2], V[1::2]
    return 0.5 * (a + b) + torch.nn.functional.gelu(torch.cat([a, b], -1) @ w1 + b1) @ w2 + b2


def _sample_all(F, d, H, W, k, scene):
    return torch.stack([_bilinear(F[m], *_project(d, H, W, k, scene.target, cam)) for m, cam in enumerate(scene.cams)],
                       -2)  # [L, H, W, V, C]


def _attend(x, Delta, Wq, Wo, heads, C):
    outs = []
    for i in range(heads):
        q = x @ Wq[:, i * C:(i + 1) * C]
        p = torch.softmax(torch.einsum("lyxc,lyxmc->lyxm", q, Delta) / math.sqrt(C), -1)
        outs.append(torch.einsum("lyxm,lyxmc->lyxc", p, Delta))
    return torch.cat(outs, -1) @ Wo


def _render(cfg, scene, V_out, beta, Wt, L, k):
    s = k
    t_up = _resize((V_out @ Wt["w_d"] + Wt["b_d"][0])[..., None], s)[..., 0]
    s_up = _resize((V_out @ Wt["w_sigma"] + Wt["b_sigma"][0])[..., None], s)[..., 0]
    b_up = _resize(beta, s)
    dr = _depth(t_up, L, cfg.near, cfg.far)
    alpha = torch.sigmoid(s_up)
    bw = torch.softmax(b_up, -1)
    col = 0.0
    for m, cam in enumerate(scene.cams):
        u, v, valid = _project(dr, cfg.out_h, cfg.out_w, 1, scene.target, cam)
        img = torch.tensor(scene.images[m], dtype=torch.float64)
        col = col + bw[..., m:m + 1] * _bilinear(img, u, v, valid)
    rgb = torch.zeros(cfg.out_h, cfg.out_w, 3, dtype=torch.float64)
    T = torch.ones(cfg.out_h, cfg.out_w, dtype=torch.float64)
    for li in range(L - 1, -1, -1):
        rgb = rgb + (T * alpha[li])[..., None] * col[li]
        T = T * (1 - alpha[li])
    return torch.cat([rgb, (1 - T)[..., None]], -1)


def network_forward(cfg, scene, Wt: Dict[str, torch.Tensor], keep: Dict = None) -> torch.Tensor:
    """RGBA of the novel view from the input images, every step of the uniform schedule (grid
    factor of step j = its pyramid factor k_j); Wt maps make_weights names to float64 tensors.
    With `keep`, each step's output volume is stored in keep[j] (for the pins)."""
    C, heads = cfg.C, cfg.heads
    images = torch.tensor(np.asarray(scene.images, np.float64))
    feats = _encode(images, Wt["enc_w"], Wt["enc_b"], {k for k, _ in cfg.scales})
    V_prev = None
    for j, (k, L) in enumerate(cfg.scales):
        H, W = cfg.out_h // k, cfg.out_w // k
        ell = torch.arange(1, L + 1, dtype=torch.float64)[:, None, None]
        if j == 0:
            # Initialization: v0 everywhere, flat layers at the depth anchors
            V_in = Wt["v0"].expand(L, H, W, C)
            d = (1.0 / ((ell - 0.5) / L * (1 / cfg.near - 1 / cfg.far) + 1 / cfg.far)).expand(L, H, W)
        else:
            kp, Lp = cfg.scales[j - 1]
            Vp = V_prev
            if Lp == 2 * L:
                Vp = _collapse(Vp, Wt[f"col_w1_{j}"], Wt[f"col_b1_{j}"], Wt[f"col_w2_{j}"], Wt[f"col_b2_{j}"])
            V_in = _resize(Vp, kp // k)
            d = _depth(V_in @ Wt["w_d"] + Wt["b_d"][0], L, cfg.near, cfg.far)
        Delta = _sample_all(feats[k], d, H, W, k, scene)
        x = _rmsnorm(V_in, Wt[f"attn_g_{j}"])
        V_attn = V_in + _attend(x, Delta, Wt[f"Wq_{j}"], Wt[f"Wo_{j}"], heads, C)
        n = _rmsnorm(V_attn, Wt[f"conv_g_{j}"])
        h1 = _conv(n, Wt[f"conv1_w_{j}"], Wt[f"conv1_b_{j}"])
        V_prev = V_attn + _conv(torch.nn.functional.gelu(h1), Wt[f"conv2_w_{j}"], Wt[f"conv2_b_{j}"])
        if keep is not None:
            keep[j] = V_prev
        if j == cfg.n_scales - 1:
            beta = torch.einsum("lyxc,lyxmc->lyxm", x @ Wt["W_beta"], Delta) / math.sqrt(C)
            return _render(cfg, scene, V_prev, beta, Wt, L, k)


def network_loss_and_grads(cfg, scene, W: Dict[str, np.ndarray], wl: np.ndarray):
    """Loss sum(wl * rgb) of the novel view and its gradient w.r.t. every weight tensor the render
    depends on (network_weight_names), float64."""
    names = network_weight_names(cfg)
    Wt = {n: torch.tensor(np.asarray(W[n], np.float64), requires_grad=True) for n in names}
    rgba = network_forward(cfg, scene, Wt)
    loss = (torch.tensor(np.asarray(wl, np.float64)) * rgba[..., :3]).sum()
    grads = torch.autograd.grad(loss, [Wt[n] for n in names], allow_unused=True)
    return float(loss.detach()), {n: (np.zeros(np.shape(W[n])) if g is None else g.numpy())
                                  for n, g in zip(names, grads)}
