"""A second, independent float64 formulation of the whole forward pass, built from torch CPU
library routines (conv2d, avg_pool2d, grid_sample, interpolate, rms_norm, gelu, softmax,
cumprod).  Test infrastructure: it exists only to pin the oracle's assembly of the steps
(which weights each scale uses, collapse before upsample, which tensor feeds which step).

It reaches the same definition by different routes: geometry through the composed
plane-induced homography A = K_m R_m R_t^T K_t^-1, b = K_m (t_m - R_m R_t^T t_t); sampling
through grid_sample; compositing as an exclusive cumulative product of (1 - alpha).
"""
import math

import numpy as np
import torch
import torch.nn.functional as TF


def _t(a):
    return torch.as_tensor(np.asarray(a, np.float64))


def _homography(cam_t, k_t, cam_m, k_m):
    Kt = np.diag([1 / k_t, 1 / k_t, 1.0]) @ cam_t.K
    Km = np.diag([1 / k_m, 1 / k_m, 1.0]) @ cam_m.K
    Rrel = cam_m.R @ cam_t.R.T
    return Km @ Rrel @ np.linalg.inv(Kt), Km @ (cam_m.t - Rrel @ cam_t.t)


def _sample(maps, cams, cam_t, k, d):
    """maps [V, C, h, w]; d [L, H, W] -> [L, H, W, V, C]."""
    L, H, W = d.shape
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64) + 0.5,
                            torch.arange(W, dtype=torch.float64) + 0.5, indexing="ij")
    p = torch.stack([xs, ys, torch.ones_like(xs)], -1)  # [H, W, 3]
    outs = []
    for m, cam in enumerate(cams):
        A, b = _homography(cam_t, k, cam, k)
        X = d[..., None] * (p @ _t(A).T)[None] + _t(b)
        z = X[..., 2]
        valid = z > 1e-6
        zs = torch.where(valid, z, torch.ones_like(z))
        u, v = X[..., 0] / zs, X[..., 1] / zs
        h, w = maps.shape[2:]
        grid = torch.stack([u / w * 2 - 1, v / h * 2 - 1], -1).reshape(1, L * H, W, 2)
        s = TF.grid_sample(maps[m:m + 1], grid, mode="bilinear", padding_mode="zeros", align_corners=False)
        s = s[0].permute(1, 2, 0).reshape(L, H, W, -1)
        outs.append(torch.where(valid[..., None], s, torch.zeros_like(s)))
    return torch.stack(outs, -2)


def _depth(t, L, near, far):
    ell = torch.arange(1, L + 1, dtype=torch.float64)[:, None, None]
    return 1.0 / (((ell - 0.5) / L + 0.5 / L * torch.tanh(t)) * (1 / near - 1 / far) + 1 / far)


def _conv_planes(x, w, b):
    """x [L, H, W, C] -> 3x3 conv per layer plane (zero pad)."""
    y = TF.conv2d(x.permute(0, 3, 1, 2), _t(w).permute(3, 2, 0, 1), _t(b), padding=1)
    return y.permute(0, 2, 3, 1)


def forward(cfg, Wt, scene):
    C, h = cfg.C, cfg.heads
    imgs = _t(scene.images).permute(0, 3, 1, 2)
    F = TF.conv2d(imgs, _t(Wt["enc_w"]).permute(3, 2, 0, 1), _t(Wt["enc_b"]), padding=1)
    levels = {1: F}
    k = 1
    while k < max(cfg.levels()):
        F = TF.avg_pool2d(F, 2)
        k *= 2
        levels[k] = F
    V = None
    for j, (k, L) in enumerate(cfg.scales):
        H, W = cfg.out_h // k, cfg.out_w // k
        if j == 0:
            V = _t(Wt["v0"]).expand(L, H, W, C).clone()
            d = _depth(torch.zeros(L, H, W, dtype=torch.float64), L, cfg.near, cfg.far)
        else:
            kp, Lp = cfg.scales[j - 1]
            if Lp == 2 * L:
                pairs = torch.cat([V[0::2], V[1::2]], -1)
                V = 0.5 * (V[0::2] + V[1::2]) + TF.gelu(pairs @ _t(Wt[f"col_w1_{j}"]) + _t(Wt[f"col_b1_{j}"])) \
                    @ _t(Wt[f"col_w2_{j}"]) + _t(Wt[f"col_b2_{j}"])
            if kp != k:
                V = TF.interpolate(V.permute(0, 3, 1, 2), scale_factor=kp // k, mode="bilinear",
                                   align_corners=False).permute(0, 2, 3, 1)
            d = _depth(V @ _t(Wt["w_d"]) + _t(Wt["b_d"])[0], L, cfg.near, cfg.far)
        D = _sample(levels[k], scene.cams, scene.target, k, d)  # [L, H, W, V, C]
        x = TF.rms_norm(V, (C,), _t(Wt[f"attn_g_{j}"]), eps=1e-6)
        q = (x @ _t(Wt[f"Wq_{j}"])).reshape(L, H, W, h, C)
        logits = torch.einsum("lyxhc,lyxvc->lyxhv", q, D) / math.sqrt(C)
        p = torch.softmax(logits, -1)
        o = torch.einsum("lyxhv,lyxvc->lyxhc", p, D).reshape(L, H, W, h * C)
        V = V + o @ _t(Wt[f"Wo_{j}"])
        if j == cfg.n_scales - 1:
            beta = torch.einsum("lyxc,lyxvc->lyxv", x @ _t(Wt["W_beta"]), D) / math.sqrt(C)
        n = TF.rms_norm(V, (C,), _t(Wt[f"conv_g_{j}"]), eps=1e-6)
        V = V + _conv_planes(TF.gelu(_conv_planes(n, Wt[f"conv1_w_{j}"], Wt[f"conv1_b_{j}"])),
                             Wt[f"conv2_w_{j}"], Wt[f"conv2_b_{j}"])
    k, L = cfg.scales[-1]
    t = V @ _t(Wt["w_d"]) + _t(Wt["b_d"])[0]
    s = V @ _t(Wt["w_sigma"]) + _t(Wt["b_sigma"])[0]
    up = lambda a: TF.interpolate(a, scale_factor=k, mode="bilinear", align_corners=False) if k > 1 else a
    t_up = up(t[None])[0]
    s_up = up(s[None])[0]
    b_up = up(beta.permute(3, 0, 1, 2))[:, :, :, :].permute(1, 2, 3, 0)  # [L, Ho, Wo, V]
    d = _depth(t_up, L, cfg.near, cfg.far)
    alpha = torch.sigmoid(s_up)
    bw = torch.softmax(b_up, -1)
    col = (bw[..., None] * _sample(imgs, scene.cams, scene.target, 1, d)).sum(-2)  # [L, Ho, Wo, 3]
    # front to back: nearest layer (index L-1) first
    a_f = alpha.flip(0)
    c_f = col.flip(0)
    T = torch.cumprod(torch.cat([torch.ones_like(a_f[:1]), 1 - a_f[:-1]], 0), 0)
    rgb = (T[..., None] * a_f[..., None] * c_f).sum(0)
    A = 1 - torch.prod(1 - a_f, 0)
    return torch.cat([rgb, A[..., None]], -1).numpy()
