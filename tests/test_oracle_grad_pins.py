"""Pins of the FP64 reference gradient (oracle/quark_grad.py), CPU only.

Its forward must equal the numpy oracle's last step and render; its autograd gradient must
equal central finite differences of that forward (float64, eps 1e-6) for entries drawn from
every differentiated tensor, including w_d, which moves the sample coordinates through the
decoded depth."""
import numpy as np
import pytest
import torch

from oracle import quark_grad as G
from oracle import quark_oracle as O
from paper_2411_16680_b300 import synth


def _case(s=2):
    cfg = synth.QuarkConfig(C=8, heads=2, scales=[(2, 4), (1, 2)], near=1.0, far=40.0, out_h=12 * s, out_w=16 * s)
    sc = synth.scene_raycast(seed=4, V=3, W=16 * s, H=12 * s, f=14.0 * s, arc=0.3)
    W = synth.make_weights(cfg, seed=8, sharp=True)
    rgba, steps = O.forward(cfg, W, sc)
    k = cfg.scales[-1][0]
    F = np.stack([O.encode_level(sc.images[m], W["enc_w"], W["enc_b"], k) for m in range(len(sc.cams))])
    return cfg, sc, W, rgba, steps[-1].V_in, F


def test_stage_forward_equals_numpy_oracle():
    cfg, sc, W, rgba, V_in, F = _case()
    j = cfg.n_scales - 1
    Wt = {n.format(j=j): torch.tensor(np.asarray(W[n.format(j=j)], np.float64)) for n in G.STAGE_WEIGHTS}
    out = G.stage_forward(cfg, sc, torch.tensor(V_in), torch.tensor(F), Wt).numpy()
    np.testing.assert_allclose(out, rgba, atol=1e-12)


def test_stage_gradient_equals_central_differences():
    cfg, sc, W, rgba, V_in, F = _case()
    j = cfg.n_scales - 1
    rng = np.random.default_rng(3)
    wl = rng.standard_normal((cfg.out_h, cfg.out_w, 3))
    loss0, g = G.stage_loss_and_grads(cfg, sc, V_in, F, W, wl)
    names = [n.format(j=j) for n in G.STAGE_WEIGHTS]
    Wt = {n: torch.tensor(np.asarray(W[n], np.float64)) for n in names}

    def loss(Vx, Fx, Wx):
        return float((torch.tensor(wl) * G.stage_forward(cfg, sc, torch.tensor(Vx), torch.tensor(Fx), Wx)[..., :3]).sum())

    eps = 1e-6
    checked = 0
    for name in ["V_in", "F"] + names:
        for _ in range(3):
            if name == "V_in":
                base = V_in
            elif name == "F":
                base = F
            else:
                base = np.asarray(W[name], np.float64)
            idx = tuple(rng.integers(0, s) for s in base.shape)
            vals = []
            for sgn in (+1, -1):
                a = np.array(base, np.float64, copy=True)
                a[idx] += sgn * eps
                if name == "V_in":
                    vals.append(loss(a, F, Wt))
                elif name == "F":
                    vals.append(loss(V_in, a, Wt))
                else:
                    W2 = dict(Wt)
                    W2[name] = torch.tensor(a)
                    vals.append(loss(V_in, F, W2))
            fd = (vals[0] - vals[1]) / (2 * eps)
            an = g[name][idx]
            assert abs(fd - an) <= 1e-5 * (1 + abs(an)), (name, idx, fd, an)
            checked += 1
    assert checked == 3 * (2 + len(names))


# ---- the whole network: encoder, every step with its transition, the render ----------------

def _net_case(s=2):
    # two steps: x2 upsample and layer collapse (4 -> 2 layers) between them, both pyramid levels
    cfg = synth.QuarkConfig(C=8, heads=2, scales=[(2, 4), (1, 2)], near=1.0, far=40.0, out_h=12 * s, out_w=16 * s)
    sc = synth.scene_raycast(seed=4, V=3, W=16 * s, H=12 * s, f=14.0 * s, arc=0.3)
    W = synth.make_weights(cfg, seed=8, sharp=True)
    return cfg, sc, W


def test_network_forward_equals_numpy_oracle():
    cfg, sc, W = _net_case()
    rgba, steps = O.forward(cfg, W, sc)
    Wt = {n: torch.tensor(np.asarray(W[n], np.float64)) for n in G.network_weight_names(cfg)}
    keep = {}
    out = G.network_forward(cfg, sc, Wt, keep).numpy()
    np.testing.assert_allclose(out, rgba, atol=1e-12)
    for j, st in enumerate(steps):
        np.testing.assert_allclose(keep[j].numpy(), st.V_out, atol=1e-12)


def test_network_weight_names_cover_what_the_render_uses():
    cfg, sc, W = _net_case()
    names = G.network_weight_names(cfg)
    # the collapse into step 1 (4 -> 2 layers) is used, step 0 has none
    assert "col_w1_1" in names and "col_w1_0" not in names
    for n in ("enc_w", "enc_b", "v0", "Wq_0", "conv2_w_0", "Wq_1", "W_beta", "w_d"):
        assert n in names


def test_network_gradient_equals_central_differences():
    """Entries of every weight tensor, through the encoder, the initialisation, both steps, the
    collapse, the upsample and the render; the appearance decoder W_a / b_a does not reach the
    render (the colours are the input images' blended by beta), so its gradient is exactly zero."""
    cfg, sc, W = _net_case()
    rng = np.random.default_rng(7)
    wl = rng.standard_normal((cfg.out_h, cfg.out_w, 3))
    names = G.network_weight_names(cfg)
    _, g = G.network_loss_and_grads(cfg, sc, W, wl)
    Wt = {n: torch.tensor(np.asarray(W[n], np.float64)) for n in names}

    def loss(Wx):
        return float((torch.tensor(wl) * G.network_forward(cfg, sc, Wx)[..., :3]).sum())

    eps = 1e-6
    for name in names:
        base = np.asarray(W[name], np.float64)
        for _ in range(2):
            idx = tuple(rng.integers(0, s) for s in base.shape)
            vals = []
            for sgn in (+1, -1):
                a = base.copy()
                a[idx] += sgn * eps
                W2 = dict(Wt)
                W2[name] = torch.tensor(a)
                vals.append(loss(W2))
            fd = (vals[0] - vals[1]) / (2 * eps)
            an = g[name][idx]
            assert abs(fd - an) <= 1e-5 * (1 + abs(an)), (name, idx, fd, an)
    assert np.all(g["W_a"] == 0) and np.all(g["b_a"] == 0)
    for name in names:
        if name not in ("W_a", "b_a"):
            assert np.abs(g[name]).max() > 0, f"{name} has no gradient"
