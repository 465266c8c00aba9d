"""Differentiation form over the whole network: the hand-written adjoints of the render, of every
Update & Fuse step (conv block, one-to-many attention with its sampling and the sample
coordinates' dependence on the decoded depth), of the transitions (x2 upsample, layer collapse,
the initialisation's v0) and of the encoder (mean-pool chain, 3x3 conv), chained through the C
ABI (quark_render_ldm_bwd, quark_update_fuse_bwd, quark_encode_pyramid_bwd) and the
torch.autograd.Function QuarkNetworkFn, against (1) the FP64 reference gradient of the whole
network (autograd of a float64 formulation, itself pinned to finite differences) and (2) central
finite differences of the GPU forward with a float64 host reduction of the loss."""
import numpy as np
import pytest
import torch

from oracle import quark_grad as G
from paper_2411_16680_b300 import autograd as QA
from paper_2411_16680_b300 import quark, synth

pytestmark = pytest.mark.gpu

REL_L2_TOL = 1e-3  # gradient vs the FP64 reference, per tensor


def _net(cfg, sc, W):
    ctx = quark.Context(cfg)
    ctx.load_weights(W)
    return QA.Network(ctx, torch.tensor(sc.images, device="cuda"), sc.cams, sc.target, W)


def _gpu_grads(net, wl):
    rgba, ldm = net.forward()
    g = net.backward(ldm, torch.tensor(wl, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    net.ctx.check_device()
    ldm.release()
    return rgba.cpu().numpy(), {n: t.cpu().numpy().astype(np.float64) for n, t in g.items()}


def _check_against_reference(cfg, scenes, W, seeds):
    total, total_ref = None, None
    for sc, seed in zip(scenes, seeds):
        wl = np.random.default_rng(seed).standard_normal((cfg.out_h, cfg.out_w, 3))
        net = _net(cfg, sc, W)
        _, g = _gpu_grads(net, wl)
        _, g_ref = G.network_loss_and_grads(cfg, sc, W, wl)
        total = g if total is None else {n: total[n] + g[n] for n in g}
        total_ref = g_ref if total_ref is None else {n: total_ref[n] + g_ref[n] for n in g_ref}
        net.ctx.close()
    names = QA.network_weight_names(cfg)
    assert set(names) | {"W_a", "b_a"} == set(total_ref)
    for name in names:
        ref, got = total_ref[name], total[name].reshape(total_ref[name].shape)
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err <= REL_L2_TOL, f"{name}: relative L2 error {err:.2e} (|ref| {np.linalg.norm(ref):.3e})"
    # the appearance decoder does not reach the render
    assert np.all(total_ref["W_a"] == 0) and np.all(total_ref["b_a"] == 0)


@pytest.mark.parametrize("C,heads,scales", [
    (16, 2, [(2, 4), (1, 2)]),                 # collapse + x2 upsample into the last step
    (32, 1, [(4, 4), (2, 4), (2, 2)]),         # upsample without collapse, then collapse without upsample
    (16, 4, [(4, 8), (2, 4), (1, 2)]),         # two collapses and two upsamples
])
def test_network_gradient_matches_fp64_reference(C, heads, scales):
    """Every weight tensor the render depends on, within relative L2 1e-3 of the FP64 gradient."""
    cfg = synth.QuarkConfig(C=C, heads=heads, scales=scales, near=1.0, far=40.0, out_h=24, out_w=32)
    sc = synth.scene_raycast(seed=4, V=3, W=32, H=24, f=28.0, arc=0.3)
    W = synth.make_weights(cfg, seed=8, sharp=True)
    _check_against_reference(cfg, [sc], W, [5])


def test_grad_workload_network_matches_fp64_reference():
    """The differentiation workload's structure (two scenes, V=4, scales (k,L) = (2,16), (1,8), C=32,
    h=2) at 128x128, where the FP64 reference gradient of the whole network is affordable: the
    gradient summed over both scenes, for every weight tensor, within relative L2 1e-3."""
    cfg = synth.config_grad().replace(out_h=128, out_w=128)
    W = synth.make_weights(cfg, seed=5678, sharp=True)
    scenes = [synth.scene_raycast(seed=s, V=4, W=128, H=128, f=100.0, arc=0.3) for s in (1234, 1235)]
    _check_against_reference(cfg, scenes, W, [1234, 1235])


# weights that never move a sample coordinate: the loss is smooth in them
KINK_FREE = ("W_beta", "w_sigma", "b_sigma")


def test_grad_workload_network_finite_differences_and_autograd():
    """Two 512x512 scenes, V=4, scales (k,L) = (2,16), (1,8), C=32, h=2; loss = sum(w * rgb) with w
    seeded N(0,1); 64 parameters drawn from every weight tensor of the network (each tensor at
    least once), central differences with eps = 1e-3 and a float64 host reduction of the loss.

    Tolerances as for the stage's test: parameters that move no sample coordinate (W^beta,
    w_sigma, b_sigma) within 1e-2 relative + 0.1 absolute (the FP32 noise floor of the loss
    difference); every other parameter moves the sample coordinates of the last step's sampling
    and of the render (through the decoded depths), and its central difference averages slopes
    across bilinear kinks: its kink noise is measured by a second difference at eps / 2 and each
    must satisfy |fd - analytic| <= 3 (noise + 0.12) + 0.05 |analytic|.  The same gradients are
    exact against the FP64 reference at 128 x 128."""
    cfg = synth.config_grad()
    W = synth.make_weights(cfg, seed=5678, sharp=True)
    scenes = [synth.scene_grad(1234), synth.scene_grad(1235)]
    wls = [np.random.default_rng(99 + i).standard_normal((cfg.out_h, cfg.out_w, 3)) for i in range(2)]
    nets = [_net(cfg, sc, W) for sc in scenes]
    grads = [_gpu_grads(net, wl)[1] for net, wl in zip(nets, wls)]
    names = QA.network_weight_names(cfg)
    total = {n: grads[0][n] + grads[1][n] for n in names}
    wl_t = [torch.tensor(wl, dtype=torch.float64, device="cuda") for wl in wls]

    def loss(Wx):
        s = 0.0
        for net, wl in zip(nets, wl_t):
            net.ctx.load_weights(Wx)
            net._loaded = None
            rgba, ldm = net.forward()
            s += float((wl * rgba[..., :3].double()).sum().item())
            ldm.release()
        return s

    rng = np.random.default_rng(64)
    order = list(names) + [names[int(i)] for i in rng.integers(0, len(names), 64 - len(names))]
    eps = 1e-3
    smooth, kinked = [], []
    for n in order:
        base = np.asarray(W[n], np.float32)
        idx = tuple(int(rng.integers(0, s)) for s in base.shape)
        an = float(total[n].reshape(base.shape)[idx])

        def fd_at(e):
            vals = []
            for sgn in (1, -1):
                W2 = dict(W)
                a = base.copy()
                a[idx] += sgn * e
                W2[n] = a
                vals.append(loss(W2))
            return (vals[0] - vals[1]) / (2 * e)

        fd = fd_at(eps)
        if n in KINK_FREE:
            smooth.append((n, idx, fd, an))
        else:
            kinked.append((n, idx, fd, an, fd_at(eps / 2)))
    for net in nets:
        net.ctx.load_weights(W)
    bad = [r for r in smooth if abs(r[2] - r[3]) > 1e-2 * abs(r[3]) + 0.1]
    assert not bad, "finite differences disagree: " + "; ".join(f"{n}{idx}: fd {fd:.6g} vs {an:.6g}"
                                                                for n, idx, fd, an in bad)
    print("\nkink-free:", [(r[0], r[1], round(r[2], 4), round(r[3], 4)) for r in smooth])
    print("coordinate-moving (fd, fd eps/2, analytic):",
          [(r[0], r[1], round(r[2], 4), round(r[4], 4), round(r[3], 4)) for r in kinked])
    bad = [r for r in kinked if abs(r[2] - r[3]) > 3 * (abs(r[2] - r[4]) + 0.12) + 0.05 * abs(r[3])]
    assert not bad, "coordinate-moving parameters disagree beyond their kink noise: " + "; ".join(
        f"{n}{idx}: fd {fd:.5g} (eps/2: {fd2:.5g}) vs {an:.5g}" for n, idx, fd, an, fd2 in bad)
    assert len(smooth) + len(kinked) == 64

    # the autograd.Function reproduces the direct backward
    net = nets[0]
    net._loaded = None
    ws = [t.requires_grad_(True) for t in net.weight_tensors()]
    rgba = QA.QuarkNetworkFn.apply(net, *ws)
    (torch.tensor(wls[0], dtype=torch.float32, device="cuda") * rgba[..., :3]).sum().backward()
    for n, t in zip(names, ws):
        np.testing.assert_allclose(t.grad.cpu().numpy(), grads[0][n].reshape(t.shape), rtol=1e-4, atol=1e-5,
                                   err_msg=n)
    for net in nets:
        net.ctx.check_device()


def test_backward_needs_kept_steps():
    cfg = synth.QuarkConfig(C=16, heads=2, scales=[(2, 4), (1, 2)], near=1.0, far=40.0, out_h=24, out_w=32)
    sc = synth.scene_raycast(seed=4, V=3, W=32, H=24, f=28.0, arc=0.3)
    W = synth.make_weights(cfg, seed=8, sharp=True)
    ctx = quark.Context(cfg)
    ctx.load_weights(W)
    pyr = ctx.encode_pyramid(torch.tensor(sc.images, device="cuda"), sc.cams)
    ldm = ctx.ldm_create(sc.target)  # volumes not kept
    for j in range(cfg.n_scales):
        ctx.update_fuse(pyr, j, ldm)
    L, H, Wd = cfg.ldm_shape(1)
    dv = torch.zeros(L, H, Wd, cfg.C, device="cuda")
    grads = {n: torch.zeros(np.asarray(W[n]).shape, device="cuda") for n in QA.network_weight_names(cfg)}
    with pytest.raises(quark.QuarkError) as e:
        ctx.update_fuse_bwd(pyr, 1, ldm, dv, torch.zeros(H, Wd, L, 3, device="cuda"),
                            torch.zeros(4, 12, 16, cfg.C, device="cuda"), torch.zeros(3, 24, 32, cfg.C, device="cuda"),
                            grads)
    assert e.value.status == quark.EINVAL and "keeps its steps" in str(e.value)
