"""The conv_kernel = 1 form of the fusion block (Sec. 3.3: the residual convolution block mirrors a
Transformer's MLP block; with 1x1 kernels it is that position-wise MLP, V + W2 gelu(W1 N(V) + b1)
+ b2), through the C ABI against the FP64 oracle: every step's volumes, decoded attributes and
logits in the FP32 form, the volumes and the output in the BF16 form (tcgen05), the no-allocation
step, and the whole-network gradient against the FP64 reference."""
import numpy as np
import pytest
import torch

from oracle import quark_grad as G
from oracle import quark_oracle as O
from paper_2411_16680_b300 import autograd as QA
from paper_2411_16680_b300 import quark, synth

from .test_gpu_parity import (PSNR_MIN_BF16, REL_TOL_BF16_VOLUME, RGBA_TOL_BF16, assert_rel, check_fp32, psnr,
                              run_gpu)

pytestmark = pytest.mark.gpu


def _cfg(C=32, heads=2, precision=synth.PREC_FP32):
    return synth.QuarkConfig(C=C, heads=heads, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1.0, far=60.0,
                             out_h=44, out_w=72, precision=precision, conv_kernel=1)


@pytest.mark.parametrize("C,heads", [(32, 2), (16, 4)])
def test_1x1_blocks_fp32(C, heads):
    cfg = _cfg(C, heads)
    scene = synth.scene_raycast(seed=7, V=3, W=72, H=44, f=55.0, arc=0.3)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    assert W["conv1_w_0"].shape == (1, 1, C, C)
    check_fp32(cfg, W, scene)


@pytest.mark.parametrize("C,heads", [(32, 2), (16, 1)])
def test_1x1_blocks_bf16(C, heads):
    cfg = _cfg(C, heads, synth.PREC_BF16)
    scene = synth.scene_raycast(seed=8, V=4, W=72, H=44, f=55.0, arc=0.3)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    ref, ref_steps = O.forward(cfg, W, scene)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        for name in ("V_attn", "V_out", "t", "s"):
            assert_rel(g[name], getattr(r, name), REL_TOL_BF16_VOLUME, f"bf16 1x1 step {j} {name}")
    err = np.abs(out - ref).max()
    assert err <= RGBA_TOL_BF16 and psnr(out, ref) >= PSNR_MIN_BF16, f"bf16 1x1 rgba max-abs {err:.3e}"


def test_1x1_blocks_noalloc_equals_regular_step():
    cfg = _cfg(32, 2)
    scene = synth.scene_raycast(seed=7, V=3, W=72, H=44, f=55.0, arc=0.3)
    ctx = quark.Context(cfg)
    ctx.load_weights(synth.make_weights(cfg, seed=11, sharp=True))
    pyr = ctx.encode_pyramid(torch.tensor(scene.images, device="cuda"), scene.cams)
    ldm = ctx.ldm_create(scene.target)
    prev = None
    for j in range(cfg.n_scales):
        ctx.update_fuse(pyr, j, ldm)
        L, H, W = cfg.ldm_shape(j)
        ref = ldm.read(quark.FIELD_VOLUME, (L, H, W, cfg.C))
        out = {n: torch.empty(*shape, device="cuda") for n, shape in
               (("v", (L, H, W, cfg.C)), ("c", (L, H, W, 3)), ("a", (L, H, W)), ("d", (L, H, W)), ("t", (H, W, L)),
                ("s", (H, W, L)), ("b", (H, W, L, 3)))}
        ctx.update_fuse_noalloc(pyr, j, scene.target, prev, out["v"], out["c"], out["a"], out["d"], out["t"],
                                out["s"], out["b"])
        torch.cuda.synchronize()
        assert_rel(out["v"].cpu().numpy(), ref.astype(np.float64), 1e-4, f"step {j} volume")
        prev = out["v"]


def test_1x1_blocks_network_gradient_matches_fp64_reference():
    cfg = synth.QuarkConfig(C=16, heads=2, scales=[(2, 4), (1, 2)], near=1.0, far=40.0, out_h=24, out_w=32,
                            conv_kernel=1)
    sc = synth.scene_raycast(seed=4, V=3, W=32, H=24, f=28.0, arc=0.3)
    W = synth.make_weights(cfg, seed=8, sharp=True)
    wl = np.random.default_rng(5).standard_normal((cfg.out_h, cfg.out_w, 3))
    ctx = quark.Context(cfg)
    ctx.load_weights(W)
    net = QA.Network(ctx, torch.tensor(sc.images, device="cuda"), sc.cams, sc.target, W)
    rgba, ldm = net.forward()
    g = net.backward(ldm, torch.tensor(wl, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    ctx.check_device()
    ref_rgba, _ = O.forward(cfg, W, sc)
    assert np.abs(rgba.cpu().numpy() - ref_rgba).max() <= 1e-4
    _, g_ref = G.network_loss_and_grads(cfg, sc, W, wl)
    for name in QA.network_weight_names(cfg):
        ref = g_ref[name]
        got = g[name].cpu().numpy().astype(np.float64).reshape(ref.shape)
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err <= 1e-3, f"{name}: relative L2 error {err:.2e}"
