"""C = 64 channels through the C ABI against the FP64 oracle: both precision forms with the layer
collapse and x2 upsamples on ragged tiles, the 1x1 fusion blocks, standard attention, the
no-allocation step; and the configurations refused with EINVAL (the BF16 form with four heads at
C = 64, whose 5C = 320 query columns exceed one tensor-core MMA's 256, and the backward pass,
which covers C = 16 and 32)."""
import numpy as np
import pytest
import torch

from oracle import quark_oracle as O
from paper_2411_16680_b300 import quark, synth
from tests.test_gpu_parity import (PSNR_MIN_BF16, REL_TOL_BF16_VOLUME, REL_TOL_FP32, RGBA_TOL_BF16, RGBA_TOL_FP32,
                                   assert_rel, check_fp32, psnr, run_gpu)

pytestmark = pytest.mark.gpu


def _cfg(heads, precision=synth.PREC_FP32, **kw):
    return synth.QuarkConfig(C=64, heads=heads, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1.0, far=60.0,
                             out_h=44, out_w=72, precision=precision, **kw)


def _scene(V=3, seed=7):
    return synth.scene_raycast(seed=seed, V=V, W=72, H=44, f=55.0, arc=0.3)


def _check_bf16(cfg, W, scene, mode=0):
    ref, ref_steps = O.forward(cfg, W, scene, mode=mode)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        for name in ("V_attn", "V_out", "t", "s"):
            assert_rel(g[name], getattr(r, name), REL_TOL_BF16_VOLUME, f"bf16 C=64 step {j} {name}")
        if "beta" in g:
            assert_rel(g["beta"], r.beta_logits, REL_TOL_BF16_VOLUME, f"bf16 C=64 step {j} beta")
    err = np.abs(out - ref).max()
    assert err <= RGBA_TOL_BF16 and psnr(out, ref) >= PSNR_MIN_BF16, f"bf16 C=64 rgba max-abs {err:.3e}"


@pytest.mark.parametrize("heads", [1, 2, 4])
def test_c64_fp32(heads):
    cfg = _cfg(heads)
    check_fp32(cfg, synth.make_weights(cfg, seed=11, sharp=True), _scene())


@pytest.mark.parametrize("heads", [1, 2])
def test_c64_bf16(heads):
    cfg = _cfg(heads, synth.PREC_BF16)
    _check_bf16(cfg, synth.make_weights(cfg, seed=11, sharp=True), _scene(V=4, seed=8))


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_c64_1x1_blocks(precision):
    cfg = _cfg(2, precision, conv_kernel=1)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    if precision == synth.PREC_FP32:
        check_fp32(cfg, W, _scene())
    else:
        _check_bf16(cfg, W, _scene())


def test_c64_standard_attention_fp32():
    cfg = _cfg(4, attn_mode=synth.ATTN_STANDARD)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = _scene()
    ref, ref_steps = O.forward(cfg, W, scene, mode=synth.ATTN_STANDARD)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        for name in ("V_attn", "V_out"):
            assert_rel(g[name], getattr(r, name), REL_TOL_FP32, f"standard C=64 step {j} {name}")
    assert np.abs(out - ref).max() <= RGBA_TOL_FP32


def test_c64_noalloc_step_equals_regular_step():
    cfg = _cfg(2, synth.PREC_BF16)
    scene = _scene()
    ctx = quark.Context(cfg)
    ctx.load_weights(synth.make_weights(cfg, seed=11, sharp=True))
    pyr = ctx.encode_pyramid(torch.tensor(scene.images, device="cuda"), scene.cams)
    ldm = ctx.ldm_create(scene.target)
    prev = None
    for j in range(cfg.n_scales):
        ctx.update_fuse(pyr, j, ldm)
        L, H, W = cfg.ldm_shape(j)
        ref = ldm.read(quark.FIELD_VOLUME, (L, H, W, cfg.C)).astype(np.float64)
        out = {n: torch.empty(*shape, device="cuda", dtype=dt) for n, shape, dt in
               (("v", (L, H, W, cfg.C), torch.bfloat16), ("c", (L, H, W, 3), torch.float32),
                ("a", (L, H, W), torch.float32), ("d", (L, H, W), torch.float32), ("t", (H, W, L), torch.float32),
                ("s", (H, W, L), torch.float32), ("b", (H, W, L, 3), torch.float32))}
        ctx.update_fuse_noalloc(pyr, j, scene.target, prev, out["v"], out["c"], out["a"], out["d"], out["t"],
                                out["s"], out["b"])
        torch.cuda.synchronize()
        assert_rel(out["v"].float().cpu().numpy(), ref, 1e-3, f"step {j} volume")
        prev = out["v"]
    ctx.check_device()


def test_c64_refusals():
    # the BF16 form with four heads at C = 64
    with pytest.raises(quark.QuarkError) as e:
        quark.Context(_cfg(4, synth.PREC_BF16))
    assert e.value.status == quark.EINVAL and "320" in str(e.value)
    # the backward pass covers C = 16 and 32
    cfg = synth.QuarkConfig(C=64, heads=2, scales=[(2, 4), (1, 2)], near=1.0, far=40.0, out_h=24, out_w=32)
    sc = synth.scene_raycast(seed=4, V=3, W=32, H=24, f=28.0, arc=0.3)
    ctx = quark.Context(cfg)
    ctx.load_weights(synth.make_weights(cfg, seed=8))
    pyr = ctx.encode_pyramid(torch.tensor(sc.images, device="cuda"), sc.cams)
    ldm = ctx.ldm_create(sc.target)
    ldm.keep_steps(True)
    for j in range(cfg.n_scales):
        ctx.update_fuse(pyr, j, ldm)
    L, H, W = cfg.ldm_shape(1)
    with pytest.raises(quark.QuarkError) as e:
        ctx.render_ldm_bwd(ldm, pyr, torch.zeros(24, 32, 3, device="cuda"), torch.zeros(L, H, W, 64, device="cuda"),
                           torch.zeros(H, W, L, 3, device="cuda"),
                           {n: torch.zeros(64, device="cuda") for n in ("w_d", "b_d", "w_sigma", "b_sigma")})
    assert e.value.status == quark.EINVAL
    ldm.release()
    pyr.release()
    ctx.close()
