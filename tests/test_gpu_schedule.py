"""Model schedules through the C ABI (Sec. 3.2; appendix tables "Model description for Quark /
Quark+"): per-step heads, fusion steps without attention (the CNN blocks after a fusion block's
first), one set of update features per Update & Fuse step (later blocks sample at the depths the
step's first block used), LDM grid factors relative to the output with a fractional final
upsample (3.75).  Against the oracle per step, and the paper's Quark schedule (24 fusion steps)
at a reduced output size."""
import numpy as np
import pytest
import torch

from oracle import quark_oracle as O
from paper_2411_16680_b300 import synth
from tests.test_gpu_parity import (PSNR_MIN_BF16, REL_TOL_FP32, RGBA_TOL_BF16, RGBA_TOL_FP32, assert_rel, psnr,
                                   run_gpu)

pytestmark = pytest.mark.gpu


def _cfg(C=16, precision=synth.PREC_FP32, mode=synth.ATTN_ONE_TO_MANY, **kw):
    # views 48 x 80 (levels 8, 4, 2); output 45 x 120 on grids 3x8, 6x16, 12x32 (factors 15, 7.5, 3.75)
    base = dict(C=C, heads=2, scales=[(8, 4), (8, 4), (8, 4), (4, 4), (4, 4), (2, 2), (2, 2)], near=1.0, far=30.0,
                out_h=45, out_w=120, ldm_f=[15, 15, 15, 7.5, 7.5, 3.75, 3.75], scale_heads=[4, 0, 4, 4, 0, 2, 1],
                reuse_depth=[0, 0, 1, 0, 0, 0, 1], precision=precision, attn_mode=mode)
    base.update(kw)
    return synth.QuarkConfig(**base)


def _scene(V=3):
    sc = synth.scene_raycast(seed=3, V=V, W=80, H=48, f=60, arc=0.3)
    t = sc.target
    return synth.Scene(sc.images, sc.cams, synth.Camera(120, 45, t.fx * 1.5, t.fx * 1.5, 60.0, 22.5, t.R, t.t))


def _check_steps(steps, ref_steps, names=("V_attn", "V_out", "t", "s", "depth", "alpha", "colour")):
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        for name in names:
            assert_rel(g[name], getattr(r, name), REL_TOL_FP32, f"step {j} {name}")
    assert_rel(steps[-1]["beta"], ref_steps[-1].beta_logits, REL_TOL_FP32, "beta")


@pytest.mark.parametrize("C,mode", [(16, synth.ATTN_ONE_TO_MANY), (32, synth.ATTN_ONE_TO_MANY),
                                    (16, synth.ATTN_STANDARD)])
def test_schedule_fp32_matches_oracle(C, mode):
    cfg = _cfg(C, mode=mode)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = _scene()
    ref, ref_steps = O.forward(cfg, W, scene, mode=mode)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
    _check_steps(steps, ref_steps)
    err = np.abs(out - ref).max()
    assert err <= RGBA_TOL_FP32, f"rgba max-abs {err:.3e}"


def test_schedule_bf16_within_tolerance():
    cfg = _cfg(32, precision=synth.PREC_BF16)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = _scene()
    ref, _ = O.forward(cfg.replace(precision=synth.PREC_FP32), W, scene)
    out, _, _ = run_gpu(cfg, W, scene, per_step=False)
    assert np.abs(out - ref).max() <= RGBA_TOL_BF16
    assert psnr(out, ref) >= PSNR_MIN_BF16


def test_schedule_with_ray_encoding_matches_oracle():
    cfg = _cfg(16, ray_encoding=1)
    W = synth.make_weights(cfg, seed=4, sharp=True)
    scene = _scene()
    ref, ref_steps = O.forward(cfg, W, scene)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
    _check_steps(steps, ref_steps, names=("V_attn", "V_out"))
    assert np.abs(out - ref).max() <= RGBA_TOL_FP32


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_explicit_default_schedule_is_bitwise_the_plain_pipeline(precision):
    cfg = synth.QuarkConfig(C=32, heads=2, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1.0, far=50.0, out_h=48,
                            out_w=64, precision=precision)
    W = synth.make_weights(cfg, seed=2, sharp=True)
    scene = synth.scene_raycast(seed=2, V=3, W=64, H=48, f=50, arc=0.3)
    a, _, _ = run_gpu(cfg, W, scene, per_step=False)
    b, _, _ = run_gpu(cfg.replace(scale_heads=[2] * 4, ldm_f=[4, 2, 2, 1], reuse_depth=[0] * 4), W, scene,
                      per_step=False)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("model", ["quark", "quarkplus"])
@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_quark_model_schedule_matches_oracle(precision, model):
    """The paper's Quark schedule (24 fusion steps, L 24/12/6, heads 4/2/1, factors 30 -> 3.75) and
    Quark+ (L 32/16/8, factors 20 -> 2.5) at a 240 x 120 output from 128 x 80 views."""
    make = synth.config_quark if model == "quark" else synth.config_quarkplus
    cfg = make(out_w=240, out_h=120).replace(precision=precision)
    W = synth.make_weights(cfg, seed=8, sharp=True)
    scene = synth.scene_quark(seed=8, V=3, W=128, H=80, out_w=240, out_h=120)
    ref, ref_steps = O.forward(cfg.replace(precision=synth.PREC_FP32), W, scene)
    out, steps, n = run_gpu(cfg, W, scene, per_step=precision == synth.PREC_FP32)
    if precision == synth.PREC_FP32:
        for j, (g, r) in enumerate(zip(steps, ref_steps)):
            assert_rel(g["V_out"], r.V_out, REL_TOL_FP32, f"step {j} V_out")
        assert np.abs(out - ref).max() <= RGBA_TOL_FP32
    else:
        assert np.abs(out - ref).max() <= RGBA_TOL_BF16
        assert psnr(out, ref) >= PSNR_MIN_BF16
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_aspect_adaptive_grids_match_oracle(precision):
    """Aspect-adaptive LDM dimensions (Sec. 4): a 200 x 130 output of a schedule given for
    240 x 120 gets grids 5x8 .. 40x64 (the model's area per layer at its aspect) and different
    factors along rows and columns (final upsample 3.25 x 3.125)."""
    cfg = synth.config_quark(out_w=240, out_h=120).replace(model_w=240, model_h=120, out_w=200, out_h=130,
                                                           precision=precision)
    assert cfg.upsample_syx == (3.25, 3.125)
    W = synth.make_weights(cfg, seed=9, sharp=True)
    scene = synth.scene_quark(seed=9, V=3, W=128, H=80, out_w=200, out_h=130)
    ref, ref_steps = O.forward(cfg.replace(precision=synth.PREC_FP32), W, scene)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=precision == synth.PREC_FP32)
    if precision == synth.PREC_FP32:
        for j, (g, r) in enumerate(zip(steps, ref_steps)):
            assert_rel(g["V_out"], r.V_out, REL_TOL_FP32, f"step {j} V_out")
        assert np.abs(out - ref).max() <= RGBA_TOL_FP32
    else:
        assert np.abs(out - ref).max() <= RGBA_TOL_BF16
        assert psnr(out, ref) >= PSNR_MIN_BF16


def test_aspect_adaptive_at_the_model_aspect_is_bitwise_the_plain_schedule():
    cfg = synth.config_quark(out_w=240, out_h=120)
    W = synth.make_weights(cfg, seed=10, sharp=True)
    scene = synth.scene_quark(seed=10, V=3, W=128, H=80, out_w=240, out_h=120)
    a, _, _ = run_gpu(cfg, W, scene, per_step=False)
    b, _, _ = run_gpu(cfg.replace(model_w=240, model_h=120), W, scene, per_step=False)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_quark_model_1080p_sampled_windows(precision):
    """The paper's Quark schedule at full size (V = 8 views 480x288, 1920x1080 output), in the launch
    configuration the bench times; the oracle computes two output windows from scratch through all
    24 fusion steps (their halos grow back through every conv and upsample)."""
    cfg = synth.config_quark().replace(precision=precision)
    W = synth.make_weights(cfg, sharp=True)
    scene = synth.scene_quark()
    out, _, _ = run_gpu(cfg, W, scene, per_step=False)
    assert np.isfinite(out).all()
    tol = RGBA_TOL_FP32 if precision == synth.PREC_FP32 else RGBA_TOL_BF16
    for r in [(0, 3, 0, 3), (540, 543, 958, 961)]:
        ref, _ = O.forward(cfg.replace(precision=synth.PREC_FP32), W, scene, r)
        err = np.abs(out[r[0]:r[1], r[2]:r[3]] - ref).max()
        assert err <= tol, f"{r}: max-abs {err:.3e}"
