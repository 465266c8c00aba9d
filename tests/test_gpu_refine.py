"""Render-and-refine through the C ABI (Sec. 3.2.2 "Decoding and rendering the intermediate LDM",
Eq. overcomposite-result, the Update Block): every Update & Fuse step after the first decodes the
volume entering it, splats appearance and density into the input views (float atomics), over-
composites them, and samples the Update Block's features.  Against the oracle per step, with the
model schedule, the ray encoding and standard attention; zero Update Block weights give the plain
pipeline bit for bit."""
import numpy as np
import pytest

from oracle import quark_oracle as O
from paper_2411_16680_b300 import synth
from tests.test_gpu_parity import (PSNR_MIN_BF16, REL_TOL_FP32, RGBA_TOL_BF16, RGBA_TOL_FP32, assert_rel, psnr,
                                   run_gpu)

pytestmark = pytest.mark.gpu


def _cfg(C=32, heads=2, precision=synth.PREC_FP32, **kw):
    base = dict(C=C, heads=heads, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1.0, far=60.0, out_h=44, out_w=72,
                precision=precision, render_refine=1)
    base.update(kw)
    return synth.QuarkConfig(**base)


def _scene(V=3):
    return synth.scene_raycast(seed=7, V=V, W=72, H=44, f=55.0, arc=0.3)


@pytest.mark.parametrize("C,heads,mode,ray", [(32, 2, synth.ATTN_ONE_TO_MANY, 0), (16, 1, synth.ATTN_ONE_TO_MANY, 0),
                                              (32, 2, synth.ATTN_STANDARD, 0), (16, 2, synth.ATTN_ONE_TO_MANY, 1)])
def test_refine_fp32_matches_oracle(C, heads, mode, ray):
    cfg = _cfg(C, heads, attn_mode=mode, ray_encoding=ray)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = _scene()
    ref, ref_steps = O.forward(cfg, W, scene, mode=mode)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        for name in ("V_attn", "V_out", "t", "s"):
            assert_rel(g[name], getattr(r, name), REL_TOL_FP32, f"step {j} {name}")
    err = np.abs(out - ref).max()
    assert err <= RGBA_TOL_FP32, f"rgba max-abs {err:.3e}"


def test_refine_bf16_within_tolerance():
    cfg = _cfg(precision=synth.PREC_BF16)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = _scene()
    ref, _ = O.forward(cfg.replace(precision=synth.PREC_FP32), W, scene)
    out, _, _ = run_gpu(cfg, W, scene, per_step=False)
    assert np.abs(out - ref).max() <= RGBA_TOL_BF16
    assert psnr(out, ref) >= PSNR_MIN_BF16


def test_refine_with_the_model_schedule_matches_oracle():
    """Refining first blocks, reusing later blocks (same update features) and blocks without
    attention; grid factors 15 -> 3.75."""
    cfg = synth.QuarkConfig(C=16, heads=2, scales=[(8, 4), (8, 4), (8, 4), (4, 4), (4, 4), (2, 2), (2, 2)], near=1.0,
                            far=30.0, out_h=45, out_w=120, ldm_f=[15, 15, 15, 7.5, 7.5, 3.75, 3.75],
                            scale_heads=[4, 0, 4, 4, 0, 2, 1], reuse_depth=[0, 0, 1, 0, 0, 0, 1], render_refine=1)
    W = synth.make_weights(cfg, seed=5, sharp=True)
    sc = synth.scene_raycast(seed=3, V=3, W=80, H=48, f=60, arc=0.3)
    t = sc.target
    scene = synth.Scene(sc.images, sc.cams, synth.Camera(120, 45, t.fx * 1.5, t.fx * 1.5, 60.0, 22.5, t.R, t.t))
    ref, ref_steps = O.forward(cfg, W, scene)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        assert_rel(g["V_out"], r.V_out, REL_TOL_FP32, f"step {j} V_out")
    assert np.abs(out - ref).max() <= RGBA_TOL_FP32


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_zero_update_block_is_the_plain_pipeline_bitwise(precision):
    cfg = _cfg(precision=precision)
    W = synth.make_weights(cfg, seed=6, sharp=True)
    for k in list(W):
        if k.startswith("upd"):
            W[k] = np.zeros_like(W[k])
    scene = _scene()
    a, _, _ = run_gpu(cfg, W, scene, per_step=False)
    b, _, _ = run_gpu(cfg.replace(render_refine=0), W, scene, per_step=False)
    assert np.array_equal(a, b)
