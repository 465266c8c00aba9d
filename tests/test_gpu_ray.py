"""Ray directional encoding (Sec. 3.2.1) through the C ABI: gamma_k computed on the coarsest grid
from the closed form of the near/far difference, projected, upsampled and added to the level
before sampling; against the oracle (explicit plane intersections) per step.  Zero projection
weights leave the pipeline bit for bit."""
import numpy as np
import pytest

from oracle import quark_oracle as O
from paper_2411_16680_b300 import synth
from tests.test_gpu_parity import (PSNR_MIN_BF16, REL_TOL_FP32, RGBA_TOL_BF16, RGBA_TOL_FP32, assert_rel, psnr,
                                   run_gpu)

pytestmark = pytest.mark.gpu


def _cfg(C=32, heads=2, precision=synth.PREC_FP32, mode=synth.ATTN_ONE_TO_MANY):
    return synth.QuarkConfig(C=C, heads=heads, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1.0, far=60.0,
                             out_h=44, out_w=72, precision=precision, attn_mode=mode, ray_encoding=1)


def _scene():
    return synth.scene_raycast(seed=7, V=3, W=72, H=44, f=55.0, arc=0.6)


@pytest.mark.parametrize("C,heads,mode", [(32, 2, synth.ATTN_ONE_TO_MANY), (16, 1, synth.ATTN_ONE_TO_MANY),
                                          (32, 2, synth.ATTN_STANDARD)])
def test_ray_encoding_fp32_matches_oracle(C, heads, mode):
    cfg = _cfg(C, heads, mode=mode)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = _scene()
    ref, ref_steps = O.forward(cfg, W, scene, mode=mode)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        for name in ("V_attn", "V_out"):
            assert_rel(g[name], getattr(r, name), REL_TOL_FP32, f"step {j} {name}")
    assert np.abs(out - ref).max() <= RGBA_TOL_FP32


def test_ray_encoding_bf16_within_tolerance():
    cfg = _cfg(precision=synth.PREC_BF16)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = _scene()
    ref, _ = O.forward(cfg.replace(precision=synth.PREC_FP32), W, scene)
    out, _, _ = run_gpu(cfg, W, scene, per_step=False)
    assert np.abs(out - ref).max() <= RGBA_TOL_BF16
    assert psnr(out, ref) >= PSNR_MIN_BF16


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_zero_projection_leaves_the_pipeline_bitwise(precision):
    cfg = _cfg(precision=precision)
    W = synth.make_weights(cfg, seed=5, sharp=True)
    for k in cfg.levels():
        W[f"W_ray_{k}"] = np.zeros_like(W[f"W_ray_{k}"])
    scene = _scene()
    a, _, _ = run_gpu(cfg, W, scene, per_step=False)
    b, _, _ = run_gpu(cfg.replace(ray_encoding=0), W, scene, per_step=False)
    assert np.array_equal(a, b)
