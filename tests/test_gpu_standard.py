"""STANDARD attention mode (Sec. 3.3 Eq. MultiHead: keys and values are the sampled features
times W^k and W^val, per-head width C/h) through the C ABI.  The GPU path projects keys and values
once per pyramid texel and samples the projected maps, which equals projecting the sampled
features because bilinear sampling is linear and the projections have no bias; the oracle
projects the sampled features.  Checked per step against the oracle (FP32 1e-4, BF16 2e-2 and
>= 40 dB), and against the GPU one-to-many path run with the folded weights (appendix A)."""
import math

import numpy as np
import pytest
import torch

from oracle import quark_oracle as O
from paper_2411_16680_b300 import synth
from tests.test_gpu_parity import (PSNR_MIN_BF16, REL_TOL_FP32, RGBA_TOL_BF16, RGBA_TOL_FP32, assert_rel, psnr,
                                   run_gpu)

pytestmark = pytest.mark.gpu


def _cfg(C, heads, precision=synth.PREC_FP32, mode=synth.ATTN_STANDARD):
    return synth.QuarkConfig(C=C, heads=heads, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1.0, far=60.0,
                             out_h=44, out_w=72, precision=precision, attn_mode=mode)


def _scene(V=3):
    return synth.scene_raycast(seed=7, V=V, W=72, H=44, f=55.0, arc=0.3)


@pytest.mark.parametrize("C,heads", [(32, 2), (32, 1), (16, 4), (16, 1)])
def test_standard_fp32_matches_oracle(C, heads):
    """Four steps with x2 upsamples and collapses, ragged tiles; per-head widths 16, 32, 4, 16."""
    cfg = _cfg(C, heads)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = _scene()
    ref, ref_steps = O.forward(cfg, W, scene, mode=synth.ATTN_STANDARD)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        for name in ("V_attn", "V_out", "t", "s"):
            assert_rel(g[name], getattr(r, name), REL_TOL_FP32, f"step {j} {name}")
        if "beta" in g:
            assert_rel(g["beta"], r.beta_logits, REL_TOL_FP32, f"step {j} beta")
    err = np.abs(out - ref).max()
    assert err <= RGBA_TOL_FP32, f"rgba max-abs {err:.3e}"


def test_standard_bf16_within_tolerance():
    cfg = _cfg(32, 2, precision=synth.PREC_BF16)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = _scene()
    ref, _ = O.forward(cfg.replace(precision=synth.PREC_FP32), W, scene, mode=synth.ATTN_STANDARD)
    out, _, _ = run_gpu(cfg, W, scene, per_step=False)
    assert np.abs(out - ref).max() <= RGBA_TOL_BF16
    assert psnr(out, ref) >= PSNR_MIN_BF16


def test_standard_equals_folded_one_to_many_on_gpu():
    """Appendix A fold: W^q_i' = sqrt(C / d_h) W^q_i W^k_i^T and W^O' = blockdiag(W^val_i) W^O turn
    the standard block into a one-to-many block with per-head width C; the two GPU paths (image-
    space projection + sampled keys/values, and the one-to-many kernels) agree."""
    C, h = 32, 2
    cfg = _cfg(C, h)
    W = synth.make_weights(cfg, seed=3, sharp=True)
    scene = _scene(V=4)
    std, _, _ = run_gpu(cfg, W, scene, per_step=False)
    dh = C // h
    W2 = dict(W)
    for j in range(cfg.n_scales):
        Wq, Wk, Wv, Wo = (W[f"{n}_std_{j}"].astype(np.float64) for n in ("Wq", "Wk", "Wv", "Wo"))
        W2[f"Wq_{j}"] = np.concatenate(
            [Wq[:, i * dh:(i + 1) * dh] @ Wk[:, i * dh:(i + 1) * dh].T * math.sqrt(C / dh) for i in range(h)],
            1).astype(np.float32)
        W2[f"Wo_{j}"] = np.concatenate([Wv[:, i * dh:(i + 1) * dh] @ Wo[i * dh:(i + 1) * dh] for i in range(h)],
                                       0).astype(np.float32)
    o2m, _, _ = run_gpu(cfg.replace(attn_mode=synth.ATTN_ONE_TO_MANY), W2, scene, per_step=False)
    assert np.abs(std - o2m).max() <= RGBA_TOL_FP32
    torch.cuda.synchronize()
