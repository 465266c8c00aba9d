"""Depth-map output (Sec. 3.1: the decoded depth over-composited instead of the blended input
views) through the C ABI, against the oracle: FP32 form to 1e-4 relative, BF16 form within the
volume tolerance; device and host targets give the same bits."""
import numpy as np
import pytest
import torch

from oracle import quark_oracle as O
from paper_2411_16680_b300 import quark, synth

pytestmark = pytest.mark.gpu


def _solve(cfg, W, scene):
    ctx = quark.Context(cfg)
    ctx.load_weights(W)
    pyr = ctx.encode_pyramid(torch.tensor(scene.images, device="cuda"), scene.cams)
    ldm = ctx.ldm_create(scene.target)
    for j in range(cfg.n_scales):
        ctx.update_fuse(pyr, j, ldm)
    return ctx, pyr, ldm


@pytest.mark.parametrize("precision,tol", [(synth.PREC_FP32, 1e-4), (synth.PREC_BF16, 5e-2)])
@pytest.mark.parametrize("scales", [[(4, 8), (2, 4), (2, 2), (1, 2)], [(4, 8), (2, 4)]])
def test_depth_map_matches_oracle(precision, tol, scales):
    """s = 1 (direct reads) and s = 2 (upsampled logits); ragged 72x44 output."""
    cfg = synth.QuarkConfig(C=32, heads=2, scales=scales, near=1.0, far=60.0, out_h=44, out_w=72,
                            precision=precision)
    W = synth.make_weights(cfg, seed=11, sharp=True)
    scene = synth.scene_raycast(seed=7, V=3, W=72, H=44, f=55.0, arc=0.3)
    ctx, pyr, ldm = _solve(cfg, W, scene)
    dev = torch.full((44, 72), float("nan"), device="cuda")
    ctx.render_depth(ldm, dev)
    host = np.full((44, 72), np.nan, np.float32)
    ctx.render_depth(ldm, host)
    torch.cuda.synchronize()
    ctx.check_device()
    got = dev.cpu().numpy()
    assert np.array_equal(got, host)
    _, steps = O.forward(cfg.replace(precision=synth.PREC_FP32), W, scene)
    ref = O.render_depth_rect(cfg, steps[-1], (0, 44, 0, 72))
    err = np.abs(got - ref) / (1.0 + np.abs(ref))
    assert np.isfinite(got).all() and err.max() <= tol, f"max rel err {err.max():.3e}"


def test_depth_map_needs_every_step():
    cfg = synth.QuarkConfig(C=16, heads=1, scales=[(2, 4), (1, 2)], near=1.0, far=30.0, out_h=24, out_w=40)
    W = synth.make_weights(cfg)
    scene = synth.scene_raycast(seed=3, V=2, W=40, H=24, f=30.0, arc=0.2)
    ctx = quark.Context(cfg)
    ctx.load_weights(W)
    pyr = ctx.encode_pyramid(torch.tensor(scene.images, device="cuda"), scene.cams)
    ldm = ctx.ldm_create(scene.target)
    ctx.update_fuse(pyr, 0, ldm)
    with pytest.raises(quark.QuarkError) as e:
        ctx.render_depth(ldm, torch.zeros(24, 40, device="cuda"))
    assert e.value.status == quark.EINVAL
