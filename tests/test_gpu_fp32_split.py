"""The FP32 form's dense contractions on the tensor cores: every operand split into an FP16 value
and its scaled FP16 remainder, three products per K step -- the residual conv block (Sec. 3.3) and
the sampling kernel's query and output projections (Sec. 3.3 one-to-many attention).  The context
takes those paths when the weights bound every part within FP16 range (C <= 32; the conv block with
3x3 kernels); otherwise the SIMT kernels run.  Both against the FP64 oracle at the FP32 form's
tolerances, on ragged tiles."""
import numpy as np
import pytest

from oracle import quark_oracle as O
from paper_2411_16680_b300 import quark, synth
from tests.test_gpu_parity import RGBA_TOL_FP32, check_fp32, run_gpu

pytestmark = pytest.mark.gpu

SIMT_TILE = (16, 8)


def _cfg(C):
    return synth.QuarkConfig(C=C, heads=2, scales=[(4, 8), (2, 4), (1, 2)], near=1.0, far=60.0, out_h=52, out_w=76)


def _scene(seed=5):
    return synth.scene_raycast(seed=seed, V=3, W=76, H=52, f=60.0, arc=0.3)


def _paths(cfg, W):
    """(attend, conv) on the tensor cores, and the conv kernel's tile at the last step."""
    ctx = quark.Context(cfg)
    ctx.load_weights(W)
    L = cfg.scales[-1][1]
    k = cfg.scales[-1][0]
    t = ctx.conv_tiles(L, cfg.out_h // k, cfg.out_w // k)
    at, cv = ctx.tensor_core_paths()
    ctx.close()
    return at, cv, t


@pytest.mark.parametrize("C", [16, 32])
@pytest.mark.parametrize("sharp", [False, True])
def test_split_conv_matches_oracle(C, sharp):
    cfg = _cfg(C)
    W = synth.make_weights(cfg, seed=17, sharp=sharp)
    at, cv, tile = _paths(cfg, W)
    assert at and cv and tile != SIMT_TILE, "the FP32 form should run both kernels on the tensor cores"
    check_fp32(cfg, W, _scene())


@pytest.mark.parametrize("C", [16, 32])
@pytest.mark.parametrize("heads", [1, 4])
@pytest.mark.parametrize("views", [3, 8])
def test_split_attention_heads_and_views(C, heads, views):
    """One and four heads (four: five C query columns, one CTA per SM), an odd and an even view count."""
    cfg = _cfg(C).replace(heads=heads)
    scene = synth.scene_raycast(seed=6, V=views, W=76, H=52, f=60.0, arc=0.4)
    W = synth.make_weights(cfg, seed=23, sharp=True)
    assert _paths(cfg, W)[0]
    check_fp32(cfg, W, scene)


def test_out_of_range_attention_weight_takes_the_simt_kernel():
    """A W^O entry of 4e4 (above 2^15): the split could overflow FP16, so the SIMT sampling kernel
    runs (the conv blocks stay on the tensor cores); the results still match the oracle."""
    cfg = _cfg(32)
    W = synth.make_weights(cfg, seed=17)
    wo = np.array(W["Wo_1"], dtype=np.float32)
    wo[0, 0] = 4e4
    W["Wo_1"] = wo
    at, cv, _ = _paths(cfg, W)
    assert not at and cv
    _check_scaled(cfg, W, _scene())


def _check_scaled(cfg, W, scene):
    """Volumes relative to their largest magnitude (with large terms the sums cancel), the image at
    the FP32 form's tolerance."""
    ref, ref_steps = O.forward(cfg, W, scene)
    out, steps, _ = run_gpu(cfg, W, scene)
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        for name in ("V_attn", "V_out"):
            rv = getattr(r, name)
            err = np.abs(g[name].astype(np.float64) - rv).max() / (1.0 + np.abs(rv).max())
            assert np.isfinite(g[name]).all() and err <= 1e-5, f"step {j} {name}: {err:.3e}"
    assert np.abs(out - ref).max() <= RGBA_TOL_FP32


def test_out_of_range_weights_take_the_simt_kernel():
    """An RMSNorm gain of 1e4 lets the normalised input reach sqrt(C) 1e4 > 2^15: the split could
    overflow FP16, so the context keeps the SIMT kernel, whose results still match the oracle.
    With terms this large the sums cancel, so the volumes are compared relative to their largest
    magnitude (FP32 accumulation error), the image at the FP32 form's tolerance."""
    cfg = _cfg(32)
    W = synth.make_weights(cfg, seed=17)
    W["conv_g_0"] = np.asarray(W["conv_g_0"]) * 1e4
    at, cv, tile = _paths(cfg, W)
    assert at and not cv and tile == SIMT_TILE
    _check_scaled(cfg, W, _scene())


def test_split_conv_narrow_planes():
    """Planes narrower than one tile in x and a single layer at the last step: every tile is ragged."""
    cfg = synth.QuarkConfig(C=32, heads=1, scales=[(2, 2), (1, 1)], near=1.0, far=40.0, out_h=30, out_w=18)
    scene = synth.scene_raycast(seed=9, V=2, W=18, H=30, f=20.0, arc=0.2)
    W = synth.make_weights(cfg, seed=3, sharp=True)
    at, cv, tile = _paths(cfg, W)
    assert at and cv and tile != SIMT_TILE
    check_fp32(cfg, W, scene)
