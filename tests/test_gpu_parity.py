"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances (the benchmark spec's bar, and one derived for the intermediates):
  FP32 form  output RGBA max-abs <= 1e-4 on [0, 1].  Feature volumes, logits and decoded
             attributes: |gpu - oracle| <= 1e-4 (1 + |oracle|): FP32 dot products of at most
             9C = 288 terms of O(1) size carry a few 1e-5 relative error at worst.
  BF16 form  output RGBA max-abs <= 2e-2 and PSNR >= 40 dB against the oracle.
Integer work (tap indices, layer order) has no separate output: a wrong tap or layer shows up
as an O(1) error in the values compared here.
"""
import math

import numpy as np
import pytest
import torch

from oracle import quark_oracle as O
from paper_2411_16680_b300 import quark, synth

pytestmark = pytest.mark.gpu

RGBA_TOL_FP32 = 1e-4
REL_TOL_FP32 = 1e-4
RGBA_TOL_BF16 = 2e-2
PSNR_MIN_BF16 = 40.0


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)


def run_gpu(cfg, W, scene, per_step=True, host_io=False):
    ctx = quark.Context(cfg)
    ctx.load_weights(W)
    if host_io:
        images = np.ascontiguousarray(scene.images)
    else:
        images = torch.tensor(scene.images, device="cuda")
    pyr = ctx.encode_pyramid(images, scene.cams)
    ldm = ctx.ldm_create(scene.target)
    steps = []
    for j in range(cfg.n_scales):
        ctx.update_fuse(pyr, j, ldm)
        if per_step:
            L, H, Wd = cfg.ldm_shape(j)
            st = {
                "V_attn": ldm.read(quark.FIELD_VOLUME_ATTN, (L, H, Wd, cfg.C)),
                "V_out": ldm.read(quark.FIELD_VOLUME, (L, H, Wd, cfg.C)),
                "colour": ldm.read(quark.FIELD_COLOUR, (L, H, Wd, 3)),
                "alpha": ldm.read(quark.FIELD_ALPHA, (L, H, Wd)),
                "depth": ldm.read(quark.FIELD_DEPTH, (L, H, Wd)),
                "t": ldm.read(quark.FIELD_DEPTH_LOGIT, (H, Wd, L)).transpose(2, 0, 1),
                "s": ldm.read(quark.FIELD_DENSITY_LOGIT, (H, Wd, L)).transpose(2, 0, 1),
            }
            if j == cfg.n_scales - 1:
                st["beta"] = ldm.read(quark.FIELD_BETA_LOGITS, (H, Wd, L, len(scene.cams))).transpose(2, 0, 1, 3)
            steps.append(st)
    if host_io:
        out = np.zeros((cfg.out_h, cfg.out_w, 4), np.float32)
        ctx.render_ldm(ldm, pyr, out)
        torch.cuda.synchronize()
    else:
        out_t = torch.zeros(cfg.out_h, cfg.out_w, 4, device="cuda")
        ctx.render_ldm(ldm, pyr, out_t)
        out = out_t.cpu().numpy()
    ctx.check_device()
    n = ctx.launch_count()
    return out, steps, n


def assert_rel(gpu, ref, tol, what):
    err = np.abs(gpu.astype(np.float64) - ref) / (1.0 + np.abs(ref))
    assert np.isfinite(gpu).all(), what
    assert err.max() <= tol, f"{what}: max rel err {err.max():.3e} at {np.unravel_index(err.argmax(), err.shape)}"


def check_fp32(cfg, W, scene, per_step=True):
    ref, ref_steps = O.forward(cfg, W, scene)
    out, steps, _ = run_gpu(cfg, W, scene, per_step)
    for j, (g, r) in enumerate(zip(steps, ref_steps)):
        for name in ("V_attn", "V_out", "colour", "alpha", "depth", "t", "s"):
            assert_rel(g[name], getattr(r, name), REL_TOL_FP32, f"step {j} {name}")
        if "beta" in g:
            assert_rel(g["beta"], r.beta_logits, REL_TOL_FP32, f"step {j} beta")
    err = np.abs(out - ref).max()
    assert err <= RGBA_TOL_FP32, f"rgba max-abs {err:.3e}"
    return out, ref


# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("sharp", [False, True])
def test_small_workload_fp32(sharp):
    """V=2 64x48 views, one step at k=2 with L=4, C=16, h=1, output 64x48 (s=2)."""
    cfg = synth.config_small()
    check_fp32(cfg, synth.make_weights(cfg, sharp=sharp), synth.scene_small())


def _multi_cfg(C=32, heads=2, out_w=72, out_h=44):
    return synth.QuarkConfig(C=C, heads=heads, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1.0, far=60.0,
                             out_h=out_h, out_w=out_w)


@pytest.mark.parametrize("C,heads", [(32, 2), (16, 4), (32, 1)])
def test_multiscale_collapse_upsample_fp32(C, heads):
    """Four steps: x2 upsample + collapse, collapse at the same resolution, x2 upsample; ragged
    tiles in x and y (72x44 output), sharp weights."""
    cfg = _multi_cfg(C, heads)
    scene = synth.scene_raycast(seed=7, V=3, W=72, H=44, f=55.0, arc=0.3)
    check_fp32(cfg, synth.make_weights(cfg, seed=11, sharp=True), scene)


def test_degenerate_single_view_single_layer():
    cfg = synth.QuarkConfig(C=16, heads=1, scales=[(2, 1), (1, 1)], near=1.0, far=30.0, out_h=24, out_w=40)
    scene = synth.scene_raycast(seed=3, V=1, W=40, H=24, f=30.0, arc=0.0)
    check_fp32(cfg, synth.make_weights(cfg, sharp=True), scene)


def test_views_behind_and_outside():
    """One view looks away from the scene (every sample at z <= 0: zero features, logit 0) and one
    is displaced far sideways (samples fall outside its image: zero padding)."""
    cfg = synth.QuarkConfig(C=16, heads=2, scales=[(2, 4), (1, 2)], near=1.0, far=40.0, out_h=32, out_w=48)
    scene = synth.scene_raycast(seed=5, V=3, W=48, H=32, f=40.0, arc=0.2)
    back = synth.make_camera(48, 32, 40.0, (0.0, 0.0, 0.0), target=(0.0, 0.0, -10.0))
    side = synth.make_camera(48, 32, 40.0, (30.0, 0.0, 0.0), target=(31.0, 0.0, 10.0))
    scene.cams = [scene.cams[0], back, side]
    check_fp32(cfg, synth.make_weights(cfg, seed=2, sharp=True), scene)


def test_host_buffers_match_device_buffers():
    cfg = _multi_cfg(16, 2)
    scene = synth.scene_raycast(seed=9, V=2, W=72, H=44, f=55.0, arc=0.2)
    W = synth.make_weights(cfg, sharp=True)
    a, _, _ = run_gpu(cfg, W, scene, per_step=False, host_io=False)
    b, _, _ = run_gpu(cfg, W, scene, per_step=False, host_io=True)
    assert np.array_equal(a, b)


def test_deterministic_and_launch_count():
    cfg = _multi_cfg(32, 2)
    scene = synth.scene_raycast(seed=9, V=2, W=72, H=44, f=55.0, arc=0.2)
    W = synth.make_weights(cfg, sharp=True)
    a, _, n = run_gpu(cfg, W, scene, per_step=False)
    b, _, _ = run_gpu(cfg, W, scene, per_step=False)
    assert np.array_equal(a, b)
    # encode + per step (collapse where L halves) attend + conv + render
    n_collapse = sum(1 for j in range(1, cfg.n_scales) if cfg.scales[j - 1][1] == 2 * cfg.scales[j][1])
    assert n == 1 + 2 * cfg.n_scales + n_collapse + 1


REL_TOL_BF16_VOLUME = 5e-2  # BF16 storage of V and BF16 tensor-core operands: a few 2^-8 roundings


@pytest.mark.parametrize("sharp", [False, True])
def test_bf16_form(sharp):
    """Precision form: BF16 pyramid / volumes, tcgen05 conv block (BF16 operands, FP32
    accumulation), FP32 geometry / softmax / transmittance, vs the FP64 oracle.  Each step's
    volume within 5e-2 (1 + |ref|); the output within the benchmark spec's 2e-2 max-abs, >= 40 dB."""
    for cfg, scene in ((synth.config_small().replace(precision=synth.PREC_BF16), synth.scene_small()),
                       (_multi_cfg(32, 2).replace(precision=synth.PREC_BF16),
                        synth.scene_raycast(seed=7, V=3, W=72, H=44, f=55.0, arc=0.3)),
                       (_multi_cfg(16, 4).replace(precision=synth.PREC_BF16),
                        synth.scene_raycast(seed=8, V=4, W=72, H=44, f=55.0, arc=0.3))):
        W = synth.make_weights(cfg, seed=11, sharp=sharp)
        ref, ref_steps = O.forward(cfg, W, scene)
        out, steps, _ = run_gpu(cfg, W, scene, per_step=True)
        for j, (g, r) in enumerate(zip(steps, ref_steps)):
            # the volumes after the attention block and after the conv block, and the raw depth /
            # density logits decoded from the stored BF16 volume (Sec. 3.2.3)
            for name in ("V_attn", "V_out", "t", "s"):
                assert_rel(g[name], getattr(r, name), REL_TOL_BF16_VOLUME, f"bf16 step {j} {name}")
            if "beta" in g:
                # blend logits: BF16 query and sampled features, FP32 dot product (Sec. 3.2.3)
                assert_rel(g["beta"], r.beta_logits, REL_TOL_BF16_VOLUME, f"bf16 step {j} beta")
        err = np.abs(out - ref).max()
        assert err <= RGBA_TOL_BF16, f"bf16 rgba max-abs {err:.3e}"
        assert psnr(out, ref) >= PSNR_MIN_BF16


@pytest.mark.parametrize("C", [16, 32, 64])
def test_bf16_pyramid_levels(C):
    """Every level of the BF16 form's pyramid against the oracle's (Sec. 3.2.1: F_1 the 3x3 conv of
    the image, F_2k the 2x2 means of F_k), on three views of 72 x 56 pixels (the largest factor, 8,
    divides the view): ragged 16 x 8 encoder tiles in x and a 9 x 7 level 8.  Per texel |gpu - oracle| <= 2^-8 (S + |oracle|) + 1e-6, S the same
    conv and means of |I| with |W| and no bias: the BF16 rounding of the image and weight operands
    (2^-9 each) and of the stored texel (2^-9).  A texel, channel or block misplaced by the
    pooling's lane exchanges is an error of the size of the features themselves."""
    H, Wd, V = 56, 72, 3
    cfg = synth.QuarkConfig(C=C, heads=1, scales=[(8, 4), (4, 4), (2, 2), (1, 2)], near=1.0, far=40.0,
                            out_h=H, out_w=Wd, precision=synth.PREC_BF16)
    sc = synth.scene_raycast(seed=31, V=V, W=Wd, H=H, f=50.0, arc=0.3)
    for sharp in (False, True):
        W = synth.make_weights(cfg, seed=12, sharp=sharp)
        ctx = quark.Context(cfg)
        ctx.load_weights(W)
        pyr = ctx.encode_pyramid(torch.tensor(sc.images, device="cuda"), sc.cams)
        for k in (1, 2, 4, 8):
            ref = np.stack([O.encode_level(sc.images[m], W["enc_w"], W["enc_b"], k) for m in range(V)])
            mag = np.stack([O.encode_level(np.abs(sc.images[m]), np.abs(W["enc_w"]), np.zeros_like(W["enc_b"]), k)
                            for m in range(V)])
            raw = np.zeros(ref.shape, np.uint16)
            pyr.read_level(k, raw)
            got = (raw.astype(np.uint32) << 16).view(np.float32)  # BF16 is the high half of an FP32 word
            err = np.abs(got.astype(np.float64) - ref)
            tol = 2.0 ** -8 * (mag + np.abs(ref)) + 1e-6
            bad = np.argwhere(err > tol)
            assert bad.size == 0, (f"C={C} sharp={sharp} level {k}: {len(bad)} texels out of bound, first "
                                   f"{tuple(bad[0])}: gpu {got[tuple(bad[0])]:.6g} oracle {ref[tuple(bad[0])]:.6g}")
        ctx.check_device()
        pyr.release()
        ctx.close()


def test_invalid_arguments_are_rejected():
    cfg = synth.config_small()
    ctx = quark.Context(cfg)
    ctx.load_weights(synth.make_weights(cfg))
    sc = synth.scene_small()
    images = torch.tensor(sc.images, device="cuda")
    bad = synth.Camera(64, 48, float("nan"), 60.0, 32.0, 24.0, np.eye(3), np.zeros(3))
    with pytest.raises(quark.QuarkError) as e:
        ctx.encode_pyramid(images, [sc.cams[0], bad])
    assert e.value.status == quark.EINVAL
    odd = synth.Camera(63, 48, 60.0, 60.0, 32.0, 24.0, np.eye(3), np.zeros(3))
    with pytest.raises(quark.QuarkError):
        ctx.ldm_create(odd)
    pyr = ctx.encode_pyramid(images, sc.cams)
    ldm = ctx.ldm_create(sc.target)
    out = torch.zeros(48, 64, 4, device="cuda")
    with pytest.raises(quark.QuarkError):
        ctx.render_ldm(ldm, pyr, out)  # no Update & Fuse step yet
    ctx.update_fuse(pyr, 0, ldm)
    ctx.render_ldm(ldm, pyr, out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()


def test_hbm_cap_refuses_instead_of_overcommitting():
    cfg = synth.config_small()
    ctx = quark.Context(cfg, hbm_cap_bytes=200_000)
    ctx.load_weights(synth.make_weights(cfg))
    sc = synth.scene_small()
    with pytest.raises(quark.QuarkError) as e:
        pyr = ctx.encode_pyramid(torch.tensor(sc.images, device="cuda"), sc.cams)
        ctx.ldm_create(sc.target)
    assert e.value.status == quark.ENOMEM


# --------------------------------------------------------------------------------------------
# The 1080p workload, at full size, on sampled outputs
# --------------------------------------------------------------------------------------------

FULL_RECTS = [(0, 4, 0, 4), (538, 542, 958, 962), (1076, 1080, 1916, 1920), (300, 303, 1500, 1506)]


# Attention-kernel tiles are 16 x 8 LDM pixels at every step: output pixel (1024, 512) lies on a
# tile corner of every step whose grid factor divides 8, the corner (128 j, 64 i) of each.
ATTEND_SEAM_RECTS = [(510, 514, 1022, 1026), (62, 66, 1790, 1794)]


def conv_seam_rects(ctx, cfg):
    """Output windows straddling a tile corner of the conv-block kernel at every step: the tile the
    kernel of the context's form uses for that step's plane (quark_conv_tiles), one corner near
    the middle of the plane and the last interior corner next to the ragged tiles."""
    rects = []
    for j, (k, L) in enumerate(cfg.scales):
        H, W = cfg.out_h // k, cfg.out_w // k
        cols, rows = ctx.conv_tiles(L, H, W)
        ty, tx = (H - 1) // rows, (W - 1) // cols  # index of the last (ragged) tile row / column
        for iy, ix in ((max(1, ty // 2), max(1, tx // 2)), (ty, tx)):
            if iy < 1 or ix < 1:
                continue
            y, x = iy * rows * k, ix * cols * k  # output coordinates of the corner
            rects.append((y - 2, y + 2, x - 2, x + 2))
    return rects


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_1080p_sampled_outputs(precision):
    """V=8 1920x1080 views, scales (8,32),(4,16),(2,8),(1,4), C=32, h=2, 1080p output, in the
    launch configuration the bench times; the oracle computes output windows from scratch through
    every scale: corners and the centre of the frame, windows across the attention kernel's tile
    corners, and windows across the conv-block kernel's tile corners at every step (the tensor-core
    conv kernel of either form picks its tile per plane size, so these windows sit where its tiling
    changes)."""
    cfg = synth.config_1080p().replace(precision=precision)
    scene = synth.scene_1080p()
    W = synth.make_weights(cfg, sharp=True)
    ctx = quark.Context(cfg)
    ctx.load_weights(W)  # the FP32 form's conv kernel (and tile) depends on the weights
    rects = FULL_RECTS + ATTEND_SEAM_RECTS + conv_seam_rects(ctx, cfg)
    ctx.close()
    out, _, _ = run_gpu(cfg, W, scene, per_step=False)
    assert np.isfinite(out).all()
    tol = RGBA_TOL_FP32 if precision == synth.PREC_FP32 else RGBA_TOL_BF16
    for r in rects:
        ref, _ = O.forward(cfg, W, scene, r)
        err = np.abs(out[r[0]:r[1], r[2]:r[3]] - ref).max()
        assert err <= tol, f"{r}: max-abs {err:.3e}"


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_maximum_view_count(precision):
    """QUARK_MAX_VIEWS (64) views through every step and the render; one more is refused."""
    cfg = synth.QuarkConfig(C=16, heads=2, scales=[(2, 4), (1, 2)], near=1.0, far=40.0, out_h=24, out_w=40,
                            precision=precision)
    scene = synth.scene_raycast(seed=13, V=quark.MAX_VIEWS, W=40, H=24, f=30.0, arc=0.8)
    W = synth.make_weights(cfg, seed=2, sharp=True)
    ref, ref_steps = O.forward(cfg, W, scene)
    out, steps, _ = run_gpu(cfg, W, scene, per_step=precision == synth.PREC_FP32)
    if precision == synth.PREC_FP32:
        for j, (g, r) in enumerate(zip(steps, ref_steps)):
            assert_rel(g["V_out"], r.V_out, REL_TOL_FP32, f"step {j} V_out")
        assert_rel(steps[-1]["beta"], ref_steps[-1].beta_logits, REL_TOL_FP32, "beta")
        assert np.abs(out - ref).max() <= RGBA_TOL_FP32
    else:
        assert np.abs(out - ref).max() <= RGBA_TOL_BF16 and psnr(out, ref) >= PSNR_MIN_BF16
    ctx = quark.Context(cfg)
    try:
        cams = list(scene.cams) + [scene.cams[0]]
        images = np.concatenate([scene.images, scene.images[:1]])
        with pytest.raises(quark.QuarkError) as e:
            ctx.encode_pyramid(images, cams)
        assert e.value.status == quark.EINVAL
    finally:
        ctx.close()


def test_destroy_refuses_while_handles_live():
    """A context is not destroyed under its pyramids and LDMs (their release would touch freed
    state): quark_destroy returns EBUSY until they are released; Context.close() releases them."""
    cfg = synth.config_small()
    ctx = quark.Context(cfg)
    ctx.load_weights(synth.make_weights(cfg))
    sc = synth.scene_small()
    pyr = ctx.encode_pyramid(torch.tensor(sc.images, device="cuda"), sc.cams)
    ldm = ctx.ldm_create(sc.target)
    assert quark.lib().quark_destroy(ctx.handle) == quark.EBUSY
    ldm.release()
    assert quark.lib().quark_destroy(ctx.handle) == quark.EBUSY
    pyr2 = ctx.encode_pyramid(torch.tensor(sc.images, device="cuda"), sc.cams)
    ctx.close()  # releases pyr and pyr2, then destroys
    assert ctx.handle is None and pyr.handle is None and pyr2.handle is None
    pyr.release()  # a no-op once the context is gone
