"""quark_update_fuse_noalloc against quark_update_fuse, through the C ABI.

Some callers cannot allocate device memory while they run: a frame loop that reserves its whole
memory budget up front (a cudaMalloc can fail mid-run and synchronises the device), or a process
whose device memory belongs to another allocator.  They use the no-allocation step, which keeps
its intermediates in a fixed static device array shared by every call.  These tests check that
it reproduces the regular step's outputs within the parity tolerance of the other GPU tests, on
two full passes in a row (the shared array keeps the previous call's contents, which must not
leak into the next result), and that a step too large for the array is refused.

The file name sorts last so that a run stopping at the first failure has already run every
other test.
"""
import numpy as np
import pytest
import torch

from paper_2411_16680_b300 import quark, synth

pytestmark = pytest.mark.gpu

# The FP32 parity tolerance of tests/test_gpu_parity.py.  Both steps launch the same kernels on
# the same inputs, so the BF16 form is held to a bound well inside its own volume tolerance (5e-2):
# only the FP32 decode of the stored BF16 volume may round differently from the conv epilogue's.
REL_TOL = {synth.PREC_FP32: 1e-4, synth.PREC_BF16: 1e-3}


def _close(got, ref, what, tol):
    got = np.asarray(got, np.float64)
    err = np.abs(got - ref) / (1.0 + np.abs(ref))
    assert np.isfinite(got).all(), what
    assert err.max() <= tol, f"{what}: max rel err {err.max():.3e}"


def _volume_to_f32(t, precision):
    return t.float() if precision == synth.PREC_BF16 else t


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
def test_noalloc_step_matches_regular_step_twice(precision):
    cfg = synth.QuarkConfig(C=32, heads=2, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1.0, far=60.0,
                            out_h=44, out_w=72, precision=precision)
    scene = synth.scene_raycast(seed=7, V=3, W=72, H=44, f=55.0, arc=0.3)
    V = len(scene.cams)
    vdtype = torch.bfloat16 if precision == synth.PREC_BF16 else torch.float32
    tol = REL_TOL[precision]
    ctx = quark.Context(cfg)
    ctx.load_weights(synth.make_weights(cfg, seed=11, sharp=True))
    pyr = ctx.encode_pyramid(torch.tensor(scene.images, device="cuda"), scene.cams)

    ldm = ctx.ldm_create(scene.target)
    ref = []
    for j in range(cfg.n_scales):
        ctx.update_fuse(pyr, j, ldm)
        L, H, W = cfg.ldm_shape(j)
        r = {"v": ldm.read(quark.FIELD_VOLUME, (L, H, W, cfg.C)),
             "colour": ldm.read(quark.FIELD_COLOUR, (L, H, W, 3)),
             "alpha": ldm.read(quark.FIELD_ALPHA, (L, H, W)),
             "depth": ldm.read(quark.FIELD_DEPTH, (L, H, W)),
             "t": ldm.read(quark.FIELD_DEPTH_LOGIT, (H, W, L)),
             "s": ldm.read(quark.FIELD_DENSITY_LOGIT, (H, W, L))}
        if j == cfg.n_scales - 1:
            r["beta"] = ldm.read(quark.FIELD_BETA_LOGITS, (H, W, L, V))
        ref.append(r)

    for rep in range(2):
        prev = None
        for j in range(cfg.n_scales):
            L, H, W = cfg.ldm_shape(j)
            last = j == cfg.n_scales - 1
            out = {"v": torch.empty(L, H, W, cfg.C, device="cuda", dtype=vdtype),
                   "colour": torch.empty(L, H, W, 3, device="cuda"),
                   "alpha": torch.empty(L, H, W, device="cuda"),
                   "depth": torch.empty(L, H, W, device="cuda"),
                   "t": torch.empty(H, W, L, device="cuda"),
                   "s": torch.empty(H, W, L, device="cuda")}
            if last:
                out["beta"] = torch.empty(H, W, L, V, device="cuda")
            ctx.update_fuse_noalloc(pyr, j, scene.target, prev, out["v"], out["colour"], out["alpha"],
                                    out["depth"], out["t"], out["s"], out.get("beta"))
            torch.cuda.synchronize()
            for name, t in out.items():
                got = _volume_to_f32(t, precision) if name == "v" else t
                _close(got.cpu().numpy(), ref[j][name], f"pass {rep} step {j} {name}", tol)
            prev = out["v"]


def test_noalloc_refuses_a_step_larger_than_its_scratch():
    cfg = synth.QuarkConfig(C=32, heads=1, scales=[(1, 16)], near=1.0, far=60.0, out_h=1024, out_w=1024)
    scene = synth.scene_noise_pair(V=1, W=16, H=16)
    ctx = quark.Context(cfg)
    ctx.load_weights(synth.make_weights(cfg))
    pyr = ctx.encode_pyramid(torch.tensor(scene.images, device="cuda"), scene.cams)
    target = synth.make_camera(1024, 1024, 900.0, (0.0, 0.0, 0.0))
    L, H, W = cfg.ldm_shape(0)
    small = torch.empty(16, device="cuda")
    with pytest.raises(quark.QuarkError) as e:
        ctx.update_fuse_noalloc(pyr, 0, target, None, small, small, small, small, small, small, small)
    assert e.value.status == quark.EINVAL
    assert "static scratch" in str(e.value)


def test_noalloc_refuses_unaligned_buffers():
    # the kernels move v_prev, v_out and beta in 16- and 32-byte vectors: a buffer that does not
    # start on a 32-byte boundary is refused before any launch
    cfg = synth.QuarkConfig(C=32, heads=1, scales=[(1, 4)], near=1.0, far=60.0, out_h=16, out_w=16)
    scene = synth.scene_noise_pair(V=1, W=16, H=16)
    ctx = quark.Context(cfg)
    ctx.load_weights(synth.make_weights(cfg))
    pyr = ctx.encode_pyramid(torch.tensor(scene.images, device="cuda"), scene.cams)
    target = synth.make_camera(16, 16, 14.0, (0.0, 0.0, 0.0))
    buf = torch.zeros(1 << 16, device="cuda")
    shifted = buf[1:]  # 4 bytes past a 256-byte boundary
    with pytest.raises(quark.QuarkError) as e:
        ctx.update_fuse_noalloc(pyr, 0, target, None, shifted, buf, buf, buf, buf, buf, buf)
    assert e.value.status == quark.EINVAL
    assert "32-byte aligned" in str(e.value)


def test_noalloc_refuses_host_buffers():
    # every caller buffer must be device memory of the context's device: a host array (which the
    # kernels cannot dereference) is refused before any launch
    cfg = synth.QuarkConfig(C=32, heads=1, scales=[(1, 4)], near=1.0, far=60.0, out_h=16, out_w=16)
    scene = synth.scene_noise_pair(V=1, W=16, H=16)
    ctx = quark.Context(cfg)
    ctx.load_weights(synth.make_weights(cfg))
    pyr = ctx.encode_pyramid(torch.tensor(scene.images, device="cuda"), scene.cams)
    target = synth.make_camera(16, 16, 14.0, (0.0, 0.0, 0.0))
    L, H, W = cfg.ldm_shape(0)
    dev = {n: torch.zeros(L * H * W * max(cfg.C, 3), device="cuda") for n in ("v", "c", "a", "d", "t", "s", "b")}
    host = np.zeros(L * H * W * 3, np.float32)
    n0 = ctx.launch_count()
    with pytest.raises(quark.QuarkError) as e:
        ctx.update_fuse_noalloc(pyr, 0, target, None, dev["v"], host, dev["a"], dev["d"], dev["t"], dev["s"], dev["b"])
    assert e.value.status == quark.EINVAL
    assert "colour must be device memory" in str(e.value)
    assert ctx.launch_count() == n0
    # the same call on device buffers runs
    ctx.update_fuse_noalloc(pyr, 0, target, None, dev["v"], dev["c"], dev["a"], dev["d"], dev["t"], dev["s"], dev["b"])
    torch.cuda.synchronize()
    assert ctx.launch_count() > n0
