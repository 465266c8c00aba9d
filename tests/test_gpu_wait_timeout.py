"""The error path of the tensor-core kernels' bounded waits, run without a fault or a hang.

Every mbarrier wait of the tcgen05 kernels gives up after a time limit: the kernel then records
the timeout in the context's error word, skips its outputs, waits (bounded) for its MMAs in
flight, frees its tensor memory and returns, and quark_check_device reports QUARK_ETIMEDOUT.
quark_test_wait_timeout makes one sampling launch leave its query MMA chain unissued, so that the
wait on it (an mbarrier nothing arrives at) runs out after 1 ms.  The test checks the reported
status, that the error word is cleared by the report, and that the same context then renders the
frame exactly as a context that never timed out.
"""
import numpy as np
import pytest
import torch

from paper_2411_16680_b300 import quark, synth

pytestmark = pytest.mark.gpu


def _render(ctx, pyr, scene, cfg):
    ldm = ctx.ldm_create(scene.target)
    out = torch.zeros(cfg.out_h, cfg.out_w, 4, device="cuda")
    ctx.render_novel_view(pyr, ldm, out)
    torch.cuda.synchronize()
    ldm.release()
    return out.cpu().numpy()


def test_bounded_wait_runs_out_and_the_context_recovers():
    cfg = synth.QuarkConfig(C=32, heads=2, scales=[(2, 4), (1, 2)], near=1.0, far=40.0, out_h=32, out_w=48,
                            precision=synth.PREC_BF16)
    scene = synth.scene_raycast(seed=5, V=3, W=48, H=32, f=40.0, arc=0.2)
    W = synth.make_weights(cfg, seed=2, sharp=True)
    images = torch.tensor(scene.images, device="cuda")

    clean = quark.Context(cfg)
    clean.load_weights(W)
    clean_pyr = clean.encode_pyramid(images, scene.cams)
    ref = _render(clean, clean_pyr, scene, cfg)
    clean.check_device()
    clean_pyr.release()
    clean.close()

    ctx = quark.Context(cfg)
    ctx.load_weights(W)
    pyr = ctx.encode_pyramid(images, scene.cams)
    ctx.test_wait_timeout()
    ldm = ctx.ldm_create(scene.target)
    ctx.update_fuse(pyr, 0, ldm)  # this step's sampling launch times out
    with pytest.raises(quark.QuarkError) as e:
        ctx.check_device()
    assert e.value.status == quark.ETIMEDOUT
    ctx.check_device()  # the report cleared the error word
    ldm.release()
    out = _render(ctx, pyr, scene, cfg)
    ctx.check_device()
    assert np.array_equal(out, ref)


def test_wait_timeout_test_needs_the_bf16_form():
    ctx = quark.Context(synth.config_small())
    with pytest.raises(quark.QuarkError) as e:
        ctx.test_wait_timeout()
    assert e.value.status == quark.EINVAL
    ctx.close()
