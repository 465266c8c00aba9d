"""Serving form through the C ABI: results are the same alone and in a concurrent mix, equal to
the direct call path, within the FP32 parity tolerance of the oracle; the queue, admission cap,
cancellation, timeouts and unknown tickets behave as documented.  Every failure here is made on
the host (a paused scheduler, a full queue, an unknown ticket); nothing faults the GPU."""
import numpy as np
import pytest
import torch

from oracle import quark_oracle as O
from paper_2411_16680_b300 import quark, synth

pytestmark = pytest.mark.gpu


def _setup(precision=synth.PREC_FP32, n_slots=4, cap=0, queue=64):
    cfg = synth.QuarkConfig(C=32, heads=2, scales=[(4, 8), (2, 4), (1, 2)], near=1.0, far=60.0, out_h=44, out_w=72,
                            precision=precision)
    W = synth.make_weights(cfg, seed=3, sharp=True)
    ctx = quark.Context(cfg)
    ctx.load_weights(W)
    srv = quark.Server(ctx, n_slots=n_slots, queue_capacity=queue, hbm_cap_bytes=cap)
    scenes = {}
    for t, seed in ((0, 11), (1, 12)):
        sc = synth.scene_raycast(seed=seed, V=4, W=72, H=44, f=55.0, arc=0.3)
        srv.set_timestep(t, torch.tensor(sc.images, device="cuda"), sc.cams)
        scenes[t] = sc
    return cfg, W, ctx, srv, scenes


def _requests(scenes):
    reqs = []
    rng = np.random.default_rng(0)
    for i in range(12):
        t = i % 2
        w, h = [(72, 44), (144, 88), (48, 32)][i % 3]
        base = scenes[t].target
        target = synth.Camera(w, h, base.fx * w / 72, base.fy * h / 44, w / 2, h / 2, base.R,
                              base.t + rng.uniform(-0.05, 0.05, 3))
        reqs.append((t, target, 1 + i % 4))
    return reqs


def _run(srv, reqs, concurrent):
    outs = [torch.full((tg.height, tg.width, 4), float("nan"), device="cuda") for _, tg, _ in reqs]
    results = [None] * len(reqs)
    if concurrent:
        tickets = [srv.submit(t, tg, n, outs[i], user_tag=i) for i, (t, tg, n) in enumerate(reqs)]
        for i, tk in enumerate(tickets):
            results[i] = srv.poll(tk, timeout_us=30_000_000)
    else:
        for i, (t, tg, n) in enumerate(reqs):
            results[i] = srv.poll(srv.submit(t, tg, n, outs[i], user_tag=i), timeout_us=30_000_000)
    for i, r in enumerate(results):
        assert r is not None and r.status == quark.OK and not r.cancelled and r.user_tag == i
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


def test_alone_equals_mix_equals_direct_and_oracle():
    cfg, W, ctx, srv, scenes = _setup(n_slots=6)
    try:
        reqs = _requests(scenes)
        alone = _run(srv, reqs, concurrent=False)
        mixed = _run(srv, reqs, concurrent=True)
        for a, b in zip(alone, mixed):
            assert np.array_equal(a, b)  # the same kernels on the same inputs: bitwise equal
        st = srv.stats()
        assert st.completed == 2 * len(reqs) and st.failed == 0 and st.p99_ms >= st.p50_ms > 0
    finally:
        srv.stop()
    # the direct call path on a pyramid of the first n views
    ctx2 = quark.Context(cfg)
    ctx2.load_weights(W)
    for i in (0, 4, 7):
        t, tg, n = reqs[i]
        sc = scenes[t]
        pyr = ctx2.encode_pyramid(torch.tensor(sc.images[:n], device="cuda"), sc.cams[:n])
        ldm = ctx2.ldm_create(tg)
        out = torch.zeros(tg.height, tg.width, 4, device="cuda")
        ctx2.render_novel_view(pyr, ldm, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), alone[i])
        # and the oracle on the same request
        ref, _ = O.forward(cfg.replace(out_h=tg.height, out_w=tg.width), W,
                           synth.Scene(sc.images[:n], sc.cams[:n], tg))
        assert np.abs(alone[i] - ref).max() <= 1e-4


def test_bf16_mix_within_tolerance_of_oracle():
    cfg, W, ctx, srv, scenes = _setup(precision=synth.PREC_BF16, n_slots=3)
    try:
        reqs = _requests(scenes)[:6]
        mixed = _run(srv, reqs, concurrent=True)
        alone = _run(srv, reqs, concurrent=False)
    finally:
        srv.stop()
    for i, (t, tg, n) in enumerate(reqs):
        assert np.array_equal(alone[i], mixed[i])
        sc = scenes[t]
        ref, _ = O.forward(cfg.replace(out_h=tg.height, out_w=tg.width, precision=synth.PREC_FP32), W,
                           synth.Scene(sc.images[:n], sc.cams[:n], tg))
        assert np.abs(mixed[i] - ref).max() <= 2e-2


def test_queue_cancel_timeout_and_errors():
    cfg, W, ctx, srv, scenes = _setup(n_slots=2, queue=3)
    try:
        tg = scenes[0].target
        outs = [torch.zeros(44, 72, 4, device="cuda") for _ in range(4)]
        srv.pause(True)
        tickets = [srv.submit(0, tg, 4, outs[i], user_tag=i) for i in range(3)]
        with pytest.raises(quark.QuarkError) as e:  # queue full
            srv.submit(0, tg, 4, outs[3])
        assert e.value.status == quark.EBUSY
        assert srv.poll(tickets[0], timeout_us=0) is None  # not done: EAGAIN
        assert srv.poll(tickets[0], timeout_us=20_000) is None  # paused: ETIMEDOUT
        srv.cancel(tickets[1])
        r = srv.poll(tickets[1], timeout_us=0)
        assert r.cancelled
        srv.pause(False)
        r0 = srv.poll(tickets[0], timeout_us=30_000_000)
        r2 = srv.poll(tickets[2], timeout_us=30_000_000)
        assert r0.status == quark.OK and r2.status == quark.OK
        with pytest.raises(quark.QuarkError) as e:  # consumed
            srv.poll(tickets[0])
        assert e.value.status == quark.ENOTFOUND
        with pytest.raises(quark.QuarkError) as e:
            srv.submit(7, tg, 4, outs[0])  # no such time step
        assert e.value.status == quark.ENOTFOUND
        with pytest.raises(quark.QuarkError) as e:
            srv.submit(0, tg, 5, outs[0])  # more views than resident
        assert e.value.status == quark.EINVAL
        bad = synth.Camera(70, 44, 55.0, 55.0, 35.0, 22.0, np.eye(3), np.zeros(3))
        with pytest.raises(quark.QuarkError) as e:
            srv.submit(0, bad, 4, outs[0])  # 70 not divisible by 4
        assert e.value.status == quark.EINVAL
        st = srv.stats()
        assert st.cancelled == 1 and st.rejected >= 1 and st.completed == 2
    finally:
        srv.stop()


def test_admission_cap_serialises_but_completes():
    # a cap that leaves room for about one request at a time beside the resident pyramids
    pyr_bytes = 2 * (4 * 44 * 72 * 16 + sum(4 * (44 // k) * (72 // k) * 32 * 4 for k in (1, 2, 4)))
    cfg2, W2, ctx2, srv, scenes2 = _setup(n_slots=4, cap=pyr_bytes + 6_000_000)
    try:
        reqs = _requests(scenes2)
        reqs = [r for r in reqs if r[1].width == 72]
        outs = _run(srv, reqs, concurrent=True)
        assert all(np.isfinite(o).all() for o in outs)
        st = srv.stats()
        assert st.hbm_high_water <= pyr_bytes + 6_000_000
        with pytest.raises(quark.QuarkError) as e:  # a 4x larger output can never fit
            big = _requests(scenes2)[1][1]
            srv.submit(0, big, 4, torch.zeros(big.height, big.width, 4, device="cuda"))
        assert e.value.status == quark.ENOMEM
    finally:
        srv.stop()
