"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties one oracle step to a closed form, a library routine run independently on
the CPU (torch conv2d / grid_sample / interpolate / avg_pool2d / scaled_dot_product_attention /
rms_norm / gelu), an invariant the paper states, or a hand-derived case, so that a dropped
term, a sign or index error or a transposed operand in the oracle fails at least one.
"""
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as TF

from oracle import flops
from oracle import quark_oracle as O
from paper_2411_16680_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------------------------
# Depth (Sec. 3.2.3, Eqs. depth anchors / depth_activation)
# --------------------------------------------------------------------------------------------

def test_depth_anchors_closed_form():
    # near 1 m, far 10 m, L = 4, t = 0: d = 1 / (delta * 0.9 + 0.1)
    d = O.depth_activation(np.zeros(4), np.arange(1, 5), 4, 1.0, 10.0)
    np.testing.assert_allclose(d, [1 / 0.2125, 1 / 0.4375, 1 / 0.6625, 1 / 0.8875], rtol=1e-15)
    np.testing.assert_allclose(d, [4.70588, 2.28571, 1.50943, 1.12676], atol=1e-5)


def test_depth_bands_monotone_and_contained():
    L, near, far = 8, 1.0, 100.0
    t = np.linspace(-30, 30, 2001)
    for ell in range(1, L + 1):
        d = O.depth_activation(t, ell, L, near, far)
        disp = 1 / d
        lo = (ell - 1) / L * (1 / near - 1 / far) + 1 / far
        hi = ell / L * (1 / near - 1 / far) + 1 / far
        assert np.all(disp >= lo - 1e-15) and np.all(disp <= hi + 1e-15)
        assert np.all(np.diff(d) <= 0)  # larger t -> nearer
    # extreme layers reach the planes: t -> +inf on l = L gives near, t -> -inf on l = 1 gives far
    assert abs(O.depth_activation(50.0, L, L, near, far) - near) < 1e-12
    assert abs(O.depth_activation(-50.0, 1, L, near, far) - far) < 1e-9


# --------------------------------------------------------------------------------------------
# Geometry (Sec. 3.1, operator P^T)
# --------------------------------------------------------------------------------------------

def _rand_cam(rng, W=64, H=48):
    R, t = synth.look_at(rng.normal(0, 0.3, 3), np.array([0.0, 0.0, 8.0]) + rng.normal(0, 0.5, 3))
    return synth.Camera(W, H, 50.0 + rng.uniform(0, 20), 55.0, 31.0, 25.0, R, t)


def test_identity_reprojection_returns_pixel_centre():
    rng = np.random.default_rng(0)
    cam = _rand_cam(rng)
    ys, xs = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    for d in (0.5, 3.0, 97.0):
        for k in (1, 2, 4):
            K = O.scaled_K(cam, k)
            Xw = O.unproject(ys, xs, np.full(ys.shape, d), K, cam)
            u, v, valid = O.project(Xw, K, cam)
            assert valid.all()
            np.testing.assert_allclose(u, xs + 0.5, atol=1e-9)
            np.testing.assert_allclose(v, ys + 0.5, atol=1e-9)


def test_plane_induced_shift_small_config():
    # Cameras translated on x with R = I: u_m = u_t - f_k (x_m - x_t) / d.  For the small
    # workload (f = 60 px, level 2 -> f_2 = 30 px, novel view at x = 0.05, views at 0 and 0.1)
    # the shifts at the four anchor depths are +-{0.31875, 0.65625, 0.99375, 1.33125} px.
    sc = synth.scene_small()
    cfg = synth.config_small()
    d = O.depth_activation(np.zeros(4), np.arange(1, 5), 4, cfg.near, cfg.far)
    ys, xs = np.array([[7]]), np.array([[11]])
    K_t = O.scaled_K(sc.target, 2)
    for cam, sign in ((sc.cams[0], +1), (sc.cams[1], -1)):
        for li in range(4):
            Xw = O.unproject(ys, xs, np.array([[d[li]]]), K_t, sc.target)
            u, v, _ = O.project(Xw, O.scaled_K(cam, 2), cam)
            shift = u[0, 0] - (11 + 0.5)
            assert abs(shift - sign * 30 * 0.05 / d[li]) < 1e-12
            assert abs(v[0, 0] - 7.5) < 1e-12
    np.testing.assert_allclose(30 * 0.05 / d, [0.31875, 0.65625, 0.99375, 1.33125], rtol=1e-12)


def test_unproject_project_round_trip_and_behind_camera():
    rng = np.random.default_rng(1)
    cam_t, cam_m = _rand_cam(rng), _rand_cam(rng)
    ys, xs = np.meshgrid(np.arange(0, 48, 5), np.arange(0, 64, 7), indexing="ij")
    d = rng.uniform(1, 20, ys.shape)
    Xw = O.unproject(ys, xs, d, cam_t.K, cam_t)
    # world point lies at camera depth d in the target frame
    np.testing.assert_allclose((Xw @ cam_t.R.T + cam_t.t)[..., 2], d, rtol=1e-13)
    u, v, valid = O.project(Xw, cam_m.K, cam_m)
    # back from view m at its own depth lands on the same world point
    zm = (Xw @ cam_m.R.T + cam_m.t)[..., 2]
    Xw2 = O.unproject(v - 0.5, u - 0.5, zm, cam_m.K, cam_m)
    np.testing.assert_allclose(Xw2, Xw, atol=1e-10)
    # a point behind a view is invalid
    behind = cam_m.centre - 2.0 * cam_m.R[2]
    _, _, ok = O.project(behind[None], cam_m.K, cam_m)
    assert not ok[0]


# --------------------------------------------------------------------------------------------
# Bilinear sampling, resizing, convolution, pooling: independent library routines
# --------------------------------------------------------------------------------------------

def _fetch_from(arr):
    h, w = arr.shape[:2]

    def fetch(iy, ix):
        inside = (iy >= 0) & (iy < h) & (ix >= 0) & (ix < w)
        return np.where(inside[..., None], arr[np.clip(iy, 0, h - 1), np.clip(ix, 0, w - 1)], 0.0)
    return fetch


def test_bilinear_matches_grid_sample_zeros():
    rng = np.random.default_rng(2)
    h, w, C = 9, 13, 5
    F = rng.standard_normal((h, w, C))
    u = rng.uniform(-2, w + 2, 500)
    v = rng.uniform(-2, h + 2, 500)
    ours = O.bilinear_zero(_fetch_from(F), u, v, np.ones(500, bool))
    grid = torch.tensor(np.stack([u / w * 2 - 1, v / h * 2 - 1], -1))[None, None]  # normalised, align_corners=False
    ref = TF.grid_sample(torch.tensor(F).permute(2, 0, 1)[None], grid, mode="bilinear", padding_mode="zeros",
                         align_corners=False)[0, :, 0].T.numpy()
    np.testing.assert_allclose(ours, ref, atol=1e-12)


def test_bilinear_texel_centres_and_affine():
    h, w = 6, 7
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    F = np.stack([2.0 * xs - 3.0 * ys + 1.0, np.ones_like(xs, dtype=float)], -1)
    fetch = _fetch_from(F)
    # texel centres return the texel
    out = O.bilinear_zero(fetch, xs + 0.5, ys + 0.5, np.ones(xs.shape, bool))
    np.testing.assert_allclose(out, F, atol=1e-14)
    # interior points reproduce the affine map exactly
    rng = np.random.default_rng(3)
    u = rng.uniform(0.5, w - 0.5, 200)
    v = rng.uniform(0.5, h - 0.5, 200)
    out = O.bilinear_zero(fetch, u, v, np.ones(200, bool))
    np.testing.assert_allclose(out[:, 0], 2 * (u - 0.5) - 3 * (v - 0.5) + 1, atol=1e-12)
    np.testing.assert_allclose(out[:, 1], 1.0, atol=1e-14)
    # zero padding fades linearly over the last half texel
    out = O.bilinear_zero(fetch, np.array([0.25, 0.0, -0.5]), np.array([3.5, 3.5, 3.5]), np.ones(3, bool))
    np.testing.assert_allclose(out[:, 1], [0.75, 0.5, 0.0], atol=1e-14)


def test_resize_x2_matches_interpolate():
    rng = np.random.default_rng(4)
    V = rng.standard_normal((3, 5, 7, 4))
    ours = O.resize_rect(V, (0, 5, 0, 7), 5, 7, 2, (0, 10, 0, 14))
    ref = TF.interpolate(torch.tensor(V).permute(0, 3, 1, 2), scale_factor=2, mode="bilinear",
                         align_corners=False).permute(0, 2, 3, 1).numpy()
    np.testing.assert_allclose(ours, ref, atol=1e-12)
    # constants are preserved, x1 is the identity
    np.testing.assert_allclose(O.resize_rect(np.full((1, 5, 7, 1), 3.0), (0, 5, 0, 7), 5, 7, 2, (0, 10, 0, 14)), 3.0)
    np.testing.assert_allclose(O.resize_rect(V, (0, 5, 0, 7), 5, 7, 1, (0, 5, 0, 7)), V, atol=0)


def test_conv3x3_matches_conv2d_and_delta_kernel():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 9, 11, 6))
    w = rng.standard_normal((3, 3, 6, 4))
    b = rng.standard_normal(4)
    ours = O.conv3x3_rect(x, (0, 9, 0, 11), 9, 11, w, b, (0, 9, 0, 11))
    ref = TF.conv2d(torch.tensor(x).permute(0, 3, 1, 2), torch.tensor(w).permute(3, 2, 0, 1),
                    torch.tensor(b), padding=1).permute(0, 2, 3, 1).numpy()
    np.testing.assert_allclose(ours, ref, atol=1e-12)
    # window evaluation equals the full plane
    part = O.conv3x3_rect(x[:, 2:8, 0:6], (2, 8, 0, 6), 9, 11, w, b, (3, 7, 0, 5))
    np.testing.assert_allclose(part, ours[:, 3:7, 0:5], atol=1e-12)
    # centre-tap-only kernel is a per-pixel matmul
    wd = np.zeros_like(w)
    wd[1, 1] = w[1, 1]
    np.testing.assert_allclose(O.conv3x3_rect(x, (0, 9, 0, 11), 9, 11, wd, b, (0, 9, 0, 11)), x @ w[1, 1] + b,
                               atol=1e-12)


def test_conv1x1_matches_conv2d_and_centre_tap_3x3():
    """The conv_kernel = 1 form of the fusion block's convolution (the position-wise MLP of a
    Transformer block, Sec. 3.3): torch's 1x1 conv2d, and the 3x3 path with the kernel at the
    centre tap and zeros elsewhere, on a window."""
    rng = np.random.default_rng(15)
    x = rng.standard_normal((2, 9, 11, 6))
    w = rng.standard_normal((1, 1, 6, 4))
    b = rng.standard_normal(4)
    ours = O.conv_rect(x, (0, 9, 0, 11), 9, 11, w, b, (0, 9, 0, 11))
    ref = TF.conv2d(torch.tensor(x).permute(0, 3, 1, 2), torch.tensor(w).permute(3, 2, 0, 1),
                    torch.tensor(b)).permute(0, 2, 3, 1).numpy()
    np.testing.assert_allclose(ours, ref, atol=1e-12)
    w3 = np.zeros((3, 3, 6, 4))
    w3[1, 1] = w[0, 0]
    part = O.conv_rect(x[:, 2:8, 0:6], (2, 8, 0, 6), 9, 11, w, b, (3, 7, 0, 5))
    np.testing.assert_allclose(part, O.conv3x3_rect(x, (0, 9, 0, 11), 9, 11, w3, b, (3, 7, 0, 5)), atol=1e-12)


def test_pipeline_with_1x1_blocks_equals_centre_tap_3x3_blocks():
    """A whole two-step pipeline with conv_kernel = 1 equals the default pipeline whose 3x3 conv
    weights hold the same matrices at the centre tap and zeros elsewhere (full frame and a
    window)."""
    cfg1 = synth.QuarkConfig(C=8, heads=2, scales=[(2, 4), (1, 2)], near=1.0, far=40.0, out_h=24, out_w=32,
                             conv_kernel=1)
    cfg3 = cfg1.replace(conv_kernel=3)
    sc = synth.scene_raycast(seed=4, V=3, W=32, H=24, f=28.0, arc=0.3)
    W1 = synth.make_weights(cfg1, seed=8, sharp=True)
    assert W1["conv1_w_0"].shape == (1, 1, 8, 8)
    W3 = dict(W1)
    for j in range(cfg1.n_scales):
        for n in (f"conv1_w_{j}", f"conv2_w_{j}"):
            w3 = np.zeros((3, 3, 8, 8), np.float32)
            w3[1, 1] = W1[n][0, 0]
            W3[n] = w3
    a, sa = O.forward(cfg1, W1, sc)
    b, sb = O.forward(cfg3, W3, sc)
    np.testing.assert_allclose(a, b, atol=1e-12)
    for x, y in zip(sa, sb):
        np.testing.assert_allclose(x.V_out, y.V_out, atol=1e-12)
    r = (5, 11, 7, 15)
    aw, _ = O.forward(cfg1, W1, sc, r)
    np.testing.assert_allclose(aw, a[r[0]:r[1], r[2]:r[3]], atol=1e-12)


def test_pyramid_matches_conv_then_avgpool_chain():
    sc = synth.scene_noise_pair(V=1, W=32, H=24)
    rng = np.random.default_rng(6)
    w = rng.standard_normal((3, 3, 3, 5))
    b = rng.standard_normal(5)
    img = torch.tensor(sc.images[0].astype(np.float64)).permute(2, 0, 1)[None]
    F = TF.conv2d(img, torch.tensor(w).permute(3, 2, 0, 1), torch.tensor(b), padding=1)
    for k in (1, 2, 4, 8):
        ours = O.encode_level(sc.images[0], w, b, k)
        np.testing.assert_allclose(ours, F[0].permute(1, 2, 0).numpy(), atol=1e-12)
        F = TF.avg_pool2d(F, 2)


def test_rmsnorm_gelu_match_torch():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((10, 16)) * 3
    g = rng.standard_normal(16)
    ref = TF.rms_norm(torch.tensor(x), (16,), torch.tensor(g), eps=1e-6).numpy()
    np.testing.assert_allclose(O.rmsnorm(x, g), ref, atol=1e-13)
    np.testing.assert_allclose(O.gelu(x), TF.gelu(torch.tensor(x)).numpy(), atol=1e-14)


# --------------------------------------------------------------------------------------------
# Attention (Sec. 3.3; appendix A)
# --------------------------------------------------------------------------------------------

def test_attention_identical_views_and_uniform_query():
    rng = np.random.default_rng(8)
    C, h, V = 8, 2, 5
    x = rng.standard_normal((3, C))
    Wq = rng.standard_normal((C, h * C))
    Wo = rng.standard_normal((h * C, C))
    D = rng.standard_normal((3, V, C))
    # V identical views: every head returns that view's value
    same = np.repeat(D[:, :1], V, axis=1)
    out, p = O.one_to_many_attention(x, same, Wq, Wo, h)
    np.testing.assert_allclose(out, np.concatenate([same[:, 0]] * h, -1) @ Wo, atol=1e-12)
    # softmax weights sum to 1
    _, p = O.one_to_many_attention(x, D, Wq, Wo, h)
    np.testing.assert_allclose(p.sum(-1), 1.0, atol=1e-14)
    # zero query (the "no cross attention" ablation, Sec. 5.4): plain mean across views
    out, _ = O.one_to_many_attention(x, D, np.zeros_like(Wq), Wo, h)
    np.testing.assert_allclose(out, np.concatenate([D.mean(1)] * h, -1) @ Wo, atol=1e-12)
    # h = 1, V = 1: the output is the single value
    out, _ = O.one_to_many_attention(x, D[:, :1], Wq[:, :C], np.eye(C), 1)
    np.testing.assert_allclose(out, D[:, 0], atol=1e-14)


def test_attention_logits_against_brute_force():
    rng = np.random.default_rng(9)
    C, h, V = 4, 2, 3
    x = rng.standard_normal(C)
    Wq = rng.standard_normal((C, h * C))
    Wo = rng.standard_normal((h * C, C))
    D = rng.standard_normal((V, C))
    out = np.zeros(C)
    for i in range(h):
        q = [sum(x[a] * Wq[a, i * C + c] for a in range(C)) for c in range(C)]
        s = [sum(q[c] * D[m, c] for c in range(C)) / math.sqrt(C) for m in range(V)]
        e = [math.exp(v) for v in s]
        p = [v / sum(e) for v in e]
        o = [sum(p[m] * D[m, c] for m in range(V)) for c in range(C)]
        for c in range(C):
            for a in range(C):
                out[a] += o[c] * Wo[i * C + c, a]
    ours, _ = O.one_to_many_attention(x, D, Wq, Wo, h)
    np.testing.assert_allclose(ours, out, atol=1e-12)


@pytest.mark.parametrize("heads", [1, 2, 4])
def test_fold_identity_standard_vs_one_to_many(heads):
    """Sec. 3.3 "Optimized Attention" / appendix A: folding W_i^k into the query and W_i^val into
    W^O turns standard cross attention into one-to-many attention."""
    rng = np.random.default_rng(10 + heads)
    C, V = 8, 6
    dh = C // heads
    x = rng.standard_normal((4, C))
    D = rng.standard_normal((4, V, C))
    Wq, Wk, Wv, Wo = (rng.standard_normal((C, C)) for _ in range(4))
    std = O.standard_attention(x, D, Wq, Wk, Wv, Wo, heads)
    # independent library path for the standard form
    q = torch.tensor(x @ Wq).reshape(4, 1, heads, dh).transpose(1, 2)
    k = torch.tensor(D @ Wk).reshape(4, V, heads, dh).transpose(1, 2)
    v = torch.tensor(D @ Wv).reshape(4, V, heads, dh).transpose(1, 2)
    sdpa = TF.scaled_dot_product_attention(q, k, v).transpose(1, 2).reshape(4, C).numpy() @ Wo
    np.testing.assert_allclose(std, sdpa, atol=1e-12)
    Wq1 = np.concatenate([Wq[:, i * dh:(i + 1) * dh] @ Wk[:, i * dh:(i + 1) * dh].T * math.sqrt(C) / math.sqrt(dh)
                          for i in range(heads)], axis=1)
    Wo1 = np.concatenate([Wv[:, i * dh:(i + 1) * dh] @ Wo[i * dh:(i + 1) * dh] for i in range(heads)], axis=0)
    o2m, _ = O.one_to_many_attention(x, D, Wq1, Wo1, heads)
    np.testing.assert_allclose(o2m, std, atol=1e-11)


def test_attention_flop_tables():
    """Appendix A tables, reproduced exactly by the closed forms."""
    rows = [list(map(int, ln.split())) for ln in open(os.path.join(GOLDEN, "attention_flops.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 9
    for N, h, dk, std, o2m in rows:
        assert flops.standard_macs(N, dk, h) == std
        assert flops.one_to_many_macs(N, dk, h) == o2m


def test_layer_collapse_zero_residual_is_pairwise_mean():
    rng = np.random.default_rng(11)
    V = rng.standard_normal((8, 3, 4, 5))
    z = lambda *s: np.zeros(s)
    out = O.layer_collapse(V, z(10, 5), z(5), z(5, 5), z(5))
    np.testing.assert_allclose(out, 0.5 * (V[0::2] + V[1::2]), atol=0)
    # pairing order: output layer j depends only on input layers 2j, 2j+1
    w1 = rng.standard_normal((10, 5)); b1 = rng.standard_normal(5); w2 = rng.standard_normal((5, 5))
    base = O.layer_collapse(V, w1, b1, w2, z(5))
    V2 = V.copy()
    V2[5] += 1.0
    d = np.abs(O.layer_collapse(V2, w1, b1, w2, z(5)) - base).max(axis=(1, 2, 3))
    assert d[2] > 0 and d[[0, 1, 3]].max() == 0


# --------------------------------------------------------------------------------------------
# Render and over-compositing (Sec. 3.1, Eq. 1)
# --------------------------------------------------------------------------------------------

def _fake_last(L, h, w, V, t, s, beta):
    r = (0, h, 0, w)
    z = np.zeros((L, h, w))
    return O.StepResult(r, None, None, None, None, None, r, np.zeros((L, h, w, 1)), t + z, s + z, None, None,
                        None, beta + np.zeros((L, h, w, V)))


def test_render_single_opaque_layer_and_transparent():
    sc = synth.scene_small()
    cfg = synth.config_small()
    L, h, w = 4, 24, 32
    # only the nearest layer (l = L) opaque: output = its blended colour, alpha 1
    s = np.full((L, 1, 1), -60.0)
    s[L - 1] = 60.0
    rgba, col, alpha, d, beta = O.render_rect(cfg, sc, _fake_last(L, h, w, 2, 0.0, s, 0.0), (0, 48, 0, 64), True)
    np.testing.assert_allclose(rgba[..., :3], col[L - 1], atol=1e-12)
    np.testing.assert_allclose(rgba[..., 3], 1.0, atol=1e-12)
    # a fully transparent LDM renders black with alpha 0
    rgba = O.render_rect(cfg, sc, _fake_last(L, h, w, 2, 0.0, -80.0, 0.0), (0, 48, 0, 64))
    np.testing.assert_allclose(rgba, 0.0, atol=1e-30)


def test_render_two_layer_closed_form_and_order():
    sc = synth.scene_small()
    cfg = synth.config_small().replace(scales=[(2, 2)])
    rng = np.random.default_rng(12)
    s = rng.standard_normal((2, 24, 32))
    t = rng.standard_normal((2, 24, 32))
    beta = rng.standard_normal((2, 24, 32, 2)) * 3
    rgba, col, alpha, d, bw = O.render_rect(cfg, sc, _fake_last(2, 24, 32, 2, t, s, beta), (0, 48, 0, 64), True)
    # c = c_L a_L + (1 - a_L) a_{L-1} c_{L-1}
    ref = col[1] * alpha[1][..., None] + ((1 - alpha[1]) * alpha[0])[..., None] * col[0]
    np.testing.assert_allclose(rgba[..., :3], ref, atol=1e-13)
    np.testing.assert_allclose(rgba, O.over_back_to_front(col, alpha), atol=1e-13)
    # blend weights are convex: per-layer colour inside the hull of the sampled colours (here [0, 1])
    np.testing.assert_allclose(bw.sum(-1), 1.0, atol=1e-14)
    assert col.min() >= 0 and col.max() <= 1


def test_depth_map_closed_forms():
    """Sec. 3.1 optional depth output: over-compositing the decoded depth.  One opaque nearest
    layer gives its depth; a transparent LDM gives 0; two layers give a_L d_L + (1 - a_L) a_{L-1}
    d_{L-1}, the same as the back-to-front over operator applied to depth as a colour; t = 0
    puts every layer at its anchor depth (Eq. depth_activation)."""
    cfg = synth.config_small()
    L, h, w = 4, 24, 32
    rect = (0, 48, 0, 64)
    s = np.full((L, 1, 1), -60.0)
    s[L - 1] = 60.0
    D = O.render_depth_rect(cfg, _fake_last(L, h, w, 2, 0.0, s, 0.0), rect)
    anchors = O.depth_activation(np.zeros(L), np.arange(1, L + 1), L, cfg.near, cfg.far)
    np.testing.assert_allclose(D, anchors[L - 1], rtol=1e-12)
    np.testing.assert_allclose(O.render_depth_rect(cfg, _fake_last(L, h, w, 2, 0.0, -80.0, 0.0), rect), 0.0,
                               atol=1e-30)
    cfg2 = cfg.replace(scales=[(2, 2)])
    rng = np.random.default_rng(3)
    t = rng.standard_normal((2, 24, 32))
    s2 = rng.standard_normal((2, 24, 32))
    last = _fake_last(2, 24, 32, 2, t, s2, 0.0)
    D = O.render_depth_rect(cfg2, last, rect)
    _, _, alpha, d, _ = O.render_rect(cfg2, synth.scene_small(), last, rect, True)
    np.testing.assert_allclose(D, alpha[1] * d[1] + (1 - alpha[1]) * alpha[0] * d[0], rtol=1e-12)
    np.testing.assert_allclose(D, O.over_back_to_front(d[..., None], alpha)[..., 0], rtol=1e-12)
    # the depth map lies between 0 and the farthest layer depth
    assert D.min() >= 0 and D.max() <= d.max()


def test_render_identical_views_identity_geometry():
    # every view is the target camera with the same image: each layer's colour is the image
    sc = synth.scene_small()
    img = sc.images[0]
    cam = sc.target
    sc2 = synth.Scene(np.stack([img, img, img]), [cam, cam, cam], cam)
    cfg = synth.config_small()
    rng = np.random.default_rng(13)
    s = rng.standard_normal((4, 24, 32))
    rgba = O.render_rect(cfg, sc2, _fake_last(4, 24, 32, 3, rng.standard_normal((4, 24, 32)), s,
                                              rng.standard_normal((4, 24, 32, 3))), (0, 48, 0, 64))
    np.testing.assert_allclose(rgba[..., :3], img * rgba[..., 3:], atol=1e-12)


def test_render_upsample_matches_interpolate():
    # the raw logits are resized by s with pixel-centre alignment before activation (Sec. 3.2.3)
    rng = np.random.default_rng(14)
    t = rng.standard_normal((4, 24, 32))
    up = O.resize_rect(t[..., None], (0, 24, 0, 32), 24, 32, 2, (0, 48, 0, 64))[..., 0]
    ref = TF.interpolate(torch.tensor(t)[None], scale_factor=2, mode="bilinear", align_corners=False)[0].numpy()
    np.testing.assert_allclose(up, ref, atol=1e-12)


# --------------------------------------------------------------------------------------------
# Whole pipeline
# --------------------------------------------------------------------------------------------

def _load_golden(name):
    vals = {}
    for ln in open(os.path.join(GOLDEN, name)):
        if ln.strip() and not ln.startswith("#"):
            k, v = ln.split("=")
            vals[k.strip()] = np.array([float(a) for a in v.split()])
    return vals


def hand_case():
    cam_t = synth.Camera(2, 2, 2.0, 2.0, 1.0, 1.0, np.eye(3), np.zeros(3))
    cam_2 = synth.Camera(2, 2, 2.0, 2.0, 1.0, 1.0, np.eye(3), np.array([-0.5, 0.0, 0.0]))
    img1 = np.zeros((2, 2, 3)); img2 = np.zeros((2, 2, 3))
    img1[..., 0] = [[0.1, 0.2], [0.3, 0.4]]; img1[..., 1] = 0.5; img1[..., 2] = 0.9
    img2[..., 0] = 0.8; img2[..., 1] = [[0.0, 0.4], [0.4, 0.0]]; img2[..., 2] = [[0.2, 0.6], [0.2, 0.6]]
    scene = synth.Scene(np.stack([img1, img2]).astype(np.float32), [cam_t, cam_2], cam_t)
    cfg = synth.QuarkConfig(C=2, heads=1, scales=[(2, 2)], near=0.8, far=4.0, out_h=2, out_w=2)
    W = {k: np.zeros(s, np.float32) for k, s in synth.weight_shapes(cfg).items()}
    W["enc_w"][1, 1, 0, 0] = 1.0
    W["enc_w"][1, 1, 1, 1] = 1.0
    W["v0"][:] = 2.0
    W["attn_g_0"][:] = 1.0
    W["conv_g_0"][:] = 1.0
    W["Wq_0"][:] = [[1, 0], [0, -1]]
    W["Wo_0"][:] = np.eye(2)
    W["W_beta"][:] = np.eye(2)
    W["conv1_w_0"][:] = 7.0
    W["conv1_w_0"][1, 1] = np.eye(2)
    W["conv2_w_0"][:] = 7.0
    W["conv2_w_0"][1, 1] = 0.5 * np.eye(2)
    W["b_sigma"][:] = math.log(3.0)
    return cfg, W, scene


def test_hand_case_end_to_end():
    g = _load_golden("hand_case.txt")
    cfg, W, scene = hand_case()
    rgba, steps = O.forward(cfg, W, scene)
    st = steps[0]
    tol = 1e-6  # float32 storage of the hand inputs (0.1, 0.3, ...) vs exact decimals
    np.testing.assert_allclose(st.depth_used[:, 0, 0], [g["depth_l1"][0], g["depth_l2"][0]], atol=1e-12)
    for l in (1, 2):
        for m in (1, 2):
            np.testing.assert_allclose(st.Delta[l - 1, 0, 0, m - 1], g[f"delta_l{l}_v{m}"], atol=tol)
        np.testing.assert_allclose(st.V_attn[l - 1, 0, 0], g[f"V_attn_l{l}"], atol=tol)
        np.testing.assert_allclose(st.beta_logits[l - 1, 0, 0], g[f"beta_logit_l{l}"], atol=tol)
        np.testing.assert_allclose(st.V_out[l - 1, 0, 0], g[f"V_out_l{l}"], atol=tol)
    np.testing.assert_allclose(st.alpha, 0.75, atol=1e-12)
    for Y in (0, 1):
        for X in (0, 1):
            np.testing.assert_allclose(rgba[Y, X], g[f"rgba_y{Y}_x{X}"], atol=tol)


def test_windowed_forward_equals_full_plane():
    cfg = synth.QuarkConfig(C=8, heads=2, scales=[(4, 8), (2, 4), (1, 4)], near=1, far=50, out_h=48, out_w=64)
    W = synth.make_weights(cfg, sharp=True)
    sc = synth.scene_raycast(V=3, W=64, H=48, f=50, arc=0.3)
    full, _ = O.forward(cfg, W, sc)
    for rect in [(0, 5, 0, 7), (20, 33, 41, 64), (47, 48, 0, 64), (10, 11, 30, 31)]:
        part, _ = O.forward(cfg, W, sc, rect)
        np.testing.assert_allclose(part, full[rect[0]:rect[1], rect[2]:rect[3]], atol=1e-13)


def test_standard_mode_equals_folded_one_to_many_pipeline():
    cfg = synth.QuarkConfig(C=8, heads=2, scales=[(2, 4), (1, 2)], near=1, far=20, out_h=24, out_w=32)
    W = synth.make_weights(cfg, sharp=True)
    sc = synth.scene_raycast(V=3, W=32, H=24, f=30, arc=0.3)
    std, _ = O.forward(cfg, W, sc, mode=1)
    C, h = cfg.C, cfg.heads
    dh = C // h
    W2 = dict(W)
    for j in range(cfg.n_scales):
        Wq, Wk, Wv, Wo = (W[f"{n}_std_{j}"].astype(np.float64) for n in ("Wq", "Wk", "Wv", "Wo"))
        W2[f"Wq_{j}"] = np.concatenate([Wq[:, i * dh:(i + 1) * dh] @ Wk[:, i * dh:(i + 1) * dh].T * math.sqrt(C / dh)
                                        for i in range(h)], 1)
        W2[f"Wo_{j}"] = np.concatenate([Wv[:, i * dh:(i + 1) * dh] @ Wo[i * dh:(i + 1) * dh] for i in range(h)], 0)
    o2m, _ = O.forward(cfg, W2, sc, mode=0)
    np.testing.assert_allclose(o2m, std, atol=1e-11)


@pytest.mark.parametrize("case", ["small", "three_scales"])
def test_pipeline_matches_independent_library_formulation(case):
    """Whole forward pass against a second float64 formulation built from torch CPU routines
    (tests/torch_pipeline.py): pins the assembly of the steps across scales."""
    from tests import torch_pipeline
    if case == "small":
        cfg, sc = synth.config_small(), synth.scene_small()
    else:
        cfg = synth.QuarkConfig(C=8, heads=2, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1, far=50,
                                out_h=48, out_w=64)
        sc = synth.scene_raycast(V=3, W=64, H=48, f=50, arc=0.3)
    W = synth.make_weights(cfg, sharp=True)
    ours, _ = O.forward(cfg, W, sc)
    ref = torch_pipeline.forward(cfg, W, sc)
    np.testing.assert_allclose(ours, ref, atol=1e-10)


# --------------------------------------------------------------------------------------------
# Ray directional encoding (Sec. 3.2.1)
# --------------------------------------------------------------------------------------------

def _ray_AB(cam_m, cam_t, k0):
    """Independent setup: view m's centre and its pixel-centre rays in target coordinates."""
    h0, w0 = cam_m.height // k0, cam_m.width // k0
    K0 = np.array(cam_m.K, np.float64).copy()
    K0[:2] /= k0
    centre = np.linalg.solve(cam_m.R, -cam_m.t)  # R c + t = 0
    out_A = cam_t.R @ centre + cam_t.t
    B = np.zeros((h0, w0, 3))
    for y in range(h0):
        for x in range(w0):
            d_cam = np.linalg.solve(K0, np.array([x + 0.5, y + 0.5, 1.0]))
            B[y, x] = cam_t.R @ np.linalg.solve(cam_m.R, d_cam)
    return out_A, B


def test_ray_difference_closed_form():
    """far - near in the target's normalised image plane equals (1/eta - 1/f) (A_z B_xy / B_z -
    A_xy) for the ray A + lam B in target coordinates (eliminate lam at z = eta and z = f)."""
    sc = synth.scene_raycast(V=3, W=64, H=48, f=50, arc=0.6)
    near, far = 1.5, 40.0
    for m in range(3):
        A, B = _ray_AB(sc.cams[m], sc.target, 4)
        ref = (1 / near - 1 / far) * (A[2] * B[..., :2] / B[..., 2:3] - A[:2])
        np.testing.assert_allclose(O.ray_difference(sc.cams[m], sc.target, 4, near, far), ref, atol=1e-12)


def test_ray_difference_zero_through_target_centre():
    """A view whose centre is the target camera's centre (any rotation and focal length): every
    ray is a target ray, so the encoding's input vanishes (the paper's first property)."""
    sc = synth.scene_raycast(V=2, W=64, H=48, f=50, arc=0.3)
    tgt = sc.target
    centre = np.linalg.solve(tgt.R, -tgt.t)
    view = synth.make_camera(64, 48, 37.0, tuple(centre), target=tuple(centre + np.array([0.3, -0.2, 1.0])))
    np.testing.assert_allclose(O.ray_difference(view, tgt, 2, 1.0, 30.0), 0.0, atol=1e-12)
    assert np.abs(O.ray_difference(sc.cams[0], tgt, 2, 1.0, 30.0)).max() > 1e-3


def test_ray_encoding_octaves_and_saturation():
    rng = np.random.default_rng(4)
    diff = rng.standard_normal((5, 7, 2))
    pe = O.ray_encoding(diff)
    assert pe.shape == (5, 7, 32)
    s, c = pe[..., 0::2], pe[..., 1::2]
    np.testing.assert_allclose(s ** 2 + c ** 2, 1.0, atol=1e-14)
    # octave i + 1 is the double angle of octave i: sin 2a = 2 sin a cos a, cos 2a = cos^2 a - sin^2 a
    for i in range(7):
        for j in range(2):
            a, b = 4 * i + 2 * j, 4 * (i + 1) + 2 * j
            np.testing.assert_allclose(pe[..., b], 2 * pe[..., a] * pe[..., a + 1], atol=1e-13)
            np.testing.assert_allclose(pe[..., b + 1], pe[..., a + 1] ** 2 - pe[..., a] ** 2, atol=1e-13)
    # octave 0 is sin / cos of pi tanh(diff)
    np.testing.assert_allclose(pe[..., 0], np.sin(np.pi * np.tanh(diff[..., 0])), atol=1e-15)
    # zero difference: sin 0 = 0, cos 0 = 1; a huge one saturates tanh at +-1: sin(2^i pi) = 0
    np.testing.assert_allclose(O.ray_encoding(np.zeros(2)), np.tile([0.0, 1.0], 16), atol=0)
    np.testing.assert_allclose(O.ray_encoding(np.array([1e9, -1e9]))[0::2], 0.0, atol=1e-12)


def test_ray_gamma_is_upsampled_projection():
    """gamma_k = bilinear upsample (pixel centres aligned, edge clamp) of the coarse encoding,
    projected; checked against a separable np.interp upsample."""
    sc = synth.scene_raycast(V=2, W=64, H=48, f=50, arc=0.3)
    rng = np.random.default_rng(8)
    Wr = rng.standard_normal((32, 5))
    k0, k = 8, 2
    r = k0 // k
    coarse = O.ray_encoding(O.ray_difference(sc.cams[1], sc.target, k0, 1.0, 30.0)) @ Wr  # [6, 8, 5]
    h0, w0 = coarse.shape[:2]
    H, Wd = 48 // k, 64 // k
    sy = np.clip((np.arange(H) + 0.5) / r - 0.5, 0, h0 - 1)
    sx = np.clip((np.arange(Wd) + 0.5) / r - 0.5, 0, w0 - 1)
    rows = np.stack([np.stack([np.interp(sy, np.arange(h0), coarse[:, x, c]) for c in range(5)], -1)
                     for x in range(w0)], 1)                      # [H, w0, 5]
    ref = np.stack([np.stack([np.interp(sx, np.arange(w0), rows[y, :, c]) for c in range(5)], -1)
                    for y in range(H)], 0)                        # [H, Wd, 5]
    got = O.ray_gamma(sc.cams[1], sc.target, k0, k, 1.0, 30.0, Wr, (0, H, 0, Wd))
    np.testing.assert_allclose(got, ref, atol=1e-12)
    # at the coarse level itself the upsample is the identity
    np.testing.assert_allclose(O.ray_gamma(sc.cams[1], sc.target, k0, k0, 1.0, 30.0, Wr, (0, h0, 0, w0)), coarse,
                               atol=1e-14)


def test_ray_encoding_off_or_zero_weights_leaves_the_pipeline():
    """With W_ray = 0 the encoding adds nothing: the pipeline equals the one without it; with the
    seeded weights it changes the output."""
    cfg = synth.QuarkConfig(C=8, heads=2, scales=[(4, 4), (2, 2)], near=1, far=20, out_h=48, out_w=64,
                            ray_encoding=1)
    W = synth.make_weights(cfg, sharp=True)
    sc = synth.scene_raycast(V=3, W=64, H=48, f=50, arc=0.3)
    base, _ = O.forward(cfg.replace(ray_encoding=0), W, sc)
    W0 = dict(W)
    for k in cfg.levels():
        W0[f"W_ray_{k}"] = np.zeros_like(W[f"W_ray_{k}"])
    np.testing.assert_allclose(O.forward(cfg, W0, sc)[0], base, atol=1e-14)
    assert np.abs(O.forward(cfg, W, sc)[0] - base).max() > 1e-3


# --------------------------------------------------------------------------------------------
# Model schedules: per-scale heads, blocks without attention, one Delta per step, grid factors
# --------------------------------------------------------------------------------------------

def _schedule_cfg(**kw):
    # views 48 x 80 (levels 1, 2, 4, 8); output 45 x 120; LDM factors 15, 7.5, 3.75
    base = dict(C=8, heads=2, scales=[(8, 4), (8, 4), (8, 4), (4, 4), (4, 4), (2, 2), (2, 2)], near=1.0, far=30.0,
                out_h=45, out_w=120, ldm_f=[15, 15, 15, 7.5, 7.5, 3.75, 3.75],
                scale_heads=[4, 0, 4, 4, 0, 2, 1], reuse_depth=[0, 0, 1, 0, 0, 0, 1])
    base.update(kw)
    return synth.QuarkConfig(**base)


def _schedule_scene():
    sc = synth.scene_raycast(V=3, W=80, H=48, f=60, arc=0.3)
    tgt = sc.target
    target = synth.Camera(120, 45, tgt.fx * 1.5, tgt.fx * 1.5, 60.0, 22.5, tgt.R, tgt.t)
    return synth.Scene(sc.images, sc.cams, target)


def test_schedule_grids_and_weights():
    cfg = _schedule_cfg()
    assert [cfg.ldm_shape(j) for j in range(cfg.n_scales)] == [(4, 3, 8)] * 3 + [(4, 6, 16)] * 2 + [(2, 12, 32)] * 2
    assert cfg.upsample_s == 3.75
    W = synth.make_weights(cfg)
    assert "Wq_1" not in W and "Wq_4" not in W and W["Wq_0"].shape == (8, 32) and W["Wq_6"].shape == (8, 8)


def test_schedule_one_delta_per_step_and_blocks_without_attention():
    """A block without attention leaves V_attn = V_in and carries the depths; a reusing block
    samples exactly the Delta of the step's first block (same depths, same features)."""
    cfg = _schedule_cfg()
    W = synth.make_weights(cfg, sharp=True)
    sc = _schedule_scene()
    _, steps = O.forward(cfg, W, sc)
    assert steps[1].Delta is None
    np.testing.assert_array_equal(steps[1].V_attn, steps[1].V_in)
    r0, r1 = steps[0].rect_attn, steps[1].rect_attn
    h1, w1 = steps[1].depth_used.shape[1:]
    np.testing.assert_array_equal(steps[1].depth_used,
                                  steps[0].depth_used[:, r1[0] - r0[0]:r1[0] - r0[0] + h1, r1[2] - r0[2]:r1[2] - r0[2] + w1])
    # scale 2 reuses: its Delta equals the one a fresh sampling at scale 0's depths gives
    cfg_fresh = _schedule_cfg(reuse_depth=[0] * 7)
    _, fresh = O.forward(cfg_fresh, W, sc)
    assert not np.allclose(steps[2].Delta, fresh[2].Delta)  # the refined volume moved the depths
    d0 = steps[0].depth_used
    r2 = steps[2].rect_attn
    oy, ox = r2[0] - r0[0], r2[2] - r0[2]
    h2, w2 = steps[2].depth_used.shape[1:]
    np.testing.assert_array_equal(steps[2].depth_used, d0[:, oy:oy + h2, ox:ox + w2])


def test_schedule_with_default_options_is_the_plain_pipeline():
    """Explicit per-scale options equal to the defaults reproduce the default pipeline bit for bit."""
    cfg = synth.QuarkConfig(C=8, heads=2, scales=[(4, 8), (2, 4), (2, 2), (1, 2)], near=1, far=50, out_h=48,
                            out_w=64)
    W = synth.make_weights(cfg, sharp=True)
    sc = synth.scene_raycast(V=3, W=64, H=48, f=50, arc=0.3)
    a, _ = O.forward(cfg, W, sc)
    cfg2 = cfg.replace(scale_heads=[2] * 4, ldm_f=[4, 2, 2, 1], reuse_depth=[0] * 4)
    b, _ = O.forward(cfg2, W, sc)
    np.testing.assert_array_equal(a, b)


def test_schedule_fractional_grid_render_is_windowed_exactly():
    """Windows of the output through a 3.75x final upsample equal the full frame."""
    cfg = _schedule_cfg()
    W = synth.make_weights(cfg, sharp=True)
    sc = _schedule_scene()
    full, _ = O.forward(cfg, W, sc)
    for rect in [(0, 7, 0, 11), (20, 33, 50, 77), (44, 45, 0, 120)]:
        part, _ = O.forward(cfg, W, sc, rect)
        np.testing.assert_allclose(part, full[rect[0]:rect[1], rect[2]:rect[3]], atol=1e-13)


# --------------------------------------------------------------------------------------------
# Render and refine: forward projection (splat), rendering in the input views, Update Block
# --------------------------------------------------------------------------------------------

def _refine_scene():
    return synth.scene_raycast(seed=7, V=3, W=72, H=44, f=55.0, arc=0.3)


def test_splat_is_the_transpose_of_bilinear_sampling():
    """Sec. 3.1 names P^T the adjoint of P: for any LDM values x and view map y,
    <splat(x), y> = <x, sample(y)> with the same coordinates (bilinear_zero is the sampler)."""
    sc = _refine_scene()
    rng = np.random.default_rng(0)
    L, f, k = 3, 4.0, 2
    H, Wd = 44 // 4, 72 // 4
    d = 1.0 / rng.uniform(1 / 40, 1 / 2, (L, H, Wd))
    x = rng.standard_normal((L, H, Wd, 2))
    cam = sc.cams[1]
    h, w = cam.height // k, cam.width // k
    y = rng.standard_normal((h, w, 2))
    acc, wsum = O.splat_layers(sc.target, f, cam, k, h, w, d, x)
    lhs = float(np.sum(acc.sum(axis=0) * y))
    ys = np.arange(H)[None, :, None]
    xs = np.arange(Wd)[None, None, :]
    u, v, valid = O.project(O.unproject(ys, xs, d, O.scaled_K(sc.target, f), sc.target), O.scaled_K(cam, k), cam)
    fetch = O.ArrayFetch(y)
    rhs = float(np.sum(x * O.bilinear_zero(fetch, u, v, valid)))
    assert abs(lhs - rhs) <= 1e-10 * (1 + abs(lhs))
    # the weight sums are the splat of ones: the same identity with y = 1 inside the map
    acc1, _ = O.splat_layers(sc.target, f, cam, k, h, w, d, np.ones((L, H, Wd, 1)))
    np.testing.assert_allclose(acc1[..., 0], wsum, atol=1e-12)


def test_splat_with_identical_cameras_lands_on_pixel_centres():
    """Target camera = view camera and equal grids: every sample lands on its own pixel centre at
    any depth (weight 1), so each layer's splat is the layer itself."""
    sc = _refine_scene()
    cam = sc.cams[0]
    rng = np.random.default_rng(1)
    L, H, Wd = 2, cam.height // 2, cam.width // 2
    d = rng.uniform(2, 30, (L, H, Wd))
    vals = rng.uniform(0, 1, (L, H, Wd, 4))
    acc, wsum = O.splat_layers(cam, 2.0, cam, 2, H, Wd, d, vals)
    np.testing.assert_allclose(wsum, 1.0, atol=1e-9)
    np.testing.assert_allclose(acc, vals, atol=1e-9)


def test_rendered_views_are_the_over_composite_of_the_decoded_layers():
    """With identical cameras the rendered view is the over operator applied to the decoded
    layers at each pixel; checked against the back-to-front recursion (Sec. 3.1)."""
    sc = _refine_scene()
    cam = sc.cams[0]
    single = synth.Scene(sc.images[:1], [cam], cam)
    cfg = synth.QuarkConfig(C=8, heads=1, scales=[(2, 3)], near=1.0, far=40.0, out_h=cam.height, out_w=cam.width)
    W = synth.make_weights(cfg, seed=2, sharp=True)
    rng = np.random.default_rng(2)
    Vc = rng.standard_normal((3, cam.height // 2, cam.width // 2, 8))
    It = O.render_to_views(cfg, W, single, Vc, 2.0, 2)[0]
    _, sig, a = O.decode_intermediate(Vc, W, cfg.near, cfg.far)
    ref = O.over_back_to_front(a, sig)
    np.testing.assert_allclose(It, ref, atol=1e-9)


def test_zero_update_block_is_the_plain_pipeline():
    """With every Update Block weight zero the update features are the image features: the
    render-and-refine pipeline equals the plain one bit for bit."""
    cfg = synth.QuarkConfig(C=8, heads=2, scales=[(4, 4), (2, 2), (2, 2)], near=1.0, far=60.0, out_h=44, out_w=72,
                            render_refine=1)
    W = synth.make_weights(cfg, seed=3, sharp=True)
    for k_ in list(W):
        if k_.startswith("upd"):
            W[k_] = np.zeros_like(W[k_])
    sc = _refine_scene()
    a, _ = O.forward(cfg, W, sc)
    b, _ = O.forward(cfg.replace(render_refine=0), W, sc)
    np.testing.assert_array_equal(a, b)
    W2 = synth.make_weights(cfg, seed=3, sharp=True)
    c, _ = O.forward(cfg, W2, sc)
    assert np.abs(c - b).max() > 1e-3  # the rendered views do change the result


# --------------------------------------------------------------------------------------------
# Aspect-adaptive LDM dimensions: the same area per layer for any output aspect
# --------------------------------------------------------------------------------------------

def test_aspect_adaptive_grids_keep_the_area_per_layer():
    """Sec. 4: the LDM keeps the model's number of pixels per layer whatever the output, and the
    final upsample adapts.  Quark targets 1920x1080 (grids 36x64 .. 288x512)."""
    q = synth.config_quark()
    ad = lambda w, h: q.replace(model_w=1920, model_h=1080, out_w=w, out_h=h)
    for w, h in [(1920, 1080), (1280, 720), (3840, 2160)]:
        c = ad(w, h)
        assert [c.ldm_shape(j) for j in range(24)] == [q.ldm_shape(j) for j in range(24)]
        assert c.upsample_syx == (h / 288, w / 512)
    # 4:3 outputs (the paper's 1024x768 and 2048x1536 benchmarks): coarsest grid 42x56 (2352 px,
    # 4:3 exactly, against 36x64 = 2304), final 336x448; the upsample is 2.2857 or 4.5714 per axis
    for w, h in [(1024, 768), (2048, 1536)]:
        c = ad(w, h)
        assert c.ldm_shape(0) == (24, 42, 56) and c.ldm_shape(23) == (6, 336, 448)
        assert c.upsample_syx == (h / 336, w / 448)
        assert abs(42 * 56 / 2304 - 1) < 0.03


def test_scaled_intrinsics_per_axis():
    """A grid with factors (ky, kx) maps a camera pixel (u, v) to (u / kx, v / ky)."""
    cam = synth.make_camera(64, 48, 50.0, (0.1, 0.0, 0.0), target=(0.0, 0.0, 10.0), cx=31.0, cy=25.0)
    rng = np.random.default_rng(4)
    Xw = rng.uniform(-2, 2, (20, 3)) + np.array([0, 0, 8.0])
    u1, v1, _ = O.project(Xw, O.scaled_K(cam, 1.0), cam)
    u2, v2, _ = O.project(Xw, O.scaled_K(cam, (3.25, 3.125)), cam)
    np.testing.assert_allclose(u2, u1 / 3.125, rtol=1e-13)
    np.testing.assert_allclose(v2, v1 / 3.25, rtol=1e-13)


def test_anisotropic_grids_window_exactly():
    """An output whose aspect differs from the model's gets different factors along rows and
    columns (here 3.25 and 3.125); windows of the output still equal the full frame."""
    cfg = synth.config_quark(out_w=240, out_h=120, C=8).replace(model_w=240, model_h=120, out_w=200, out_h=130)
    assert cfg.ldm_shape(0)[1:] == (5, 8) and cfg.ldm_shape(23)[1:] == (40, 64)
    assert cfg.upsample_syx == (3.25, 3.125)
    sc = synth.scene_quark(seed=8, V=2, W=128, H=80, out_w=200, out_h=130)
    W = synth.make_weights(cfg, seed=8, sharp=True)
    full, _ = O.forward(cfg, W, sc)
    for rect in [(0, 9, 0, 13), (60, 71, 97, 120), (129, 130, 0, 200)]:
        part, _ = O.forward(cfg, W, sc, rect)
        np.testing.assert_allclose(part, full[rect[0]:rect[1], rect[2]:rect[3]], atol=1e-13)


def test_update_block_lift_closed_form():
    """With its CNN zeroed the Update Block is F + up(I~) W_r + b_r; at a x2 level change the
    rendering is upsampled with edge clamp and pixel centres aligned (here written out by hand)."""
    rng = np.random.default_rng(6)
    C = 8
    F = rng.standard_normal((6, 8, C))
    It = rng.uniform(0, 1, (3, 4, 4))
    W = {"upd_Wr_1": rng.standard_normal((4, C)), "upd_br_1": rng.standard_normal(C), "upd_g_1": np.ones(C),
         "upd1_w_1": np.zeros((3, 3, C, C)), "upd1_b_1": np.zeros(C), "upd2_w_1": np.zeros((3, 3, C, C)),
         "upd2_b_1": np.zeros(C)}
    got = O.update_block(W, 1, F, It)
    up = np.zeros((6, 8, 4))
    for y in range(6):
        for x in range(8):
            sy, sx = (y + 0.5) / 2 - 0.5, (x + 0.5) / 2 - 0.5
            y0, x0 = int(np.floor(sy)), int(np.floor(sx))
            fy, fx = sy - y0, sx - x0
            cy = lambda i: min(max(i, 0), 2)
            cx = lambda i: min(max(i, 0), 3)
            up[y, x] = ((1 - fy) * (1 - fx) * It[cy(y0), cx(x0)] + (1 - fy) * fx * It[cy(y0), cx(x0 + 1)] +
                        fy * (1 - fx) * It[cy(y0 + 1), cx(x0)] + fy * fx * It[cy(y0 + 1), cx(x0 + 1)])
    np.testing.assert_allclose(got, F + up @ W["upd_Wr_1"] + W["upd_br_1"], atol=1e-12)
