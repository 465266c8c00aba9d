"""Model schedules on the host: the Quark workload follows the paper's model table (appendix,
table "Model description for Quark"), the LDM grid rule of the oracle (Sec. 3.2; Sec. 4 for the
aspect-adaptive reading) gives those tables' grids and equals the sizes the input module uses,
and the C ABI rejects schedules its steps cannot run."""
import pytest
import torch

from oracle import quark_oracle as O
from paper_2411_16680_b300 import quark, synth


def test_quark_workload_matches_the_model_table():
    """Per Update & Fuse step of the table: output layer dimensions (L, h, w) and encoded
    feature map (h, w) for 480x288 input views and a 1920x1080 output; blocks A4,C,C x3 (x3
    steps), A4,C,A4,C, A2,C,A2,C, A1,C,A1,C; final upsample 3.75."""
    cfg = synth.config_quark()
    assert cfg.n_scales == 24 and cfg.C == 32 and cfg.upsample_s == 3.75
    groups = [(0, 6), (6, 12), (12, 18), (18, 20), (20, 22), (22, 24)]
    table_out = [(24, 36, 64), (24, 36, 64), (24, 72, 128), (24, 72, 128), (12, 144, 256), (6, 288, 512)]
    table_feat = [(36, 60), (36, 60), (72, 120), (72, 120), (144, 240), (288, 480)]
    table_blocks = [[4, 0, 4, 0, 4, 0]] * 3 + [[4, 4], [2, 2], [1, 1]]
    for (a, b), out, feat, blocks in zip(groups, table_out, table_feat, table_blocks):
        assert all(O.ldm_shape(cfg, j) == out for j in range(a, b))
        assert all((288 // cfg.scales[j][0], 480 // cfg.scales[j][0]) == feat for j in range(a, b))
        assert [cfg.heads_of(j) for j in range(a, b)] == blocks
        # one set of update features per step: only the step's first block decodes depths
        assert [cfg.reuse_of(j) for j in range(a, b) if cfg.heads_of(j)] == [0] + [1] * (len([h for h in blocks if h]) - 1)
    # layer collapse at the first block of steps 3 and 4 only
    collapses = [j for j in range(1, 24) if cfg.scales[j - 1][1] == 2 * cfg.scales[j][1]]
    assert collapses == [20, 22]


def test_quarkplus_workload_matches_the_model_table():
    """Quark+ table: output layer dimensions (32, 54, 96), (32, 54, 96), (32, 108, 192),
    (32, 108, 192), (16, 216, 384), (8, 432, 768); feature maps 54x90 .. 432x720 of 720x432 views;
    the same blocks as Quark; final upsample 1080 / 432 = 2.5."""
    cfg = synth.config_quarkplus()
    assert cfg.n_scales == 24 and cfg.upsample_s == 2.5
    groups = [(0, 6), (6, 12), (12, 18), (18, 20), (20, 22), (22, 24)]
    table_out = [(32, 54, 96), (32, 54, 96), (32, 108, 192), (32, 108, 192), (16, 216, 384), (8, 432, 768)]
    table_feat = [(54, 90), (54, 90), (108, 180), (108, 180), (216, 360), (432, 720)]
    for (a, b), out, feat in zip(groups, table_out, table_feat):
        assert all(cfg.ldm_shape(j) == out for j in range(a, b))
        assert all((432 // cfg.scales[j][0], 720 // cfg.scales[j][0]) == feat for j in range(a, b))
    q = synth.config_quark()
    assert [q.heads_of(j) for j in range(24)] == [cfg.heads_of(j) for j in range(24)]
    assert [q.reuse_of(j) for j in range(24)] == [cfg.reuse_of(j) for j in range(24)]


def _bad(**kw):
    base = dict(C=16, heads=2, scales=[(8, 4), (8, 4), (4, 4)], near=1.0, far=30.0, out_h=45, out_w=120,
                ldm_f=[15, 15, 7.5], scale_heads=[4, 0, 2], reuse_depth=[0, 0, 0])
    base.update(kw)
    return synth.QuarkConfig(**base)


@pytest.mark.parametrize("kw", [
    dict(scale_heads=[0, 4, 2]),                                   # step 0 without attention
    dict(scale_heads=[4, 4, 0]),                                   # last step without attention
    dict(reuse_depth=[1, 0, 0]),                                   # step 0 reusing depths
    dict(scales=[(8, 4), (4, 4), (4, 4)], ldm_f=[15, 7.5, 7.5]),  # no-attention after a grid change
    dict(scales=[(8, 4), (8, 2), (4, 2)]),                         # no-attention across a layer collapse
    dict(reuse_depth=[0, 0, 1]),                                   # reuse across a grid change
    dict(ldm_f=[15, 15, 5]),                                       # grid ratio 3
    dict(scale_heads=[4, 0, 3]),                                   # 3 heads
    dict(ldm_f=[15, -15, 7.5]),                                    # negative grid factor
])
def test_schedule_validation_rejects(kw):
    with pytest.raises(quark.QuarkError) as e:
        quark.Context(_bad(**kw))
    assert e.value.status == quark.EINVAL, kw


def test_valid_schedules_pass_validation():
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: creation would succeed")
    for cfg in (_bad(), synth.config_quark(), synth.config_quarkplus(), _bad(scale_heads=[4, 0, 2], reuse_depth=[0, 0, 0])):
        with pytest.raises(quark.QuarkError) as e:
            quark.Context(cfg)
        assert e.value.status == quark.ECUDA  # past validation, stopped only by the missing device


@pytest.mark.parametrize("cfg", [
    synth.config_1080p(), synth.config_small(), synth.config_grad(), synth.config_quark(), synth.config_quarkplus(),
    synth.config_quark(out_w=1024, out_h=768).replace(model_w=1920, model_h=1080),
    synth.config_quark(out_w=2048, out_h=1536).replace(model_w=1920, model_h=1080),
    synth.config_quarkplus(out_w=1024, out_h=768).replace(model_w=1920, model_h=1080),
    synth.config_quark(out_w=200, out_h=130).replace(model_w=240, model_h=120),
], ids=["1080p", "small", "grad", "quark", "quarkplus", "quark_1024x768", "quark_2048x1536", "quarkplus_1024x768",
        "anisotropic_200x130"])
def test_input_sizes_follow_the_oracle_grid_rule(cfg):
    """The input module sizes buffers and reads with its own copy of the grid rule; it must give the
    oracle's grids and factors at every step (the CUDA path computes them a third time, in the ABI)."""
    for j in range(cfg.n_scales):
        assert cfg.ldm_shape(j) == O.ldm_shape(cfg, j)
        assert cfg.fyx_of(j) == pytest.approx(O.grid_factors(cfg, j), rel=0, abs=0)


def test_aspect_adaptive_grids_keep_the_model_area():
    """Sec. 4: at another aspect the LDM keeps the model's pixel count per layer (to rounding) and
    its grids stay x2 multiples of the coarsest; at the model's own size the rule is the identity."""
    model = synth.config_quark()
    for w, h in ((1024, 768), (2048, 1536), (1280, 720), (3840, 2160)):
        cfg = synth.config_quark(out_w=w, out_h=h).replace(model_w=1920, model_h=1080)
        for j in range(cfg.n_scales):
            _, H, W = O.ldm_shape(cfg, j)
            _, Hm, Wm = O.ldm_shape(model, j)
            assert abs(H * W - Hm * Wm) / (Hm * Wm) < 0.05
            assert abs(W / H - w / h) < 0.05 * w / h
            _, H0, W0 = O.ldm_shape(cfg, 0)
            assert H % H0 == 0 and W % W0 == 0 and H // H0 == W // W0
    same = synth.config_quark().replace(model_w=1920, model_h=1080)
    assert [O.ldm_shape(same, j) for j in range(same.n_scales)] == [O.ldm_shape(model, j) for j in range(model.n_scales)]
