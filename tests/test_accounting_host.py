"""Host checks of the roofline accounting: the algorithmic FLOPs of the sampling step split into
the tensor-core projections and the SIMT per-view work, and the bench's choice of the reported
and the binding roofline.  No GPU."""
import pytest

import bench
from paper_2411_16680_b300 import accounting, synth

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2000.0, "source": "test"}


def _cfg(precision):
    return synth.QuarkConfig(C=32, heads=2, scales=[(8, 32), (4, 16), (2, 8), (1, 4)], near=1.0, far=100.0,
                             out_h=1080, out_w=1920, precision=precision)


def test_sampling_flops_split_into_projections_and_per_view_work():
    cfg, V = _cfg(synth.PREC_BF16), 8
    w = accounting.per_view_work(cfg, V, 1080, 1920)["attend"]
    C, h = cfg.C, 2
    proj = simt = 0
    for j, (k, L) in enumerate(cfg.scales):
        E = L * (1080 // k) * (1920 // k)
        last = j == len(cfg.scales) - 1
        # X W^q (+ X W^beta on the last step) and O W^O per element
        proj += 2 * E * (2 * h * C * C + (C * C if last else 0))
        # per view: bilinear sample (4 taps x C), h logits and h weighted sums (h C each), blend logit
        simt += 2 * E * V * (4 * C + 2 * h * C + (C if last else 0))
    assert w["tensor_flops"] == proj
    assert w["flops"] - w["tensor_flops"] == simt


def test_fp32_form_tensor_flops_follow_its_paths():
    # SIMT kernels only: no tensor FLOPs
    work = accounting.per_view_work(_cfg(synth.PREC_FP32), 8, 1080, 1920, (False, False))
    assert all(v["tensor_flops"] == 0 for v in work.values())
    conv = accounting.per_view_work(_cfg(synth.PREC_BF16), 8, 1080, 1920)["conv_block"]
    E = sum(L * (1080 // k) * (1920 // k) for k, L in _cfg(1).scales)
    assert conv["tensor_flops"] == 2 * 18 * 32 * 32 * E and conv["tensor_products"] == 1
    # split FP16 operands: the same definition FLOPs on the tensor cores, three products each
    split = accounting.per_view_work(_cfg(synth.PREC_FP32), 8, 1080, 1920, (True, True))
    bf = accounting.per_view_work(_cfg(synth.PREC_BF16), 8, 1080, 1920)
    for fam in ("attend", "conv_block"):
        assert split[fam]["tensor_flops"] == bf[fam]["tensor_flops"] > 0
        assert split[fam]["tensor_products"] == 3
    assert split["collapse"]["tensor_flops"] == 0 and split["encode"]["tensor_flops"] == 0


def test_split_roofline_takes_a_third_of_the_dense_peak():
    cfg = _cfg(synth.PREC_FP32)
    res = {"ktimes": {"conv_block": (4, 4.0), "render": (1, 0.3)}, "tc_paths": (True, True)}
    r = bench.roofline(cfg, 8, 1080, 1920, res, PEAKS)
    assert r["bound"] == "tensor" and r["peak"] == round(PEAKS["bf16_tflops_sustained"] / 3, 1)


@pytest.mark.parametrize("fam,precision,bound", [("attend", synth.PREC_BF16, "hbm"),
                                                 ("conv_block", synth.PREC_BF16, "tensor"),
                                                 ("conv_block", synth.PREC_FP32, "alu")])
def test_roofline_reports_the_stated_bound_and_names_the_binding_one(fam, precision, bound):
    cfg = _cfg(precision)
    res = {"ktimes": {fam: (4, 4.0), "render": (1, 0.3)}}  # FP32: the SIMT kernels (no tc_paths)
    r = bench.roofline(cfg, 8, 1080, 1920, res, PEAKS)
    assert r["kernel"] == fam and r["bound"] == bound
    assert r["frac"] == r["fractions"][bound]
    w = accounting.per_view_work(cfg, 8, 1080, 1920)[fam]
    alu = (w["flops"] - w["tensor_flops"]) / w["launches"]
    t_at_peak = {"hbm": w["bytes"] / w["launches"] / (PEAKS["hbm_gbs"] * 1e9),
                 "alu": alu / (accounting.fp32_alu_peak_tflops(PEAKS["sm_max_mhz"]) * 1e12)}
    if w["tensor_flops"]:
        t_at_peak["tensor"] = w["tensor_flops"] / w["launches"] / (PEAKS["bf16_tflops_sustained"] * 1e12)
    assert set(r["fractions"]) == set(t_at_peak)
    assert r["binding"] == max(t_at_peak, key=t_at_peak.get)
