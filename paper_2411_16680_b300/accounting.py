"""Algorithmic (compulsory) bytes and FLOPs of each kernel family for one novel view.

Bytes count every tensor a kernel must read or write once: the feature volume entering and
leaving a step, the pyramid level it samples (each texel once), the decoded attributes, the
blend logits, the images and the output.  FLOPs count the multiply-adds of the definition
(2 per MAC) plus nothing for activations.  These are the numerators of the roofline fractions
the bench reports; measured DRAM traffic above them means re-reads.
"""
from __future__ import annotations

from typing import Dict


def per_view_work(cfg, V: int, img_h: int, img_w: int, tc_paths=None) -> Dict[str, Dict[str, float]]:
    """tc_paths: (attend, conv) on the tensor cores, as quark_tensor_core_paths reports them for the
    loaded weights; default: both in the BF16 form, neither in the FP32 form."""
    C = cfg.C
    bf16 = cfg.precision == 1
    elt = 2 if bf16 else 4
    # "tensor_flops": the part of "flops" that runs on the tensor cores; the rest runs on the FP32
    # SIMT pipes.  "tensor_products": tensor-core products per FLOP of the definition: 1 in the BF16
    # form, 3 where the FP32 form splits each operand into two FP16 parts (x_h w_h, x_h w_l, x_l w_h)
    out: Dict[str, Dict[str, float]] = {k: {"bytes": 0.0, "flops": 0.0, "tensor_flops": 0.0, "launches": 0,
                                            "tensor_products": 1 if bf16 else 3}
                                        for k in ("encode", "collapse", "attend", "conv_block", "render", "refine")}
    attend_tc, conv_tc = (bf16, bf16) if tc_paths is None else (bool(tc_paths[0]), bool(tc_paths[1]))
    tc = bf16
    # encode: images in, every used level out, RGBA copy out
    e = out["encode"]
    e["bytes"] += V * img_h * img_w * (3 * 4 + 16)
    for k in cfg.levels():
        e["bytes"] += V * (img_h // k) * (img_w // k) * C * elt
    e["flops"] += 2 * 27 * C * V * img_h * img_w
    e["launches"] += 1
    for j, (k, L) in enumerate(cfg.scales):
        _, H, W = cfg.ldm_shape(j)
        E = L * H * W
        h = cfg.heads_of(j)
        last = j == cfg.n_scales - 1
        a = out["attend"]
        vin = 0
        if j > 0:
            Lp, Hp, Wp = cfg.ldm_shape(j - 1)
            vin = L * Hp * Wp * C * elt
            if Lp == 2 * L:
                c = out["collapse"]
                c["bytes"] += (Lp + L) * Hp * Wp * C * elt
                c["flops"] += 2 * 3 * C * C * L * Hp * Wp
                c["tensor_flops"] += 2 * 3 * C * C * L * Hp * Wp if tc else 0
                c["launches"] += 1
        cb = out["conv_block"]
        cb["bytes"] += 2 * E * C * elt + (2 * E * 4 if last else 0)  # V in and out; raw logits of the last step
        cb["flops"] += 2 * (18 * C * C + 5 * C) * E
        cb["tensor_flops"] += 2 * 18 * C * C * E if conv_tc else 0
        cb["launches"] += 1
        if h == 0:
            continue  # a block without attention: its conv block only
        texels = V * (img_h // k) * (img_w // k)
        if cfg.refines(j):
            # render-and-refine: decode of the entering volume (its C channels in, 5 floats out), the
            # splat (5 floats in; V x (colour, density, weight) sums written and read back by the
            # composite), the rendered views, then F' = F + up(I~) W_r and the Update Block's conv
            # block (F' in, Delta out); the attention then reads Delta in place of the level
            r = out["refine"]
            Lp, Hp, Wp = cfg.ldm_shape(j - 1)
            kp = cfg.scales[j - 1][0]
            Ep = L * Hp * Wp
            rtex = V * (img_h // kp) * (img_w // kp)
            r["bytes"] += Ep * C * elt + Ep * 5 * 4 + Ep * 5 * 4 + 2 * rtex * L * 5 * 4 + rtex * 16
            r["bytes"] += 2 * texels * C * elt + rtex * 16 + 2 * texels * C * elt
            r["flops"] += 2 * Ep * 5 * C + 2 * texels * (4 * C + (18 * C * C + 5 * C))
            r["launches"] += 5
        # the sampled depths: read by a block that reuses them, written for the next sampling block
        # when that one reuses them
        nxt = next((i for i in range(j + 1, cfg.n_scales) if cfg.heads_of(i)), None)
        writes = nxt is not None and cfg.reuse_of(nxt) and not cfg.reuse_of(j)
        a["bytes"] += E * 4 * (int(bool(cfg.reuse_of(j))) + int(bool(writes)))
        if getattr(cfg, "ray_encoding", 0):
            # gamma_k: the level read and written once more (the coarse encoding is negligible)
            k0 = max(cfg.levels())
            out["attend"]["bytes"] += 2 * texels * C * elt
            out["attend"]["flops"] += 2 * V * (img_h // k0) * (img_w // k0) * 32 * C + 2 * 4 * texels * C
            out["attend"]["launches"] += 2
        if getattr(cfg, "attn_mode", 0) == 1:
            # standard: keys / values (and the features on the last step) projected once per texel
            # (written, then read by the sampling), per element q = x W^q, q_i . k_i and p v_i per
            # view and head, W^O
            nc = (3 if last else 2) * C
            a["bytes"] += vin + texels * C * elt + 2 * texels * nc * elt + E * C * elt + (E * V * 4 if last else 0)
            a["flops"] += 2 * (texels * 2 * C * C + E * (2 * C * C + 2 * V * C + (C * C + V * C if last else 0)))
            a["launches"] += 2
        else:
            a["bytes"] += vin + texels * C * elt + E * C * elt + (E * V * 4 if last else 0)
            # per element: the projections X W^q (+ the blend query X W^beta) and O W^O (tensor cores
            # when attend_tc), per view the bilinear sample, h logits, h weighted sums and the
            # blend logit (SIMT)
            proj = 2 * h * C * C + (C * C if last else 0)
            macs = proj + 2 * V * h * C + 4 * V * C + (V * C if last else 0)
            a["flops"] += 2 * macs * E
            a["tensor_flops"] += 2 * proj * E if attend_tc else 0
            a["launches"] += 1
    L, Hl, Wl = cfg.ldm_shape(cfg.n_scales - 1)
    r = out["render"]
    r["bytes"] += L * Hl * Wl * (2 + V) * 4 + V * img_h * img_w * 16 + cfg.out_h * cfg.out_w * 16
    r["flops"] += 2 * cfg.out_h * cfg.out_w * L * V * 16
    r["launches"] += 1
    return out


def fp32_alu_peak_tflops(sm_mhz: float, n_sm: int = 148, lanes: int = 128) -> float:
    """FP32 SIMT peak: n_sm SMs x `lanes` FP32 FMA lanes x 2 FLOP x clock."""
    return n_sm * lanes * 2 * sm_mhz * 1e6 / 1e12
