"""Hand derivation of a tiny end-to-end case; writes hand_case.txt.

Uses only `math`: every number below is a closed form worked out by hand for this
specific set-up (no oracle and no CUDA code is involved).  The set-up is chosen so that
each step of the method reduces to a few scalars:

  output 2x2, one scale (k=2, L=2) -> a 1x1 LDM; V=2 views of 2x2 pixels; C=2; h=1.
  near 0.8 m, far 4 m  ->  1/near - 1/far = 1, 1/far = 0.25.
  Depth anchors (Eq. depth anchors): delta_1 = 0.25, delta_2 = 0.75; with tanh(0) = 0 the
  disparities (Eq. depth_activation) are 0.5 and 1.0, so d_1 = 2 m (far), d_2 = 1 m (near).
  Target = view 1: f = 2 px, c = (1, 1), R = I, at the origin.  View 2: same intrinsics,
  centre (0.5, 0, 0).
  Encoder: centre tap maps (R, G) -> channels (0, 1), zero bias, so the level-2 map of a
  view is the mean of its R and G planes: view 1 (0.25, 0.5), view 2 (0.8, 0.2).
  Level-2 intrinsics f = 1, c = 0.5.  The LDM pixel centre (0.5, 0.5) looks down the
  optical axis: X = (0, 0, d).  View 1 sees it at u = 0.5 (texel centre, weight 1).
  View 2 sees it at u = 0.5 - 0.5/d: u = 0.25 (d=2) and u = 0 (d=1); with zero padding
  the 1x1 map contributes 0.75 F and 0.5 F.
  v0 = (2, 2), gains 1 -> N(v0) = r (1, 1) with r = 2/sqrt(4 + 1e-6).
  Wq = [[1, 0], [0, -1]], Wo = I, W_beta = I.
  Conv block: centre taps I and 0.5 I, every other tap 7.0 (they only ever see zero
  padding on a 1x1 plane), zero biases -> V_out = V_attn + 0.5 gelu(N(V_attn)).
  Decoders: w_d = 0, b_d = 0 (depth stays at the anchors), w_sigma = 0, b_sigma = ln 3
  (alpha = 0.75), W_a = 0, b_a = 0 (colour 0.5).
  Render (s = 2): every output pixel reads the single LDM pixel.  Full-resolution ray of
  pixel (X, Y) is ((X - 0.5)/2, (Y - 0.5)/2, 1).  View 1 samples its own pixel (X, Y).
  View 2 sees it at u = X + 0.5 - 1/d, v = Y + 0.5: for d = 2 it averages pixels X-1 and
  X of row Y; for d = 1 it reads pixel X-1 (zero outside the image).
  Over, front (l = 2) to back (l = 1): RGB = 0.75 c_2 + 0.25 * 0.75 c_1, A = 1 - 0.25^2.
"""
import math
import os

r = 2.0 / math.sqrt(4.0 + 1e-6)
s2 = math.sqrt(2.0)
F1 = (0.25, 0.5)
F2 = (0.8, 0.2)


def gelu(x):
    return 0.5 * x * (1.0 + math.erf(x / s2))


lines = []
lines.append("# Hand-derived tiny end-to-end case; see hand_case_derivation.py for the set-up.")
lines.append("# Sec. 3.1 Eq. (1); Sec. 3.2.3 Eqs. (depth anchors, depth_activation); Sec. 3.3 attention,")
lines.append("# fusion block and conv block.  key = value (float64).")
lines.append("depth_l1 = 2.0")
lines.append("depth_l2 = 1.0")
Delta = {1: [F1, (0.75 * F2[0], 0.75 * F2[1])], 2: [F1, (0.5 * F2[0], 0.5 * F2[1])]}
V_attn = {}
for l in (1, 2):
    d1, d2 = Delta[l]
    for m, dm in ((1, d1), (2, d2)):
        lines.append(f"delta_l{l}_v{m} = {dm[0]!r} {dm[1]!r}")
    # q = r (1, -1); logits q . Delta_m / sqrt(2)
    s_1 = r * (d1[0] - d1[1]) / s2
    s_2 = r * (d2[0] - d2[1]) / s2
    p2 = 1.0 / (1.0 + math.exp(s_1 - s_2))
    p1 = 1.0 - p2
    lines.append(f"p_l{l} = {p1!r} {p2!r}")
    o = (p1 * d1[0] + p2 * d2[0], p1 * d1[1] + p2 * d2[1])
    va = (2.0 + o[0], 2.0 + o[1])
    V_attn[l] = va
    lines.append(f"V_attn_l{l} = {va[0]!r} {va[1]!r}")
    # beta logits: (N(v0) W_beta) . Delta_m / sqrt(2) = r (Delta_m0 + Delta_m1) / sqrt(2)
    lines.append(f"beta_logit_l{l} = {r * (d1[0] + d1[1]) / s2!r} {r * (d2[0] + d2[1]) / s2!r}")
    ms = (va[0] ** 2 + va[1] ** 2) / 2.0
    n = (va[0] / math.sqrt(ms + 1e-6), va[1] / math.sqrt(ms + 1e-6))
    vo = (va[0] + 0.5 * gelu(n[0]), va[1] + 0.5 * gelu(n[1]))
    lines.append(f"V_out_l{l} = {vo[0]!r} {vo[1]!r}")
lines.append("alpha = 0.75")

# blend weights at the output: layer 1 logits equal -> (0.5, 0.5); layer 2 logits
# r*0.75/sqrt2 and r*0.5/sqrt2 -> beta_1 = 1 / (1 + exp(-0.25 r / sqrt2))
b1_l2 = 1.0 / (1.0 + math.exp(-0.25 * r / s2))
b2_l2 = 1.0 - b1_l2
img1 = {(0, 0): (0.1, 0.5, 0.9), (0, 1): (0.2, 0.5, 0.9), (1, 0): (0.3, 0.5, 0.9), (1, 1): (0.4, 0.5, 0.9)}
img2 = {(0, 0): (0.8, 0.0, 0.2), (0, 1): (0.8, 0.4, 0.6), (1, 0): (0.8, 0.4, 0.2), (1, 1): (0.8, 0.0, 0.6)}
zero = (0.0, 0.0, 0.0)
for Y in (0, 1):
    for X in (0, 1):
        v1 = img1[(Y, X)]
        left = img2.get((Y, X - 1), zero)
        here = img2[(Y, X)]
        v2_l1 = tuple(0.5 * a + 0.5 * b for a, b in zip(left, here))
        v2_l2 = left
        c1 = tuple(0.5 * a + 0.5 * b for a, b in zip(v1, v2_l1))
        c2 = tuple(b1_l2 * a + b2_l2 * b for a, b in zip(v1, v2_l2))
        rgb = tuple(0.75 * a + 0.1875 * b for a, b in zip(c2, c1))
        lines.append(f"rgba_y{Y}_x{X} = {rgb[0]!r} {rgb[1]!r} {rgb[2]!r} 0.9375")

with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "hand_case.txt"), "w") as fh:
    fh.write("\n".join(lines) + "\n")
