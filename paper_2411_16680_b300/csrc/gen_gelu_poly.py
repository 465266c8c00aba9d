"""Coefficients of the polynomial GELUs in device_common.cuh: gelu_poly2 (B = 5, degree 11, for
the BF16 form's layer collapse) and gelu_fine2 (B = 6, degree 16, for the FP32 form: its error is
FP32 rounding, about 2 ulp).

gelu(x) = x Phi(x) with Phi(x) = 0.5 + x S(x^2) and S(u) = erf(sqrt(u / 2)) / (2 sqrt(u)).
S is fitted by weighted least squares on Chebyshev nodes of u in [0, B^2], as a polynomial of
degree DEG in t = 2 u / B^2 - 1 (a well-conditioned basis on [-1, 1]).  The kernel clamps u to
B^2 and saturates Phi to [0, 1], so |x| > B gives gelu = x or 0.  Printed: the coefficients
(lowest order first) and the maximum absolute error of an FP32 evaluation against the exact
erf form on [-12, 12], for both fits.  Run: python gen_gelu_poly.py
"""
import numpy as np
from scipy.special import erf

B, DEG = 5.0, 11


def fit():
    u = (np.cos(np.linspace(0, np.pi, 4000)) + 1) * 0.5 * B * B
    su = np.sqrt(np.maximum(u, 1e-300))
    S = np.where(u > 1e-12, erf(su / np.sqrt(2)) / (2 * su), 1 / np.sqrt(2 * np.pi))
    t = u * (2 / (B * B)) - 1
    return np.polynomial.polynomial.polyfit(t, S, DEG, w=su + 1e-3)


def eval_f32(co, x):
    c = co.astype(np.float32)
    xf = x.astype(np.float32)
    u = np.minimum(xf * xf, np.float32(B * B))
    t = (u * np.float32(2 / (B * B)) - np.float32(1)).astype(np.float32)
    acc = np.full_like(t, c[-1])
    for ci in c[-2::-1]:
        acc = (acc * t + ci).astype(np.float32)
    phi = np.clip((xf * acc + np.float32(0.5)).astype(np.float32), 0, 1)
    return (xf * phi).astype(np.float32)


if __name__ == "__main__":
    for B, DEG in ((5.0, 11), (6.0, 16)):
        co = fit()
        x = np.linspace(-12, 12, 600001)
        ref = 0.5 * x * (1 + erf(x / np.sqrt(2)))
        err = np.abs(eval_f32(co, x) - ref)
        print("B =", B, "degree", DEG, "max abs error", f"{err.max():.2e}",
              "max error relative to max(1, |x|)", f"{np.max(err / np.maximum(1.0, np.abs(x))):.2e}")
        print(", ".join(f"{float(np.float32(c)):.9e}f" for c in co))
