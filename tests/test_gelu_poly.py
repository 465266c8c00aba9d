"""Host checks of the packed polynomial GELUs the kernels evaluate (device_common.cuh): the
coefficients as compiled, evaluated in FP32 the way the kernels do (u = x^2 clamped to B^2,
t = u (2 / B^2) - 1 fused, Horner on t, Phi = 0.5 + x S saturated to [0, 1]), against the exact
erf form of GELU (Sec. 3.3's conv block uses GELU).  No GPU."""
import os
import re

import numpy as np
import pytest
from scipy.special import erf

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2411_16680_b300", "csrc", "device_common.cuh")


def _coefficients(name):
    text = open(SRC).read()
    body = text[text.index(f"float2 {name}(float2 x)"):]
    arr = re.search(r"constexpr float c\[(\d+)\] = \{([^}]*)\}", body)
    vals = [float(v.strip().rstrip("f")) for v in arr.group(2).split(",")]
    assert len(vals) == int(arr.group(1))
    return np.asarray(vals, np.float32)


def _eval(c, x, B):
    x = x.astype(np.float32)
    u = np.minimum(x * x, np.float32(B * B))
    # the kernels fuse u * (2 / B^2) - 1 into one FMA: evaluate it in float64 and round once
    t = (u.astype(np.float64) * np.float64(np.float32(2.0 / (B * B))) - 1.0).astype(np.float32)
    acc = np.full_like(t, c[-1])
    for ci in c[-2::-1]:
        acc = (acc.astype(np.float64) * t + ci).astype(np.float32)
    phi = np.clip((x.astype(np.float64) * acc + 0.5).astype(np.float32), 0, 1)
    return (x * phi).astype(np.float32)


@pytest.mark.parametrize("name,B,abs_tol,rel_tol", [("gelu_poly2", 5.0, 4e-6, 1.1e-6),
                                                     ("gelu_fine2", 6.0, 1.2e-6, 3e-7)])
def test_polynomial_gelu_matches_the_erf_form(name, B, abs_tol, rel_tol):
    c = _coefficients(name)
    x = np.concatenate([np.linspace(-12, 12, 400001), [0.0, -0.0, 1e-8, -1e-8, 40.0, -40.0]])
    ref = 0.5 * x * (1 + erf(x / np.sqrt(2)))
    err = np.abs(_eval(c, x, B).astype(np.float64) - ref)
    assert err.max() <= abs_tol
    assert np.max(err / np.maximum(1.0, np.abs(x))) <= rel_tol
