"""Integer work of the sampling (Sec. 3.1 operator P^T): the origins of the bilinear taps,
floor(u - 0.5) and floor(v - 0.5), that the kernels compute (quark_sample_coords: each precision
form's own device arithmetic -- IEEE divide in FP32, one reciprocal in BF16) equal the FP64
oracle's for every sample of a 960x540 eight-view rig at the grids of the workloads, except where
the oracle's coordinate lies within 1e-3 px of a texel boundary: there FP32 rounding may decide
either way, and bilinear sampling is continuous across the boundary.  Those samples are counted
and printed; the continuous coordinates agree to 1e-3 px everywhere."""
import numpy as np
import pytest

from oracle import quark_oracle as O
from paper_2411_16680_b300 import quark, synth

pytestmark = pytest.mark.gpu

NEAR_PX = 1e-3


@pytest.mark.parametrize("precision", [synth.PREC_FP32, synth.PREC_BF16])
@pytest.mark.parametrize("k_t,k_m", [(8.0, 8), (2.0, 2), (3.75, 1)])
def test_tap_origins_match_the_oracle(precision, k_t, k_m):
    sc = synth.scene_1080p(W=960, H=540)
    H, W, L = int(round(540 / k_t)), int(round(960 / k_t)), 4
    rng = np.random.default_rng(int(k_t * 100) + k_m)
    ell = np.arange(1, L + 1, dtype=np.float64)[:, None, None]
    t = rng.uniform(-3.0, 3.0, (L, H, W))
    d32 = O.depth_activation(t, ell, L, 1.0, 100.0).astype(np.float32)
    ys = np.broadcast_to(np.arange(H)[None, :, None], (L, H, W))
    xs = np.broadcast_to(np.arange(W)[None, None, :], (L, H, W))
    ctx = quark.Context(synth.config_small().replace(precision=precision))
    near_total = total = 0
    try:
        for cam in sc.cams:
            uv, taps, valid = ctx.sample_coords(sc.target, k_t, k_t, cam, float(k_m), xs + 0.5, ys + 0.5, d32)
            Xw = O.unproject(ys, xs, d32.astype(np.float64), O.scaled_K(sc.target, k_t), sc.target)
            u, v, ok = O.project(Xw, O.scaled_K(cam, float(k_m)), cam)
            u, v, ok = u.ravel(), v.ravel(), ok.ravel()
            assert np.array_equal(valid.astype(bool), ok)
            xr, yr = u - 0.5, v - 0.5
            near = (np.abs(xr - np.round(xr)) < NEAR_PX) | (np.abs(yr - np.round(yr)) < NEAR_PX)
            exact = ok & ~near
            assert np.array_equal(taps[exact, 0], np.floor(xr[exact]).astype(np.int64))
            assert np.array_equal(taps[exact, 1], np.floor(yr[exact]).astype(np.int64))
            assert np.abs(uv[ok, 0] - u[ok]).max() <= NEAR_PX and np.abs(uv[ok, 1] - v[ok]).max() <= NEAR_PX
            near_total += int((ok & near).sum())
            total += int(ok.sum())
    finally:
        ctx.close()
    print(f"\ntap origins: form {'bf16' if precision else 'fp32'}, grid factor {k_t} -> level {k_m}: {total} samples "
          f"equal the FP64 oracle; {near_total} ({near_total / max(total, 1):.2e}) lie within {NEAR_PX} px of a "
          f"texel boundary and are exempt")
