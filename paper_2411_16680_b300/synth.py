"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *makes inputs*: workload descriptions, pinhole cameras, input
images (value-noise textures or a small ray-cast scene) and random-init network
weights.  It holds none of the method's arithmetic (no reprojection, sampling,
attention, convolution or compositing); each side implements those itself.

Workloads follow the shapes of the paper's experiments (Sec. 1: 8 input views
up to ~30 cm apart, 1080p output; Tables "Model description for Quark / Quark+":
LDM layer counts 4..32, C = 32, 1..4 heads).  The paper's datasets and trained
weights are not available, so seeded synthetic scenes and N(0, std) weights
stand in for them.
"""
from __future__ import annotations

import dataclasses
import os
import tempfile
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


# --------------------------------------------------------------------------------------------
# Workload description
# --------------------------------------------------------------------------------------------

ATTN_ONE_TO_MANY = 0
ATTN_STANDARD = 1
PREC_FP32 = 0
PREC_BF16 = 1


@dataclass
class QuarkConfig:
    """Shape of one Quark network instance.

    scales: list of (k, L) from coarse to fine.  Scale j uses pyramid level k_j (relative to
    the input views) and an LDM of L_j layers on a grid of (out_h / f_j, out_w / f_j) pixels,
    f_j = k_j unless ldm_f gives it.  Consecutive scales have f_{j-1} / f_j and k_{j-1} / k_j in
    {1, 2} and L_{j-1} / L_j in {1, 2} (layer collapse, Sec. 3.2).  The final render upsamples
    the last scale by s = f_last (Sec. 3.2.3, factor s).

    Per-scale options of the full model schedule (the paper's model tables), None = defaults:
      scale_heads  attention heads of each scale's fusion block; 0 = a block with no attention
                   (the second residual CNN block of an "A, C, C" group)
      ldm_f        LDM grid factor of each scale relative to the output (e.g. 30, 15, 7.5, 3.75)
      reuse_depth  1 = the scale samples the views at the depths of the latest scale that
                   sampled (one set of update features Delta per Update & Fuse step, fused by
                   several blocks)
    """

    C: int = 16
    heads: int = 1
    scales: List[Tuple[int, int]] = field(default_factory=lambda: [(2, 4)])
    near: float = 1.0
    far: float = 10.0
    out_h: int = 48
    out_w: int = 64
    attn_mode: int = ATTN_ONE_TO_MANY
    precision: int = PREC_FP32
    ray_encoding: int = 0  # 1: add the ray directional encoding gamma_k to the sampled features
    scale_heads: Optional[List[int]] = None
    ldm_f: Optional[List[float]] = None
    reuse_depth: Optional[List[int]] = None
    render_refine: int = 0  # 1: update features from rendered input views (render-and-refine)
    # aspect-adaptive LDM dims: the output size the grid factors are given for (e.g. 1920 x 1080);
    # other outputs get grids of the same area per layer at their own aspect (None: off)
    model_w: Optional[int] = None
    model_h: Optional[int] = None
    # kernel size of the fusion blocks' residual convolutions: 3 (Sec. 3.3) or 1 (the position-wise
    # MLP block of a Transformer, which the residual convolution block mirrors)
    conv_kernel: int = 3

    @property
    def n_scales(self) -> int:
        return len(self.scales)

    def heads_of(self, j: int) -> int:
        return self.heads if self.scale_heads is None else int(self.scale_heads[j])

    def f_of(self, j: int) -> float:
        return float(self.scales[j][0]) if self.ldm_f is None else float(self.ldm_f[j])

    def reuse_of(self, j: int) -> int:
        return 0 if self.reuse_depth is None else int(self.reuse_depth[j])

    def refines(self, j: int) -> bool:
        """Step j renders the intermediate LDM into the input views and runs the Update Block: the
        first sampling block of every Update & Fuse step after the initialisation."""
        return bool(self.render_refine) and j > 0 and self.heads_of(j) > 0 and not self.reuse_of(j)

    @property
    def upsample_s(self) -> float:
        return self.f_of(self.n_scales - 1)

    @property
    def upsample_syx(self) -> Tuple[float, float]:
        """Final upsample factors (rows, columns): out_h / H and out_w / W of the last grid."""
        return self.fyx_of(self.n_scales - 1)

    def fyx_of(self, j: int) -> Tuple[float, float]:
        """Grid factors of step j along rows and columns: output size over grid size."""
        _, H, W = self.ldm_shape(j)
        return self.out_h / H, self.out_w / W

    def ldm_shape(self, j: int) -> Tuple[int, int, int]:
        L = self.scales[j][1]
        if self.model_w:
            # same area per layer as the model's grids, at the output's aspect (Sec. 4: the LDM
            # keeps its pixel count for any output, the final upsample adapts); the coarsest grid
            # is rounded, the finer ones are its x2 multiples
            f0 = self.f_of(0)
            area = (self.model_h / f0) * (self.model_w / f0)
            aspect = self.out_w / self.out_h
            h0 = max(1, int(np.floor(np.sqrt(area / aspect) + 0.5)))
            w0 = max(1, int(np.floor(h0 * aspect + 0.5)))
            m = int(round(f0 / self.f_of(j)))
            return L, h0 * m, w0 * m
        f = self.f_of(j)
        H, W = int(round(self.out_h / f)), int(round(self.out_w / f))
        assert abs(H * f - self.out_h) < 1e-6 and abs(W * f - self.out_w) < 1e-6, "output not divisible by f"
        return L, H, W

    def levels(self) -> List[int]:
        return sorted({k for k, _ in self.scales})

    def replace(self, **kw) -> "QuarkConfig":
        return dataclasses.replace(self, **kw)


@dataclass
class Camera:
    """Pinhole camera, world->camera extrinsics X_c = R X_w + t; x right, y down, z forward."""

    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray  # (3, 3) float64
    t: np.ndarray  # (3,) float64

    @property
    def K(self) -> np.ndarray:
        return np.array([[self.fx, 0.0, self.cx], [0.0, self.fy, self.cy], [0.0, 0.0, 1.0]])

    @property
    def centre(self) -> np.ndarray:
        return -self.R.T @ self.t


def look_at(centre: Sequence[float], target: Sequence[float]) -> Tuple[np.ndarray, np.ndarray]:
    """Rotation/translation of a camera at `centre` aimed at `target` (y down, z forward)."""
    c = np.asarray(centre, np.float64)
    z = np.asarray(target, np.float64) - c
    z = z / np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    x = x / np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    return R, -R @ c


def make_camera(width, height, f, centre, target=None, cx=None, cy=None) -> Camera:
    if target is None:
        R, t = np.eye(3), -np.asarray(centre, np.float64)
    else:
        R, t = look_at(centre, target)
    return Camera(width, height, float(f), float(f),
                  float(width / 2 if cx is None else cx), float(height / 2 if cy is None else cy), R, t)


# --------------------------------------------------------------------------------------------
# Value noise (input textures only)
# --------------------------------------------------------------------------------------------

def _lattice(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.random((n, n, 3))


def value_noise_2d(lat: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Smooth (smoothstep-interpolated) periodic value noise; lat is (n, n, 3) in [0, 1)."""
    n = lat.shape[0]
    flat = lat.reshape(n * n, 3).astype(np.float32)
    u0 = np.floor(u)
    v0 = np.floor(v)
    fu = (u - u0).astype(np.float32)
    fv = (v - v0).astype(np.float32)
    fu = fu * fu * (3 - 2 * fu)
    fv = fv * fv * (3 - 2 * fv)
    i0 = u0.astype(np.int64) % n
    j0 = v0.astype(np.int64) % n
    i1 = (i0 + 1) % n
    j1 = (j0 + 1) % n
    a = np.take(flat, j0 * n + i0, axis=0)
    b = np.take(flat, j0 * n + i1, axis=0)
    c = np.take(flat, j1 * n + i0, axis=0)
    d = np.take(flat, j1 * n + i1, axis=0)
    fu = fu[..., None]
    fv = fv[..., None]
    return (a + (b - a) * fu) * (1 - fv) + (c + (d - c) * fu) * fv


def fbm_2d(rng: np.random.Generator, u: np.ndarray, v: np.ndarray, octaves: int,
           lattice_n: int = 64) -> np.ndarray:
    """Sum of `octaves` value-noise octaves (frequency x2, amplitude x0.5), normalised to [0, 1]."""
    out = np.zeros(u.shape + (3,), np.float32)
    amp, tot, freq = 1.0, 0.0, 1.0
    for _ in range(octaves):
        lat = _lattice(rng, lattice_n)
        out += amp * value_noise_2d(lat, u * freq, v * freq)
        tot += amp
        amp *= 0.5
        freq *= 2.0
    return out / tot


# --------------------------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------------------------

@dataclass
class Scene:
    images: np.ndarray           # (V, H, W, 3) float32 in [0, 1]
    cams: List[Camera]           # input views
    target: Camera               # novel view (output resolution)
    depth: Optional[np.ndarray] = None  # (V, H, W) ground-truth z of the ray-cast scene


def scene_noise_pair(seed: int = 1234, V: int = 2, W: int = 64, H: int = 48, f: float = 60.0,
                     baseline: float = 0.1, octaves: int = 3, period: float = 16.0,
                     out_w: Optional[int] = None, out_h: Optional[int] = None) -> Scene:
    """Smooth value-noise images (base period `period` px), cameras spaced `baseline` apart on x,
    all looking down +z (R = I), novel view at the midpoint of the rig."""
    rng = np.random.default_rng(seed)
    ys, xs = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    imgs = []
    for _ in range(V):
        imgs.append(fbm_2d(rng, xs / period, ys / period, octaves, lattice_n=max(8, int(np.ceil(max(W, H) / period)) + 2)))
    images = np.stack(imgs).astype(np.float32)
    xs_c = np.linspace(0.0, baseline * (V - 1), V)
    cams = [make_camera(W, H, f, (x, 0.0, 0.0)) for x in xs_c]
    ow = W if out_w is None else out_w
    oh = H if out_h is None else out_h
    sx, sy = ow / W, oh / H
    target = Camera(ow, oh, f * sx, f * sy, W / 2 * sx, H / 2 * sy, np.eye(3),
                    -np.array([xs_c.mean(), 0.0, 0.0]))
    return Scene(images, cams, target)


def _ray_dirs(cam: Camera) -> np.ndarray:
    ys, xs = np.meshgrid(np.arange(cam.height, dtype=np.float64) + 0.5,
                         np.arange(cam.width, dtype=np.float64) + 0.5, indexing="ij")
    d_cam = np.stack([(xs - cam.cx) / cam.fx, (ys - cam.cy) / cam.fy, np.ones_like(xs)], -1)
    return d_cam @ cam.R  # camera -> world (R^T d), z_cam = 1 along each ray


def scene_raycast(seed: int = 1234, V: int = 8, W: int = 1920, H: int = 1080, f: float = 1400.0,
                  arc: float = 0.6, radius: float = 10.0, n_planes: int = 10, n_spheres: int = 10,
                  zmin: float = 1.0, zmax: float = 100.0, octaves: int = 5,
                  out_w: Optional[int] = None, out_h: Optional[int] = None) -> Scene:
    """Ray-cast scene: `n_planes` textured quads and `n_spheres` textured spheres placed uniformly in
    inverse depth over [zmin, zmax] m in front of the rig, over a textured backdrop plane at zmax.
    Cameras sit evenly on an `arc` m arc of a circle of `radius` m around (0, 0, radius), aimed at it;
    the novel view is the arc midpoint.  One ray per pixel, no antialiasing."""
    rng = np.random.default_rng(seed)
    centre = np.array([0.0, 0.0, radius])
    half = arc / radius / 2.0
    thetas = np.linspace(-half, half, V)
    cams = []
    for th in thetas:
        c = np.array([radius * np.sin(th), 0.0, radius - radius * np.cos(th)])
        R, t = look_at(c, centre)
        cams.append(Camera(W, H, f, f, W / 2, H / 2, R, t))
    ow = W if out_w is None else out_w
    oh = H if out_h is None else out_h
    target = Camera(ow, oh, f * ow / W, f * oh / H, ow / 2, oh / 2, np.eye(3), np.zeros(3))

    tan_x = (W / 2) / f
    tan_y = (H / 2) / f
    prims = []
    for i in range(n_planes + n_spheres):
        z = 1.0 / rng.uniform(1.0 / zmax, 1.0 / zmin)
        px = rng.uniform(-0.8, 0.8) * tan_x * z
        py = rng.uniform(-0.8, 0.8) * tan_y * z
        size = rng.uniform(0.05, 0.25) * tan_x * z
        tex = rng.integers(0, 2**31)
        if i < n_planes:
            # quad with normal tilted away from -z, spanned by two unit axes
            nrm = np.array([rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4), -1.0])
            nrm /= np.linalg.norm(nrm)
            a1 = np.cross(np.array([0.0, 1.0, 0.0]), nrm)
            a1 /= np.linalg.norm(a1)
            a2 = np.cross(nrm, a1)
            prims.append(("quad", np.array([px, py, z]), nrm, a1, a2, size, tex))
        else:
            prims.append(("sphere", np.array([px, py, z]), size * 0.7, tex))
    back_tex = rng.integers(0, 2**31)

    key = None
    cache_dir = os.environ.get("QUARK_SCENE_CACHE", os.path.join(tempfile.gettempdir(), "quark_scene_cache"))
    if W * H * V >= 1_000_000:
        key = os.path.join(cache_dir, f"raycast_{seed}_{V}_{W}x{H}_{f}_{arc}_{radius}_{n_planes}_{n_spheres}_"
                                      f"{zmin}_{zmax}_{octaves}.npz")
        if os.path.exists(key):
            z = np.load(key)
            return Scene(z["images"], cams, target, z["depth"])
    args = [(cam, prims, back_tex, zmax, octaves) for cam in cams]
    if V >= 4 and W * H >= 1_000_000:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=min(V, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_render_view_star, args))
    else:
        res = [_render_view(*a) for a in args]
    images = np.stack([r[0] for r in res]).astype(np.float32)
    depth = np.stack([r[1] for r in res]).astype(np.float32)
    if key is not None:
        os.makedirs(cache_dir, exist_ok=True)
        tmp = key + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, images=images, depth=depth)
        os.replace(tmp, key)
    return Scene(images, cams, target, depth)


def _render_view(cam: Camera, prims, back_tex, zmax: float, octaves: int):
    """Nearest hit per pixel (ray parameter = camera depth, since rays have unit camera z),
    then one texture lookup per pixel from the primitive hit."""
    H, W = cam.height, cam.width
    o = cam.centre
    d = _ray_dirs(cam).reshape(-1, 3)
    n = d.shape[0]
    best = np.full(n, np.inf)
    pid = np.full(n, -1, np.int64)      # -1: backdrop
    ta = np.zeros(n)                    # texture coordinates of the nearest hit
    tb = np.zeros(n)
    s_back = (zmax - o[2]) / d[:, 2]
    hit = s_back > 0
    best[hit] = s_back[hit]
    for i, pr in enumerate(prims):
        if pr[0] == "quad":
            _, c0, nrm, a1, a2, size, tex = pr
            den = d @ nrm
            s = ((c0 - o) @ nrm) / np.where(np.abs(den) < 1e-12, 1e-12, den)
            P = o + d * s[:, None] - c0
            lu = P @ a1
            lv = P @ a2
            m = (s > 0) & (s < best) & (np.abs(lu) < size) & (np.abs(lv) < size)
            best[m] = s[m]
            pid[m] = i
            ta[m] = lu[m] / size * 4.0
            tb[m] = lv[m] / size * 4.0
        else:
            _, c0, r, tex = pr
            oc = o - c0
            b = d @ oc
            a = np.einsum("ij,ij->i", d, d)
            cc = oc @ oc - r * r
            disc = b * b - a * cc
            ok = disc > 0
            s = np.full(n, np.inf)
            s[ok] = (-b[ok] - np.sqrt(disc[ok])) / a[ok]
            m = ok & (s > 0) & (s < best)
            best[m] = s[m]
            pid[m] = i
            P = o + d[m] * s[m, None] - c0
            ta[m] = np.arctan2(P[:, 0], -P[:, 2]) * 3.0
            tb[m] = np.arcsin(np.clip(P[:, 1] / r, -1, 1)) * 3.0
    col = np.zeros((n, 3), np.float32)
    back = pid < 0
    P = o + d[back] * best[back, None]
    col[back] = fbm_2d(np.random.default_rng(back_tex), P[:, 0] / 4.0, P[:, 1] / 4.0, octaves)
    for i, pr in enumerate(prims):
        m = pid == i
        if m.any():
            col[m] = fbm_2d(np.random.default_rng(pr[-1]), ta[m], tb[m], octaves)
    return col.reshape(H, W, 3), best.reshape(H, W)


def _render_view_star(a):
    return _render_view(*a)


def perturb_target(scene: Scene, rng: np.random.Generator, jitter: float) -> Camera:
    """Novel view jittered by U(-jitter, jitter) m per axis, same orientation."""
    c = scene.target.centre + rng.uniform(-jitter, jitter, 3)
    return dataclasses.replace(scene.target, t=-scene.target.R @ c)


# --------------------------------------------------------------------------------------------
# Weights
# --------------------------------------------------------------------------------------------

def weight_shapes(cfg: QuarkConfig) -> Dict[str, Tuple[int, ...]]:
    """Every tensor of the network, row-vector convention (y = x @ W + b).

    enc_w (3, 3, 3, C): 3x3 encoder conv [dy, dx, c_in, c_out]; enc_b (C,)
    v0 (C,): learned initial feature (Sec. 3.2.2, Initialization)
    per scale j: attn_g_j (C,), Wq_j (C, h*C), Wo_j (h*C, C)          one-to-many attention (Sec. 3.3)
                 conv_g_j (C,), conv1_w_j (k,k,C,C), conv1_b_j, conv2_w_j, conv2_b_j   residual conv block (k = conv_kernel)
                 col_w1_j (2C, C), col_b1_j (C,), col_w2_j (C, C), col_b2_j (C,)      layer collapse MLP
                 Wq_std_j, Wk_std_j, Wv_std_j, Wo_std_j (C, C)         standard cross-attention mode
    w_d (C,), b_d (1,), w_sigma (C,), b_sigma (1,), W_a (C, 3), b_a (3,)   LDM decoders
    W_beta (C, C): blend-weight query projection of the final block (Sec. 3.2.3)
    W_ray_k (32, C) per pyramid level k used: projection of the ray directional encoding (Sec. 3.2.1)
    """
    C = cfg.C
    s = {"enc_w": (3, 3, 3, C), "enc_b": (C,), "v0": (C,)}
    for j in range(cfg.n_scales):
        h = cfg.heads_of(j)
        if h > 0:
            s.update({f"attn_g_{j}": (C,), f"Wq_{j}": (C, h * C), f"Wo_{j}": (h * C, C)})
        ks = cfg.conv_kernel
        s.update({
            f"conv_g_{j}": (C,), f"conv1_w_{j}": (ks, ks, C, C), f"conv1_b_{j}": (C,),
            f"conv2_w_{j}": (ks, ks, C, C), f"conv2_b_{j}": (C,),
            f"col_w1_{j}": (2 * C, C), f"col_b1_{j}": (C,), f"col_w2_{j}": (C, C), f"col_b2_{j}": (C,),
        })
        if h > 0:
            s.update({f"Wq_std_{j}": (C, C), f"Wk_std_{j}": (C, C), f"Wv_std_{j}": (C, C), f"Wo_std_{j}": (C, C)})
        if cfg.refines(j):
            # Update Block: the rendered view (RGB + alpha) lifted to C channels, then a residual CNN
            s.update({f"upd_Wr_{j}": (4, C), f"upd_br_{j}": (C,), f"upd_g_{j}": (C,),
                      f"upd1_w_{j}": (3, 3, C, C), f"upd1_b_{j}": (C,), f"upd2_w_{j}": (3, 3, C, C),
                      f"upd2_b_{j}": (C,)})
    s.update({"w_d": (C,), "b_d": (1,), "w_sigma": (C,), "b_sigma": (1,), "W_a": (C, 3), "b_a": (3,),
              "W_beta": (C, C)})
    for k in cfg.levels():
        s[f"W_ray_{k}"] = (32, C)
    return s


def make_weights(cfg: QuarkConfig, seed: int = 5678, std: float = 0.02, sharp: bool = False) -> Dict[str, np.ndarray]:
    """Random-init weights.  Default: every tensor N(0, std) (gains 1 + N(0, std)).

    sharp=True draws fan-in-scaled weights (N(0, 1/fan_in) x gain: query and blend projections
    x4, residual-branch outputs x0.4) so that the softmax over views, the blend weights, the depth tanh and
    the gelu are far from their linear regimes."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, shp in weight_shapes(cfg).items():
        if not sharp:
            if name.startswith(("attn_g", "conv_g", "upd_g")):
                w = 1.0 + std * rng.standard_normal(shp)
            else:
                w = std * rng.standard_normal(shp)
        else:
            if name.startswith(("attn_g", "conv_g", "upd_g")):
                w = 1.0 + 0.2 * rng.standard_normal(shp)
            elif name in ("v0",):
                w = rng.standard_normal(shp)
            elif name.startswith(("enc_b", "conv1_b", "conv2_b", "col_b", "upd1_b", "upd2_b", "upd_br")) or \
                    name in ("b_d", "b_sigma", "b_a"):
                w = 0.3 * rng.standard_normal(shp)
            else:
                fan_in = int(np.prod(shp[:-1])) if len(shp) > 1 else shp[0]
                if name.startswith(("Wq", "W_beta")):
                    gain = 4.0
                elif name.startswith(("Wo_", "conv2_w", "col_w2", "upd2_w")):
                    gain = 0.4  # residual branches scaled down so the volume does not drift
                else:
                    gain = 1.0
                w = gain * rng.standard_normal(shp) / np.sqrt(fan_in)
        out[name] = w.astype(np.float32)
    return out


# --------------------------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------------------------

def config_small() -> QuarkConfig:
    """V=2 views 64x48, f=60, 16-channel level-2 map from one 3x3 conv, LDM 32x24 L=4,
    depths in inverse depth over 1..10 m, C=16, one head, output 64x48 (s=2)."""
    return QuarkConfig(C=16, heads=1, scales=[(2, 4)], near=1.0, far=10.0, out_h=48, out_w=64)


def scene_small(seed: int = 1234) -> Scene:
    return scene_noise_pair(seed=seed)


def config_1080p() -> QuarkConfig:
    """V=8 views 1920x1080, scales (k, L) = (8,32),(4,16),(2,8),(1,4), C=32, two heads,
    near 1 m, far 100 m, 1080p output (s=1)."""
    return QuarkConfig(C=32, heads=2, scales=[(8, 32), (4, 16), (2, 8), (1, 4)], near=1.0, far=100.0,
                       out_h=1080, out_w=1920)


def scene_1080p(seed: int = 1234, V: int = 8, W: int = 1920, H: int = 1080) -> Scene:
    return scene_raycast(seed=seed, V=V, W=W, H=H, f=1400.0 * W / 1920.0)


def config_quark(out_w: int = 1920, out_h: int = 1080, C: int = 32) -> QuarkConfig:
    """The paper's Quark model (appendix table "Model description for Quark"): an Initialize step
    and five Update & Fuse steps, 24 fusion steps in all.  Per step: pyramid level k, layers L,
    LDM grid factor f (36x64 -> 288x512 for a 1920x1080 output), the heads of each fusion block
    and its residual CNN blocks.  A fusion block "A_h, C, C" is one step with attention and a
    conv block, then one step with a conv block only; the first block of an Update & Fuse step
    samples the views at the depths decoded from its input, the later blocks reuse them (one
    set of update features per step).  The final render upsamples by s = 3.75."""
    return _schedule(24, 30.0, out_w, out_h, C)


def config_quarkplus(out_w: int = 1920, out_h: int = 1080, C: int = 32) -> QuarkConfig:
    """The paper's Quark+ model (appendix table "Model description for Quark+"): the Quark schedule
    with 32 -> 16 -> 8 layers on LDM grids 54x96 -> 432x768 for a 1920x1080 output (grid factors
    20, 10, 5, 2.5; the table's 432x768 output LDM gives the final upsample 2.5), from 720x432 views."""
    return _schedule(32, 20.0, out_w, out_h, C)


def _schedule(L0: int, f0: float, out_w: int, out_h: int, C: int) -> QuarkConfig:
    groups = [  # (k, L, f, heads of each fusion block, CNN blocks per fusion block)
        (8, L0, f0, [4, 4, 4], 2),               # Initialize (flat layers at the depth anchors)
        (8, L0, f0, [4, 4, 4], 2),               # Update & Fuse 0
        (4, L0, f0 / 2, [4, 4, 4], 2),           # Update & Fuse 1 (x2 upsample)
        (4, L0, f0 / 2, [4, 4], 1),              # Update & Fuse 2
        (2, L0 // 2, f0 / 4, [2, 2], 1),         # Update & Fuse 3 (layer collapse, x2 upsample)
        (1, L0 // 4, f0 / 8, [1, 1], 1),         # Update & Fuse 4 (layer collapse, x2 upsample)
    ]
    scales, f, heads, reuse = [], [], [], []
    for k, L, ff, hs, n_cnn in groups:
        for b, h in enumerate(hs):
            for i in range(n_cnn):
                scales.append((k, L))
                f.append(ff)
                heads.append(h if i == 0 else 0)
                reuse.append(1 if i == 0 and b > 0 else 0)
    return QuarkConfig(C=C, heads=4, scales=scales, near=1.0, far=100.0, out_h=out_h, out_w=out_w,
                       scale_heads=heads, ldm_f=f, reuse_depth=reuse)


def scene_quark(seed: int = 1234, V: int = 8, W: int = 480, H: int = 288, out_w: int = 1920,
                out_h: int = 1080) -> Scene:
    """Input views at the Quark table's resolution (480x288: a 36x60 level-8 feature map; Quark+:
    720x432, a 54x90 map) and a 1920x1080 novel view covering the same frustum."""
    return scene_raycast(seed=seed, V=V, W=W, H=H, f=350.0 * W / 480.0, out_w=out_w, out_h=out_h)


def config_grad() -> QuarkConfig:
    """Differentiation workload: V=4 views 512x512, scales (2,16), (1,8), C=32, two heads."""
    return QuarkConfig(C=32, heads=2, scales=[(2, 16), (1, 8)], near=1.0, far=100.0, out_h=512, out_w=512)


def scene_grad(seed: int) -> Scene:
    return scene_raycast(seed=seed, V=4, W=512, H=512, f=400.0, arc=0.3)
