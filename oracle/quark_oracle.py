"""FP64 CPU oracle of Quark's Update & Fuse steps and final LDM render.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import this module.  The CUDA path never does, and this module
shares no code with it: it only reads the seeded inputs made by the synth module.

Plain numpy float64, written from the paper step by step (Flynn et al., "Quark:
Real-time, High-resolution, and General Neural View Synthesis", 2024):

  encode        Sec. 3.2.1 and the "Encode Input Images" figure: a 3x3 conv (3 -> C,
                zero pad, bias) at full resolution, then strided 2x2 mean pooling;
                level k holds the k x k block mean of the conv output.
  transition    Sec. 3.2.2 "Initialization" (broadcast learned v0, flat layers at the
                depth anchors) and "Layer Collapse" (mean of adjacent layers plus a
                residual MLP of their concatenation), then a x2 bilinear upsample when
                the resolution changes (caption of the Update & Fuse figure).
  depth         Sec. 3.2.3, Eq. (depth anchors) and Eq. (depth_activation).
  back-project  Sec. 3.1 (operator P^T): unproject each LDM pixel at its layer depth,
                project into each input view, bilinearly sample the view's feature map.
  attention     Sec. 3.3: One-to-many attention, head_i = Attention(N(V) W_i^q, D, D),
                MultiHead = concat(heads) W^O, V' = V + MultiHead(N(V), D); N = RMSNorm.
  conv block    Sec. 3.3: V' = V + Conv(gelu(Conv(N(V)))), 3x3 per layer plane; with the
                conv_kernel option 1 the convolutions are 1x1, i.e. the position-wise MLP block
                of a Transformer that the residual convolution block mirrors.
  decode        Sec. 3.2.2 "Decoding": sigma = sigmoid(V W_sigma), c = sigmoid(V W_a),
                depth by Eq. (depth_activation).
  blend logits  Sec. 3.2.3: the one-to-many attention logits of the final block against
                its update features, softmax delayed until after upsampling.
  render        Sec. 3.1, Eq. (1): upsample the unactivated depth / density / blend
                logits, activate, back-project the input images, blend with beta, over
                composite (front to back, equivalent to the paper's back to front).
  render and    Sec. 3.2.2 "Decoding and rendering the intermediate LDM", Eq.
  refine        (overcomposite-result), and the Update Block: decode the volume entering an
                Update & Fuse step (activated), bilinearly splat appearance and density into
                every input view (operator P), over-composite there, and turn the rendered
                views and the image features into the update features Delta that the step
                samples instead of the image features.

Conventions (the paper is silent on them; the same readings bind the CUDA path):
pixel centres at (x + 0.5, y + 0.5); camera x right, y down, z forward; world->camera
X_c = R X_w + t; depth = camera z; level-k intrinsics diag(1/k, 1/k, 1) K; layer
index l = 1..L with l = 1 farthest and l = L nearest; bilinear sampling with zero
padding (grid_sample "zeros", align_corners=False); bilinear resizing with edge
clamp; a sample with camera z <= 1e-6 in the source view is invalid and reads zero.

Every computation runs on rectangular windows of a plane ("rects").  A full plane is
one rect; sampled outputs of a large frame are computed by growing the requested rect
backwards through each step's halo (render upsample, two 3x3 convs, x2 upsample).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
from scipy.special import erf

Z_MIN = 1e-6
RMS_EPS = 1e-6

Rect = Tuple[int, int, int, int]  # y0, y1, x0, x1 (half-open), in plane coordinates


# ---------------------------------------------------------------------------------------------
# LDM grids (Sec. 3.2: the step's grid factor relative to the output; Sec. 4: for outputs whose
# aspect differs from the model's, the LDM keeps its pixel count and the final upsample adapts)
# ---------------------------------------------------------------------------------------------

def ldm_shape(cfg, j: int) -> Tuple[int, int, int]:
    """(L, H, W) of step j's LDM.  By default H = out_h / f_j and W = out_w / f_j for the step's
    grid factor f_j.  With a model size (model_w x model_h, aspect-adaptive): the coarsest grid has
    the model's area per layer at the output's aspect, h0 = round(sqrt(area / aspect)) and
    w0 = round(h0 * aspect), and step j's grid is that times f_0 / f_j (the finer grids are its x2
    multiples)."""
    L = cfg.scales[j][1]
    f = cfg.f_of(j)
    if cfg.model_w:
        f0 = cfg.f_of(0)
        area = (cfg.model_h / f0) * (cfg.model_w / f0)
        aspect = cfg.out_w / cfg.out_h
        h0 = max(1, int(math.floor(math.sqrt(area / aspect) + 0.5)))
        w0 = max(1, int(math.floor(h0 * aspect + 0.5)))
        m = int(round(f0 / f))
        return L, h0 * m, w0 * m
    H, W = int(round(cfg.out_h / f)), int(round(cfg.out_w / f))
    assert abs(H * f - cfg.out_h) < 1e-6 and abs(W * f - cfg.out_w) < 1e-6, "output not divisible by f"
    return L, H, W


def grid_factors(cfg, j: int) -> Tuple[float, float]:
    """Step j's grid factors (rows, columns): the output size over the grid size."""
    _, H, W = ldm_shape(cfg, j)
    return cfg.out_h / H, cfg.out_w / W


# ---------------------------------------------------------------------------------------------
# Elementwise definitions
# ---------------------------------------------------------------------------------------------

def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def gelu(x):
    """erf form of gelu (the paper does not say which form; reading: exact erf)."""
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def rmsnorm(v, g):
    """RMSNorm (Zhang & Sennrich 2019), the normalisation N of Sec. 3.3: g * v / rms(v)."""
    return g * v / np.sqrt(np.mean(v * v, axis=-1, keepdims=True) + RMS_EPS)


def depth_anchor(ell, L):
    """Eq. (depth anchors): delta = (l - 0.5) / L for l = 1..L."""
    return (np.asarray(ell, np.float64) - 0.5) / L


def depth_activation(t, ell, L, near, far):
    """Eq. (depth_activation): d = [(delta + 0.5/L tanh t)(1/near - 1/far) + 1/far]^-1."""
    disparity = (depth_anchor(ell, L) + 0.5 / L * np.tanh(t)) * (1.0 / near - 1.0 / far) + 1.0 / far
    return 1.0 / disparity


def grow(r: Rect, n: int, H: int, W: int) -> Rect:
    return (max(r[0] - n, 0), min(r[1] + n, H), max(r[2] - n, 0), min(r[3] + n, W))


# ---------------------------------------------------------------------------------------------
# Cameras and the back-projection geometry (Sec. 3.1, operator P^T)
# ---------------------------------------------------------------------------------------------

def scaled_K(cam, k) -> np.ndarray:
    """Intrinsics of a grid k times coarser than the camera's own pixels; k is one factor, or
    (k_rows, k_cols) for a grid whose factors differ along the two axes."""
    ky, kx = (k, k) if np.isscalar(k) else k
    return np.diag([1.0 / kx, 1.0 / ky, 1.0]) @ cam.K


def unproject(ys, xs, d, K_t, cam_t):
    """World point of target pixel (ys, xs) at camera depth d (arrays broadcast together)."""
    p = np.stack(np.broadcast_arrays(xs + 0.5, ys + 0.5, np.ones_like(xs, dtype=np.float64)), -1)
    ray = p @ np.linalg.inv(K_t).T          # camera-space point at z = 1
    Xc = ray * np.asarray(d)[..., None]      # scale to depth d
    return (Xc - cam_t.t) @ cam_t.R          # R^T (X_c - t)


def project(Xw, K_m, cam_m):
    """Continuous pixel coordinates of world points in view m, and their validity (z > 1e-6)."""
    Xc = Xw @ cam_m.R.T + cam_m.t
    z = Xc[..., 2]
    valid = z > Z_MIN
    zs = np.where(valid, z, 1.0)
    uvw = Xc @ K_m.T
    return uvw[..., 0] / zs, uvw[..., 1] / zs, valid


# ---------------------------------------------------------------------------------------------
# Bilinear operators
# ---------------------------------------------------------------------------------------------

def bilinear_zero(fetch, u, v, valid):
    """Bilinear sample at continuous pixel coords (u, v); taps outside the map read zero.

    fetch(iy, ix) returns the texels at integer indices (zero outside the map), shape
    idx.shape + (C,).  Invalid samples return zero."""
    x = u - 0.5
    y = v - 0.5
    x0 = np.floor(x)
    y0 = np.floor(y)
    fx = (x - x0)[..., None]
    fy = (y - y0)[..., None]
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    out = ((1 - fy) * (1 - fx) * fetch(y0, x0) + (1 - fy) * fx * fetch(y0, x0 + 1)
           + fy * (1 - fx) * fetch(y0 + 1, x0) + fy * fx * fetch(y0 + 1, x0 + 1))
    return np.where(valid[..., None], out, 0.0)


def resize_taps(dst, ratio, n_src):
    """Edge-clamped linear taps of a resize by `ratio` (pixel centres aligned):
    src = (dst + 0.5) / ratio - 0.5.  Returns (i0, i1, w1)."""
    src = (np.asarray(dst, np.float64) + 0.5) / ratio - 0.5
    i0 = np.floor(src)
    w1 = src - i0
    i0 = i0.astype(np.int64)
    return np.clip(i0, 0, n_src - 1), np.clip(i0 + 1, 0, n_src - 1), w1


def resize_rect(src: np.ndarray, src_rect: Rect, H_src: int, W_src: int, ratio, out_rect: Rect):
    """Bilinear resize (edge clamp) of src [..., h, w, C] held on src_rect, evaluated on out_rect;
    ratio is one factor or (rows, columns)."""
    ry, rx = (ratio, ratio) if np.isscalar(ratio) else ratio
    ys = np.arange(out_rect[0], out_rect[1])
    xs = np.arange(out_rect[2], out_rect[3])
    y0, y1, wy = resize_taps(ys, ry, H_src)
    x0, x1, wx = resize_taps(xs, rx, W_src)
    for a in (y0, y1):
        assert a.min() >= src_rect[0] and a.max() < src_rect[1], "resize source rect too small"
    for a in (x0, x1):
        assert a.min() >= src_rect[2] and a.max() < src_rect[3], "resize source rect too small"
    y0 -= src_rect[0]; y1 -= src_rect[0]; x0 -= src_rect[2]; x1 -= src_rect[2]
    wy = wy[:, None, None]
    wx = wx[None, :, None]
    r0 = src[..., y0, :, :]
    r1 = src[..., y1, :, :]
    top = r0[..., :, x0, :] * (1 - wx) + r0[..., :, x1, :] * wx
    bot = r1[..., :, x0, :] * (1 - wx) + r1[..., :, x1, :] * wx
    return top * (1 - wy) + bot * wy


def conv3x3_rect(x: np.ndarray, x_rect: Rect, H: int, W: int, w: np.ndarray, b: np.ndarray, out_rect: Rect):
    """3x3 convolution, zero padding at the plane border, per leading index (layer).

    x: [..., h, w, Cin] on x_rect; w: [3, 3, Cin, Cout] indexed [dy, dx]; returns
    [..., out_h, out_w, Cout] on out_rect.  Every in-plane neighbour of out_rect must lie
    in x_rect."""
    oy0, oy1, ox0, ox1 = out_rect
    need = (oy0 - 1, oy1 + 1, ox0 - 1, ox1 + 1)
    lead = x.shape[:-3]
    padded = np.zeros(lead + (need[1] - need[0], need[3] - need[2], x.shape[-1]))
    # copy the in-plane part of the needed window
    iy0, iy1 = max(need[0], 0), min(need[1], H)
    ix0, ix1 = max(need[2], 0), min(need[3], W)
    assert iy0 >= x_rect[0] and iy1 <= x_rect[1] and ix0 >= x_rect[2] and ix1 <= x_rect[3], "conv halo missing"
    padded[..., iy0 - need[0]:iy1 - need[0], ix0 - need[2]:ix1 - need[2], :] = \
        x[..., iy0 - x_rect[0]:iy1 - x_rect[0], ix0 - x_rect[2]:ix1 - x_rect[2], :]
    oh, ow = oy1 - oy0, ox1 - ox0
    out = np.zeros(lead + (oh, ow, w.shape[-1])) + b
    for dy in range(3):
        for dx in range(3):
            out += padded[..., dy:dy + oh, dx:dx + ow, :] @ w[dy, dx]
    return out


def conv_rect(x: np.ndarray, x_rect: Rect, H: int, W: int, w: np.ndarray, b: np.ndarray, out_rect: Rect):
    """The fusion block's convolution with kernel w [k, k, Cin, Cout]: k = 3 is conv3x3_rect; k = 1
    is the position-wise linear map of a Transformer's MLP block, which the residual convolution
    block of Sec. 3.3 mirrors (the conv_kernel option): y = x w[0, 0] + b on out_rect."""
    if w.shape[0] == 3:
        return conv3x3_rect(x, x_rect, H, W, w, b, out_rect)
    assert w.shape[:2] == (1, 1)
    oy, ox = out_rect[0] - x_rect[0], out_rect[2] - x_rect[2]
    assert oy >= 0 and ox >= 0 and out_rect[1] <= x_rect[1] and out_rect[3] <= x_rect[3], "conv input missing"
    xs = x[..., oy:oy + out_rect[1] - out_rect[0], ox:ox + out_rect[3] - out_rect[2], :]
    return xs @ w[0, 0] + b


# ---------------------------------------------------------------------------------------------
# Encoder (Sec. 3.2.1): conv3x3 at full resolution, then 2x2 mean pooling per level
# ---------------------------------------------------------------------------------------------

def encode_box(image: np.ndarray, enc_w, enc_b, k: int, box: Rect) -> np.ndarray:
    """Level-k feature map of one view on box (level coordinates): the k x k block mean of
    F_1 = conv3x3(image) (zero pad, bias).  Returns [h, w, C]."""
    H, W = image.shape[:2]
    full = (box[0] * k, box[1] * k, box[2] * k, box[3] * k)
    F1 = conv3x3_rect(image.astype(np.float64), (0, H, 0, W), H, W,
                      enc_w.astype(np.float64), enc_b.astype(np.float64), full)
    h, w = box[1] - box[0], box[3] - box[2]
    return F1.reshape(h, k, w, k, -1).mean(axis=(1, 3))


def encode_level(image, enc_w, enc_b, k):
    """The whole level-k map of one view, [H/k, W/k, C]."""
    H, W = image.shape[:2]
    return encode_box(image, enc_w, enc_b, k, (0, H // k, 0, W // k))


# ---------------------------------------------------------------------------------------------
# Ray directional encoding (Sec. 3.2.1)
# ---------------------------------------------------------------------------------------------

RAY_OCTAVES = 8


def ray_difference(cam_m, cam_t, k0, near, far):
    """For the pixel centres of view m on its k0-times coarser grid: the ray's intersections with
    the near and far planes of the LDM frustum (target-camera depth `near` and `far`), each taken
    to the target's normalised image plane (x / z, y / z), and their difference, far minus near.
    [h0, w0, 2].  Zero for a ray through the target camera's centre (a target ray)."""
    h0, w0 = cam_m.height // k0, cam_m.width // k0
    ys, xs = np.meshgrid(np.arange(h0) + 0.5, np.arange(w0) + 0.5, indexing="ij")
    p = np.stack([xs, ys, np.ones_like(xs)], -1)
    d_w = (p @ np.linalg.inv(scaled_K(cam_m, k0)).T) @ cam_m.R  # ray direction, world
    c_w = -cam_m.R.T @ cam_m.t                                  # view m's centre, world
    A = cam_t.R @ c_w + cam_t.t                                 # ray in target coordinates: A + lam B
    B = d_w @ cam_t.R.T
    Bz = B[..., 2]
    Bz = np.where(np.abs(Bz) < 1e-300, 1e-300, Bz)
    planes = []
    for z in (near, far):
        lam = (z - A[2]) / Bz
        X = A + lam[..., None] * B  # X.z == z
        planes.append(X[..., :2] / z)
    return planes[1] - planes[0]


def ray_encoding(diff):
    """tanh of the difference vector, then a sinusoidal encoding with 8 octaves: feature
    4 i + 2 j + {0, 1} = {sin, cos}(2^i pi tanh(diff_j)), i = 0..7, j = x, y.  [..., 32]."""
    e = np.tanh(diff)
    feats = []
    for i in range(RAY_OCTAVES):
        for j in range(2):
            a = (2.0 ** i) * math.pi * e[..., j]
            feats += [np.sin(a), np.cos(a)]
    return np.stack(feats, -1)


def ray_gamma(cam_m, cam_t, k0, k, near, far, W_ray, box):
    """gamma_k of view m on `box` (y0, y1, x0, x1) of level k: the encoding computed once on the
    coarse grid k0, bilinearly upsampled by k0 / k (pixel centres aligned, edge clamp) and
    projected to C channels by the level's own matrix W_ray [32][C]."""
    coarse = ray_encoding(ray_difference(cam_m, cam_t, k0, near, far))
    h0, w0 = coarse.shape[:2]
    up = resize_rect(coarse, (0, h0, 0, w0), h0, w0, k0 // k, box)
    return up @ W_ray


class LevelFetch:
    """Texel fetch from level k of view m with zero padding; evaluates the encoder lazily on
    the bounding box of the texels asked for (all fetches are declared first by `need`)."""

    def __init__(self, image, enc_w, enc_b, k, gamma=None):
        self.image, self.enc_w, self.enc_b, self.k = image, enc_w, enc_b, k
        self.gamma = gamma  # optional: box -> ray directional encoding added to the features
        self.h, self.w = image.shape[0] // k, image.shape[1] // k
        self.box = None
        self.data = None

    def prepare(self, ys_list, xs_list):
        ys = np.concatenate([np.ravel(a) for a in ys_list])
        xs = np.concatenate([np.ravel(a) for a in xs_list])
        inside = (ys >= 0) & (ys < self.h) & (xs >= 0) & (xs < self.w)
        if not inside.any():
            self.box = (0, 0, 0, 0)
            self.data = np.zeros((0, 0, self.enc_b.shape[0]))
            return
        box = (int(ys[inside].min()), int(ys[inside].max()) + 1, int(xs[inside].min()), int(xs[inside].max()) + 1)
        self.box = box
        self.data = encode_box(self.image, self.enc_w, self.enc_b, self.k, box)
        if self.gamma is not None:
            self.data = self.data + self.gamma(box)

    def __call__(self, iy, ix):
        inside = (iy >= 0) & (iy < self.h) & (ix >= 0) & (ix < self.w)
        by = np.clip(iy - self.box[0], 0, max(self.data.shape[0] - 1, 0))
        bx = np.clip(ix - self.box[2], 0, max(self.data.shape[1] - 1, 0))
        if self.data.size == 0:
            return np.zeros(iy.shape + (self.enc_b.shape[0],))
        vals = self.data[by, bx]
        return np.where(inside[..., None], vals, 0.0)


def sample_views(fetchers: Sequence, cams, cam_t, k_t: float, k_m: float, d, ys, xs):
    """Back-projection P^T (Sec. 3.1): for target pixels (ys, xs) at depth d, sample each view.

    d: [L, h, w]; ys [h, 1], xs [1, w] target grid indices at scale k_t.  Returns Delta
    [L, h, w, V, C]."""
    K_t = scaled_K(cam_t, k_t)
    Xw = unproject(ys[None], xs[None], d, K_t, cam_t)  # [L, h, w, 3]
    coords = []
    for m, cam in enumerate(cams):
        u, v, valid = project(Xw, scaled_K(cam, k_m), cam)
        coords.append((u, v, valid))
        x0 = np.floor(u - 0.5).astype(np.int64)
        y0 = np.floor(v - 0.5).astype(np.int64)
        x0 = np.where(valid, x0, -2)
        y0 = np.where(valid, y0, -2)
        fetchers[m].prepare([y0, y0, y0 + 1, y0 + 1], [x0, x0 + 1, x0, x0 + 1])
    out = []
    for m in range(len(cams)):
        u, v, valid = coords[m]
        out.append(bilinear_zero(fetchers[m], u, v, valid))
    return np.stack(out, axis=-2)


# ---------------------------------------------------------------------------------------------
# Fusion block pieces (Sec. 3.3)
# ---------------------------------------------------------------------------------------------

def one_to_many_attention(x, Delta, Wq, Wo, heads):
    """MultiHead(x, Delta) with head_i = softmax(x W_i^q Delta^T / sqrt(C)) Delta (Sec. 3.3,
    "Optimized Attention"); per-head query dimension C (appendix A).  Returns (out, p)."""
    C = x.shape[-1]
    outs, ps = [], []
    for i in range(heads):
        q = x @ Wq[:, i * C:(i + 1) * C]                          # [..., C]
        logits = np.einsum("...c,...mc->...m", q, Delta) / math.sqrt(C)
        logits = logits - logits.max(axis=-1, keepdims=True)
        p = np.exp(logits)
        p = p / p.sum(axis=-1, keepdims=True)
        outs.append(np.einsum("...m,...mc->...c", p, Delta))
        ps.append(p)
    return np.concatenate(outs, axis=-1) @ Wo, np.stack(ps, axis=-2)


def standard_attention(x, Delta, Wq, Wk, Wv, Wo, heads):
    """Textbook multi-head cross attention (Sec. 3.3, Preliminaries; appendix A): queries x W^q,
    keys Delta W^k, values Delta W^val, each split into `heads` heads of C/heads channels,
    softmax(q k^T / sqrt(C/heads)) per head, concat, times W^O."""
    C = x.shape[-1]
    dh = C // heads
    q = x @ Wq
    k = Delta @ Wk
    v = Delta @ Wv
    outs = []
    for i in range(heads):
        sl = slice(i * dh, (i + 1) * dh)
        logits = np.einsum("...c,...mc->...m", q[..., sl], k[..., sl]) / math.sqrt(dh)
        logits = logits - logits.max(axis=-1, keepdims=True)
        p = np.exp(logits)
        p = p / p.sum(axis=-1, keepdims=True)
        outs.append(np.einsum("...m,...mc->...c", p, v[..., sl]))
    return np.concatenate(outs, axis=-1) @ Wo


def layer_collapse(V, w1, b1, w2, b2):
    """Layer Collapse (Sec. 3.2.2): pairs (l=2j-1, 2j) -> mean + MLP(concat); MLP = 2C -> C,
    gelu, C -> C (the paper does not give the MLP depth; reading: one hidden layer)."""
    a = V[0::2]
    b = V[1::2]
    cat = np.concatenate([a, b], axis=-1)
    return 0.5 * (a + b) + gelu(cat @ w1 + b1) @ w2 + b2


# ---------------------------------------------------------------------------------------------
# One Update & Fuse step on windows
# ---------------------------------------------------------------------------------------------

@dataclass
class StepResult:
    rect_attn: Rect
    V_in: np.ndarray       # [L, h, w, C] on rect_attn
    V_attn: np.ndarray     # after the attention block, on rect_attn
    depth_used: np.ndarray  # depth the views were sampled at, on rect_attn
    Delta: np.ndarray      # [L, h, w, V, C]
    x_norm: np.ndarray     # N(V_in) of the attention block
    rect_out: Rect
    V_out: np.ndarray      # after the conv block, on rect_out
    t: np.ndarray          # raw depth logit [L, h, w]
    s: np.ndarray          # raw density logit [L, h, w]
    colour: np.ndarray     # [L, h, w, 3]
    alpha: np.ndarray      # [L, h, w]
    depth: np.ndarray      # [L, h, w]
    beta_logits: Optional[np.ndarray]  # [L, h, w, V] on rect_attn (last scale only)


def update_fuse_step(cfg, W, scene, fetchers, j, prev: Optional[StepResult],
                     rect_attn: Rect, rect_out: Rect, last: bool, mode: int = 0, delta_fetch=None) -> StepResult:
    """One fusion step.  The views' update features are the level-k image features (fetchers[k]),
    or, with render-and-refine, the Update Block's output (delta_fetch, one fetcher per view)."""
    f64 = lambda a: np.asarray(a, np.float64)
    k, L = cfg.scales[j]          # pyramid level of the views, layers
    f = grid_factors(cfg, j)      # LDM grid factors (rows, columns) relative to the output
    _, H, Wd = ldm_shape(cfg, j)
    heads = cfg.heads_of(j)
    C = cfg.C
    ys = np.arange(rect_attn[0], rect_attn[1])[:, None]
    xs = np.arange(rect_attn[2], rect_attn[3])[None, :]
    h, w = rect_attn[1] - rect_attn[0], rect_attn[3] - rect_attn[2]
    ell = np.arange(1, L + 1, dtype=np.float64)[:, None, None]

    # ---- transition: initialisation, or layer collapse then x2 upsample ----
    if j == 0:
        V_in = np.broadcast_to(f64(W["v0"]), (L, h, w, C)).copy()
        d = np.broadcast_to(1.0 / ((ell - 0.5) / L * (1 / cfg.near - 1 / cfg.far) + 1 / cfg.far), (L, h, w)).copy()
    else:
        Lp, Hp, Wp = ldm_shape(cfg, j - 1)
        Vp, rp = prev.V_out, prev.rect_out
        if Lp == 2 * L:
            Vp = layer_collapse(Vp, f64(W[f"col_w1_{j}"]), f64(W[f"col_b1_{j}"]),
                                f64(W[f"col_w2_{j}"]), f64(W[f"col_b2_{j}"]))
        else:
            assert Lp == L
        ratio = H // Hp  # 1, or 2 for a x2 upsample (both axes)
        assert ratio * Hp == H and ratio * Wp == Wd
        V_in = resize_rect(Vp, rp, Hp, Wp, ratio, rect_attn)
        if cfg.reuse_of(j) or heads == 0:
            # the depths of the latest scale that sampled (same grid and layers): reused for the
            # sampling, or carried through a block without attention
            assert ratio == 1 and Lp == L
            oy, ox = rect_attn[0] - prev.rect_attn[0], rect_attn[2] - prev.rect_attn[2]
            d = prev.depth_used[:, oy:oy + h, ox:ox + w]
        else:
            t_in = V_in @ f64(W["w_d"]) + f64(W["b_d"])[0]
            d = depth_activation(t_in, ell, L, cfg.near, cfg.far)

    if heads == 0:
        # a fusion block without attention (its residual CNN block only)
        Delta, x, V_attn = None, None, V_in
    else:
        # ---- back-project the views' level-k features at the current depths ----
        src = fetchers[k] if delta_fetch is None else delta_fetch
        Delta = sample_views(src, scene.cams, scene.target, f, k, d, ys, xs)  # [L,h,w,V,C]

        # ---- fusion block: one-to-many attention ----
        x = rmsnorm(V_in, f64(W[f"attn_g_{j}"]))
        if mode == 0:
            upd, _ = one_to_many_attention(x, Delta, f64(W[f"Wq_{j}"]), f64(W[f"Wo_{j}"]), heads)
        else:
            upd = standard_attention(x, Delta, f64(W[f"Wq_std_{j}"]), f64(W[f"Wk_std_{j}"]),
                                     f64(W[f"Wv_std_{j}"]), f64(W[f"Wo_std_{j}"]), heads)
        V_attn = V_in + upd

    beta = None
    if last:
        assert heads > 0, "the blend logits come from the last block's attention"
        qb = x @ f64(W["W_beta"])
        beta = np.einsum("...c,...mc->...m", qb, Delta) / math.sqrt(C)

    # ---- fusion block: residual conv block V + Conv(gelu(Conv(N(V)))) ----
    n = rmsnorm(V_attn, f64(W[f"conv_g_{j}"]))
    mid_rect = grow(rect_out, 1, H, Wd)
    h1 = conv_rect(n, rect_attn, H, Wd, f64(W[f"conv1_w_{j}"]), f64(W[f"conv1_b_{j}"]), mid_rect)
    h2 = conv_rect(gelu(h1), mid_rect, H, Wd, f64(W[f"conv2_w_{j}"]), f64(W[f"conv2_b_{j}"]), rect_out)
    oy, ox = rect_out[0] - rect_attn[0], rect_out[2] - rect_attn[2]
    V_out = V_attn[:, oy:oy + h2.shape[1], ox:ox + h2.shape[2]] + h2

    # ---- decode the LDM attributes ----
    ello = np.arange(1, L + 1, dtype=np.float64)[:, None, None]
    t = V_out @ f64(W["w_d"]) + f64(W["b_d"])[0]
    s = V_out @ f64(W["w_sigma"]) + f64(W["b_sigma"])[0]
    colour = sigmoid(V_out @ f64(W["W_a"]) + f64(W["b_a"]))
    return StepResult(rect_attn, V_in, V_attn, d, Delta, x, rect_out, V_out, t, s, colour, sigmoid(s),
                      depth_activation(t, ello, L, cfg.near, cfg.far), beta)


# ---------------------------------------------------------------------------------------------
# Final render (Sec. 3.1 Eq. 1, Sec. 3.2.3 Upsampling & Activation)
# ---------------------------------------------------------------------------------------------

def render_rect(cfg, scene, last: StepResult, out_rect: Rect, return_layers: bool = False):
    """RGBA of the novel view on out_rect (full output resolution)."""
    L, Hl, Wl = ldm_shape(cfg, cfg.n_scales - 1)
    s = grid_factors(cfg, cfg.n_scales - 1)
    rect_beta = last.rect_attn
    ob = (last.rect_out[0] - rect_beta[0], last.rect_out[2] - rect_beta[2])
    hb, wb = last.V_out.shape[1], last.V_out.shape[2]
    beta_on_out = last.beta_logits[:, ob[0]:ob[0] + hb, ob[1]:ob[1] + wb]
    t_up = resize_rect(last.t[..., None], last.rect_out, Hl, Wl, s, out_rect)[..., 0]
    s_up = resize_rect(last.s[..., None], last.rect_out, Hl, Wl, s, out_rect)[..., 0]
    b_up = resize_rect(beta_on_out, last.rect_out, Hl, Wl, s, out_rect)  # [L, h, w, V]
    ell = np.arange(1, L + 1, dtype=np.float64)[:, None, None]
    d = depth_activation(t_up, ell, L, cfg.near, cfg.far)
    alpha = sigmoid(s_up)
    bl = b_up - b_up.max(axis=-1, keepdims=True)
    beta = np.exp(bl)
    beta = beta / beta.sum(axis=-1, keepdims=True)

    ys = np.arange(out_rect[0], out_rect[1])[:, None]
    xs = np.arange(out_rect[2], out_rect[3])[None, :]
    K_t = scene.target.K
    Xw = unproject(ys[None], xs[None], d, K_t, scene.target)
    col = np.zeros(d.shape + (3,))
    for m, cam in enumerate(scene.cams):
        img = scene.images[m].astype(np.float64)
        Hi, Wi = img.shape[:2]

        def fetch(iy, ix, img=img, Hi=Hi, Wi=Wi):
            inside = (iy >= 0) & (iy < Hi) & (ix >= 0) & (ix < Wi)
            return np.where(inside[..., None], img[np.clip(iy, 0, Hi - 1), np.clip(ix, 0, Wi - 1)], 0.0)

        u, v, valid = project(Xw, cam.K, cam)
        col += beta[..., m:m + 1] * bilinear_zero(fetch, u, v, valid)
    rgb = np.zeros(d.shape[1:] + (3,))
    T = np.ones(d.shape[1:])
    for li in range(L - 1, -1, -1):        # front (l = L, nearest) to back (l = 1)
        rgb += (T * alpha[li])[..., None] * col[li]
        T = T * (1.0 - alpha[li])
    rgba = np.concatenate([rgb, (1.0 - T)[..., None]], axis=-1)
    if return_layers:
        return rgba, col, alpha, d, beta
    return rgba


def render_depth_rect(cfg, last: StepResult, out_rect: Rect):
    """Depth map of the novel view on out_rect (Sec. 3.1: the optional output, the decoded depth
    over-composited instead of the blended input views).  The raw depth and density logits of the
    last LDM are upsampled and activated exactly as for the colour render; then, front (l = L) to
    back, D += T alpha_l d_l and T *= 1 - alpha_l, with 0 behind the last layer.  Reading: the
    over-composite itself, not normalised by the accumulated alpha."""
    L, Hl, Wl = ldm_shape(cfg, cfg.n_scales - 1)
    s = grid_factors(cfg, cfg.n_scales - 1)
    t_up = resize_rect(last.t[..., None], last.rect_out, Hl, Wl, s, out_rect)[..., 0]
    s_up = resize_rect(last.s[..., None], last.rect_out, Hl, Wl, s, out_rect)[..., 0]
    ell = np.arange(1, L + 1, dtype=np.float64)[:, None, None]
    d = depth_activation(t_up, ell, L, cfg.near, cfg.far)
    alpha = sigmoid(s_up)
    D = np.zeros(d.shape[1:])
    T = np.ones(d.shape[1:])
    for li in range(L - 1, -1, -1):
        D += T * alpha[li] * d[li]
        T = T * (1.0 - alpha[li])
    return D


def over_back_to_front(col, alpha):
    """Over operator applied back to front (l = 1 first), as the paper states it (Sec. 3.1)."""
    rgb = np.zeros(col.shape[1:])
    a_acc = np.zeros(alpha.shape[1:])
    for li in range(col.shape[0]):
        rgb = alpha[li][..., None] * col[li] + (1 - alpha[li])[..., None] * rgb
        a_acc = alpha[li] + (1 - alpha[li]) * a_acc
    return np.concatenate([rgb, a_acc[..., None]], axis=-1)


# ---------------------------------------------------------------------------------------------
# Render and refine (Sec. 3.2.2 "Decoding and rendering the intermediate LDM", Eq.
# (overcomposite-result), the Update Block of the Update & Fuse figure)
# ---------------------------------------------------------------------------------------------

SPLAT_EPS = 1e-2  # reading: splats are normalised by max(weight sum, SPLAT_EPS)


def decode_intermediate(V, W, near, far):
    """Intermediate LDM of a feature volume V [L, H, W, C], activated before projection:
    depth by Eq. (depth_activation), density sigmoid(V w_sigma + b_sigma), appearance
    sigmoid(V W_a + b_a).  Returns d [L, H, W], sigma [L, H, W], a [L, H, W, 3]."""
    f64 = lambda x: np.asarray(x, np.float64)
    L = V.shape[0]
    ell = np.arange(1, L + 1, dtype=np.float64)[:, None, None]
    t = V @ f64(W["w_d"]) + f64(W["b_d"])[0]
    sig = sigmoid(V @ f64(W["w_sigma"]) + f64(W["b_sigma"])[0])
    a = sigmoid(V @ f64(W["W_a"]) + f64(W["b_a"]))
    return depth_activation(t, ell, L, near, far), sig, a


def splat_layers(cam_t, f, cam_m, k, h, w, d, vals):
    """Forward projection P (Sec. 3.2.2): every LDM pixel x layer (grid factor f of the target)
    at its depth d lands at continuous coordinates (u, v) of view m's level-k grid (h x w) and
    adds its values, times the bilinear weights, to the four nearest pixel centres -- the
    transpose of bilinear sampling, nothing outside the map or behind the camera.
    d [L, H, W], vals [L, H, W, n] -> weighted sums [L, h, w, n] and weight sums [L, h, w]."""
    L, H, Wd = d.shape
    ys = np.arange(H, dtype=np.float64)[None, :, None]
    xs = np.arange(Wd, dtype=np.float64)[None, None, :]
    Xw = unproject(ys, xs, d, scaled_K(cam_t, f), cam_t)
    u, v, valid = project(Xw, scaled_K(cam_m, k), cam_m)
    # clamp far-away coordinates (their taps are outside the map either way) before the floor
    x = np.clip(np.where(valid, u, -10.0) - 0.5, -3.0, w + 2.0)
    y = np.clip(np.where(valid, v, -10.0) - 0.5, -3.0, h + 2.0)
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = x - x0, y - y0
    x0, y0 = x0.astype(np.int64), y0.astype(np.int64)
    li = np.broadcast_to(np.arange(L)[:, None, None], d.shape)
    acc = np.zeros((L, h, w, vals.shape[-1]))
    wsum = np.zeros((L, h, w))
    for dy, dx, wt in ((0, 0, (1 - fy) * (1 - fx)), (0, 1, (1 - fy) * fx), (1, 0, fy * (1 - fx)), (1, 1, fy * fx)):
        iy, ix = y0 + dy, x0 + dx
        ok = valid & (iy >= 0) & (iy < h) & (ix >= 0) & (ix < w)
        np.add.at(acc, (li[ok], iy[ok], ix[ok]), wt[ok][:, None] * vals[ok])
        np.add.at(wsum, (li[ok], iy[ok], ix[ok]), wt[ok])
    return acc, wsum


def render_to_views(cfg, W, scene, Vc, f, k):
    """Eq. (overcomposite-result): I~ = O(P(a, d), P(sigma, d)) in every input view, at level k.
    Vc [L, H, W, C] is the volume entering the step (after any layer collapse) on its grid of
    factor f.  Each layer's splat is normalised by its weight sum (reading: clamped below at
    SPLAT_EPS, so sparsely covered pixels fade out), then the layers are over-composited front to
    back in LDM order (l = L nearest first).  Returns [V, h, w, 4]: RGB and accumulated alpha."""
    d, sig, a = decode_intermediate(Vc, W, cfg.near, cfg.far)
    vals = np.concatenate([a, sig[..., None]], axis=-1)
    out = []
    for cam in scene.cams:
        h, w = cam.height // k, cam.width // k
        acc, wsum = splat_layers(scene.target, f, cam, k, h, w, d, vals)
        lay = acc / np.maximum(wsum, SPLAT_EPS)[..., None]
        rgb, T = np.zeros((h, w, 3)), np.ones((h, w))
        for li in range(Vc.shape[0] - 1, -1, -1):
            al = lay[li, ..., 3]
            rgb = rgb + (T * al)[..., None] * lay[li, ..., :3]
            T = T * (1.0 - al)
        out.append(np.concatenate([rgb, (1.0 - T)[..., None]], axis=-1))
    return np.stack(out)


def update_block(W, j, F, It):
    """Update Block of step j (reading; the paper calls it a small CNN on [I~, I_k, rho_k]):
    F' = F + up(I~) W_r + b_r, Delta = F' + Conv(gelu(Conv(N(F')))) with 3x3 convs (zero pad),
    the residual CNN block of Sec. 3.3 in image space.  F [h, w, C] are the view's level-k
    features (with the ray directional encoding when it is on), It [h', w', 4] its rendering at
    the previous step's level, upsampled x h / h' (1 or 2) with edge clamp."""
    f64 = lambda x: np.asarray(x, np.float64)
    h, w = F.shape[:2]
    hp, wp = It.shape[:2]
    Iu = resize_rect(It, (0, hp, 0, wp), hp, wp, h // hp, (0, h, 0, w))
    Fp = F + Iu @ f64(W[f"upd_Wr_{j}"]) + f64(W[f"upd_br_{j}"])
    n = rmsnorm(Fp, f64(W[f"upd_g_{j}"]))
    full = (0, h, 0, w)
    h1 = conv3x3_rect(n, full, h, w, f64(W[f"upd1_w_{j}"]), f64(W[f"upd1_b_{j}"]), full)
    return Fp + conv3x3_rect(gelu(h1), full, h, w, f64(W[f"upd2_w_{j}"]), f64(W[f"upd2_b_{j}"]), full)


class ArrayFetch:
    """Texel fetch from a whole per-view map [h, w, C] (zero outside it)."""

    def __init__(self, data):
        self.data = data
        self.h, self.w = data.shape[:2]

    def prepare(self, ys_list, xs_list):
        pass

    def __call__(self, iy, ix):
        inside = (iy >= 0) & (iy < self.h) & (ix >= 0) & (ix < self.w)
        vals = self.data[np.clip(iy, 0, self.h - 1), np.clip(ix, 0, self.w - 1)]
        return np.where(inside[..., None], vals, 0.0)


def refine_features(cfg, W, scene, fetchers, j, prev: StepResult):
    """Update features of step j with render-and-refine: the volume entering the step (collapsed
    when L halves) rendered into the views at step j-1's level, then the Update Block on each
    view's level-k_j features.  Whole frames only.  Returns one fetcher per view."""
    f64 = lambda a: np.asarray(a, np.float64)
    k, L = cfg.scales[j]
    kp, Lp = cfg.scales[j - 1]
    Vc = prev.V_out
    if Lp == 2 * L:
        Vc = layer_collapse(Vc, f64(W[f"col_w1_{j}"]), f64(W[f"col_b1_{j}"]), f64(W[f"col_w2_{j}"]),
                            f64(W[f"col_b2_{j}"]))
    It = render_to_views(cfg, W, scene, Vc, grid_factors(cfg, j - 1), kp)
    out = []
    for m, lf in enumerate(fetchers[k]):
        lf.prepare([np.array([0, lf.h - 1])], [np.array([0, lf.w - 1])])  # the whole level (+ gamma)
        out.append(ArrayFetch(update_block(W, j, lf.data, It[m])))
    return out


# ---------------------------------------------------------------------------------------------
# Whole forward pass on a window of the output
# ---------------------------------------------------------------------------------------------

def plan_rects(cfg, out_rect: Rect):
    """Windows each scale must compute so that out_rect of the final render is exact."""
    n = cfg.n_scales
    _, Hl, Wl = ldm_shape(cfg, n - 1)
    sy, sx = grid_factors(cfg, n - 1)
    ys = np.arange(out_rect[0], out_rect[1])
    xs = np.arange(out_rect[2], out_rect[3])
    y0, y1, _ = resize_taps(ys, sy, Hl)
    x0, x1, _ = resize_taps(xs, sx, Wl)
    need = (int(y0.min()), int(y1.max()) + 1, int(x0.min()), int(x1.max()) + 1)
    rect_out = [None] * n
    rect_attn = [None] * n
    for j in range(n - 1, -1, -1):
        _, H, W = ldm_shape(cfg, j)
        rect_out[j] = need
        rect_attn[j] = grow(need, 2, H, W)
        if j > 0:
            _, Hp, Wp = ldm_shape(cfg, j - 1)
            ratio = H // Hp
            ys = np.arange(rect_attn[j][0], rect_attn[j][1])
            xs = np.arange(rect_attn[j][2], rect_attn[j][3])
            a0, a1, _ = resize_taps(ys, ratio, Hp)
            b0, b1, _ = resize_taps(xs, ratio, Wp)
            need = (int(a0.min()), int(a1.max()) + 1, int(b0.min()), int(b1.max()) + 1)
    return rect_attn, rect_out


def make_fetchers(cfg, scene, W):
    """Level-k texel fetchers of every view; with the ray directional encoding on, the fetched
    update features are F_k + gamma_k (reading: the encoding is added to the image features; the
    encoding is computed at the coarsest level the network uses)."""
    k0 = max(cfg.levels())
    ray = getattr(cfg, "ray_encoding", 0)

    def gamma(m, k):
        if not ray:
            return None
        Wr = np.asarray(W[f"W_ray_{k}"], np.float64)
        return lambda box: ray_gamma(scene.cams[m], scene.target, k0, k, cfg.near, cfg.far, Wr, box)

    return {k: [LevelFetch(scene.images[m], np.asarray(W["enc_w"], np.float64),
                           np.asarray(W["enc_b"], np.float64), k, gamma(m, k)) for m in range(len(scene.cams))]
            for k in cfg.levels()}


def forward(cfg, W, scene, out_rect: Optional[Rect] = None, mode: int = 0):
    """Novel-view RGBA on out_rect (default: the whole frame) plus every scale's step result."""
    if out_rect is None:
        out_rect = (0, cfg.out_h, 0, cfg.out_w)
    rect_attn, rect_out = plan_rects(cfg, out_rect)
    fetchers = make_fetchers(cfg, scene, W)
    refine = getattr(cfg, "render_refine", 0)
    if refine:
        assert out_rect == (0, cfg.out_h, 0, cfg.out_w), "render-and-refine renders whole views: whole frames only"
    steps: List[StepResult] = []
    prev = None
    delta = None  # update features of the current Update & Fuse step (render-and-refine)
    for j in range(cfg.n_scales):
        if refine and cfg.refines(j):
            delta = refine_features(cfg, W, scene, fetchers, j, prev)
        prev = update_fuse_step(cfg, W, scene, fetchers, j, prev, rect_attn[j], rect_out[j],
                                last=(j == cfg.n_scales - 1), mode=mode, delta_fetch=delta)
        steps.append(prev)
    rgba = render_rect(cfg, scene, steps[-1], out_rect)
    return rgba, steps


def encode_pyramid(cfg, W, scene) -> Dict[int, np.ndarray]:
    """All levels of all views, {k: [V, H/k, W/k, C]} (small cases)."""
    return {k: np.stack([encode_level(scene.images[m], np.asarray(W["enc_w"], np.float64),
                                      np.asarray(W["enc_b"], np.float64), k)
                         for m in range(len(scene.cams))]) for k in cfg.levels()}
