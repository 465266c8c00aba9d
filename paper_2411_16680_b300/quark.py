"""Python binding of libquark.so (include/quark.h).  Argument marshalling only: every step of the
path runs in the library's CUDA kernels.  Device buffers are torch CUDA tensors (or any object
with data_ptr()); host buffers are numpy arrays or CPU tensors (pinned for asynchronous copies).

The names mirror the C ABI: Context.encode_pyramid -> quark_encode_pyramid, etc.
"""
from __future__ import annotations

import ctypes as ct
import os
import weakref
from typing import Dict, List, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libquark.so")

MAX_SCALES = 32
MAX_VIEWS = 64

OK, EINVAL, ENOMEM, ECUDA, EAGAIN, ETIMEDOUT, ENOTFOUND, EBUSY, EINTERNAL = range(9)
FP32, BF16 = 0, 1
FIELD_VOLUME, FIELD_VOLUME_ATTN, FIELD_COLOUR, FIELD_ALPHA, FIELD_DEPTH, FIELD_BETA_LOGITS, \
    FIELD_DEPTH_LOGIT, FIELD_DENSITY_LOGIT = range(8)


class QuarkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"quark status {status}: {msg}")
        self.status = status


class Camera(ct.Structure):
    _fields_ = [("width", ct.c_int), ("height", ct.c_int), ("fx", ct.c_double), ("fy", ct.c_double),
                ("cx", ct.c_double), ("cy", ct.c_double), ("R", ct.c_double * 9), ("t", ct.c_double * 3)]


class Config(ct.Structure):
    _fields_ = [("C", ct.c_int), ("heads", ct.c_int), ("n_scales", ct.c_int), ("k", ct.c_int * MAX_SCALES),
                ("L", ct.c_int * MAX_SCALES), ("near_m", ct.c_float), ("far_m", ct.c_float),
                ("precision", ct.c_int), ("attn_mode", ct.c_int), ("ray_encoding", ct.c_int),
                ("render_refine", ct.c_int), ("scale_heads", ct.c_int * MAX_SCALES), ("ldm_f", ct.c_float * MAX_SCALES),
                ("reuse_depth", ct.c_int * MAX_SCALES), ("model_width", ct.c_int), ("model_height", ct.c_int),
                ("conv_kernel", ct.c_int),
                ("hbm_cap_bytes", ct.c_size_t)]


_FP = ct.POINTER(ct.c_float)
_PER = ct.POINTER(ct.c_float) * MAX_SCALES


class Weights(ct.Structure):
    _fields_ = [("enc_w", _FP), ("enc_b", _FP), ("v0", _FP), ("attn_g", _PER), ("Wq", _PER), ("Wo", _PER),
                ("conv_g", _PER), ("conv1_w", _PER), ("conv1_b", _PER), ("conv2_w", _PER), ("conv2_b", _PER),
                ("col_w1", _PER), ("col_b1", _PER), ("col_w2", _PER), ("col_b2", _PER),
                ("w_d", _FP), ("b_d", ct.c_float), ("w_sigma", _FP), ("b_sigma", ct.c_float),
                ("W_a", _FP), ("b_a", _FP), ("W_beta", _FP),
                ("Wq_std", _PER), ("Wk_std", _PER), ("Wv_std", _PER), ("Wo_std", _PER),
                ("W_ray", _FP * 4),
                ("upd_Wr", _PER), ("upd_br", _PER), ("upd_g", _PER), ("upd1_w", _PER), ("upd1_b", _PER),
                ("upd2_w", _PER), ("upd2_b", _PER)]


class ServeConfig(ct.Structure):
    _fields_ = [("n_slots", ct.c_int), ("queue_capacity", ct.c_int), ("hbm_cap_bytes", ct.c_size_t)]


class Request(ct.Structure):
    _fields_ = [("timestep", ct.c_int), ("target", Camera), ("n_views", ct.c_int), ("rgba", ct.c_void_p),
                ("user_tag", ct.c_uint64)]


class Result(ct.Structure):
    _fields_ = [("status", ct.c_int), ("cancelled", ct.c_int), ("user_tag", ct.c_uint64), ("queue_ms", ct.c_double),
                ("gpu_ms", ct.c_double), ("total_ms", ct.c_double)]


class Stats(ct.Structure):
    _fields_ = [("submitted", ct.c_uint64), ("completed", ct.c_uint64), ("failed", ct.c_uint64),
                ("cancelled", ct.c_uint64), ("rejected", ct.c_uint64), ("in_flight", ct.c_int), ("queued", ct.c_int),
                ("p50_ms", ct.c_double), ("p99_ms", ct.c_double), ("mean_ms", ct.c_double), ("fps", ct.c_double),
                ("hbm_in_use", ct.c_size_t), ("hbm_high_water", ct.c_size_t)]


STAGE_GRAD_FIELDS = ("attn_g", "Wq", "Wo", "W_beta", "conv_g", "conv1_w", "conv1_b", "conv2_w", "conv2_b", "w_d",
                     "b_d", "w_sigma", "b_sigma")


class StageGrads(ct.Structure):
    _fields_ = [(n, ct.c_void_p) for n in STAGE_GRAD_FIELDS]


# quark_grads: whole-network weight gradients (shared fields, then per-step arrays)
GRAD_SHARED_HEAD = ("enc_w", "enc_b", "v0")
GRAD_PER_STEP = ("attn_g", "Wq", "Wo", "conv_g", "conv1_w", "conv1_b", "conv2_w", "conv2_b", "col_w1", "col_b1",
                 "col_w2", "col_b2")
GRAD_SHARED_TAIL = ("w_d", "b_d", "w_sigma", "b_sigma", "W_beta")


class Grads(ct.Structure):
    _fields_ = ([(n, ct.c_void_p) for n in GRAD_SHARED_HEAD] +
                [(n, ct.c_void_p * MAX_SCALES) for n in GRAD_PER_STEP] +
                [(n, ct.c_void_p) for n in GRAD_SHARED_TAIL])


def make_grads(grads: Dict) -> Grads:
    """quark_grads from a dict of device tensors keyed by make_weights names (e.g. "Wq_1", "w_d");
    absent names are NULL."""
    g = Grads()
    for n in GRAD_SHARED_HEAD + GRAD_SHARED_TAIL:
        if n in grads:
            setattr(g, n, _ptr(grads[n]))
    for n in GRAD_PER_STEP:
        arr = getattr(g, n)
        for j in range(MAX_SCALES):
            key = f"{n}_{j}"
            if key in grads:
                arr[j] = _ptr(grads[key])
    return g


_lib = None


def lib():
    """The loaded library; raises when it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2411_16680_b300.build`")
        L = ct.CDLL(LIB_PATH)
        vp = ct.c_void_p
        sig = {
            "quark_create": ([ct.POINTER(Config), ct.c_int, ct.POINTER(vp)], ct.c_int),
            "quark_destroy": ([vp], ct.c_int),
            "quark_load_weights": ([vp, ct.POINTER(Weights)], ct.c_int),
            "quark_encode_pyramid": ([vp, vp, ct.POINTER(Camera), ct.c_int, vp, ct.POINTER(vp)], ct.c_int),
            "quark_ldm_create": ([vp, ct.POINTER(Camera), ct.POINTER(vp)], ct.c_int),
            "quark_update_fuse": ([vp, vp, ct.c_int, vp, vp], ct.c_int),
            "quark_render_ldm": ([vp, vp, vp, vp, vp], ct.c_int),
            "quark_render_novel_view": ([vp, vp, vp, vp, vp], ct.c_int),
            "quark_render_depth": ([vp, vp, vp, vp], ct.c_int),
            "quark_ldm_read": ([vp, ct.c_int, vp, ct.c_size_t], ct.c_int),
            "quark_ldm_field_bytes": ([vp, ct.c_int], ct.c_size_t),
            "quark_release_pyramid": ([vp], ct.c_int),
            "quark_release_ldm": ([vp], ct.c_int),
            "quark_last_error": ([vp], ct.c_char_p),
            "quark_launch_count": ([vp], ct.c_uint64),
            "quark_reset_counters": ([vp], None),
            "quark_set_profiling": ([vp, ct.c_int], ct.c_int),
            "quark_kernel_times": ([vp, ct.POINTER(ct.c_char_p), ct.POINTER(ct.c_double), ct.POINTER(ct.c_uint64),
                                    ct.c_int], ct.c_int),
            "quark_check_device": ([vp], ct.c_int),
            "quark_pyramid_read": ([vp, ct.c_int, vp, ct.c_size_t], ct.c_int),
            "quark_step_input": ([vp, vp, ct.c_int, vp, vp], ct.c_int),
            "quark_stage_forward": ([vp, vp, vp, vp, vp, vp, vp], ct.c_int),
            "quark_stage_backward": ([vp, vp, vp, vp, vp, vp, vp, vp, ct.POINTER(StageGrads), vp], ct.c_int),
            "quark_serve_start": ([vp, ct.POINTER(ServeConfig), ct.POINTER(vp)], ct.c_int),
            "quark_serve_set_timestep": ([vp, ct.c_int, vp, ct.POINTER(Camera), ct.c_int], ct.c_int),
            "quark_serve_submit": ([vp, ct.POINTER(Request), ct.POINTER(ct.c_uint64)], ct.c_int),
            "quark_serve_poll": ([vp, ct.c_uint64, ct.c_int, ct.POINTER(Result)], ct.c_int),
            "quark_serve_cancel": ([vp, ct.c_uint64], ct.c_int),
            "quark_serve_pause": ([vp, ct.c_int], ct.c_int),
            "quark_serve_stats": ([vp, ct.POINTER(Stats)], ct.c_int),
            "quark_serve_stop": ([vp], ct.c_int),
            "quark_update_fuse_noalloc": ([vp, vp, ct.c_int, ct.POINTER(Camera), vp, vp, vp, vp, vp, vp, vp, vp, vp],
                                          ct.c_int),
            "quark_sample_coords": ([vp, ct.POINTER(Camera), ct.c_double, ct.c_double, ct.POINTER(Camera), ct.c_double,
                                     ct.c_int, vp, vp, vp, vp, vp, vp], ct.c_int),
            "quark_test_wait_timeout": ([vp], ct.c_int),
            "quark_measure_fp32_peak": ([ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)], ct.c_int),
            "quark_ldm_keep_steps": ([vp, ct.c_int], ct.c_int),
            "quark_render_ldm_bwd": ([vp, vp, vp, vp, vp, vp, ct.POINTER(Grads), vp], ct.c_int),
            "quark_update_fuse_bwd": ([vp, vp, ct.c_int, vp, vp, vp, vp, vp, ct.POINTER(Grads), vp], ct.c_int),
            "quark_encode_pyramid_bwd": ([vp, vp, ct.POINTER(vp), ct.POINTER(Grads), vp], ct.c_int),
            "quark_conv_tiles": ([vp, ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)],
                                 ct.c_int),
            "quark_tensor_core_paths": ([vp, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)], ct.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols() -> List[str]:
    return [n for n in ("quark_create", "quark_destroy", "quark_load_weights", "quark_encode_pyramid",
                        "quark_ldm_create", "quark_update_fuse", "quark_render_ldm", "quark_render_novel_view",
                        "quark_render_depth",
                        "quark_ldm_read", "quark_ldm_field_bytes", "quark_release_pyramid", "quark_release_ldm",
                        "quark_last_error", "quark_launch_count", "quark_reset_counters", "quark_set_profiling",
                        "quark_kernel_times")]


def measure_fp32_peak(device: int = 0):
    """quark_measure_fp32_peak: (scalar FMA, packed FP32x2 FMA) TFLOP/s of the device's FP32 lanes."""
    a, b = ct.c_double(0.0), ct.c_double(0.0)
    _check(lib().quark_measure_fp32_peak(device, ct.byref(a), ct.byref(b)))
    return a.value, b.value


def _check(status: int, ctx=None):
    if status != OK:
        msg = lib().quark_last_error(ctx)
        raise QuarkError(status, msg.decode() if msg else "")


def make_camera(cam) -> Camera:
    c = Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float64).reshape(9)
    t = np.asarray(cam.t, np.float64).reshape(3)
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
    return c


def make_config(cfg, hbm_cap_bytes: int = 0) -> Config:
    c = Config()
    c.C, c.heads, c.n_scales = cfg.C, cfg.heads, len(cfg.scales)
    for j, (k, L) in enumerate(cfg.scales):
        c.k[j], c.L[j] = k, L
    c.near_m, c.far_m = cfg.near, cfg.far
    c.precision = cfg.precision
    c.attn_mode = cfg.attn_mode
    c.ray_encoding = getattr(cfg, "ray_encoding", 0)
    c.render_refine = getattr(cfg, "render_refine", 0)
    # model schedule: per-step heads (0 in the workload = a block without attention, -1 here),
    # LDM grid factors and reused depths; unset = the uniform schedule (zero-filled)
    if getattr(cfg, "scale_heads", None) is not None:
        for j, h in enumerate(cfg.scale_heads):
            c.scale_heads[j] = int(h) if int(h) > 0 else -1
    if getattr(cfg, "ldm_f", None) is not None:
        for j, f in enumerate(cfg.ldm_f):
            c.ldm_f[j] = float(f)
    if getattr(cfg, "reuse_depth", None) is not None:
        for j, r in enumerate(cfg.reuse_depth):
            c.reuse_depth[j] = int(r)
    if getattr(cfg, "model_w", None):
        c.model_width, c.model_height = int(cfg.model_w), int(cfg.model_h)
    c.conv_kernel = int(getattr(cfg, "conv_kernel", 3))
    c.hbm_cap_bytes = hbm_cap_bytes
    return c


def _ptr(x) -> int:
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Pyramid:
    def __init__(self, ctx: "Context", handle: ct.c_void_p, V: int):
        self.ctx, self.handle, self.V = ctx, handle, V
        ctx._handles.add(self)

    def read_level(self, k: int, dst):
        """Copy level k into dst (a tensor or array of exactly the level's size)."""
        n = dst.numel() * dst.element_size() if hasattr(dst, "numel") else dst.nbytes
        _check(lib().quark_pyramid_read(self.handle, k, _ptr(dst), n), self.ctx.handle)

    def release(self):
        # a pyramid outlives no context: Context.close() releases it first
        if self.handle and getattr(self.ctx, "handle", None):
            lib().quark_release_pyramid(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class LDM:
    def __init__(self, ctx: "Context", handle: ct.c_void_p):
        self.ctx, self.handle = ctx, handle
        ctx._handles.add(self)

    def keep_steps(self, keep: bool = True):
        """quark_ldm_keep_steps: keep every step's volumes for the backward pass."""
        _check(lib().quark_ldm_keep_steps(self.handle, int(keep)), self.ctx.handle)

    def field_bytes(self, field: int) -> int:
        return lib().quark_ldm_field_bytes(self.handle, field)

    def read(self, field: int, shape=None) -> np.ndarray:
        n = self.field_bytes(field)
        out = np.empty(n // 4, np.float32)
        _check(lib().quark_ldm_read(self.handle, field, out.ctypes.data, n), self.ctx.handle)
        return out if shape is None else out.reshape(shape)

    def release(self):
        if self.handle and getattr(self.ctx, "handle", None):
            lib().quark_release_ldm(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Context:
    """quark_ctx: one network configuration and its weights on one device."""

    def __init__(self, cfg, device: int = 0, hbm_cap_bytes: int = 0):
        self.cfg = cfg
        self._handles = weakref.WeakSet()  # live Pyramid / LDM objects, released by close()
        self._ccfg = make_config(cfg, hbm_cap_bytes)
        h = ct.c_void_p()
        _check(lib().quark_create(ct.byref(self._ccfg), device, ct.byref(h)))
        self.handle = h

    def close(self):
        """quark_destroy, after releasing every pyramid and LDM made from this context (the library
        refuses to destroy a context whose handles are alive)."""
        if getattr(self, "handle", None):
            for h in list(getattr(self, "_handles", ())):
                h.release()
            lib().quark_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return lib().quark_last_error(self.handle).decode()

    def load_weights(self, W: Dict[str, np.ndarray]):
        keep = {}

        def p(name):
            a = np.ascontiguousarray(W[name], np.float32)
            keep[name] = a
            return a.ctypes.data_as(_FP)

        w = Weights()
        w.enc_w, w.enc_b, w.v0 = p("enc_w"), p("enc_b"), p("v0")
        n = len(self.cfg.scales)
        for j in range(n):
            if f"Wq_{j}" in W:  # absent for a block without attention
                w.attn_g[j], w.Wq[j], w.Wo[j] = p(f"attn_g_{j}"), p(f"Wq_{j}"), p(f"Wo_{j}")
            w.conv_g[j], w.conv1_w[j], w.conv1_b[j] = p(f"conv_g_{j}"), p(f"conv1_w_{j}"), p(f"conv1_b_{j}")
            w.conv2_w[j], w.conv2_b[j] = p(f"conv2_w_{j}"), p(f"conv2_b_{j}")
            if f"col_w1_{j}" in W:
                w.col_w1[j], w.col_b1[j] = p(f"col_w1_{j}"), p(f"col_b1_{j}")
                w.col_w2[j], w.col_b2[j] = p(f"col_w2_{j}"), p(f"col_b2_{j}")
            if f"upd_Wr_{j}" in W:  # render-and-refine: the step's Update Block
                w.upd_Wr[j], w.upd_br[j], w.upd_g[j] = p(f"upd_Wr_{j}"), p(f"upd_br_{j}"), p(f"upd_g_{j}")
                w.upd1_w[j], w.upd1_b[j] = p(f"upd1_w_{j}"), p(f"upd1_b_{j}")
                w.upd2_w[j], w.upd2_b[j] = p(f"upd2_w_{j}"), p(f"upd2_b_{j}")
            if f"Wq_std_{j}" in W:
                w.Wq_std[j], w.Wk_std[j] = p(f"Wq_std_{j}"), p(f"Wk_std_{j}")
                w.Wv_std[j], w.Wo_std[j] = p(f"Wv_std_{j}"), p(f"Wo_std_{j}")
        w.w_d, w.w_sigma, w.W_a, w.b_a, w.W_beta = p("w_d"), p("w_sigma"), p("W_a"), p("b_a"), p("W_beta")
        for i, k in enumerate((1, 2, 4, 8)):
            if f"W_ray_{k}" in W:
                w.W_ray[i] = p(f"W_ray_{k}")
        w.b_d = float(np.asarray(W["b_d"]).reshape(-1)[0])
        w.b_sigma = float(np.asarray(W["b_sigma"]).reshape(-1)[0])
        _check(lib().quark_load_weights(self.handle, ct.byref(w)), self.handle)

    def encode_pyramid(self, images, cams: Sequence, stream=None, into: Optional[Pyramid] = None) -> Pyramid:
        """images: [V, H, W, 3] float32, device tensor or host array/tensor.  `into` re-encodes an
        existing pyramid in place (same V and resolution) instead of allocating a new one."""
        V = len(cams)
        arr = (Camera * V)(*[make_camera(c) for c in cams])
        h = ct.c_void_p(into.handle.value if into is not None else None)
        _check(lib().quark_encode_pyramid(self.handle, _ptr(images), arr, V, _stream(stream), ct.byref(h)),
               self.handle)
        return into if into is not None else Pyramid(self, h, V)

    def ldm_create(self, target) -> LDM:
        cam = make_camera(target)
        h = ct.c_void_p()
        _check(lib().quark_ldm_create(self.handle, ct.byref(cam), ct.byref(h)), self.handle)
        return LDM(self, h)

    def update_fuse(self, pyr: Pyramid, scale: int, ldm: LDM, stream=None):
        _check(lib().quark_update_fuse(self.handle, pyr.handle, scale, ldm.handle, _stream(stream)), self.handle)

    def update_fuse_noalloc(self, pyr: Pyramid, scale: int, target, v_prev, v_out, colour, alpha, depth, t_raw,
                            s_raw, beta=None, stream=None):
        """quark_update_fuse_noalloc: one step on caller-owned device buffers; the library allocates
        nothing (its intermediates use a fixed static device array, see quark.h)."""
        cam = make_camera(target)
        p = lambda x: None if x is None else _ptr(x)
        _check(lib().quark_update_fuse_noalloc(self.handle, pyr.handle, scale, ct.byref(cam), p(v_prev), p(v_out),
                                               p(colour), p(alpha), p(depth), p(t_raw), p(s_raw), p(beta),
                                               _stream(stream)), self.handle)

    def render_ldm(self, ldm: LDM, pyr: Pyramid, rgba, stream=None):
        _check(lib().quark_render_ldm(self.handle, ldm.handle, pyr.handle, _ptr(rgba), _stream(stream)), self.handle)

    def render_depth(self, ldm: LDM, depth, stream=None):
        """Depth map [H_out, W_out] of the solved LDM (device tensor or host array)."""
        _check(lib().quark_render_depth(self.handle, ldm.handle, _ptr(depth), _stream(stream)), self.handle)

    def render_novel_view(self, pyr: Pyramid, ldm: LDM, rgba, stream=None):
        _check(lib().quark_render_novel_view(self.handle, pyr.handle, ldm.handle, _ptr(rgba), _stream(stream)),
               self.handle)

    # ---- differentiable stage (FP32): last Update & Fuse step + render ----
    def step_input(self, ldm: LDM, scale: int, v_in, stream=None):
        _check(lib().quark_step_input(self.handle, ldm.handle, scale, _ptr(v_in), _stream(stream)), self.handle)

    def stage_forward(self, pyr: Pyramid, feat, v_in, ldm: LDM, rgba, stream=None):
        _check(lib().quark_stage_forward(self.handle, pyr.handle, _ptr(feat), _ptr(v_in), ldm.handle, _ptr(rgba),
                                         _stream(stream)), self.handle)

    def stage_backward(self, pyr: Pyramid, feat, v_in, ldm: LDM, dl_drgb, dv_in, dfeat, grads: Dict, stream=None):
        g = StageGrads(*[_ptr(grads[n]) for n in STAGE_GRAD_FIELDS])
        _check(lib().quark_stage_backward(self.handle, pyr.handle, _ptr(feat), _ptr(v_in), ldm.handle, _ptr(dl_drgb),
                                          _ptr(dv_in), _ptr(dfeat), ct.byref(g), _stream(stream)), self.handle)

    # ---- backward pass through the whole network ----
    def render_ldm_bwd(self, ldm: LDM, pyr: Pyramid, dl_drgb, dv_out, dbeta, grads: Dict, stream=None):
        """quark_render_ldm_bwd: writes dv_out, dbeta; accumulates the decoder gradients in `grads`."""
        g = make_grads(grads)
        _check(lib().quark_render_ldm_bwd(self.handle, ldm.handle, pyr.handle, _ptr(dl_drgb), _ptr(dv_out),
                                          _ptr(dbeta), ct.byref(g), _stream(stream)), self.handle)

    def update_fuse_bwd(self, pyr: Pyramid, scale: int, ldm: LDM, dv_out, dbeta, dv_prev, dfeat, grads: Dict,
                        stream=None):
        """quark_update_fuse_bwd: writes dv_prev; accumulates dfeat and the step's weight gradients."""
        g = make_grads(grads)
        p = lambda x: None if x is None else _ptr(x)
        _check(lib().quark_update_fuse_bwd(self.handle, pyr.handle, scale, ldm.handle, _ptr(dv_out), p(dbeta),
                                           p(dv_prev), _ptr(dfeat), ct.byref(g), _stream(stream)), self.handle)

    def encode_pyramid_bwd(self, pyr: Pyramid, dfeat: Dict, grads: Dict, stream=None):
        """quark_encode_pyramid_bwd: dfeat maps pyramid factors k (1, 2, 4, 8) to level gradients;
        accumulates enc_w, enc_b in `grads`."""
        arr = (ct.c_void_p * 4)(*[_ptr(dfeat[k]) if k in dfeat else None for k in (1, 2, 4, 8)])
        g = make_grads(grads)
        _check(lib().quark_encode_pyramid_bwd(self.handle, pyr.handle, arr, ct.byref(g), _stream(stream)),
               self.handle)

    def sample_coords(self, target, k_tx: float, k_ty: float, view, k_m: float, px, py, depth):
        """quark_sample_coords: (u, v) [n, 2] float32, tap origins [n, 2] int32 and validity [n] of target
        grid pixel centres (px, py) at depths `depth` in `view`'s level-k_m grid, as the kernels compute them."""
        px, py, depth = (np.ascontiguousarray(x, np.float32).ravel() for x in (px, py, depth))
        n = px.size
        uv = np.zeros((n, 2), np.float32)
        taps = np.zeros((n, 2), np.int32)
        valid = np.zeros(n, np.int32)
        t, v = make_camera(target), make_camera(view)
        _check(lib().quark_sample_coords(self.handle, ct.byref(t), k_tx, k_ty, ct.byref(v), k_m, n, _ptr(px), _ptr(py),
                                         _ptr(depth), _ptr(uv), _ptr(taps), _ptr(valid)), self.handle)
        return uv, taps, valid

    def conv_tiles(self, L: int, H: int, W: int):
        """quark_conv_tiles: (columns, rows) of the conv-block kernel's output tile for an L x H x W volume."""
        cols, rows = ct.c_int(0), ct.c_int(0)
        _check(lib().quark_conv_tiles(self.handle, L, H, W, ct.byref(cols), ct.byref(rows)), self.handle)
        return cols.value, rows.value

    def tensor_core_paths(self):
        """quark_tensor_core_paths: (attend, conv) -- whether the sampling kernel's projections and the
        conv block's convolutions run on the tensor cores for the loaded weights."""
        at, cv = ct.c_int(0), ct.c_int(0)
        _check(lib().quark_tensor_core_paths(self.handle, ct.byref(at), ct.byref(cv)), self.handle)
        return bool(at.value), bool(cv.value)

    def test_wait_timeout(self):
        """quark_test_wait_timeout: the next BF16 sampling launch's bounded wait runs out (error-path test)."""
        _check(lib().quark_test_wait_timeout(self.handle), self.handle)

    def check_device(self):
        """Synchronise and raise if a kernel's bounded device-side wait ran out."""
        _check(lib().quark_check_device(self.handle), self.handle)

    # ---- accounting ----
    def launch_count(self) -> int:
        return int(lib().quark_launch_count(self.handle))

    def reset_counters(self):
        lib().quark_reset_counters(self.handle)

    def set_profiling(self, on: bool):
        _check(lib().quark_set_profiling(self.handle, 1 if on else 0), self.handle)

    def kernel_times(self) -> Dict[str, tuple]:
        cap = 16
        names = (ct.c_char_p * cap)()
        ms = (ct.c_double * cap)()
        n = (ct.c_uint64 * cap)()
        k = lib().quark_kernel_times(self.handle, names, ms, n, cap)
        return {names[i].decode(): (int(n[i]), float(ms[i])) for i in range(k)}


class Server:
    """quark_server: continuous-batching request loop over resident time steps (see quark.h)."""

    def __init__(self, ctx: Context, n_slots: int = 8, queue_capacity: int = 1024, hbm_cap_bytes: int = 0):
        self.ctx = ctx
        cfg = ServeConfig(n_slots, queue_capacity, hbm_cap_bytes)
        h = ct.c_void_p()
        _check(lib().quark_serve_start(ctx.handle, ct.byref(cfg), ct.byref(h)), ctx.handle)
        self.handle = h

    def set_timestep(self, timestep: int, images, cams: Sequence):
        V = len(cams)
        arr = (Camera * V)(*[make_camera(c) for c in cams])
        _check(lib().quark_serve_set_timestep(self.handle, timestep, _ptr(images), arr, V), self.ctx.handle)

    def submit(self, timestep: int, target, n_views: int, rgba, user_tag: int = 0) -> int:
        req = Request(timestep, make_camera(target), n_views, _ptr(rgba), user_tag)
        t = ct.c_uint64()
        _check(lib().quark_serve_submit(self.handle, ct.byref(req), ct.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0) -> Optional[Result]:
        """The ticket's result, or None if not done within timeout_us (EAGAIN / ETIMEDOUT)."""
        r = Result()
        st = lib().quark_serve_poll(self.handle, ticket, timeout_us, ct.byref(r))
        if st in (EAGAIN, ETIMEDOUT):
            return None
        _check(st)
        return r

    def cancel(self, ticket: int):
        _check(lib().quark_serve_cancel(self.handle, ticket))

    def pause(self, paused: bool):
        _check(lib().quark_serve_pause(self.handle, 1 if paused else 0))

    def stats(self) -> Stats:
        st = Stats()
        _check(lib().quark_serve_stats(self.handle, ct.byref(st)))
        return st

    def stop(self):
        if getattr(self, "handle", None):
            lib().quark_serve_stop(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
