// Device helpers shared by the kernels: storage-type vector loads/stores (FP32 or BF16
// storage, FP32 arithmetic), the depth activation, and the bilinear tap rule.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <math.h>

#include "quark_internal.cuh"

namespace quark {

// ---- division by a launch constant -----------------------------------------------------------
// n / d for 0 <= n < 2^31 by a multiply-high with a magic number m and shift l computed on the host
// for the divisor d (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994: l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1), instead of a
// runtime integer division (a few instructions against a couple of dozen).
struct FastDiv {
    uint32_t d, m, l;
};
static inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    return FastDiv{d, (uint32_t)m, l};
}
__device__ __forceinline__ int fdiv(int n, const FastDiv& q) {
    return (int)((__umulhi((uint32_t)n, q.m) + (uint32_t)n) >> q.l);
}

// ---- 16-channel vector loads/stores in the storage type --------------------------------------

// 32 bytes of read-only data in one 256-bit load (sm_100 family; global memory only; `p` 32-byte
// aligned): a whole L1 sector per thread, half the load instructions of two 128-bit loads.
__device__ __forceinline__ void ldg256(const void* p, uint4& a, uint4& b) {
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                 : "l"(p));
}

// 32 bytes stored in one 256-bit store (sm_100 family; global memory only; `p` 32-byte aligned);
// stcs256 with the streaming (evict-first) hint, for data the next kernel reads once.
__device__ __forceinline__ void stg256(void* p, const uint4& a, const uint4& b) {
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(a.x), "r"(a.y), "r"(a.z),
                 "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
                 : "memory");
}
__device__ __forceinline__ void stcs256(void* p, const uint4& a, const uint4& b) {
    asm volatile("st.global.cs.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(a.x), "r"(a.y), "r"(a.z),
                 "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
                 : "memory");
}

__device__ __forceinline__ void load16(const float* __restrict__ p, float (&o)[16]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float4 v = __ldg(q + i);
        o[4 * i + 0] = v.x; o[4 * i + 1] = v.y; o[4 * i + 2] = v.z; o[4 * i + 3] = v.w;
    }
}

__device__ __forceinline__ void load16(const __nv_bfloat16* __restrict__ p, float (&o)[16]) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        uint4 v = __ldg(q + i);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float2 f = __bfloat1622float2(h[j]);
            o[8 * i + 2 * j] = f.x;
            o[8 * i + 2 * j + 1] = f.y;
        }
    }
}

// accumulate w * p[0..16) into o
__device__ __forceinline__ void fma16(const float* __restrict__ p, float w, float (&o)[16]) {
    float t[16];
    load16(p, t);
#pragma unroll
    for (int i = 0; i < 16; ++i) o[i] = fmaf(w, t[i], o[i]);
}
__device__ __forceinline__ void fma16(const __nv_bfloat16* __restrict__ p, float w, float (&o)[16]) {
    float t[16];
    load16(p, t);
#pragma unroll
    for (int i = 0; i < 16; ++i) o[i] = fmaf(w, t[i], o[i]);
}

__device__ __forceinline__ void store16(float* p, const float (&v)[16]) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

__device__ __forceinline__ void store16(__nv_bfloat16* p, const float (&v)[16]) {
    uint4 u[2];
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(u);
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    uint4* q = reinterpret_cast<uint4*>(p);
    q[0] = u[0];
    q[1] = u[1];
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ void from_f(float& d, float x) { d = x; }
__device__ __forceinline__ void from_f(__nv_bfloat16& d, float x) { d = __float2bfloat16_rn(x); }

// acc[0..16) += a * r[0..16) with r 16-byte aligned (shared-memory weight rows)
__device__ __forceinline__ void fma_row16(const float* r, float a, float (&acc)[16]) {
    const float4* r4 = reinterpret_cast<const float4*>(r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float4 w = r4[i];
        acc[4 * i + 0] = fmaf(a, w.x, acc[4 * i + 0]);
        acc[4 * i + 1] = fmaf(a, w.y, acc[4 * i + 1]);
        acc[4 * i + 2] = fmaf(a, w.z, acc[4 * i + 2]);
        acc[4 * i + 3] = fmaf(a, w.w, acc[4 * i + 3]);
    }
}

// ---- elementwise definitions ------------------------------------------------------------------

// Eq. (depth_activation): d = 1 / ((delta + 0.5/L tanh t) (1/near - 1/far) + 1/far),
// delta = (l - 0.5) / L with l = li + 1.
__device__ __forceinline__ float depth_from_logit(float t, int li, int L, DepthParams dp) {
    float delta = (li + 0.5f) / L;
    return 1.0f / fmaf(delta + 0.5f / L * tanhf(t), dp.span, dp.inv_far);
}
__device__ __forceinline__ float depth_anchor(int li, int L, DepthParams dp) {
    return 1.0f / fmaf((li + 0.5f) / L, dp.span, dp.inv_far);
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// erf-GELU of two values on packed FP32x2 arithmetic, for the BF16 form (whose outputs are rounded
// to BF16): gelu(x) = x Phi(x), Phi(x) = 0.5 + x S(x^2), with S a degree-11 least-squares
// polynomial in t = 2 x^2 / 25 - 1 for |x| <= 5; beyond, x^2 is clamped to 25 and Phi saturates
// to 1 or 0.  Maximum absolute error 3.6e-6 against the exact erf form (coefficients and error
// from gen_gelu_poly.py).
// GELU in its tanh form (Hendrycks & Gimpel, 2016), 0.5 x (1 + tanh(sqrt(2 / pi) (x + 0.044715 x^3))),
// on packed FP32x2 with the tanh on the special-function unit (PTX tanh.approx).  It stays within
// 5e-4 of the erf form everywhere (4.7e-4 at x = 2.7, where a BF16 value's half-ulp is 5.3e-3), so
// the BF16 form uses it where the result is rounded to BF16 (the conv block's mid tile).
__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 gelu_tanh2(float2 x) {
    constexpr float K0 = 0.7978845608028654f;    // sqrt(2 / pi)
    constexpr float K1 = 0.035677408136300125f;  // 0.044715 sqrt(2 / pi)
    const float2 x2 = __fmul2_rn(x, x);
    const float2 inner = __fmul2_rn(x, __ffma2_rn(x2, make_float2(K1, K1), make_float2(K0, K0)));
    const float2 hx = __fmul2_rn(x, make_float2(0.5f, 0.5f));
    return __ffma2_rn(hx, make_float2(tanh_approx(inner.x), tanh_approx(inner.y)), hx);
}

__device__ __forceinline__ float2 gelu_poly2(float2 x) {
    constexpr float c[12] = {1.413636357e-01f, -7.029806077e-02f, 5.153302103e-02f, -4.040101916e-02f,
                             3.127557412e-02f, -2.353477105e-02f, 1.720164344e-02f, -1.048013940e-02f,
                             4.697760567e-03f, -3.445686540e-03f, 3.397131106e-03f, -1.309263054e-03f};
    float2 u = __fmul2_rn(x, x);
    u.x = fminf(u.x, 25.f);
    u.y = fminf(u.y, 25.f);
    const float2 t = __ffma2_rn(u, make_float2(0.08f, 0.08f), make_float2(-1.f, -1.f));
    float2 acc = make_float2(c[11], c[11]);
#pragma unroll
    for (int i = 10; i >= 0; --i) acc = __ffma2_rn(acc, t, make_float2(c[i], c[i]));
    float2 phi = __ffma2_rn(x, acc, make_float2(0.5f, 0.5f));
    phi.x = __saturatef(phi.x);
    phi.y = __saturatef(phi.y);
    return __fmul2_rn(x, phi);
}

// erf-GELU of two values on packed FP32x2 arithmetic, for the FP32 form: the construction of
// gelu_poly2 on |x| <= 6 with a degree-16 polynomial in t = x^2 / 18 - 1, whose error is FP32
// rounding: 8.7e-7 absolute, 2.1e-7 relative to max(1, |x|), against the exact erf form (beyond
// |x| = 6 the exact Phi is within 1e-9 of 0 or 1).  Coefficients and error from gen_gelu_poly.py.
__device__ __forceinline__ float2 gelu_fine2(float2 x) {
    constexpr float c[17] = {1.178485230e-01f, -5.889960751e-02f, 4.406414181e-02f, -3.638968989e-02f,
                             3.108768910e-02f, -2.660531178e-02f, 2.242538892e-02f, -1.841114089e-02f,
                             1.405856665e-02f, -9.705077857e-03f, 7.379670627e-03f, -6.239356007e-03f,
                             3.092317842e-03f, -2.200730378e-04f, 6.576618762e-04f, -1.334174885e-03f,
                             5.238011363e-04f};
    float2 u = __fmul2_rn(x, x);
    u.x = fminf(u.x, 36.f);
    u.y = fminf(u.y, 36.f);
    const float2 t = __ffma2_rn(u, make_float2(1.0f / 18.f, 1.0f / 18.f), make_float2(-1.f, -1.f));
    float2 acc = make_float2(c[16], c[16]);
#pragma unroll
    for (int i = 15; i >= 0; --i) acc = __ffma2_rn(acc, t, make_float2(c[i], c[i]));
    float2 phi = __ffma2_rn(x, acc, make_float2(0.5f, 0.5f));
    phi.x = __saturatef(phi.x);
    phi.y = __saturatef(phi.y);
    return __fmul2_rn(x, phi);
}

// Map target-grid pixel (px, py) at depth d into a view; returns false when the point is
// at or behind the view's camera plane (z <= 1e-6).
__device__ __forceinline__ bool reproject(const ViewMap& m, float px, float py, float d, float& u, float& v) {
    float X = fmaf(d, fmaf(m.A[0], px, fmaf(m.A[1], py, m.A[2])), m.b[0]);
    float Y = fmaf(d, fmaf(m.A[3], px, fmaf(m.A[4], py, m.A[5])), m.b[1]);
    float Z = fmaf(d, fmaf(m.A[6], px, fmaf(m.A[7], py, m.A[8])), m.b[2]);
    if (!(Z > 1e-6f)) return false;
    float iz = 1.0f / Z;
    u = X * iz;
    v = Y * iz;
    return true;
}

// 2^x and 1/x on the special-function unit (PTX ex2.approx / rcp.approx, flush-to-zero).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// reproject with the perspective divide as one reciprocal (the BF16 form's sampling and the render)
__device__ __forceinline__ bool reproject_rcp(const ViewMap& m, float px, float py, float d, float& u, float& v) {
    const float X = fmaf(d, fmaf(m.A[0], px, fmaf(m.A[1], py, m.A[2])), m.b[0]);
    const float Y = fmaf(d, fmaf(m.A[3], px, fmaf(m.A[4], py, m.A[5])), m.b[1]);
    const float Z = fmaf(d, fmaf(m.A[6], px, fmaf(m.A[7], py, m.A[8])), m.b[2]);
    if (!(Z > 1e-6f)) return false;
    const float iz = rcp_approx(Z);
    u = X * iz;
    v = Y * iz;
    return true;
}

// Bilinear taps with zero padding at continuous pixel coordinates (u, v) of an h x w map
// (pixel centres at +0.5).  Returns false when no tap can touch the map (the sample is 0).
struct Taps {
    int x0, y0;
    float fx, fy;
};
__device__ __forceinline__ bool bilinear_taps(float u, float v, int h, int w, Taps& t) {
    float xs = u - 0.5f, ys = v - 0.5f;
    if (!(xs > -1.0f && xs < (float)w && ys > -1.0f && ys < (float)h)) return false;
    float x0 = floorf(xs), y0 = floorf(ys);
    t.fx = xs - x0;
    t.fy = ys - y0;
    t.x0 = (int)x0;
    t.y0 = (int)y0;
    return true;
}

// The same four taps as in-map texel indices (row-major, h x w) and weights.  A tap outside the map,
// or every tap of a sample that cannot touch it (ok false, or no tap inside), keeps an in-map index
// and gets weight zero, so the four fetches need no branch and can be in flight together.
struct Taps4 {
    int i00, i01, i10, i11;
    float w00, w01, w10, w11;
};
__device__ __forceinline__ Taps4 bilinear_taps4(bool ok, float u, float v, int h, int w) {
    Taps t{0, 0, 0.f, 0.f};
    ok = ok && bilinear_taps(u, v, h, w, t);
    const float gx0 = ok && t.x0 >= 0 ? 1 - t.fx : 0.f, gx1 = ok && t.x0 + 1 < w ? t.fx : 0.f;
    const float gy0 = ok && t.y0 >= 0 ? 1 - t.fy : 0.f, gy1 = ok && t.y0 + 1 < h ? t.fy : 0.f;
    const int cx0 = max(t.x0, 0), cx1 = min(t.x0 + 1, w - 1);
    const int ry0 = max(t.y0, 0) * w, ry1 = min(t.y0 + 1, h - 1) * w;
    return Taps4{ry0 + cx0, ry0 + cx1, ry1 + cx0, ry1 + cx1, gy0 * gx0, gy0 * gx1, gy1 * gx0, gy1 * gx1};
}

// Edge-clamped linear taps of a resize by `ratio` (pixel centres aligned; e.g. 2 or 3.75):
// src = (dst + 0.5) / ratio - 0.5.
__device__ __forceinline__ void resize_taps(int dst, float ratio, int n, int& i0, int& i1, float& w1) {
    float src = (dst + 0.5f) / ratio - 0.5f;
    float f = floorf(src);
    w1 = src - f;
    int a = (int)f;
    i0 = min(max(a, 0), n - 1);
    i1 = min(max(a + 1, 0), n - 1);
}

}  // namespace quark
