// Final render (Sec. 3.1 Eq. 1; Sec. 3.2.3 "Upsampling & Activation").  One thread per output
// pixel: bilinear upsample by s of the raw depth / density / blend logits of the last LDM (a
// direct read when s = 1), activation (Eq. depth_activation, sigmoid, softmax over views in one
// online pass on ex2.approx), back-projection of every input image onto each layer (zero padding), blend, and
// the over operator front to back (l = L nearest first): C += T alpha c, T *= (1 - alpha).
// Output RGBA with A = 1 - T.
#include "device_common.cuh"

namespace quark {

constexpr int RD_THREADS = 128;

__device__ __forceinline__ float4 sample_rgba(const float4* __restrict__ img, int h, int w, bool ok, float u, float v) {
    const Taps4 t = bilinear_taps4(ok, u, v, h, w);
    const float4 p00 = __ldg(img + t.i00), p01 = __ldg(img + t.i01);
    const float4 p10 = __ldg(img + t.i10), p11 = __ldg(img + t.i11);
    float4 r;
    r.x = fmaf(t.w11, p11.x, fmaf(t.w10, p10.x, fmaf(t.w01, p01.x, t.w00 * p00.x)));
    r.y = fmaf(t.w11, p11.y, fmaf(t.w10, p10.y, fmaf(t.w01, p01.y, t.w00 * p00.y)));
    r.z = fmaf(t.w11, p11.z, fmaf(t.w10, p10.z, fmaf(t.w01, p01.z, t.w00 * p00.z)));
    r.w = 0.f;
    return r;
}

// The blend softmax runs in log2 units (ex2_approx); the perspective divide is one reciprocal
// (reproject_rcp).
constexpr float RD_LOG2E = 1.4426950408889634f;

// One layer's contribution: blend-weighted colour of the V views with an online softmax over the
// views (running maximum, rescaled sums, in log2 units), so the logits are read once.  logit4(m0,
// b) fills the logits of views m0 .. m0 + 3 (V a multiple of 4: one 16-byte load per LDM corner),
// logit1(m) one view's.
template <bool VEC4, typename Logit4, typename Logit1>
__device__ __forceinline__ void blend_layer(const RenderArgs& a, Logit4 logit4, Logit1 logit1, float pxc, float pyc,
                                            float d, float& cr, float& cg, float& cb) {
    const size_t img_stride = (size_t)a.Hi * a.Wi;
    float mx = -INFINITY, sum = 0.f, lr = 0.f, lg = 0.f, lb = 0.f;
    auto view = [&](int m, float b) {
        const float mn = fmaxf(mx, b);
        const float sc = ex2_approx(mx - mn), p = ex2_approx(b - mn);
        sum = fmaf(sum, sc, p);
        lr *= sc;
        lg *= sc;
        lb *= sc;
        float u = 0.f, v = 0.f;
        const bool ok = reproject_rcp(a.geo.v[m], pxc, pyc, d, u, v);
        const float4 c = sample_rgba(a.rgba + m * img_stride, a.Hi, a.Wi, ok, u, v);
        lr = fmaf(p, c.x, lr);
        lg = fmaf(p, c.y, lg);
        lb = fmaf(p, c.z, lb);
        mx = mn;
    };
    if constexpr (VEC4) {
        for (int m0 = 0; m0 < a.V; m0 += 4) {
            float b[4];
            logit4(m0, b);
#pragma unroll
            for (int i = 0; i < 4; ++i) view(m0 + i, b[i] * RD_LOG2E);
        }
    } else {
        for (int m = 0; m < a.V; ++m) view(m, logit1(m) * RD_LOG2E);
    }
    const float is = 1.0f / sum;
    cr = lr * is;
    cg = lg * is;
    cb = lb * is;
}

template <bool VEC4>
__global__ void __launch_bounds__(RD_THREADS) render_kernel(const RenderArgs a) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)a.Hout * a.Wout) return;
    const int X = (int)((uint32_t)idx % (uint32_t)a.Wout), Y = (int)((uint32_t)idx / (uint32_t)a.Wout);  // < 2^32 pixels
    const int L = a.L, V = a.V;
    const float pxc = X + 0.5f, pyc = Y + 0.5f;
    float cr = 0.f, cg = 0.f, cb = 0.f, T = 1.f;
    if (a.sx == 1.f && a.sy == 1.f) {
        // the LDM grid is the output grid: the upsample is the identity
        for (int li = L - 1; li >= 0; --li) {
            const float d = depth_from_logit(a.t_raw[idx * L + li], li, L, a.dp);
            const float al = sigmoidf_(a.s_raw[idx * L + li]);
            const float* bl = a.beta + (idx * L + li) * V;
            float r, g, b;
            blend_layer<VEC4>(
                a,
                [&](int m0, float (&o)[4]) {
                    const float4 t = __ldg(reinterpret_cast<const float4*>(bl + m0));
                    o[0] = t.x;
                    o[1] = t.y;
                    o[2] = t.z;
                    o[3] = t.w;
                },
                [&](int m) { return __ldg(bl + m); }, pxc, pyc, d, r, g, b);
            const float w = T * al;
            cr = fmaf(w, r, cr);
            cg = fmaf(w, g, cg);
            cb = fmaf(w, b, cb);
            T *= 1.f - al;
        }
    } else {
        int y0, y1, x0, x1;
        float wy, wx;
        resize_taps(Y, a.sy, a.Hl, y0, y1, wy);
        resize_taps(X, a.sx, a.Wl, x0, x1, wx);
        const size_t q00 = (size_t)y0 * a.Wl + x0, q01 = (size_t)y0 * a.Wl + x1;
        const size_t q10 = (size_t)y1 * a.Wl + x0, q11 = (size_t)y1 * a.Wl + x1;
        auto up = [&](const float* f, size_t stride, size_t off) {
            float top = f[q00 * stride + off] * (1 - wx) + f[q01 * stride + off] * wx;
            float bot = f[q10 * stride + off] * (1 - wx) + f[q11 * stride + off] * wx;
            return top * (1 - wy) + bot * wy;
        };
        for (int li = L - 1; li >= 0; --li) {
            const float d = depth_from_logit(up(a.t_raw, L, li), li, L, a.dp);
            const float al = sigmoidf_(up(a.s_raw, L, li));
            const size_t bstride = (size_t)L * V, boff = (size_t)li * V;
            float r, g, b;
            blend_layer<VEC4>(
                a,
                [&](int m0, float (&o)[4]) {
                    const float4 t00 = __ldg(reinterpret_cast<const float4*>(a.beta + q00 * bstride + boff + m0));
                    const float4 t01 = __ldg(reinterpret_cast<const float4*>(a.beta + q01 * bstride + boff + m0));
                    const float4 t10 = __ldg(reinterpret_cast<const float4*>(a.beta + q10 * bstride + boff + m0));
                    const float4 t11 = __ldg(reinterpret_cast<const float4*>(a.beta + q11 * bstride + boff + m0));
                    auto lerp2 = [&](float v00, float v01, float v10, float v11) {
                        const float top = v00 * (1 - wx) + v01 * wx, bot = v10 * (1 - wx) + v11 * wx;
                        return top * (1 - wy) + bot * wy;
                    };
                    o[0] = lerp2(t00.x, t01.x, t10.x, t11.x);
                    o[1] = lerp2(t00.y, t01.y, t10.y, t11.y);
                    o[2] = lerp2(t00.z, t01.z, t10.z, t11.z);
                    o[3] = lerp2(t00.w, t01.w, t10.w, t11.w);
                },
                [&](int m) { return up(a.beta, bstride, boff + m); }, pxc, pyc, d, r, g, b);
            const float w = T * al;
            cr = fmaf(w, r, cr);
            cg = fmaf(w, g, cg);
            cb = fmaf(w, b, cb);
            T *= 1.f - al;
        }
    }
    a.out[idx] = make_float4(cr, cg, cb, 1.f - T);
}

// Depth map (Sec. 3.1, the optional output): the decoded depth over-composited instead of the
// blended input views, D += T alpha_l d_l front to back, 0 behind the last layer.  The raw logits
// are upsampled and activated as in render_kernel.
__global__ void __launch_bounds__(RD_THREADS) render_depth_kernel(const RenderArgs a, float* __restrict__ depth) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)a.Hout * a.Wout) return;
    const int X = (int)((uint32_t)idx % (uint32_t)a.Wout), Y = (int)((uint32_t)idx / (uint32_t)a.Wout);  // < 2^32 pixels
    const int L = a.L;
    float D = 0.f, T = 1.f;
    if (a.sx == 1.f && a.sy == 1.f) {
        for (int li = L - 1; li >= 0; --li) {
            const float d = depth_from_logit(a.t_raw[idx * L + li], li, L, a.dp);
            const float al = sigmoidf_(a.s_raw[idx * L + li]);
            D = fmaf(T * al, d, D);
            T *= 1.f - al;
        }
    } else {
        int y0, y1, x0, x1;
        float wy, wx;
        resize_taps(Y, a.sy, a.Hl, y0, y1, wy);
        resize_taps(X, a.sx, a.Wl, x0, x1, wx);
        const size_t q00 = (size_t)y0 * a.Wl + x0, q01 = (size_t)y0 * a.Wl + x1;
        const size_t q10 = (size_t)y1 * a.Wl + x0, q11 = (size_t)y1 * a.Wl + x1;
        auto up = [&](const float* f, int li) {
            const float top = f[q00 * L + li] * (1 - wx) + f[q01 * L + li] * wx;
            const float bot = f[q10 * L + li] * (1 - wx) + f[q11 * L + li] * wx;
            return top * (1 - wy) + bot * wy;
        };
        for (int li = L - 1; li >= 0; --li) {
            const float d = depth_from_logit(up(a.t_raw, li), li, L, a.dp);
            const float al = sigmoidf_(up(a.s_raw, li));
            D = fmaf(T * al, d, D);
            T *= 1.f - al;
        }
    }
    depth[idx] = D;
}

cudaError_t launch_render_depth(const RenderArgs& a, float* depth, cudaStream_t st) {
    const size_t n = (size_t)a.Hout * a.Wout;
    render_depth_kernel<<<(unsigned)((n + RD_THREADS - 1) / RD_THREADS), RD_THREADS, 0, st>>>(a, depth);
    return cudaGetLastError();
}

cudaError_t launch_render(const RenderArgs& a, cudaStream_t st) {
    const size_t n = (size_t)a.Hout * a.Wout;
    const unsigned grid = (unsigned)((n + RD_THREADS - 1) / RD_THREADS);
    // V a multiple of 4: a pixel's logits of 4 views are 16 contiguous, 16-byte-aligned bytes
    if (a.V % 4 == 0) render_kernel<true><<<grid, RD_THREADS, 0, st>>>(a);
    else render_kernel<false><<<grid, RD_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace quark
