// Render-and-refine of an Update & Fuse step (Sec. 3.2.2 "Decoding and rendering the
// intermediate LDM", Eq. overcomposite-result; the Update Block of the Update & Fuse figure).
//
// splat_kernel      one thread per LDM element (layer plane x pixel of the previous step's grid):
//                   its decoded appearance and density, at its decoded depth, projected into every
//                   input view (operator P) and added with the four bilinear weights to the nearest
//                   pixel centres of the view's grid -- float4 atomics for (colour, density), one
//                   float atomic for the weight.  The transpose of bilinear sampling.
// composite_kernel  one thread per view pixel: each layer's splat normalised by max(weight sum,
//                   1e-2) (sparsely covered pixels fade out), then the over operator front to back
//                   in LDM layer order -> I~ (RGB, accumulated alpha).
// refine_add_kernel one thread per 16 channels of a level-k texel: F' = F + up(I~) W_r + b_r, the
//                   rendered view (x2 bilinear upsample, edge clamp, when the level changes) lifted
//                   to C channels; the Update Block's residual CNN block then runs on F' with the
//                   conv-block kernels and its output is the step's update features.
#include "device_common.cuh"

namespace quark {

constexpr float SPLAT_EPS = 1e-2f;

__global__ void __launch_bounds__(256) splat_kernel(const SplatArgs a) {
    const size_t plane = (size_t)a.H * a.W;
    const size_t el = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (el >= (size_t)a.L * plane) return;
    const int li = (int)(el / plane);
    const int pix = (int)(el % plane);
    const float px = (pix % a.W) + 0.5f, py = (pix / a.W) + 0.5f;
    const float d = a.depth[el], al = a.alpha[el];
    const float c0 = a.colour[3 * el], c1 = a.colour[3 * el + 1], c2 = a.colour[3 * el + 2];
    const size_t vplane = (size_t)a.h * a.w;
    for (int m = 0; m < a.V; ++m) {
        float u, v;
        if (!reproject(a.geo.v[m], px, py, d, u, v)) continue;
        // far-away coordinates are clamped before the conversion (their taps are outside anyway)
        const float x = fminf(fmaxf(u - 0.5f, -3.f), (float)a.w + 2.f);
        const float y = fminf(fmaxf(v - 0.5f, -3.f), (float)a.h + 2.f);
        const float xf = floorf(x), yf = floorf(y);
        const float fx = x - xf, fy = y - yf;
        const int x0 = (int)xf, y0 = (int)yf;
        const size_t base = ((size_t)m * a.L + li) * vplane;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int iy = y0 + (t >> 1), ix = x0 + (t & 1);
            const float wt = ((t >> 1) ? fy : 1.f - fy) * ((t & 1) ? fx : 1.f - fx);
            if (iy < 0 || iy >= a.h || ix < 0 || ix >= a.w || !(wt > 0.f)) continue;
            const size_t o = base + (size_t)iy * a.w + ix;
            atomicAdd(a.acc + o, make_float4(wt * c0, wt * c1, wt * c2, wt * al));
            atomicAdd(a.wsum + o, wt);
        }
    }
}

__global__ void __launch_bounds__(256) composite_kernel(const SplatArgs a) {
    const size_t vplane = (size_t)a.h * a.w;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)a.V * vplane) return;
    const size_t m = idx / vplane, pix = idx % vplane;
    float r = 0.f, g = 0.f, b = 0.f, T = 1.f;
    for (int li = a.L - 1; li >= 0; --li) {
        const size_t o = (m * a.L + li) * vplane + pix;
        const float4 s = a.acc[o];
        const float in = 1.0f / fmaxf(a.wsum[o], SPLAT_EPS);
        const float al = s.w * in, w = T * al * in;
        r = fmaf(w, s.x, r);
        g = fmaf(w, s.y, g);
        b = fmaf(w, s.z, b);
        T *= 1.f - al;
    }
    a.out[idx] = make_float4(r, g, b, 1.f - T);
}

template <typename T, int C>
__global__ void __launch_bounds__(256) refine_add_kernel(const RefineArgs a) {
    constexpr int G = C / 16;
    const size_t n = (size_t)a.V * a.h * a.w * G;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int c0 = (int)(idx % G) * 16;
    const size_t t = idx / G;  // texel of the level
    const int m = (int)(t / ((size_t)a.h * a.w));
    const int r = (int)(t % ((size_t)a.h * a.w));
    const int y = r / a.w, x = r % a.w;
    int y0, y1, x0, x1;
    float wy, wx;
    resize_taps(y, (float)a.ratio, a.hr, y0, y1, wy);
    resize_taps(x, (float)a.ratio, a.wr, x0, x1, wx);
    const float4* I = a.rend + (size_t)m * a.hr * a.wr;
    const float4 p00 = I[(size_t)y0 * a.wr + x0], p01 = I[(size_t)y0 * a.wr + x1];
    const float4 p10 = I[(size_t)y1 * a.wr + x0], p11 = I[(size_t)y1 * a.wr + x1];
    auto lerp2 = [&](float v00, float v01, float v10, float v11) {
        const float top = v00 * (1 - wx) + v01 * wx, bot = v10 * (1 - wx) + v11 * wx;
        return top * (1 - wy) + bot * wy;
    };
    const float iu[4] = {lerp2(p00.x, p01.x, p10.x, p11.x), lerp2(p00.y, p01.y, p10.y, p11.y),
                         lerp2(p00.z, p01.z, p10.z, p11.z), lerp2(p00.w, p01.w, p10.w, p11.w)};
    float f[16];
    load16(reinterpret_cast<const T*>(a.feat) + t * C + c0, f);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int c = c0 + i;
        float lift = __ldg(a.wr_b + 4 * C + c);
#pragma unroll
        for (int q = 0; q < 4; ++q) lift = fmaf(iu[q], __ldg(a.wr_b + q * C + c), lift);
        f[i] += lift;
    }
    store16(reinterpret_cast<T*>(a.out) + t * C + c0, f);
}

cudaError_t launch_splat(const SplatArgs& a, cudaStream_t st) {
    const size_t n = (size_t)a.L * a.H * a.W;
    if (n == 0 || a.V == 0) return cudaSuccess;
    splat_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_composite_views(const SplatArgs& a, cudaStream_t st) {
    const size_t n = (size_t)a.V * a.h * a.w;
    if (n == 0) return cudaSuccess;
    composite_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int C>
static cudaError_t launch_refine_t(const RefineArgs& a, cudaStream_t st) {
    const size_t n = (size_t)a.V * a.h * a.w * (C / 16);
    refine_add_kernel<T, C><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_refine_add(const RefineArgs& a, bool bf16, cudaStream_t st) {
    if ((size_t)a.V * a.h * a.w == 0) return cudaSuccess;
    if (a.C == 16) return bf16 ? launch_refine_t<__nv_bfloat16, 16>(a, st) : launch_refine_t<float, 16>(a, st);
    if (a.C == 32) return bf16 ? launch_refine_t<__nv_bfloat16, 32>(a, st) : launch_refine_t<float, 32>(a, st);
    if (a.C == 64) return bf16 ? launch_refine_t<__nv_bfloat16, 64>(a, st) : launch_refine_t<float, 64>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
