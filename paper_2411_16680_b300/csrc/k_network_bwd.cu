// Adjoints of the transitions between Update & Fuse steps and of the encoder (FP32 form), for the
// backward pass through the whole network (the paper trains end to end through its
// differentiable render, Sec. 3.1, Sec. 3.4):
//
//   upsample2_bwd_kernel  adjoint of the x2 bilinear upsample (edge clamp, pixel centres aligned;
//                         caption of the Update & Fuse figure), as a gather: each source texel sums
//                         the weights it received from the destination pixels that read it, so the
//                         result is deterministic.
//   collapse_bwd_kernel   adjoint of Layer Collapse (Sec. 3.2.2): V'_j = (a + b) / 2 +
//                         gelu([a, b] W1 + b1) W2 + b2 with a, b the layers 2j, 2j + 1; writes the
//                         gradients of a and b and the per-element factors of the MLP's weight
//                         gradients (gelu output, pre-activation gradient, concatenated input).
//   pool_chain_bwd_kernel adjoint of the encoder's mean-pool chain (Sec. 3.2.1): F_2k is the 2x2
//                         mean of F_k, so the full-resolution conv output receives
//                         sum_k dF_k(y / k, x / k) / k^2 over the levels in use.
#include "device_common.cuh"
#include "bwd_internal.cuh"

namespace quark {

// weight of destination index `dst` on source index `src` in the x2 resize of one axis
__device__ __forceinline__ float up2_weight(int dst, int src, int n_src) {
    int i0, i1;
    float w1;
    resize_taps(dst, 2.f, n_src, i0, i1, w1);
    return (i0 == src ? 1.f - w1 : 0.f) + (i1 == src ? w1 : 0.f);
}

__global__ void upsample2_bwd_kernel(const float* __restrict__ dout, float* din, int L, int Hp, int Wp, int C) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)L * Hp * Wp * C) return;
    const int c = (int)(i % C);
    const size_t e = i / C;
    const int xp = (int)(e % Wp), yp = (int)((e / Wp) % Hp), li = (int)(e / ((size_t)Wp * Hp));
    const int H = 2 * Hp, W = 2 * Wp;
    const float* base = dout + (size_t)li * H * W * C + c;
    float s = 0.f;
    // destination pixels 2p - 2 .. 2p + 2 are the only ones whose taps can reach source p
    for (int y = max(2 * yp - 2, 0); y <= min(2 * yp + 2, H - 1); ++y) {
        const float wy = up2_weight(y, yp, Hp);
        if (wy == 0.f) continue;
        for (int x = max(2 * xp - 2, 0); x <= min(2 * xp + 2, W - 1); ++x) {
            const float wx = up2_weight(x, xp, Wp);
            if (wx == 0.f) continue;
            s = fmaf(wy * wx, base[((size_t)y * W + x) * C], s);
        }
    }
    din[i] = s;
}

template <int C>
__global__ void __launch_bounds__(128) collapse_bwd_kernel(const float* __restrict__ vprev, const float* __restrict__ dcol,
                                                           int L, int H, int W, const float* __restrict__ w,
                                                           float* dvprev, float* g_out, float* dh_out, float* cat_out) {
    __shared__ float sw[3 * C * C + 2 * C];  // W1 [2C][C], b1 [C], W2 [C][C], b2 [C]
    const CollapseLayout cl{C};
    for (int i = threadIdx.x; i < cl.total(); i += blockDim.x) sw[i] = w[i];
    __syncthreads();
    const size_t plane = (size_t)H * W;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // element of the collapsed volume
    if (e >= (size_t)L * plane) return;
    const int j = (int)(e / plane);
    const size_t pix = e % plane;
    const float* pa = vprev + ((size_t)(2 * j) * plane + pix) * C;
    const float* pb = vprev + ((size_t)(2 * j + 1) * plane + pix) * C;
    const float* w1 = sw + cl.w1();
    const float* b1 = sw + cl.b1();
    const float* w2 = sw + cl.w2();
    float cat[2 * C], h[C], dg[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        cat[c] = pa[c];
        cat[C + c] = pb[c];
    }
#pragma unroll
    for (int o = 0; o < C; ++o) h[o] = b1[o];
    for (int i = 0; i < 2 * C; ++i)
#pragma unroll
        for (int o = 0; o < C; ++o) h[o] = fmaf(cat[i], w1[i * C + o], h[o]);
    const float* dy = dcol + e * C;
    // dg = dy W2^T
#pragma unroll
    for (int i = 0; i < C; ++i) {
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < C; ++o) s = fmaf(dy[o], w2[i * C + o], s);
        dg[i] = s;
    }
    // dh = dg gelu'(h); the gelu output is kept for the W2 gradient
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const float z = h[i];
        const float cdf = 0.5f * (1.f + erff(z * 0.70710678118654752f));
        const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
        g_out[e * C + i] = z * cdf;
        dg[i] *= cdf + z * pdf;
        dh_out[e * C + i] = dg[i];
    }
    // d[a, b] = dy / 2 + dh W1^T
    float* da = dvprev + ((size_t)(2 * j) * plane + pix) * C;
    float* db = dvprev + ((size_t)(2 * j + 1) * plane + pix) * C;
    for (int i = 0; i < 2 * C; ++i) {
        float s = 0.5f * dy[i % C];
#pragma unroll
        for (int o = 0; o < C; ++o) s = fmaf(dg[o], w1[i * C + o], s);
        if (i < C) da[i] = s;
        else db[i - C] = s;
        cat_out[e * 2 * C + i] = cat[i];
    }
}

__global__ void pool_chain_bwd_kernel(const float* __restrict__ d1, const float* __restrict__ d2,
                                      const float* __restrict__ d4, const float* __restrict__ d8, int V, int H, int W,
                                      int C, float* out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)V * H * W * C) return;
    const int c = (int)(i % C);
    const size_t p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H), m = (int)(p / ((size_t)W * H));
    float s = d1 ? d1[i] : 0.f;
    const float* lv[3] = {d2, d4, d8};
    for (int q = 0; q < 3; ++q) {
        const int k = 2 << q;
        if (!lv[q]) continue;
        const int h = H / k, w = W / k;
        s += lv[q][(((size_t)m * h + y / k) * w + x / k) * C + c] / (float)(k * k);
    }
    out[i] = s;
}

static unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_upsample2_bwd(const float* dout, float* din, int L, int Hp, int Wp, int C, cudaStream_t st) {
    const size_t n = (size_t)L * Hp * Wp * C;
    upsample2_bwd_kernel<<<nblk(n, 256), 256, 0, st>>>(dout, din, L, Hp, Wp, C);
    return cudaGetLastError();
}

cudaError_t launch_collapse_bwd(const float* vprev, const float* dcol, int L, int H, int W, int C, const float* w,
                                float* dvprev, float* g_out, float* dh_out, float* cat_out, cudaStream_t st) {
    const unsigned g = nblk((size_t)L * H * W, 128);
    if (C == 16) collapse_bwd_kernel<16><<<g, 128, 0, st>>>(vprev, dcol, L, H, W, w, dvprev, g_out, dh_out, cat_out);
    else if (C == 32) collapse_bwd_kernel<32><<<g, 128, 0, st>>>(vprev, dcol, L, H, W, w, dvprev, g_out, dh_out, cat_out);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_pool_chain_bwd(const float* const dlev[4], int V, int H, int W, int C, float* out, cudaStream_t st) {
    const size_t n = (size_t)V * H * W * C;
    pool_chain_bwd_kernel<<<nblk(n, 256), 256, 0, st>>>(dlev[0], dlev[1], dlev[2], dlev[3], V, H, W, C, out);
    return cudaGetLastError();
}

}  // namespace quark
