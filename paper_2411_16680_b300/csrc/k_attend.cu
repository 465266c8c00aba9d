// Transition and one-to-many attention of an Update & Fuse step.
//
// collapse_kernel  Layer Collapse (Sec. 3.2.2): pairs (l = 2j-1, 2j) of the previous step's
//                  volume -> 0.5 (a + b) + W2^T gelu(W1^T [a; b] + b1) + b2.
// attend_kernel    the fused sample-attend step: volume entering the step (broadcast v0, or the
//                  previous volume, bilinearly x2-upsampled on the fly) -> decode depth
//                  (Eq. depth_activation) -> per view: reproject, bilinear-sample the level-k
//                  feature map (operator P^T, Sec. 3.1) -> RMSNorm, query projection, online
//                  softmax over views, weighted sum, output projection, residual (Sec. 3.3).
//                  On the last step it also writes the blend logits (Sec. 3.2.3).
//
// Thread mapping: C/16 threads per LDM element, each owning 16 channels of the query, the
// sampled features and the head outputs; dot products are finished with shuffles inside the
// group.  Consecutive elements are consecutive x of one layer row, so a warp's samples land
// on neighbouring texels of each view.
//
// Layout of the sources: this file holds the layer collapse and the dispatch; the attention
// kernels' templates are in k_attend_impl.cuh, instantiated per channel count in
// k_attend_c{16,32,64}.cu (one-to-many) and k_attend_std_c{16,32,64}.cu (standard mode).
#include <algorithm>

#include "k_attend_impl.cuh"

namespace quark {

// -------------------------------------------------------------------------------------------
// Layer collapse
// -------------------------------------------------------------------------------------------

template <typename T, int C>
__global__ void __launch_bounds__(128) collapse_kernel(CollapseArgs a) {
    extern __shared__ float4 w4[];
    float* w = reinterpret_cast<float*>(w4);  // the MLP's weights (dynamic: 49 KB at C = 64)
    const CollapseLayout lay{C};
    for (int i = threadIdx.x; i < lay.total(); i += blockDim.x) w[i] = a.w[i];
    __syncthreads();
    const size_t plane = (size_t)a.H * a.W;
    const size_t n = (size_t)a.L * plane;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const size_t j = e / plane, pix = e % plane;
    const T* pa = reinterpret_cast<const T*>(a.in) + ((2 * j) * plane + pix) * C;
    const T* pb = reinterpret_cast<const T*>(a.in) + ((2 * j + 1) * plane + pix) * C;
    float va[C], vb[C];
#pragma unroll
    for (int c0 = 0; c0 < C; c0 += 16) {
        float t[16];
        load16(pa + c0, t);
#pragma unroll
        for (int i = 0; i < 16; ++i) va[c0 + i] = t[i];
        load16(pb + c0, t);
#pragma unroll
        for (int i = 0; i < 16; ++i) vb[c0 + i] = t[i];
    }
    // packed FP32x2 arithmetic on rows of weights read as float4 (the weight rows are 16-byte
    // aligned: C is a multiple of 16 and every block of the layout starts at a multiple of C)
    float2 h[C / 2];
#pragma unroll
    for (int c = 0; c < C; c += 2) h[c / 2] = make_float2(w[lay.b1() + c], w[lay.b1() + c + 1]);
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const float4* r0 = reinterpret_cast<const float4*>(&w[lay.w1() + i * C]);
        const float4* r1 = reinterpret_cast<const float4*>(&w[lay.w1() + (C + i) * C]);
        const float2 xa = make_float2(va[i], va[i]), xb = make_float2(vb[i], vb[i]);
#pragma unroll
        for (int c4 = 0; c4 < C / 4; ++c4) {
            const float4 p = r0[c4], q = r1[c4];
            h[2 * c4] = __ffma2_rn(xa, make_float2(p.x, p.y), __ffma2_rn(xb, make_float2(q.x, q.y), h[2 * c4]));
            h[2 * c4 + 1] = __ffma2_rn(xa, make_float2(p.z, p.w), __ffma2_rn(xb, make_float2(q.z, q.w), h[2 * c4 + 1]));
        }
    }
    float2 o2[C / 2];
#pragma unroll
    for (int c = 0; c < C; c += 2)
        o2[c / 2] = make_float2(0.5f * (va[c] + vb[c]) + w[lay.b2() + c], 0.5f * (va[c + 1] + vb[c + 1]) + w[lay.b2() + c + 1]);
#pragma unroll
    for (int i2 = 0; i2 < C / 2; ++i2) {
        const float2 g = gelu_fine2(h[i2]);  // the erf form to FP32 rounding
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float gk = k ? g.y : g.x;
            const float2 gg = make_float2(gk, gk);
            const float4* r = reinterpret_cast<const float4*>(&w[lay.w2() + (2 * i2 + k) * C]);
#pragma unroll
            for (int c4 = 0; c4 < C / 4; ++c4) {
                const float4 p = r[c4];
                o2[2 * c4] = __ffma2_rn(gg, make_float2(p.x, p.y), o2[2 * c4]);
                o2[2 * c4 + 1] = __ffma2_rn(gg, make_float2(p.z, p.w), o2[2 * c4 + 1]);
            }
        }
    }
    float o[C];
#pragma unroll
    for (int c = 0; c < C; c += 2) {
        o[c] = o2[c / 2].x;
        o[c + 1] = o2[c / 2].y;
    }
    T* po = reinterpret_cast<T*>(a.out) + e * C;
#pragma unroll
    for (int c0 = 0; c0 < C; c0 += 16) {
        float t[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) t[i] = o[c0 + i];
        store16(po + c0, t);
    }
}

// BF16 form: both MLP layers on tcgen05 (k_collapse_tc.cu).  FP32 form: the same kernel on split
// FP16 operands when the context packed them (C <= 32), else this SIMT kernel.
cudaError_t launch_collapse(const CollapseArgs& a, int C, bool bf16, cudaStream_t st) {
    if (bf16) return launch_collapse_tc(a, C, false, st);
    if (a.wtc && C <= 32) return launch_collapse_tc(a, C, true, st);
    size_t n = (size_t)a.L * a.H * a.W;
    unsigned grid = (unsigned)((n + 127) / 128);
    auto run = [&](auto k, int Cv) {
        const int smem = (3 * Cv * Cv + 2 * Cv) * (int)sizeof(float);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k<<<grid, 128, smem, st>>>(a);
        return cudaGetLastError();
    };
    if (C == 16) return run(collapse_kernel<float, 16>, 16);
    if (C == 32) return run(collapse_kernel<float, 32>, 32);
    if (C == 64) return run(collapse_kernel<float, 64>, 64);
    return cudaErrorInvalidValue;
}

cudaError_t launch_kv_project(const void* feat, size_t texels, int C, const float* wkv, void* out, bool with_f, bool bf16,
                              cudaStream_t st) {
    if (texels == 0) return cudaSuccess;
    if (C == 16) return bf16 ? launch_kv_t<__nv_bfloat16, 16>(feat, texels, wkv, out, with_f, st)
                             : launch_kv_t<float, 16>(feat, texels, wkv, out, with_f, st);
    if (C == 32) return bf16 ? launch_kv_t<__nv_bfloat16, 32>(feat, texels, wkv, out, with_f, st)
                             : launch_kv_t<float, 32>(feat, texels, wkv, out, with_f, st);
    if (C == 64) return bf16 ? launch_kv_t<__nv_bfloat16, 64>(feat, texels, wkv, out, with_f, st)
                             : launch_kv_t<float, 64>(feat, texels, wkv, out, with_f, st);
    return cudaErrorInvalidValue;
}

// Standard mode, both precisions (SIMT; BF16 storage of the maps and volumes in the BF16 form).
// a.feat is the projected map of launch_kv_project (2C channels per texel, 3C on the last step).
cudaError_t launch_attend_std(const AttendArgs& a, int C, int heads, Transition tr, bool last, bool bf16,
                              cudaStream_t st) {
    if (reinterpret_cast<uintptr_t>(a.feat) % 32) return cudaErrorMisalignedAddress;  // 256-bit tap loads
    if (!a.w_std) return cudaErrorInvalidValue;
    if (C == 16) return attend_std_c16(a, heads, tr, last, bf16, st);
    if (C == 32) return attend_std_c32(a, heads, tr, last, bf16, st);
    if (C == 64) return attend_std_c64(a, heads, tr, last, bf16, st);
    return cudaErrorInvalidValue;
}

// BF16 form: projections on tcgen05 (k_attend_tc.cu).  FP32 form: the same kernel with split FP16
// operands when the context packed them (C <= 32, weights within the split's range), else this
// SIMT kernel.
cudaError_t launch_attend(const AttendArgs& a, int C, int heads, Transition tr, bool last, bool bf16,
                          cudaStream_t st) {
    if (bf16) return launch_attend_tc(a, C, heads, tr, last, false, st);
    if (a.wtc && C <= 32) return launch_attend_tc(a, C, heads, tr, last, true, st);
    if (reinterpret_cast<uintptr_t>(a.feat) % 32) return cudaErrorMisalignedAddress;  // 256-bit tap loads
    if (C == 16) return attend_fp32_c16(a, heads, tr, last, st);
    if (C == 32) return attend_fp32_c32(a, heads, tr, last, st);
    if (C == 64) return attend_fp32_c64(a, heads, tr, last, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
