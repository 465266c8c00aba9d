// Decode of the LDM attributes from a stored volume V (Sec. 3.2.2 "Decoding"; Sec. 3.2.3
// Eq. depth_activation): colour = sigmoid(V W_a + b_a), alpha = sigmoid(V w_sigma + b_sigma),
// depth from t = V w_d + b_d, plus the raw logits t and V w_sigma + b_sigma in pixel-major
// [H][W][L] order.  Run on demand when the decoded attributes are read; the dot products run
// in channel order from the stored values, exactly as the conv block computes the two logits
// of the rendered step, so both give the same bits.  One thread per element.
#include "device_common.cuh"

namespace quark {

template <typename T, int C>
__global__ void __launch_bounds__(256) decode_kernel(const DecodeArgs a) {
    const ConvLayout lay{C};
    const size_t plane = (size_t)a.H * a.W;
    const size_t el = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (el >= (size_t)a.L * plane) return;
    const int li = (int)(el / plane);
    const size_t pix = el % plane;
    const T* v = reinterpret_cast<const T*>(a.vol) + el * C;
    const float* w = a.w;
    float t = w[lay.bd()], s = w[lay.bs()];
    float rgb[3] = {w[lay.ba()], w[lay.ba() + 1], w[lay.ba() + 2]};
#pragma unroll
    for (int c0 = 0; c0 < C; c0 += 16) {
        float o[16];
        load16(v + c0, o);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            t = fmaf(o[i], __ldg(w + lay.wd() + c), t);
            s = fmaf(o[i], __ldg(w + lay.ws() + c), s);
            rgb[0] = fmaf(o[i], __ldg(w + lay.wa() + 3 * c + 0), rgb[0]);
            rgb[1] = fmaf(o[i], __ldg(w + lay.wa() + 3 * c + 1), rgb[1]);
            rgb[2] = fmaf(o[i], __ldg(w + lay.wa() + 3 * c + 2), rgb[2]);
        }
    }
    a.colour[3 * el + 0] = sigmoidf_(rgb[0]);
    a.colour[3 * el + 1] = sigmoidf_(rgb[1]);
    a.colour[3 * el + 2] = sigmoidf_(rgb[2]);
    a.alpha[el] = sigmoidf_(s);
    a.depth[el] = depth_from_logit(t, li, a.L, a.dp);
    if (a.t_raw) a.t_raw[pix * a.L + li] = t;
    if (a.s_raw) a.s_raw[pix * a.L + li] = s;
}

cudaError_t launch_decode(const DecodeArgs& a, int C, bool bf16, cudaStream_t st) {
    const size_t n = (size_t)a.L * a.H * a.W;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (C == 16) {
        if (bf16) decode_kernel<__nv_bfloat16, 16><<<grid, 256, 0, st>>>(a);
        else decode_kernel<float, 16><<<grid, 256, 0, st>>>(a);
    } else if (C == 32) {
        if (bf16) decode_kernel<__nv_bfloat16, 32><<<grid, 256, 0, st>>>(a);
        else decode_kernel<float, 32><<<grid, 256, 0, st>>>(a);
    } else if (C == 64) {
        if (bf16) decode_kernel<__nv_bfloat16, 64><<<grid, 256, 0, st>>>(a);
        else decode_kernel<float, 64><<<grid, 256, 0, st>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace quark
