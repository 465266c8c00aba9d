// Residual conv block of the fusion block (Sec. 3.3): V' = V + Conv2(gelu(Conv1(N(V)))), 3x3
// convolutions per layer plane (zero padding), N = RMSNorm.  When asked (the last step, whose
// LDM is rendered), it also writes the raw depth and density logits t = V' w_d + b_d and
// V' w_sigma + b_sigma (Sec. 3.2.2 "Decoding") in pixel-major [H][W][L] order; the other decoded
// attributes are produced on demand by k_decode.cu.
//
// FP32 SIMT form.  One CTA per 16x8 output tile of one layer plane: the normalised input tile
// with a 2-pixel halo and the gelu(Conv1) tile with a 1-pixel halo stay in shared memory, so
// V is read once and written once; the 3x3 weights of each conv are staged in shared memory in
// turn.  Each thread produces all C output channels of one pixel.
#include "device_common.cuh"

namespace quark {

constexpr int CV_TW = 16, CV_TH = 8;
constexpr int CV_IW = CV_TW + 4, CV_IH = CV_TH + 4;  // input tile incl. halo 2
constexpr int CV_MW = CV_TW + 2, CV_MH = CV_TH + 2;  // mid tile incl. halo 1
constexpr int CV_THREADS = CV_TW * CV_TH;

template <int C>
struct ConvSmem {
    static constexpr int P = C + 1;  // padded pixel stride (bank spread)
    static constexpr int in_off = 0;
    static constexpr int mid_off = in_off + CV_IH * CV_IW * P;
    static constexpr int w_off = ((mid_off + CV_MH * CV_MW * P) + 3) & ~3;
    static constexpr int misc_off = w_off + 9 * C * C;
    static constexpr int total = misc_off + 8 * C + 8;
};

// acc[j] += x * (w[2j], w[2j+1]) over a row of C weights: packed FP32x2, two channels per FMA
template <int C>
__device__ __forceinline__ void fma_row_x2(const float* w, float x, float2 (&acc)[C / 2]) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
    const float2 x2 = make_float2(x, x);
#pragma unroll
    for (int i = 0; i < C / 4; ++i) {
        const float4 t = w4[i];
        acc[2 * i] = __ffma2_rn(x2, make_float2(t.x, t.y), acc[2 * i]);
        acc[2 * i + 1] = __ffma2_rn(x2, make_float2(t.z, t.w), acc[2 * i + 1]);
    }
}

template <typename T, int C>
__global__ void __launch_bounds__(CV_THREADS) conv_block_kernel(const ConvArgs a) {
    using S = ConvSmem<C>;
    constexpr int P = S::P;
    const ConvLayout lay{C};
    extern __shared__ float4 sm4[];
    float* sm = reinterpret_cast<float*>(sm4);
    float* sin = sm + S::in_off;
    float* smid = sm + S::mid_off;
    float* sw = sm + S::w_off;
    float* misc = sm + S::misc_off;  // g, b1, b2, w_d, w_s, (unused 3C + 3), b_d, b_s

    const int tid = threadIdx.x;
    const int H = a.H, W = a.W, L = a.L;
    const int X0 = blockIdx.x * CV_TW, Y0 = blockIdx.y * CV_TH, li = blockIdx.z;
    const size_t plane = (size_t)H * W;
    const T* vin = reinterpret_cast<const T*>(a.in) + (size_t)li * plane * C;

    for (int i = tid; i < C; i += CV_THREADS) {
        misc[i] = a.w[lay.g() + i];
        misc[C + i] = a.w[lay.b1() + i];
        misc[2 * C + i] = a.w[lay.b2() + i];
        misc[3 * C + i] = a.w[lay.wd() + i];
        misc[4 * C + i] = a.w[lay.ws() + i];
    }
    if (tid == 3) misc[8 * C + 3] = a.w[lay.bd()];
    if (tid == 4) misc[8 * C + 4] = a.w[lay.bs()];
    {
        const float4* src = reinterpret_cast<const float4*>(a.w + lay.w1());
        float4* dst = reinterpret_cast<float4*>(sw);
        for (int i = tid; i < 9 * C * C / 4; i += CV_THREADS) dst[i] = src[i];
    }
    __syncthreads();

    // ---- normalised input tile (zero outside the plane) ----
    for (int p = tid; p < CV_IH * CV_IW; p += CV_THREADS) {
        const int gy = Y0 - 2 + p / CV_IW, gx = X0 - 2 + p % CV_IW;
        float* dst = sin + p * P;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            float v[C];
            const T* src = vin + ((size_t)gy * W + gx) * C;
#pragma unroll
            for (int c0 = 0; c0 < C; c0 += 16) {
                float t[16];
                load16(src + c0, t);
#pragma unroll
                for (int i = 0; i < 16; ++i) v[c0 + i] = t[i];
            }
            float ms = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) ms = fmaf(v[c], v[c], ms);
            const float r = 1.0f / sqrtf(ms / C + 1e-6f);
#pragma unroll
            for (int c = 0; c < C; ++c) dst[c] = v[c] * r * misc[c];
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) dst[c] = 0.f;
        }
    }
    __syncthreads();

    // ---- gelu(Conv1) on the mid tile (zero outside the plane: Conv2's padding) ----
    for (int p = tid; p < CV_MH * CV_MW; p += CV_THREADS) {
        const int my = p / CV_MW, mx = p % CV_MW;
        const int gy = Y0 - 1 + my, gx = X0 - 1 + mx;
        float* dst = smid + p * P;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            float2 acc[C / 2];
#pragma unroll
            for (int j = 0; j < C / 2; ++j) acc[j] = make_float2(misc[C + 2 * j], misc[C + 2 * j + 1]);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const float* src = sin + ((my + tap / 3) * CV_IW + mx + tap % 3) * P;
                const float* wt = sw + tap * C * C;
#pragma unroll 4
                for (int ci = 0; ci < C; ++ci) fma_row_x2<C>(wt + ci * C, src[ci], acc);
            }
#pragma unroll
            for (int j = 0; j < C / 2; ++j) {
                dst[2 * j] = gelu_erf(acc[j].x);
                dst[2 * j + 1] = gelu_erf(acc[j].y);
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) dst[c] = 0.f;
        }
    }
    __syncthreads();
    {
        const float4* src = reinterpret_cast<const float4*>(a.w + lay.w2());
        float4* dst = reinterpret_cast<float4*>(sw);
        for (int i = tid; i < 9 * C * C / 4; i += CV_THREADS) dst[i] = src[i];
    }
    __syncthreads();

    // ---- Conv2, residual, decode ----
    const int oy = tid / CV_TW, ox = tid % CV_TW;
    const int gy = Y0 + oy, gx = X0 + ox;
    if (gy >= H || gx >= W) return;
    float2 acc[C / 2];
#pragma unroll
    for (int j = 0; j < C / 2; ++j) acc[j] = make_float2(misc[2 * C + 2 * j], misc[2 * C + 2 * j + 1]);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const float* src = smid + ((oy + tap / 3) * CV_MW + ox + tap % 3) * P;
        const float* wt = sw + tap * C * C;
#pragma unroll 4
        for (int ci = 0; ci < C; ++ci) fma_row_x2<C>(wt + ci * C, src[ci], acc);
    }
    const size_t pix = (size_t)gy * W + gx;
    const T* res = vin + pix * C;
    T* out = reinterpret_cast<T*>(a.out) + ((size_t)li * plane + pix) * C;
    float t = misc[8 * C + 3], s = misc[8 * C + 4];
#pragma unroll
    for (int c0 = 0; c0 < C; c0 += 16) {
        float r[16], o[16];
        load16(res + c0, r);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            o[i] = r[i] + (i & 1 ? acc[c / 2].y : acc[c / 2].x);
            t = fmaf(o[i], misc[3 * C + c], t);
            s = fmaf(o[i], misc[4 * C + c], s);
        }
        store16(out + c0, o);
    }
    if (a.t_raw) {
        a.t_raw[pix * L + li] = t;
        a.s_raw[pix * L + li] = s;
    }
}

template <typename T, int C>
static cudaError_t launch_t(const ConvArgs& a, cudaStream_t st) {
    const size_t smem = (size_t)ConvSmem<C>::total * sizeof(float);
    auto k = conv_block_kernel<T, C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + CV_TW - 1) / CV_TW, (a.H + CV_TH - 1) / CV_TH, a.L);
    k<<<grid, CV_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// FP32 form: this SIMT kernel.  BF16 form: the tcgen05 kernel (k_conv_tc.cu).  1x1 kernels: k_mlp.cu.
cudaError_t launch_conv_block(const ConvArgs& a, int C, bool bf16, cudaStream_t st) {
    if (a.ks == 1) return launch_mlp_block(a, C, bf16, st);  // 1x1 convolutions: per element
    if (bf16) return launch_conv_block_tc(a, C, st);
    if (C == 16) return launch_t<float, 16>(a, st);
    if (C == 32) return launch_t<float, 32>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
