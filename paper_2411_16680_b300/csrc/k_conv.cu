// Residual conv block of the fusion block (Sec. 3.3): V' = V + Conv2(gelu(Conv1(N(V)))), 3x3
// convolutions per layer plane (zero padding), N = RMSNorm.  When asked (the last step, whose
// LDM is rendered), it also writes the raw depth and density logits t = V' w_d + b_d and
// V' w_sigma + b_sigma (Sec. 3.2.2 "Decoding") in pixel-major [H][W][L] order; the other decoded
// attributes are produced on demand by k_decode.cu.
//
// FP32 SIMT form.  One CTA per 16x8 output tile of one layer plane: the normalised input tile
// with a 2-pixel halo and the gelu(Conv1) tile with a 1-pixel halo stay in shared memory, so
// V is read once and written once; the 3x3 weights of each conv are staged in shared memory in
// turn.  Each work item is a register tile of 2 x 2 pixels x 8 output channels.
#include "device_common.cuh"

namespace quark {

constexpr int CV_TW = 16, CV_TH = 8;
constexpr int CV_IW = CV_TW + 4, CV_IH = CV_TH + 4;  // input tile incl. halo 2
constexpr int CV_MW = CV_TW + 2, CV_MH = CV_TH + 2;  // mid tile incl. halo 1
constexpr int CV_THREADS = CV_TW * CV_TH;

constexpr int CV_TAPS = 3;  // taps of weights staged in shared memory at a time

template <int C>
struct ConvSmem {
    static constexpr int P = C + 1;  // padded pixel stride (bank spread)
    static constexpr int in_off = 0;
    static constexpr int mid_off = in_off + CV_IH * CV_IW * P;
    static constexpr int w_off = ((mid_off + CV_MH * CV_MW * P) + 3) & ~3;
    static constexpr int misc_off = w_off + CV_TAPS * C * C;
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

// threads of a CTA: 128 (256 at C = 64, where the tile has twice the channel groups to cover)
template <int C>
constexpr int cv_threads() { return C == 64 ? 2 * CV_THREADS : CV_THREADS; }

template <typename T, int C>
__global__ void __launch_bounds__(cv_threads<C>()) conv_block_kernel(const ConvArgs a) {
    constexpr int NT = cv_threads<C>();
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

    for (int i = tid; i < C; i += NT) {
        misc[i] = a.w[lay.g() + i];
        misc[C + i] = a.w[lay.b1() + i];
        misc[2 * C + i] = a.w[lay.b2() + i];
        misc[3 * C + i] = a.w[lay.wd() + i];
        misc[4 * C + i] = a.w[lay.ws() + i];
    }
    if (tid == 3) misc[8 * C + 3] = a.w[lay.bd()];
    if (tid == 4) misc[8 * C + 4] = a.w[lay.bs()];
    __syncthreads();
    // taps [t0, t0 + CV_TAPS) of a conv's weights into shared memory (the caller synchronises)
    auto stage = [&](int woff, int t0) {
        const float4* src = reinterpret_cast<const float4*>(a.w + woff + (size_t)t0 * C * C);
        float4* dst = reinterpret_cast<float4*>(sw);
        for (int i = tid; i < CV_TAPS * C * C / 4; i += NT) dst[i] = src[i];
    };

    // ---- normalised input tile (zero outside the plane) ----
    for (int p = tid; p < CV_IH * CV_IW; p += NT) {
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
    // Register tiles: a work item is a 2 x 2 block of pixels x 8 output channels (32 FP32
    // accumulators); per tap and input channel it reads four inputs and two float4 weight quads
    // from shared memory for 16 packed FMAs.  Items: block-major with the channel group fastest, so
    // a warp's lanes read 8 blocks' inputs (each broadcast to 4 lanes) and one 128-byte weight row.
    // The weights come in chunks of CV_TAPS taps, so each thread keeps its items' accumulators
    // (at most two items: 9 x 5 blocks x G groups <= 2 x 128) across the chunks.
    constexpr int G = C / 8;  // output-channel groups
    auto accumulate = [&](float2 (&acc)[4][4], const float* s00, int rowp, const float* wt) {
#pragma unroll 4
        for (int ci = 0; ci < C; ++ci) {
            const float x[4] = {s00[ci], s00[P + ci], s00[rowp + ci], s00[rowp + P + ci]};
            const float4 w0 = *reinterpret_cast<const float4*>(wt + ci * C);
            const float4 w1 = *reinterpret_cast<const float4*>(wt + ci * C + 4);
            const float2 wp[4] = {make_float2(w0.x, w0.y), make_float2(w0.z, w0.w), make_float2(w1.x, w1.y),
                                  make_float2(w1.z, w1.w)};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 x2 = make_float2(x[q], x[q]);
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[q][j] = __ffma2_rn(x2, wp[j], acc[q][j]);
            }
        }
    };
    {
        constexpr int MBX = CV_MW / 2, MBY = CV_MH / 2;  // 9 x 5 blocks of the mid tile
        constexpr int NIT = MBX * MBY * G;
        static_assert(NIT <= 2 * NT, "at most two conv1 items per thread");
        float2 acc[2][4][4];
        int bx[2], by[2], gi[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int it = min(tid + k * NT, NIT - 1);
            gi[k] = it % G;
            bx[k] = (it / G) % MBX;
            by[k] = (it / G) / MBX;
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[k][q][j] = make_float2(misc[C + gi[k] * 8 + 2 * j], misc[C + gi[k] * 8 + 2 * j + 1]);
        }
        const bool second = tid + NT < NIT;
        for (int t0 = 0; t0 < 9; t0 += CV_TAPS) {
            stage(lay.w1(), t0);
            __syncthreads();
#pragma unroll
            for (int tt = 0; tt < CV_TAPS; ++tt) {
                const int dy = (t0 + tt) / 3, dx = (t0 + tt) % 3;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (k == 1 && !second) break;
                    accumulate(acc[k], sin + ((2 * by[k] + dy) * CV_IW + 2 * bx[k] + dx) * P, CV_IW * P,
                               sw + tt * C * C + gi[k] * 8);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k == 1 && !second) break;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int my = 2 * by[k] + (q >> 1), mx = 2 * bx[k] + (q & 1);
                const int gy = Y0 - 1 + my, gx = X0 - 1 + mx;
                const bool inside = gy >= 0 && gy < H && gx >= 0 && gx < W;
                float* dst = smid + (my * CV_MW + mx) * P + gi[k] * 8;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    dst[2 * j] = inside ? gelu_erf(acc[k][q][j].x) : 0.f;
                    dst[2 * j + 1] = inside ? gelu_erf(acc[k][q][j].y) : 0.f;
                }
            }
        }
    }
    __syncthreads();

    // ---- Conv2, residual, decode: 8 x 4 blocks of 2 x 2 output pixels x G channel groups ----
    constexpr int OBX = CV_TW / 2, OBY = CV_TH / 2;
    static_assert(OBX * OBY * G <= NT, "one conv2 item per thread");
    {
        const bool active = tid < OBX * OBY * G;
        const int it = active ? tid : 0;
        const int g = it % G, b = it / G;
        const int bx = b % OBX, by = b / OBX;
        float2 acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                acc[q][j] = make_float2(misc[2 * C + g * 8 + 2 * j], misc[2 * C + g * 8 + 2 * j + 1]);
        for (int t0 = 0; t0 < 9; t0 += CV_TAPS) {
            stage(lay.w2(), t0);
            __syncthreads();
            if (active) {
#pragma unroll
                for (int tt = 0; tt < CV_TAPS; ++tt) {
                    const int dy = (t0 + tt) / 3, dx = (t0 + tt) % 3;
                    accumulate(acc, smid + ((2 * by + dy) * CV_MW + 2 * bx + dx) * P, CV_MW * P,
                               sw + tt * C * C + g * 8);
                }
            }
            __syncthreads();
        }
        if (!active) return;  // whole warps (64 or 128 items): the shuffles below see full warps
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gy = Y0 + 2 * by + (q >> 1), gx = X0 + 2 * bx + (q & 1);
            const bool inside = gy < H && gx < W;
            const size_t pix = (size_t)(inside ? gy : 0) * W + (inside ? gx : 0);
            float t = 0.f, sd = 0.f;
            if (inside) {
                const float* res = reinterpret_cast<const float*>(vin) + pix * C + g * 8;
                float* out = reinterpret_cast<float*>(a.out) + ((size_t)li * plane + pix) * C + g * 8;
                const float4 r0 = __ldg(reinterpret_cast<const float4*>(res));
                const float4 r1 = __ldg(reinterpret_cast<const float4*>(res) + 1);
                const float o[8] = {r0.x + acc[q][0].x, r0.y + acc[q][0].y, r0.z + acc[q][1].x, r0.w + acc[q][1].y,
                                    r1.x + acc[q][2].x, r1.y + acc[q][2].y, r1.z + acc[q][3].x, r1.w + acc[q][3].y};
                reinterpret_cast<float4*>(out)[0] = make_float4(o[0], o[1], o[2], o[3]);
                reinterpret_cast<float4*>(out)[1] = make_float4(o[4], o[5], o[6], o[7]);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    t = fmaf(o[i], misc[3 * C + g * 8 + i], t);
                    sd = fmaf(o[i], misc[4 * C + g * 8 + i], sd);
                }
            }
            // the logits sum over the G channel groups, held by consecutive lanes
#pragma unroll
            for (int off = 1; off < G; off <<= 1) {
                t += __shfl_xor_sync(0xffffffffu, t, off);
                sd += __shfl_xor_sync(0xffffffffu, sd, off);
            }
            if (inside && g == 0 && a.t_raw) {
                a.t_raw[pix * L + li] = t + misc[8 * C + 3];
                a.s_raw[pix * L + li] = sd + misc[8 * C + 4];
            }
        }
    }
}

template <typename T, int C>
static cudaError_t launch_t(const ConvArgs& a, cudaStream_t st) {
    const size_t smem = (size_t)ConvSmem<C>::total * sizeof(float);
    auto k = conv_block_kernel<T, C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + CV_TW - 1) / CV_TW, (a.H + CV_TH - 1) / CV_TH, a.L);
    k<<<grid, cv_threads<C>(), smem, st>>>(a);
    return cudaGetLastError();
}

// BF16 form: the tcgen05 kernel (k_conv_tc.cu).  FP32 form: the same kernel on split FP16 operands
// when the context packed them (C <= 32, weights within the split's range), else this SIMT kernel.
// 1x1 kernels: k_mlp.cu.
cudaError_t launch_conv_block(const ConvArgs& a, int C, bool bf16, cudaStream_t st) {
    if (a.ks == 1) return launch_mlp_block(a, C, bf16, st);  // 1x1 convolutions: per element
    if (bf16) return launch_conv_block_tc(a, C, false, st);
    if (a.wtc && C <= 32) return launch_conv_block_tc(a, C, true, st);
    if (C == 16) return launch_t<float, 16>(a, st);
    if (C == 32) return launch_t<float, 32>(a, st);
    if (C == 64) return launch_t<float, 64>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
