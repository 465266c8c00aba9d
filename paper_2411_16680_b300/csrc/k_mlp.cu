// The fusion block's residual block with 1x1 convolutions (config conv_kernel = 1):
// V' = V + W2 gelu(W1 N(V) + b1) + b2 per LDM element -- the position-wise MLP block of a
// Transformer, which the paper's residual 3x3 convolution block mirrors (Sec. 3.3).  As the conv
// block, it writes the raw depth and density logits of V' when asked (Sec. 3.2.2 "Decoding").
// The 1x1 weights sit at the centre tap of the packed 3x3 weight layout (zeros elsewhere), so the
// decode, the backward pass and the packing are shared with the 3x3 block.
//
//   mlp_block_kernel     FP32 form: one thread per element, both C x C matrices in shared
//                        memory, packed FP32x2 FMAs, erf GELU.
//   mlp_block_tc_kernel  BF16 form on tcgen05: persistent CTAs stride over tiles of 128
//                        consecutive elements; N(V) (BF16) -> X W1 (TMEM) -> + b1, GELU (tanh
//                        form, as the BF16 conv block) -> BF16 -> G W2 (TMEM) -> + b2 + V,
//                        stored as BF16 (and the logits from V' as stored).  Every wait bounded.
#include <algorithm>

#include "device_common.cuh"
#include "umma.cuh"

namespace quark {

constexpr int MB_THREADS = 128;
constexpr uint64_t MB_WAIT_NS = 1000000000ull;

// acc[j] += x * (w[2j], w[2j+1]) over a row of C weights (packed FP32x2)
template <int C>
__device__ __forceinline__ void mlp_fma_row(const float* w, float x, float2 (&acc)[C / 2]) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
    const float2 x2 = make_float2(x, x);
#pragma unroll
    for (int i = 0; i < C / 4; ++i) {
        const float4 t = w4[i];
        acc[2 * i] = __ffma2_rn(x2, make_float2(t.x, t.y), acc[2 * i]);
        acc[2 * i + 1] = __ffma2_rn(x2, make_float2(t.z, t.w), acc[2 * i + 1]);
    }
}

template <int C>
__global__ void __launch_bounds__(MB_THREADS) mlp_block_kernel(const ConvArgs a) {
    const ConvLayout lay{C};
    __shared__ __align__(16) float sw1[C * C];
    __shared__ __align__(16) float sw2[C * C];
    __shared__ float misc[6 * C + 2];  // g, b1, b2, w_d, w_s, b_d, b_s
    for (int i = threadIdx.x; i < C * C; i += blockDim.x) {
        sw1[i] = a.w[lay.w1() + 4 * C * C + i];  // the centre tap
        sw2[i] = a.w[lay.w2() + 4 * C * C + i];
    }
    for (int i = threadIdx.x; i < C; i += blockDim.x) {
        misc[i] = a.w[lay.g() + i];
        misc[C + i] = a.w[lay.b1() + i];
        misc[2 * C + i] = a.w[lay.b2() + i];
        misc[3 * C + i] = a.w[lay.wd() + i];
        misc[4 * C + i] = a.w[lay.ws() + i];
    }
    if (threadIdx.x == 0) {
        misc[5 * C] = a.w[lay.bd()];
        misc[5 * C + 1] = a.w[lay.bs()];
    }
    __syncthreads();
    const size_t plane = (size_t)a.H * a.W;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)a.L * plane) return;
    const float* vin = reinterpret_cast<const float*>(a.in) + e * C;
    float v[C];
#pragma unroll
    for (int i = 0; i < C / 4; ++i) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(vin) + i);
        v[4 * i] = q.x;
        v[4 * i + 1] = q.y;
        v[4 * i + 2] = q.z;
        v[4 * i + 3] = q.w;
    }
    float ms = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) ms = fmaf(v[c], v[c], ms);
    const float r = 1.0f / sqrtf(ms / C + 1e-6f);
    float2 acc[C / 2];
#pragma unroll
    for (int j = 0; j < C / 2; ++j) acc[j] = make_float2(misc[C + 2 * j], misc[C + 2 * j + 1]);
#pragma unroll 4
    for (int ci = 0; ci < C; ++ci) mlp_fma_row<C>(sw1 + ci * C, v[ci] * r * misc[ci], acc);
    float g[C];
#pragma unroll
    for (int j = 0; j < C / 2; ++j) {
        g[2 * j] = gelu_erf(acc[j].x);
        g[2 * j + 1] = gelu_erf(acc[j].y);
    }
#pragma unroll
    for (int j = 0; j < C / 2; ++j) acc[j] = make_float2(misc[2 * C + 2 * j], misc[2 * C + 2 * j + 1]);
#pragma unroll 4
    for (int ci = 0; ci < C; ++ci) mlp_fma_row<C>(sw2 + ci * C, g[ci], acc);
    float* out = reinterpret_cast<float*>(a.out) + e * C;
    float t = misc[5 * C], s = misc[5 * C + 1];
#pragma unroll
    for (int c0 = 0; c0 < C; c0 += 16) {
        float o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            o[i] = v[c] + (i & 1 ? acc[c / 2].y : acc[c / 2].x);
            t = fmaf(o[i], misc[3 * C + c], t);
            s = fmaf(o[i], misc[4 * C + c], s);
        }
        store16(out + c0, o);
    }
    if (a.t_raw) {
        const int li = (int)(e / plane);
        const size_t pix = e % plane;
        a.t_raw[pix * a.L + li] = t;
        a.s_raw[pix * a.L + li] = s;
    }
}

// ---- BF16 form on tcgen05 ----

template <int C>
struct MbSmem {
    static constexpr int x_off = 0;                          // A: 128 x C bf16 (N(V), then gelu)
    static constexpr int w1_off = x_off + MB_THREADS * C * 2;  // B: C x C bf16
    static constexpr int w2_off = w1_off + C * C * 2;          // B: C x C bf16
    static constexpr int misc_off = w2_off + C * C * 2;        // g, b1, b2, w_d, w_s, b_d, b_s fp32
    static constexpr int bar_off = (misc_off + (6 * C + 2) * 4 + 7) / 8 * 8;
    static constexpr int total = bar_off + 16;
    static constexpr uint32_t tmem_cols = 2 * C;  // X W1 in [0, C), G W2 in [C, 2C)
};

template <int C>
__global__ void __launch_bounds__(MB_THREADS) mlp_block_tc_kernel(const ConvArgs a) {
    using S = MbSmem<C>;
    const ConvLayout lay{C};
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* s_x = sm + S::x_off;
    float* misc = reinterpret_cast<float*>(sm + S::misc_off);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::bar_off + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    const size_t plane = (size_t)a.H * a.W;
    const size_t E = (size_t)a.L * plane;
    const long ntiles = (long)((E + MB_THREADS - 1) / MB_THREADS);

    // the centre taps of the packed conv weights (tcgen05 B operands: W1 block, then W2 block)
    {
        constexpr int n16 = C * C * 2 / 16, tap16 = 4 * C * C * 2 / 16, blk16 = 9 * C * C * 2 / 16;
        const uint4* src = reinterpret_cast<const uint4*>(a.wtc);
        uint4* d1 = reinterpret_cast<uint4*>(sm + S::w1_off);
        uint4* d2 = reinterpret_cast<uint4*>(sm + S::w2_off);
        for (int i = tid; i < n16; i += MB_THREADS) {
            d1[i] = __ldg(src + tap16 + i);
            d2[i] = __ldg(src + blk16 + tap16 + i);
        }
        for (int i = tid; i < C; i += MB_THREADS) {
            misc[i] = a.w[lay.g() + i];
            misc[C + i] = a.w[lay.b1() + i];
            misc[2 * C + i] = a.w[lay.b2() + i];
            misc[3 * C + i] = a.w[lay.wd() + i];
            misc[4 * C + i] = a.w[lay.ws() + i];
        }
        if (tid == 0) {
            misc[5 * C] = a.w[lay.bd()];
            misc[5 * C + 1] = a.w[lay.bs()];
        }
    }
    if (warp == 0) umma::tmem_alloc(tslot, S::tmem_cols);
    if (tid == 0) umma::mbar_init(mbar, 1);
    umma::fence_smem_to_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(MB_THREADS, C);
    constexpr uint32_t LBO_A = MB_THREADS * 16, LBO_B = C * 16;
    uint32_t phase = 0;
    bool failed = false;
    int fail_code = 0;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const size_t e = (size_t)tile * MB_THREADS + tid;
        const bool live = e < E;
        const size_t ec = live ? e : E - 1;
        const __nv_bfloat16* vin = reinterpret_cast<const __nv_bfloat16*>(a.in) + ec * C;
        // the element's channels as BF16 pairs (256-bit loads), kept for the residual
        uint32_t vpk[C / 2];
#pragma unroll
        for (int g = 0; g < C / 16; ++g) {
            uint4 u0, u1;
            ldg256(vin + 16 * g, u0, u1);
            vpk[8 * g + 0] = u0.x; vpk[8 * g + 1] = u0.y; vpk[8 * g + 2] = u0.z; vpk[8 * g + 3] = u0.w;
            vpk[8 * g + 4] = u1.x; vpk[8 * g + 5] = u1.y; vpk[8 * g + 6] = u1.z; vpk[8 * g + 7] = u1.w;
        }
        float ms = 0.f;
#pragma unroll
        for (int j = 0; j < C / 2; ++j) {
            const float lo = __uint_as_float(vpk[j] << 16), hi = __uint_as_float(vpk[j] & 0xffff0000u);
            ms = fmaf(lo, lo, fmaf(hi, hi, ms));
        }
        const float r = 1.0f / sqrtf(ms / C + 1e-6f);
        // X = N(V) as the K-major A operand (channel group g of row m at g * 128 * 16 + m * 16)
#pragma unroll
        for (int g = 0; g < C / 8; ++g) {
            uint4 u;
            __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t w = vpk[4 * g + i];
                const int c = 8 * g + 2 * i;
                hh[i] = __floats2bfloat162_rn(__uint_as_float(w << 16) * r * misc[c],
                                              __uint_as_float(w & 0xffff0000u) * r * misc[c + 1]);
            }
            *reinterpret_cast<uint4*>(s_x + ((size_t)g * MB_THREADS + tid) * 16) = u;
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (tid == 0) {
            const uint64_t ad = umma::desc(umma::smem_u32(s_x), LBO_A, 128);
            const uint64_t bd = umma::desc(umma::smem_u32(sm + S::w1_off), LBO_B, 128);
#pragma unroll
            for (int kk = 0; kk < C / 16; ++kk)
                umma::mma_bf16(tmem, ad + ((2 * kk * LBO_A) >> 4), bd + ((2 * kk * LBO_B) >> 4), idesc, kk > 0);
            umma::commit(mbar);
        }
        failed = __syncthreads_or(!umma::mbar_wait(mbar, phase, MB_WAIT_NS));
        umma::fence_after_sync();
        if (failed) {
            fail_code = 7;
            break;
        }
        phase ^= 1;
        // G = gelu(H + b1) -> BF16 A operand (X has been read by the MMA)
#pragma unroll
        for (int ch = 0; ch < C / 16; ++ch) {
            float hv[16];
            umma::ld_32x32b_x16(tmem + lane_base + ch * 16, hv);
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                uint4 u;
                __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = ch * 16 + 8 * g + 2 * i;
                    const float2 ge = gelu_tanh2(make_float2(hv[8 * g + 2 * i] + misc[C + c],
                                                             hv[8 * g + 2 * i + 1] + misc[C + c + 1]));
                    hh[i] = __floats2bfloat162_rn(ge.x, ge.y);
                }
                *reinterpret_cast<uint4*>(s_x + ((size_t)(2 * ch + g) * MB_THREADS + tid) * 16) = u;
            }
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (tid == 0) {
            const uint64_t ad = umma::desc(umma::smem_u32(s_x), LBO_A, 128);
            const uint64_t bd = umma::desc(umma::smem_u32(sm + S::w2_off), LBO_B, 128);
#pragma unroll
            for (int kk = 0; kk < C / 16; ++kk)
                umma::mma_bf16(tmem + C, ad + ((2 * kk * LBO_A) >> 4), bd + ((2 * kk * LBO_B) >> 4), idesc, kk > 0);
            umma::commit(mbar);
        }
        failed = __syncthreads_or(!umma::mbar_wait(mbar, phase, MB_WAIT_NS));
        umma::fence_after_sync();
        if (failed) {
            fail_code = 8;
            break;
        }
        phase ^= 1;
        {
            __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(a.out) + ec * C;
            float t = misc[5 * C], s = misc[5 * C + 1];
#pragma unroll
            for (int ch = 0; ch < C / 16; ++ch) {
                float ov[16];
                umma::ld_32x32b_x16(tmem + lane_base + C + ch * 16, ov);
                uint4 u[2];
                __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(u);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = ch * 16 + 2 * j;
                    const uint32_t w = vpk[c / 2];
                    hh[j] = __floats2bfloat162_rn(__uint_as_float(w << 16) + ov[2 * j] + misc[2 * C + c],
                                                  __uint_as_float(w & 0xffff0000u) + ov[2 * j + 1] + misc[2 * C + c + 1]);
                    // the logits from V' as stored, as the on-demand decode computes them
                    const float2 o = __bfloat1622float2(hh[j]);
                    t = fmaf(o.y, misc[3 * C + c + 1], fmaf(o.x, misc[3 * C + c], t));
                    s = fmaf(o.y, misc[4 * C + c + 1], fmaf(o.x, misc[4 * C + c], s));
                }
                if (live) stg256(out + ch * 16, u[0], u[1]);
            }
            if (live && a.t_raw) {
                const int li = (int)(e / plane);
                const size_t pix = e % plane;
                a.t_raw[pix * a.L + li] = t;
                a.s_raw[pix * a.L + li] = s;
            }
        }
        // this tile's TMEM reads and X-tile use before the next tile's writes and MMAs
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
    }
    if (failed && tid == 0) {
        atomicExch(a.err, fail_code);
        umma::mbar_wait(mbar, phase, MB_WAIT_NS);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(tmem, S::tmem_cols);
}

cudaError_t launch_mlp_block(const ConvArgs& a, int C, bool bf16, cudaStream_t st) {
    const size_t E = (size_t)a.L * a.H * a.W;
    if (E == 0) return cudaSuccess;
    if (!bf16) {
        const unsigned g = (unsigned)((E + MB_THREADS - 1) / MB_THREADS);
        if (C == 16) mlp_block_kernel<16><<<g, MB_THREADS, 0, st>>>(a);
        else if (C == 32) mlp_block_kernel<32><<<g, MB_THREADS, 0, st>>>(a);
        else if (C == 64) mlp_block_kernel<64><<<g, MB_THREADS, 0, st>>>(a);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    if (!a.wtc || !a.err) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(a.in) % 32 || reinterpret_cast<uintptr_t>(a.out) % 32) return cudaErrorMisalignedAddress;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const long ntiles = (long)((E + MB_THREADS - 1) / MB_THREADS);
    // persistent: eight CTAs per SM, fewer where their TMEM columns (2 C each) would exceed the 512
    const unsigned grid = (unsigned)std::min<long>(ntiles, (long)std::min(8, 256 / C) * sms);
#define QK_MB_LAUNCH(CV)                                                                               \
    do {                                                                                               \
        auto k = mlp_block_tc_kernel<CV>;                                                              \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, MbSmem<CV>::total); \
        if (e != cudaSuccess) return e;                                                                \
        k<<<grid, MB_THREADS, MbSmem<CV>::total, st>>>(a);                                             \
    } while (0)
    if (C == 16) QK_MB_LAUNCH(16);
    else if (C == 32) QK_MB_LAUNCH(32);
    else if (C == 64) QK_MB_LAUNCH(64);
    else return cudaErrorInvalidValue;
#undef QK_MB_LAUNCH
    return cudaGetLastError();
}

}  // namespace quark
