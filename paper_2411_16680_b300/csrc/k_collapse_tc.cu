// Layer Collapse of the BF16 form on tcgen05 tensor cores (Sec. 3.2.2): each pair (l = 2j-1, 2j)
// of the previous step's volume becomes 0.5 (a + b) + gelu([a; b] W1 + b1) W2 + b2.
//
// Persistent CTAs (six per SM; weights staged and TMEM allocated once) stride over tiles of 128
// pixels of one layer pair (M = 128, one element per thread):
//   1. a and b (BF16) are copied as they are into shared memory as the K-major A operand
//      X = [a | b] (K = 2C); 0.5 (a + b) is kept in FP32 registers.
//   2. X W1 (N = C) into TMEM; + b1, GELU (polynomial erf form), BF16 -> shared memory as the
//      A operand G (K = C).
//   3. G W2 (N = C) into the next TMEM columns; + b2 + 0.5 (a + b); stored as BF16.
// Each MMA chain signals an mbarrier through tcgen05.commit; every wait is bounded.
//
// FP32 form (SPLIT): X, G and the packed weights as FP16 parts, the rounded value and the scaled
// remainder fp16((x - fp16(x)) 2^11), three kind::f16 MMAs per K step into a high and a low
// accumulator (FP32 accuracy); each element's rows are scaled by a power of two into [-1, 1)
// before the split ([a | b] by that of max |a|, |b|; G by that of max |G|) and the MMA results
// scaled back, so any volume magnitude is exact to FP32 rounding; GELU gelu_fine2; FP32 in and out.
#include <cuda_fp16.h>

#include <algorithm>

#include "device_common.cuh"
#include "umma.cuh"

namespace quark {

constexpr int CL_M = 128;
constexpr uint64_t CL_WAIT_NS = 1000000000ull;

template <int C, bool SPLIT>
struct ClSmem {
    static constexpr int P = SPLIT ? 2 : 1;                     // operand parts
    static constexpr int x_off = 0;                             // A: 128 x 2C (per part)
    static constexpr int g_off = x_off + P * CL_M * 2 * C * 2;  // A: 128 x C (per part)
    static constexpr int w1_off = g_off + P * CL_M * C * 2;     // B: C x 2C (per part)
    static constexpr int w2_off = w1_off + P * 2 * C * C * 2;   // B: C x C (per part)
    static constexpr int b_off = w2_off + P * C * C * 2;        // b1 [C], b2 [C] fp32
    static constexpr int bar_off = b_off + 2 * C * 4;
    static constexpr int total = bar_off + 16;
    // X W1 in [0, C), G W2 in [C, 2C); SPLIT: their low accumulators in [2C, 3C), [3C, 4C)
    static constexpr uint32_t tmem_cols = P * 2 * C;
    static constexpr uint32_t LO = 2 * C;
};

// FP32 form: eight values as their FP16 parts
__device__ __forceinline__ void cl_split8(const float* v, uint4& hi, uint4& lo) {
    __half2* h = reinterpret_cast<__half2*>(&hi);
    __half2* l = reinterpret_cast<__half2*>(&lo);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __half2 hh = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
        const float2 f = __half22float2(hh);
        h[j] = hh;
        l[j] = __floats2half2_rn((v[2 * j] - f.x) * 2048.f, (v[2 * j + 1] - f.y) * 2048.f);
    }
}

// 16 consecutive TMEM columns of this warp's lanes
__device__ __forceinline__ void tmem_row16(uint32_t tmem, int warp, int col, float (&v)[16]) {
    umma::ld_32x32b_x16(tmem + ((uint32_t)(warp * 32) << 16) + col, v);
}

template <int C, bool SPLIT>
__global__ void __launch_bounds__(CL_M) collapse_tc_kernel(const CollapseArgs a, const FastDiv tiles_p_div) {
    using S = ClSmem<C, SPLIT>;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* s_x = sm + S::x_off;
    uint8_t* s_g = sm + S::g_off;
    float* s_b = reinterpret_cast<float*>(sm + S::b_off);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::bar_off + 8);

    const int tid = threadIdx.x, warp = tid >> 5;
    const size_t plane = (size_t)a.H * a.W;
    const int tiles_p = (int)((plane + CL_M - 1) / CL_M);
    const int ntiles = tiles_p * a.L;

    // weights (once per CTA): packed BF16 B operands (W1 then W2, contiguous), FP32 biases
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.wtc);
        uint4* dst = reinterpret_cast<uint4*>(sm + S::w1_off);
        constexpr int n16 = S::P * 3 * C * C * 2 / 16;  // W1 then W2, each part by part
        for (int i = tid; i < n16; i += CL_M) dst[i] = __ldg(src + i);
        const CollapseLayout lay{C};
        for (int i = tid; i < C; i += CL_M) {
            s_b[i] = a.w[lay.b1() + i];
            s_b[C + i] = a.w[lay.b2() + i];
        }
    }
    if (warp == 0) umma::tmem_alloc(tslot, S::tmem_cols);
    if (tid == 0) umma::mbar_init(mbar, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = SPLIT ? umma::idesc_f16_f32(CL_M, C) : umma::idesc_bf16_f32(CL_M, C);
    constexpr uint32_t LBO_A1 = CL_M * 16, LBO_B = C * 16;
    uint32_t phase = 0;
    bool failed = false;
    int fail_code = 0;

    // persistent: tiles of 128 pixels of one output layer j, the layer pair (2j, 2j+1) in
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j = fdiv(tile, tiles_p_div);
        const size_t pix = (size_t)(tile - j * tiles_p) * CL_M + tid;
        const bool live = pix < plane;
        const size_t pixc = live ? pix : plane - 1;
        // X row of this element: channel group g (8 bf16) of row m at g * 128 * 16 + m * 16
        // (the previous tile's MMAs, which read X and G, completed before its epilogue)
        float avg[C];
        int xe = 0;  // SPLIT: the exponent X was scaled by
        if constexpr (SPLIT) {
            // FP32 form: both layers' channels (two 256-bit loads per 16 channels), scaled by 2^-xe
            // into [-1, 1), split into FP16 parts
            const float* pa = reinterpret_cast<const float*>(a.in) + ((size_t)(2 * j) * plane + pixc) * C;
            const float* pb = reinterpret_cast<const float*>(a.in) + ((size_t)(2 * j + 1) * plane + pixc) * C;
            float va[C], vb[C];
#pragma unroll
            for (int g = 0; g < C / 8; ++g) {
                uint4 u0, u1, w0, w1;
                ldg256(pa + 8 * g, u0, u1);
                ldg256(pb + 8 * g, w0, w1);
                const float fa[8] = {__uint_as_float(u0.x), __uint_as_float(u0.y), __uint_as_float(u0.z), __uint_as_float(u0.w),
                                     __uint_as_float(u1.x), __uint_as_float(u1.y), __uint_as_float(u1.z), __uint_as_float(u1.w)};
                const float fb[8] = {__uint_as_float(w0.x), __uint_as_float(w0.y), __uint_as_float(w0.z), __uint_as_float(w0.w),
                                     __uint_as_float(w1.x), __uint_as_float(w1.y), __uint_as_float(w1.z), __uint_as_float(w1.w)};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    va[8 * g + i] = fa[i];
                    vb[8 * g + i] = fb[i];
                }
            }
            float mx = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                avg[c] = 0.5f * (va[c] + vb[c]);
                mx = fmaxf(mx, fmaxf(fabsf(va[c]), fabsf(vb[c])));
            }
            frexpf(mx, &xe);
#pragma unroll
            for (int g = 0; g < C / 8; ++g) {
                float ta[8], tb[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    ta[i] = ldexpf(va[8 * g + i], -xe);
                    tb[i] = ldexpf(vb[8 * g + i], -xe);
                }
                uint4 ha, la, hb, lb;
                cl_split8(ta, ha, la);
                cl_split8(tb, hb, lb);
                *reinterpret_cast<uint4*>(s_x + ((size_t)g * CL_M + tid) * 16) = ha;
                *reinterpret_cast<uint4*>(s_x + ((size_t)(C / 8 + g) * CL_M + tid) * 16) = hb;
                *reinterpret_cast<uint4*>(s_x + ((size_t)(2 * C / 8 + g) * CL_M + tid) * 16) = la;
                *reinterpret_cast<uint4*>(s_x + ((size_t)(3 * C / 8 + g) * CL_M + tid) * 16) = lb;
            }
        } else {
            // the pixel's channels of both layers in 256-bit loads (whole sectors)
            const __nv_bfloat16* pa = reinterpret_cast<const __nv_bfloat16*>(a.in) + ((size_t)(2 * j) * plane + pixc) * C;
            const __nv_bfloat16* pb = reinterpret_cast<const __nv_bfloat16*>(a.in) + ((size_t)(2 * j + 1) * plane + pixc) * C;
            uint4 ua[C / 8], ub[C / 8];
#pragma unroll
            for (int g = 0; g < C / 16; ++g) {
                ldg256(pa + 16 * g, ua[2 * g], ua[2 * g + 1]);
                ldg256(pb + 16 * g, ub[2 * g], ub[2 * g + 1]);
            }
#pragma unroll
            for (int g = 0; g < C / 8; ++g) {
                *reinterpret_cast<uint4*>(s_x + ((size_t)g * CL_M + tid) * 16) = ua[g];
                *reinterpret_cast<uint4*>(s_x + ((size_t)(C / 8 + g) * CL_M + tid) * 16) = ub[g];
                const __nv_bfloat162* ha = reinterpret_cast<const __nv_bfloat162*>(&ua[g]);
                const __nv_bfloat162* hb = reinterpret_cast<const __nv_bfloat162*>(&ub[g]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float2 fa = __bfloat1622float2(ha[i]), fb = __bfloat1622float2(hb[i]);
                    avg[8 * g + 2 * i] = 0.5f * (fa.x + fb.x);
                    avg[8 * g + 2 * i + 1] = 0.5f * (fa.y + fb.y);
                }
            }
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();

        // ---- H = X W1 ----
        if (tid == 0) {
            const uint64_t ad = umma::desc(umma::smem_u32(s_x), LBO_A1, 128);
            const uint64_t bd = umma::desc(umma::smem_u32(sm + S::w1_off), LBO_B, 128);
#pragma unroll
            for (int kk = 0; kk < 2 * C / 16; ++kk) {
                const uint64_t ak = ad + ((2 * kk * LBO_A1) >> 4), bk = bd + ((2 * kk * LBO_B) >> 4);
                umma::mma_bf16(tmem, ak, bk, idesc, kk > 0);
                if constexpr (SPLIT) {  // the low parts: X at 2C / 8 groups on, W1 after its high part
                    umma::mma_bf16(tmem + S::LO, ak, bk + ((2 * C * C * 2) >> 4), idesc, kk > 0);
                    umma::mma_bf16(tmem + S::LO, ak + ((2 * C / 8 * LBO_A1) >> 4), bk, idesc, 1);
                }
            }
            umma::commit(mbar);
        }
        failed = __syncthreads_or(!umma::mbar_wait(mbar, phase, CL_WAIT_NS));
        umma::fence_after_sync();
        if (failed) {
            fail_code = 5;
            break;
        }
        phase ^= 1;
        int ge_exp = 0;  // SPLIT: the exponent G was scaled by
        if constexpr (SPLIT) {
            // G = gelu(2^xe (H_hi + 2^-11 H_lo) + b1), scaled by 2^-ge_exp into [-1, 1), as FP16 parts
            float gv[C];
            float mg = 0.f;
#pragma unroll
            for (int ch = 0; ch < C / 16; ++ch) {
                float hv[16], hl[16];
                tmem_row16(tmem, warp, ch * 16, hv);
                tmem_row16(tmem, warp, S::LO + ch * 16, hl);
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const int c = ch * 16 + i;
                    const float2 ge = gelu_fine2(make_float2(ldexpf(fmaf(hl[i], 1.0f / 2048.f, hv[i]), xe) + s_b[c],
                                                             ldexpf(fmaf(hl[i + 1], 1.0f / 2048.f, hv[i + 1]), xe) + s_b[c + 1]));
                    gv[c] = ge.x;
                    gv[c + 1] = ge.y;
                    mg = fmaxf(mg, fmaxf(fabsf(ge.x), fabsf(ge.y)));
                }
            }
            frexpf(mg, &ge_exp);
#pragma unroll
            for (int g = 0; g < C / 8; ++g) {
                float t[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) t[i] = ldexpf(gv[8 * g + i], -ge_exp);
                uint4 hi, lo;
                cl_split8(t, hi, lo);
                *reinterpret_cast<uint4*>(s_g + ((size_t)g * CL_M + tid) * 16) = hi;
                *reinterpret_cast<uint4*>(s_g + ((size_t)(C / 8 + g) * CL_M + tid) * 16) = lo;
            }
        } else {
            // G = gelu(H + b1) -> BF16 A operand (K = C)
#pragma unroll
            for (int ch = 0; ch < C / 16; ++ch) {
                float hv[16];
                tmem_row16(tmem, warp, ch * 16, hv);
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    uint4 u;
                    __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int c = ch * 16 + 8 * g + 2 * i;
                        const float2 ge = gelu_poly2(make_float2(hv[8 * g + 2 * i] + s_b[c], hv[8 * g + 2 * i + 1] + s_b[c + 1]));
                        hh[i] = __floats2bfloat162_rn(ge.x, ge.y);
                    }
                    *reinterpret_cast<uint4*>(s_g + ((size_t)(2 * ch + g) * CL_M + tid) * 16) = u;
                }
            }
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();

        // ---- G W2 into TMEM columns [C, 2C) ----
        if (tid == 0) {
            const uint64_t ad = umma::desc(umma::smem_u32(s_g), LBO_A1, 128);
            const uint64_t bd = umma::desc(umma::smem_u32(sm + S::w2_off), LBO_B, 128);
#pragma unroll
            for (int kk = 0; kk < C / 16; ++kk) {
                const uint64_t ak = ad + ((2 * kk * LBO_A1) >> 4), bk = bd + ((2 * kk * LBO_B) >> 4);
                umma::mma_bf16(tmem + C, ak, bk, idesc, kk > 0);
                if constexpr (SPLIT) {  // the low parts: G at C / 8 groups on, W2 after its high part
                    umma::mma_bf16(tmem + S::LO + C, ak, bk + ((C * C * 2) >> 4), idesc, kk > 0);
                    umma::mma_bf16(tmem + S::LO + C, ak + ((C / 8 * LBO_A1) >> 4), bk, idesc, 1);
                }
            }
            umma::commit(mbar);
        }
        failed = __syncthreads_or(!umma::mbar_wait(mbar, phase, CL_WAIT_NS));
        umma::fence_after_sync();
        if (failed) {
            fail_code = 6;
            break;
        }
        phase ^= 1;
        if constexpr (SPLIT) {
            // out = 0.5 (a + b) + b2 + 2^ge_exp (O_hi + 2^-11 O_lo), FP32
            float* po = reinterpret_cast<float*>(a.out) + ((size_t)j * plane + pixc) * C;
#pragma unroll
            for (int ch = 0; ch < C / 16; ++ch) {
                float ov[16], ol[16];
                tmem_row16(tmem, warp, C + ch * 16, ov);
                tmem_row16(tmem, warp, S::LO + C + ch * 16, ol);
                uint4 u[4];
                float* f = reinterpret_cast<float*>(u);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int c = ch * 16 + i;
                    f[i] = avg[c] + s_b[C + c] + ldexpf(fmaf(ol[i], 1.0f / 2048.f, ov[i]), ge_exp);
                }
                if (live) {
                    stg256(po + ch * 16, u[0], u[1]);
                    stg256(po + ch * 16 + 8, u[2], u[3]);
                }
            }
        } else {
            __nv_bfloat16* po = reinterpret_cast<__nv_bfloat16*>(a.out) + ((size_t)j * plane + pixc) * C;
#pragma unroll
            for (int ch = 0; ch < C / 16; ++ch) {
                float ov[16];
                tmem_row16(tmem, warp, C + ch * 16, ov);
                uint4 u[2];
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&u[g]);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int c = ch * 16 + 8 * g + 2 * i;
                        hh[i] = __floats2bfloat162_rn(avg[c] + s_b[C + c] + ov[8 * g + 2 * i],
                                                      avg[c + 1] + s_b[C + c + 1] + ov[8 * g + 2 * i + 1]);
                    }
                }
                if (live) stg256(po + ch * 16, u[0], u[1]);  // 16 channels, one 256-bit store
            }
        }
        // this tile's TMEM reads before the next tile's MMAs
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
    }
    if (failed && tid == 0) {
        atomicExch(a.err, fail_code);
        umma::mbar_wait(mbar, phase, CL_WAIT_NS);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(tmem, S::tmem_cols);
}

cudaError_t launch_collapse_tc(const CollapseArgs& a, int C, bool split, cudaStream_t st) {
    if (!a.wtc || !a.err) return cudaErrorInvalidValue;
    // 256-bit pixel loads and stores
    if (reinterpret_cast<uintptr_t>(a.in) % 32 || reinterpret_cast<uintptr_t>(a.out) % 32) return cudaErrorMisalignedAddress;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const size_t plane = (size_t)a.H * a.W;
    const long ntiles = (long)((plane + CL_M - 1) / CL_M) * a.L;
    if (ntiles == 0) return cudaSuccess;
    // persistent CTAs per SM, as shared memory and TMEM columns allow: BF16 six (C <= 32) or three
    // (C = 64: 72 KB and 128 columns each); FP32 split (C <= 32) three (62 KB, 4C columns each)
    const long per_sm = split ? 3L : (C == 64 ? 3L : 6L);
    const unsigned grid = (unsigned)std::min<long>(ntiles, per_sm * sms);
#define QK_CL_LAUNCH(CV, SV)                                                                           \
    do {                                                                                               \
        auto k = collapse_tc_kernel<CV, SV>;                                                           \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, ClSmem<CV, SV>::total); \
        if (e != cudaSuccess) return e;                                                                \
        k<<<grid, CL_M, ClSmem<CV, SV>::total, st>>>(a, make_fastdiv((uint32_t)((plane + CL_M - 1) / CL_M))); \
    } while (0)
    if (split) {
        if (C == 16) QK_CL_LAUNCH(16, true);
        else if (C == 32) QK_CL_LAUNCH(32, true);
        else return cudaErrorInvalidValue;
    } else {
        if (C == 16) QK_CL_LAUNCH(16, false);
        else if (C == 32) QK_CL_LAUNCH(32, false);
        else if (C == 64) QK_CL_LAUNCH(64, false);
        else return cudaErrorInvalidValue;
    }
#undef QK_CL_LAUNCH
    return cudaGetLastError();
}

}  // namespace quark
