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
#include <algorithm>

#include "device_common.cuh"
#include "umma.cuh"

namespace quark {

constexpr int CL_M = 128;
constexpr uint64_t CL_WAIT_NS = 1000000000ull;

template <int C>
struct ClSmem {
    static constexpr int x_off = 0;                        // A: 128 x 2C bf16
    static constexpr int g_off = x_off + CL_M * 2 * C * 2;  // A: 128 x C bf16
    static constexpr int w1_off = g_off + CL_M * C * 2;     // B: C x 2C bf16
    static constexpr int w2_off = w1_off + 2 * C * C * 2;   // B: C x C bf16
    static constexpr int b_off = w2_off + C * C * 2;        // b1 [C], b2 [C] fp32
    static constexpr int bar_off = b_off + 2 * C * 4;
    static constexpr int total = bar_off + 16;
    static constexpr uint32_t tmem_cols = 2 * C;  // X W1 in [0, C), G W2 in [C, 2C)
};

// 16 consecutive TMEM columns of this warp's lanes
__device__ __forceinline__ void tmem_row16(uint32_t tmem, int warp, int col, float (&v)[16]) {
    umma::ld_32x32b_x16(tmem + ((uint32_t)(warp * 32) << 16) + col, v);
}

template <int C>
__global__ void __launch_bounds__(CL_M) collapse_tc_kernel(const CollapseArgs a) {
    using S = ClSmem<C>;
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
        constexpr int n16 = 3 * C * C * 2 / 16;
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
    constexpr uint32_t idesc = umma::idesc_bf16_f32(CL_M, C);
    constexpr uint32_t LBO_A1 = CL_M * 16, LBO_B = C * 16;
    uint32_t phase = 0;
    bool failed = false;
    int fail_code = 0;

    // persistent: tiles of 128 pixels of one output layer j, the layer pair (2j, 2j+1) in
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int j = tile / tiles_p;
        const size_t pix = (size_t)(tile % tiles_p) * CL_M + tid;
        const bool live = pix < plane;
        const size_t pixc = live ? pix : plane - 1;
        // X row of this element: channel group g (8 bf16) of row m at g * 128 * 16 + m * 16
        // (the previous tile's MMAs, which read X and G, completed before its epilogue)
        float avg[C];
        {
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
            for (int kk = 0; kk < 2 * C / 16; ++kk)
                umma::mma_bf16(tmem, ad + ((2 * kk * LBO_A1) >> 4), bd + ((2 * kk * LBO_B) >> 4), idesc, kk > 0);
            umma::commit(mbar);
        }
        failed = __syncthreads_or(!umma::mbar_wait(mbar, phase, CL_WAIT_NS));
        umma::fence_after_sync();
        if (failed) {
            fail_code = 5;
            break;
        }
        phase ^= 1;
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
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();

        // ---- G W2 into TMEM columns [C, 2C) ----
        if (tid == 0) {
            const uint64_t ad = umma::desc(umma::smem_u32(s_g), LBO_A1, 128);
            const uint64_t bd = umma::desc(umma::smem_u32(sm + S::w2_off), LBO_B, 128);
#pragma unroll
            for (int kk = 0; kk < C / 16; ++kk)
                umma::mma_bf16(tmem + C, ad + ((2 * kk * LBO_A1) >> 4), bd + ((2 * kk * LBO_B) >> 4), idesc, kk > 0);
            umma::commit(mbar);
        }
        failed = __syncthreads_or(!umma::mbar_wait(mbar, phase, CL_WAIT_NS));
        umma::fence_after_sync();
        if (failed) {
            fail_code = 6;
            break;
        }
        phase ^= 1;
        {
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

cudaError_t launch_collapse_tc(const CollapseArgs& a, int C, cudaStream_t st) {
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
    // persistent CTAs: six per SM (shared memory and TMEM columns allow it at C <= 32; at C = 64,
    // 72 KB of shared memory and 128 TMEM columns each: three)
    const unsigned grid = (unsigned)std::min<long>(ntiles, (C == 64 ? 3L : 6L) * sms);
#define QK_CL_LAUNCH(CV)                                                                               \
    do {                                                                                               \
        auto k = collapse_tc_kernel<CV>;                                                               \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, ClSmem<CV>::total); \
        if (e != cudaSuccess) return e;                                                                \
        k<<<grid, CL_M, ClSmem<CV>::total, st>>>(a);                                                   \
    } while (0)
    if (C == 16) QK_CL_LAUNCH(16);
    else if (C == 32) QK_CL_LAUNCH(32);
    else if (C == 64) QK_CL_LAUNCH(64);
    else return cudaErrorInvalidValue;
#undef QK_CL_LAUNCH
    return cudaGetLastError();
}

}  // namespace quark
