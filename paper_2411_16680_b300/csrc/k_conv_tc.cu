// Residual conv block on 5th-generation tensor cores (BF16 form): V' = V + Conv2(gelu(Conv1(N(V))))
// with 3x3 convolutions per layer plane (Sec. 3.3); when asked (the last step), also the raw
// depth and density logits of V' as stored in BF16 (Sec. 3.2.2 "Decoding").  BF16 operands, FP32
// accumulation in TMEM; normalisation, gelu and residual in FP32 registers.
//
// Implicit GEMM.  An output tile is TC_R rows x 126 columns of one layer plane; two persistent
// CTAs share an SM and stride over the tiles (the packed weights are staged once per CTA), so one
// CTA's tile loads overlap the other's MMAs and epilogues.  Each
// tile row is one M = 128 MMA block (pixels), N = C (output channels), K = 9 taps x C input
// channels.  The normalised input tile (TC_R + 4 rows x 130 columns) is stored channel-group
// major -- pixel p, channel c at (c / 8) * NPIX * 16 + p * 16 + (c % 8) * 2 -- so the A operand of
// tap (dy, dx) for row r is the same layout started (r + dy) * 130 + dx pixels further on: a
// 16-byte-aligned shift of the descriptor start, no data movement.  Conv1 fills TC_R + 2 mid rows
// of 128 pixels in TMEM (columns r * C ..), the epilogue writes gelu(conv1 + b1) back to shared
// memory as BF16 in the same layout (zero outside the plane: conv2's padding), and conv2 reuses
// the TMEM columns for TC_R output rows; its 128-row blocks read two mid pixels past the 126
// valid outputs, whose results are discarded.  One thread issues the MMAs; completion is
// signalled through an mbarrier with a bounded wait.
#include <algorithm>

#include "device_common.cuh"
#include "umma.cuh"

namespace quark {

constexpr int TC_R = 4;  // output rows per tile: two CTAs fit on an SM
constexpr int TC_M = 128;
constexpr int TC_OUT_W = TC_M - 2;
constexpr int TC_IN_W = TC_M + 2;
constexpr int TC_IN_H = TC_R + 4;
constexpr int TC_MID_H = TC_R + 2;
constexpr int TC_THREADS = 256;
constexpr uint64_t TC_WAIT_NS = 1000000000ull;  // 1 s bound on every MMA wait

template <int C>
struct TcSmem {
    static constexpr int G = C / 8;
    static constexpr int NPIX_IN = TC_IN_H * TC_IN_W + 8;
    static constexpr int NPIX_MID = TC_MID_H * TC_M + 8;
    // the mid tile reuses the input tile's memory: conv1 has finished reading it when the
    // first epilogue writes gelu(conv1)
    static constexpr int in_off = 0;
    static constexpr int mid_off = 0;
    static_assert(NPIX_MID <= NPIX_IN, "mid tile must fit in the input tile");
    static constexpr int w1_off = in_off + G * NPIX_IN * 16;
    static constexpr int w2_off = w1_off + 9 * C * C * 2;
    static constexpr int misc_off = w2_off + 9 * C * C * 2;
    static constexpr int misc_n = 8 * C + 8;
    static constexpr int bar_off = misc_off + misc_n * 4;
    static constexpr int total = bar_off + 16;
    static_assert(2 * (total + 1024) <= 233472, "two CTAs per SM");
};

template <int C>
__device__ __forceinline__ void store_pixel_bf16(uint8_t* base, int npix, int p, const float (&v)[C]) {
#pragma unroll
    for (int g = 0; g < C / 8; ++g) {
        uint4 u;
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(v[8 * g + 2 * j], v[8 * g + 2 * j + 1]);
        *reinterpret_cast<uint4*>(base + ((size_t)g * npix + p) * 16) = u;
    }
}

template <int C>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float (&v)[C]) {
    if constexpr (C == 32) {
        umma::ld_32x32b_x32(taddr, v);
    } else {
        umma::ld_32x32b_x16(taddr, v);
    }
}

template <int C>
__global__ void __launch_bounds__(TC_THREADS, 2) conv_block_tc_kernel(const ConvArgs a) {
    using S = TcSmem<C>;
    constexpr uint32_t TMEM_COLS = TC_MID_H * C <= 128 ? 128 : 256;  // conv1 accumulators, per CTA
    static_assert(TC_MID_H * C <= 256, "TMEM budget of two CTAs");
    const ConvLayout lay{C};
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* s_in = sm + S::in_off;
    uint8_t* s_mid = sm + S::mid_off;
    uint8_t* s_w1 = sm + S::w1_off;
    uint8_t* s_w2 = sm + S::w2_off;
    float* misc = reinterpret_cast<float*>(sm + S::misc_off);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::bar_off + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W, L = a.L;
    const size_t plane = (size_t)H * W;
    const int tiles_x = (W + TC_OUT_W - 1) / TC_OUT_W, tiles_y = (H + TC_R - 1) / TC_R;
    const int ntiles = tiles_x * tiles_y * L;

    // ---- constants and packed BF16 weights ----
    for (int i = tid; i < C; i += TC_THREADS) {
        misc[i] = a.w[lay.g() + i];
        misc[C + i] = a.w[lay.b1() + i];
        misc[2 * C + i] = a.w[lay.b2() + i];
        misc[3 * C + i] = a.w[lay.wd() + i];
        misc[4 * C + i] = a.w[lay.ws() + i];
    }
    if (tid == 3) misc[8 * C + 3] = a.w[lay.bd()];
    if (tid == 4) misc[8 * C + 4] = a.w[lay.bs()];
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.wtc);
        uint4* d1 = reinterpret_cast<uint4*>(s_w1);
        uint4* d2 = reinterpret_cast<uint4*>(s_w2);
        constexpr int n = 9 * C * C * 2 / 16;
        for (int i = tid; i < n; i += TC_THREADS) {
            d1[i] = __ldg(src + i);
            d2[i] = __ldg(src + n + i);
        }
    }
    if (warp == 0) umma::tmem_alloc(tslot, TMEM_COLS);
    if (tid == 0) umma::mbar_init(mbar, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(TC_M, C);
    constexpr uint32_t LBO_W = C * 16;  // B: N = C rows of 16 B per core-matrix column
    const int q = warp & 3, half = warp >> 2;
    const int col = q * 32 + lane;  // the pixel (TMEM lane) this thread reads
    uint32_t phase = 0;             // parity of the next completion of mbar
    bool failed = false;
    int fail_code = 0;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * TC_OUT_W, y0 = ((tile / tiles_x) % tiles_y) * TC_R;
        const int li = tile / (tiles_x * tiles_y);
        const __nv_bfloat16* vin = reinterpret_cast<const __nv_bfloat16*>(a.in) + (size_t)li * plane * C;

        // ---- normalised input tile: rows y0-2 .. y0+TC_R+1, columns x0-2 .. x0+127 ----
        // (the mid tile of the previous tile, which shares this memory, was last read by its conv2,
        // complete before that tile's epilogue)
        // two pixels per thread per iteration: both pixels' loads are in flight before either is used
        constexpr int NPIX = TC_IN_H * TC_IN_W;
        for (int p0 = tid; p0 < NPIX; p0 += 2 * TC_THREADS) {
            uint4 raw[2][C / 8];
            bool in[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int p = p0 + u * TC_THREADS;
                const int gy = y0 - 2 + p / TC_IN_W, gx = x0 - 2 + p % TC_IN_W;
                in[u] = p < NPIX && gy >= 0 && gy < H && gx >= 0 && gx < W;
                const uint4* src = reinterpret_cast<const uint4*>(vin + ((size_t)(in[u] ? gy : 0) * W + (in[u] ? gx : 0)) * C);
#pragma unroll
                for (int g = 0; g < C / 8; ++g) raw[u][g] = in[u] ? __ldg(src + g) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int p = p0 + u * TC_THREADS;
                if (p >= NPIX) break;
                float v[C];
#pragma unroll
                for (int g = 0; g < C / 8; ++g) {
                    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw[u][g]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float2 f = __bfloat1622float2(h[j]);
                        v[8 * g + 2 * j] = f.x;
                        v[8 * g + 2 * j + 1] = f.y;
                    }
                }
                float ms = 0.f;
#pragma unroll
                for (int c = 0; c < C; ++c) ms = fmaf(v[c], v[c], ms);
                const float r = in[u] ? 1.0f / sqrtf(ms / C + 1e-6f) : 0.f;
#pragma unroll
                for (int c = 0; c < C; ++c) v[c] = v[c] * r * misc[c];
                store_pixel_bf16<C>(s_in, S::NPIX_IN, p, v);
            }
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();

        // ---- conv1: TC_MID_H row blocks ----
        if (tid == 0) {
            // descriptors built once; each MMA adds its constant start offset (in 16-byte units) to
            // the start-address field, which stays below 2^14 for any shared-memory address
            constexpr uint32_t LBO_A = S::NPIX_IN * 16;
            const uint64_t ad0 = umma::desc(umma::smem_u32(s_in), LBO_A, 128);
            const uint64_t bd0 = umma::desc(umma::smem_u32(s_w1), LBO_W, 128);
#pragma unroll
            for (int r = 0; r < TC_MID_H; ++r)
#pragma unroll
                for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                    for (int kk = 0; kk < C / 16; ++kk) {
                        const int dy = tap / 3, dx = tap % 3;
                        const uint32_t ao = (((r + dy) * TC_IN_W + dx) * 16 + 2 * kk * LBO_A) >> 4;
                        const uint32_t bo = (tap * C * C * 2 + 2 * kk * LBO_W) >> 4;
                        umma::mma_bf16(tmem + r * C, ad0 + ao, bd0 + bo, idesc, (tap | kk) != 0);
                    }
            umma::commit(mbar);
        }
        failed = __syncthreads_or(!umma::mbar_wait(mbar, phase, TC_WAIT_NS));
        umma::fence_after_sync();
        if (failed) {
            fail_code = 1;
            break;
        }
        phase ^= 1;
        {
            // ---- epilogue 1: gelu(conv1 + b1) -> BF16 mid tile, zero outside the plane ----
            for (int r = half; r < TC_MID_H; r += 2) {
                float v[C];
                tmem_load_row<C>(tmem + ((uint32_t)(q * 32) << 16) + r * C, v);
                const int gy = y0 - 1 + r, gx = x0 - 1 + col;
                const bool inside = gy >= 0 && gy < H && gx >= 0 && gx < W;
#pragma unroll
                for (int c = 0; c < C; c += 2) {
                    const float2 g = gelu_poly2(__fadd2_rn(make_float2(v[c], v[c + 1]), make_float2(misc[C + c], misc[C + c + 1])));
                    v[c] = inside ? g.x : 0.f;
                    v[c + 1] = inside ? g.y : 0.f;
                }
                store_pixel_bf16<C>(s_mid, S::NPIX_MID, r * TC_M + col, v);
            }
            umma::fence_smem_to_async();
            umma::fence_before_sync();
            __syncthreads();
            umma::fence_after_sync();

            // ---- conv2: TC_R row blocks, reusing TMEM columns ----
            if (tid == 0) {
                constexpr uint32_t LBO_A = S::NPIX_MID * 16;
                const uint64_t ad0 = umma::desc(umma::smem_u32(s_mid), LBO_A, 128);
                const uint64_t bd0 = umma::desc(umma::smem_u32(s_w2), LBO_W, 128);
#pragma unroll
                for (int r = 0; r < TC_R; ++r)
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                        for (int kk = 0; kk < C / 16; ++kk) {
                            const int dy = tap / 3, dx = tap % 3;
                            const uint32_t ao = (((r + dy) * TC_M + dx) * 16 + 2 * kk * LBO_A) >> 4;
                            const uint32_t bo = (tap * C * C * 2 + 2 * kk * LBO_W) >> 4;
                            umma::mma_bf16(tmem + r * C, ad0 + ao, bd0 + bo, idesc, (tap | kk) != 0);
                        }
                umma::commit(mbar);
            }
            failed = __syncthreads_or(!umma::mbar_wait(mbar, phase, TC_WAIT_NS));
            umma::fence_after_sync();
            if (failed) {
                fail_code = 2;
                break;
            }
            phase ^= 1;
            {
                // ---- epilogue 2: residual, V_out, decode ----
                for (int r = half; r < TC_R; r += 2) {
                    float v[C];
                    tmem_load_row<C>(tmem + ((uint32_t)(q * 32) << 16) + r * C, v);
                    const int gy = y0 + r, gx = x0 + col;
                    if (col >= TC_OUT_W || gy >= H || gx >= W) continue;
                    const size_t pix = (size_t)gy * W + gx;
                    const size_t el = (size_t)li * plane + pix;
                    float t = misc[8 * C + 3], s = misc[8 * C + 4];
                    uint4* out = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.out) + el * C);
#pragma unroll
                    for (int c0 = 0; c0 < C; c0 += 16) {
                        float rr[16];
                        load16(vin + pix * C + c0, rr);
                        uint4 u[2];
                        __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(u);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int c = c0 + 2 * j;
                            hh[j] = __floats2bfloat162_rn(rr[2 * j] + v[c] + misc[2 * C + c],
                                                          rr[2 * j + 1] + v[c + 1] + misc[2 * C + c + 1]);
                            // the logits from V' as stored, as the on-demand decode computes them
                            const float2 o = __bfloat1622float2(hh[j]);
                            t = fmaf(o.y, misc[3 * C + c + 1], fmaf(o.x, misc[3 * C + c], t));
                            s = fmaf(o.y, misc[4 * C + c + 1], fmaf(o.x, misc[4 * C + c], s));
                        }
                        out[c0 / 8] = u[0];
                        out[c0 / 8 + 1] = u[1];
                    }
                    if (a.t_raw) {
                        a.t_raw[pix * L + li] = t;
                        a.s_raw[pix * L + li] = s;
                    }
                }
            }
        }
        umma::fence_before_sync();  // this tile's TMEM reads before the next tile's MMAs
    }
    // on a timeout, give the MMAs still in flight another bounded wait before freeing TMEM
    if (failed && tid == 0) {
        atomicExch(a.err, fail_code);
        umma::mbar_wait(mbar, phase, TC_WAIT_NS);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(tmem, TMEM_COLS);
}

template <int C>
static cudaError_t launch_tc(const ConvArgs& a, cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = TcSmem<C>::total;
    auto k = conv_block_tc_kernel<C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long ntiles = (long)((a.W + TC_OUT_W - 1) / TC_OUT_W) * ((a.H + TC_R - 1) / TC_R) * a.L;
    const int grid = (int)std::min<long>(ntiles, 2L * sms);
    k<<<grid, TC_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conv_block_tc(const ConvArgs& a, int C, cudaStream_t st) {
    if (!a.wtc || !a.err) return cudaErrorInvalidValue;
    if (C == 16) return launch_tc<16>(a, st);
    if (C == 32) return launch_tc<32>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
