// Encode Input Images (Sec. 3.2.1) in the BF16 form with the convolution on tcgen05 tensor cores:
// F_1 = conv3x3(I) (3 -> C, zero pad, bias, no activation) as a GEMM of the image patches
// (M = 128 pixels, K = 27 taps x channels padded to 32, N = C) with BF16 operands and FP32
// accumulation in TMEM; F_2k = 2x2 mean pool of F_k, taken from the FP32 accumulators.  Also
// writes the RGBA-padded copy of the images used by the render.
//
// Persistent CTAs of 128 threads stride over 16 x 8 pixel tiles of the views (a thread per pixel,
// which is also its TMEM lane):
//   1. the tile's 18 x 10 x 3 image patch (prefetched with cp.async during the previous tile);
//   2. each thread writes its pixel's 27 patch values (and 5 zeros) as a K-major row of the A
//      operand; one thread issues the two K = 16 MMAs into TMEM and commits to an mbarrier;
//   3. each thread reads its pixel's C accumulators, adds the bias and stores the level-1 texel
//      (BF16, 256-bit stores); the 2x2 means of level 2 are taken with shuffles within the warp
//      (a warp holds two tile rows), levels 4 and 8 from level-2 texels staged in shared memory.
// Every wait is bounded; on a timeout the CTA records the error and stops.
#include <algorithm>

#include "device_common.cuh"
#include "umma.cuh"

namespace quark {

constexpr int ET_W = 16, ET_H = 8, ET_M = ET_W * ET_H;  // tile (pixels) = M
constexpr int ET_PW = ET_W + 2, ET_PH = ET_H + 2;       // image patch incl. the 1-pixel halo
constexpr int ET_K = 32;                                // 27 taps x channels, zero-padded
// Row stride of the image patch in shared memory, in floats: 80 = 16 (mod 32), so that the two tile
// rows of a warp (16 pixels at a 3-float stride each) read 32 distinct banks
constexpr int ET_PROW = 80;
constexpr uint64_t ET_WAIT_NS = 1000000000ull;

template <int C>
struct EtSmem {
    static constexpr int a_off = 0;                                 // A: 128 x 32 bf16, K-major
    static constexpr int b_off = a_off + ET_M * ET_K * 2;           // B: C x 32 bf16
    static constexpr int patch_off = b_off + C * ET_K * 2;          // fp32 [2][10][ET_PROW] (18 x 3 used)
    // level-2 texels at a stride of C + 4 floats: the eight texels a warp stages fall on distinct banks
    static constexpr int L2S = C + 4;
    static constexpr int l2_off = patch_off + 2 * ET_PH * ET_PROW * 4;  // fp32 level-2 texels [4][8][L2S]
    static constexpr int l4_off = l2_off + 4 * 8 * L2S * 4;         // fp32 level-4 texels [2][4][C]
    static constexpr int bias_off = l4_off + 2 * 4 * C * 4;         // fp32 [C]
    static constexpr int bar_off = (bias_off + C * 4 + 7) / 8 * 8;
    static constexpr int total = bar_off + 16;
    static constexpr uint32_t tmem_cols = C <= 32 ? 32 : 64;
};

// a tile's view and pixel origin (divisions by the launch's tile counts: FastDiv)
struct EtTile {
    int v, X0, Y0;
};
__device__ __forceinline__ EtTile et_tile(int tile, const FastDiv& per_view, const FastDiv& tiles_x) {
    const int v = fdiv(tile, per_view), r = tile - v * (int)per_view.d;
    const int ty = fdiv(r, tiles_x);
    return EtTile{v, (r - ty * (int)tiles_x.d) * ET_W, ty * ET_H};
}

__device__ __forceinline__ void et_cp_async4(float* smem, const float* gmem, bool valid) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0) : "memory");
}

// the tile's image patch (rows Y0-1 .. Y0+8, columns X0-1 .. X0+16, zero outside the image)
__device__ __forceinline__ void et_fetch_patch(const EncodeArgs& a, const EtTile& t, float* patch) {
    const int X0 = t.X0, Y0 = t.Y0;
    const float* img = a.images + (size_t)t.v * a.H * a.W * 3;
    for (int i = threadIdx.x; i < ET_PH * ET_PW * 3; i += ET_M) {
        const int c = i % 3, px = (i / 3) % ET_PW, py = i / (3 * ET_PW);
        const int gy = Y0 - 1 + py, gx = X0 - 1 + px;
        const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
        et_cp_async4(patch + py * ET_PROW + px * 3 + c, in ? img + ((size_t)gy * a.W + gx) * 3 + c : img, in);
    }
}

// store 16 channels (fp32 values) of a texel as BF16 in one 256-bit store
__device__ __forceinline__ void et_store16(__nv_bfloat16* p, const float* v) {
    uint4 u[2];
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(u);
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    stg256(p, u[0], u[1]);
}

template <int C>
__global__ void __launch_bounds__(ET_M, C == 64 ? 4 : 8) encode_tc_kernel(const EncodeArgs a, const void* wtc, int* err,
                                                                          const FastDiv per_view, const FastDiv tiles_x) {
    using S = EtSmem<C>;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* s_a = sm + S::a_off;
    float* s_patch = reinterpret_cast<float*>(sm + S::patch_off);
    float* s_l2 = reinterpret_cast<float*>(sm + S::l2_off);
    float* s_l4 = reinterpret_cast<float*>(sm + S::l4_off);
    float* s_bias = reinterpret_cast<float*>(sm + S::bias_off);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::bar_off + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W;
    const int ntiles = (int)per_view.d * a.V;
    {
        const uint4* src = reinterpret_cast<const uint4*>(wtc);
        uint4* dst = reinterpret_cast<uint4*>(sm + S::b_off);
        for (int i = tid; i < C * ET_K * 2 / 16; i += ET_M) dst[i] = __ldg(src + i);
        for (int i = tid; i < C; i += ET_M) s_bias[i] = a.w[27 * C + i];
    }
    if (warp == 0) umma::tmem_alloc(tslot, S::tmem_cols);
    if (tid == 0) umma::mbar_init(mbar, 1);
    umma::fence_smem_to_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(ET_M, C);
    constexpr uint32_t LBO_A = ET_M * 16, LBO_B = C * 16;
    const int px = tid % ET_W, py = tid / ET_W;  // this thread's pixel in the tile
    uint32_t phase = 0;
    bool failed = false;

    int tile = blockIdx.x;
    EtTile cur = et_tile(tile, per_view, tiles_x);
    if (tile < ntiles) et_fetch_patch(a, cur, s_patch);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        float* patch = s_patch + (it & 1) * (ET_PH * ET_PROW);
        const EtTile nxt = et_tile(tile + gridDim.x, per_view, tiles_x);
        if (tile + (int)gridDim.x < ntiles) et_fetch_patch(a, nxt, s_patch + ((it + 1) & 1) * (ET_PH * ET_PROW));
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this tile's patch has landed
        __syncthreads();
        const int v = cur.v, X0 = cur.X0, Y0 = cur.Y0;
        const int X = X0 + px, Y = Y0 + py;
        const bool inside = X < W && Y < H;

        // ---- A row of this pixel: patch values in (dy, dx, ci) order, then zeros ----
        {
            float k[ET_K];
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                    for (int ci = 0; ci < 3; ++ci) k[(dy * 3 + dx) * 3 + ci] = patch[(py + dy) * ET_PROW + (px + dx) * 3 + ci];
#pragma unroll
            for (int i = 27; i < ET_K; ++i) k[i] = 0.f;
#pragma unroll
            for (int g = 0; g < ET_K / 8; ++g) {
                uint4 u;
                __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
                for (int j = 0; j < 4; ++j) hh[j] = __floats2bfloat162_rn(k[8 * g + 2 * j], k[8 * g + 2 * j + 1]);
                *reinterpret_cast<uint4*>(s_a + ((size_t)g * ET_M + tid) * 16) = u;
            }
            if (inside)
                a.rgba[((size_t)v * H + Y) * W + X] = make_float4(k[12], k[13], k[14], 0.f);  // the centre tap
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (tid == 0) {
            const uint64_t ad = umma::desc(umma::smem_u32(s_a), LBO_A, 128);
            const uint64_t bd = umma::desc(umma::smem_u32(sm + S::b_off), LBO_B, 128);
#pragma unroll
            for (int kk = 0; kk < ET_K / 16; ++kk)
                umma::mma_bf16(tmem, ad + ((2 * kk * LBO_A) >> 4), bd + ((2 * kk * LBO_B) >> 4), idesc, kk > 0);
            umma::commit(mbar);
        }
        // one thread polls the MMA's mbarrier; the others wait at the CTA barrier, leaving the issue
        // slots to the SM's other CTAs (the fence after the barrier orders their TMEM reads)
        failed = __syncthreads_or(tid == 0 && !umma::mbar_wait_suspend(mbar, phase, ET_WAIT_NS));
        umma::fence_after_sync();
        if (failed) break;
        phase ^= 1;

        // ---- level 1 and the 2x2 means (lanes ^ 1: x + 1, ^ 16: y + 1) ----
        float f[C];
        if constexpr (C == 64) {
            float hi[32];
            umma::ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16), *reinterpret_cast<float(*)[32]>(f));
            umma::ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + 32, hi);
#pragma unroll
            for (int c = 0; c < 32; ++c) f[32 + c] = hi[c];
        } else if constexpr (C == 32) {
            umma::ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16), f);
        } else {
            umma::ld_32x32b_x16(tmem + ((uint32_t)(warp * 32) << 16), f);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) f[c] += s_bias[c];
        if (a.level[0] && inside) {
            __nv_bfloat16* l1 = reinterpret_cast<__nv_bfloat16*>(a.level[0]) + (((size_t)v * H + Y) * W + X) * C;
#pragma unroll
            for (int c0 = 0; c0 < C; c0 += 16) et_store16(l1 + c0, f + c0);
        }
        // The 2x2 block's four lanes split its sums: the x partners (lane ^ 1) exchange halves of the
        // channels, then the y partners (lane ^ 16) halves of those halves, so that each lane ends
        // with a quarter of the channels of the block's sum (C / 2 + C / 4 shuffles instead of 2 C;
        // the pairings, and so the rounded sums, are those of (f00 + f01) + (f10 + f11)).
        constexpr int HC = C / 2, QC = C / 4;
        const bool xo = px & 1, yo = lane & 16;
        float g[HC];
#pragma unroll
        for (int i = 0; i < HC; ++i) {
            const float r = __shfl_xor_sync(0xffffffffu, xo ? f[i] : f[HC + i], 1);
            g[i] = (xo ? f[HC + i] : f[i]) + r;
        }
        float q[QC];
#pragma unroll
        for (int i = 0; i < QC; ++i) {
            const float r = __shfl_xor_sync(0xffffffffu, yo ? g[i] : g[QC + i], 16);
            q[i] = 0.25f * ((yo ? g[QC + i] : g[i]) + r);
        }
        // every lane of the block stores its quarter of the level-2 texel (channels cq .. cq + C / 4)
        const int cq = (xo ? HC : 0) + (yo ? QC : 0);
        const int x2 = px >> 1, y2 = warp;  // level-2 texel within the tile (8 x 4)
        {
            const int X2 = X0 / 2 + x2, Y2 = Y0 / 2 + y2;
            if (a.level[1] && X2 < W / 2 && Y2 < H / 2) {
                __nv_bfloat16* l2 =
                    reinterpret_cast<__nv_bfloat16*>(a.level[1]) + (((size_t)v * (H / 2) + Y2) * (W / 2) + X2) * C + cq;
                if constexpr (QC == 16) {
                    et_store16(l2, q);
                } else {
                    uint32_t u[QC / 2];
#pragma unroll
                    for (int j = 0; j < QC / 2; ++j) {
                        const __nv_bfloat162 h = __floats2bfloat162_rn(q[2 * j], q[2 * j + 1]);
                        u[j] = *reinterpret_cast<const uint32_t*>(&h);
                    }
                    if constexpr (QC == 8) *reinterpret_cast<uint4*>(l2) = make_uint4(u[0], u[1], u[2], u[3]);
                    else *reinterpret_cast<uint2*>(l2) = make_uint2(u[0], u[1]);
                }
            }
#pragma unroll
            for (int c = 0; c < QC; c += 4)
                *reinterpret_cast<float4*>(s_l2 + (y2 * 8 + x2) * S::L2S + cq + c) = make_float4(q[c], q[c + 1], q[c + 2], q[c + 3]);
        }
        // this tile's TMEM reads, before the next tile's MMA; the level-2 texels for the next means
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();

        // ---- level 4 (4 x 2 texels of the tile): thread = texel (t / 16) x channel pair (t % 16) ----
        if (a.level[2] || a.level[3]) {
            constexpr int PAIRS = C / 2;
            for (int i = tid; i < 8 * PAIRS; i += ET_M) {
                const int q = i / PAIRS, cp = 2 * (i % PAIRS);
                const int x4 = q % 4, y4 = q / 4;
                float2 s = make_float2(0.f, 0.f);
#pragma unroll
                for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const float2 t = *reinterpret_cast<const float2*>(s_l2 + ((2 * y4 + dy) * 8 + 2 * x4 + dx) * S::L2S + cp);
                        s.x += t.x;
                        s.y += t.y;
                    }
                s = make_float2(0.25f * s.x, 0.25f * s.y);
                s_l4[(y4 * 4 + x4) * C + cp] = s.x;
                s_l4[(y4 * 4 + x4) * C + cp + 1] = s.y;
                const int X4 = X0 / 4 + x4, Y4 = Y0 / 4 + y4;
                if (a.level[2] && X4 < W / 4 && Y4 < H / 4)
                    *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(a.level[2]) +
                                                       (((size_t)v * (H / 4) + Y4) * (W / 4) + X4) * C + cp) =
                        __floats2bfloat162_rn(s.x, s.y);
            }
            __syncthreads();
            // ---- level 8 (2 x 1 texels of the tile) ----
            if (a.level[3]) {
                for (int i = tid; i < 2 * PAIRS; i += ET_M) {
                    const int x8 = i / PAIRS, cp = 2 * (i % PAIRS);
                    float2 s = make_float2(0.f, 0.f);
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            const float* p = s_l4 + (dy * 4 + 2 * x8 + dx) * C + cp;
                            s.x += p[0];
                            s.y += p[1];
                        }
                    const int X8 = X0 / 8 + x8, Y8 = Y0 / 8;
                    if (X8 < W / 8 && Y8 < H / 8)
                        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(a.level[3]) +
                                                           (((size_t)v * (H / 8) + Y8) * (W / 8) + X8) * C + cp) =
                            __floats2bfloat162_rn(0.25f * s.x, 0.25f * s.y);
                }
            }
        }
        __syncthreads();  // the patch buffer and the staged texels are reused by the next tile
        cur = nxt;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (failed) {
        if (tid == 0) atomicExch(err, 9);
        umma::mbar_wait_suspend(mbar, phase, ET_WAIT_NS);  // nothing of ours may still run when TMEM is freed
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(tmem, S::tmem_cols);
}

// CTAs of 128 threads resident per SM: registers (64 K per SM, allocated per warp in units of 256),
// shared memory (228 KB per SM, 1 KB reserved per CTA) and TMEM (512 columns, 32 or 64 per CTA)
static int et_ctas_per_sm(int regs, int smem, int tmem_cols) {
    const int warp_regs = (regs * 32 + 255) / 256 * 256;
    const int by_regs = 65536 / (warp_regs * (ET_M / 32));
    const int by_smem = (228 * 1024) / (smem + 1024);
    return std::max(1, std::min(std::min(by_regs, by_smem), 512 / tmem_cols));
}

cudaError_t launch_encode_tc(const EncodeArgs& a, int C, const void* wtc, int* err, cudaStream_t st) {
    if (!wtc || !err) return cudaErrorInvalidValue;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const int tiles_x = (a.W + ET_W - 1) / ET_W, tiles_y = (a.H + ET_H - 1) / ET_H;
    const long ntiles = (long)tiles_x * tiles_y * a.V;
    if (ntiles == 0) return cudaSuccess;
    // persistent: as many CTAs per SM as fit at once (registers bind; ~20 KB of shared memory and 32
    // TMEM columns each), striding over the tiles
#define QK_ET_LAUNCH(CV)                                                                               \
    do {                                                                                               \
        auto k = encode_tc_kernel<CV>;                                                                 \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, EtSmem<CV>::total); \
        if (e == cudaSuccess)                                                                          \
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared); \
        cudaFuncAttributes fa{};                                                                       \
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);                                       \
        if (e != cudaSuccess) return e;                                                                \
        const int per_sm = et_ctas_per_sm(fa.numRegs, EtSmem<CV>::total, (int)EtSmem<CV>::tmem_cols);                               \
        const int grid = (int)std::min<long>(ntiles, (long)per_sm * sms);                              \
        k<<<grid, ET_M, EtSmem<CV>::total, st>>>(a, wtc, err, make_fastdiv((uint32_t)(tiles_x * tiles_y)), \
                                                 make_fastdiv((uint32_t)tiles_x));                      \
    } while (0)
    if (C == 16) QK_ET_LAUNCH(16);
    else if (C == 32) QK_ET_LAUNCH(32);
    else if (C == 64) QK_ET_LAUNCH(64);
    else return cudaErrorInvalidValue;
#undef QK_ET_LAUNCH
    return cudaGetLastError();
}

}  // namespace quark
