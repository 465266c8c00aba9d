// Residual conv block on 5th-generation tensor cores (BF16 form): V' = V + Conv2(gelu(Conv1(N(V))))
// with 3x3 convolutions per layer plane (Sec. 3.3); when asked (the last step), also the raw
// depth and density logits of V' as stored in BF16 (Sec. 3.2.2 "Decoding").  BF16 operands, FP32
// accumulation in TMEM; normalisation, gelu and residual in FP32 registers.
//
// Implicit GEMM on a flattened tile.  An output tile is R rows x OW columns of one layer plane; its
// input (R + 4 rows) and mid (R + 2 rows) tiles are stored with one pitch P = OW + 4 pixels,
// channel-group major -- pixel idx = row * P + column, channel c at (c / 8) * NPIX * 16 + idx * 16 +
// (c % 8) * 2 -- so tap (dy, dx) of any pixel is the pixel dy * P + dx further on, and the A operand
// of a block of 128 consecutive pixels for that tap is the same layout started that many pixels
// later: a 16-byte-aligned shift of the descriptor start, no data movement.  Blocks run across row
// ends; the two columns past each row's last valid mid column and the pixels past the last row are
// computed and discarded (a valid pixel's taps never reach them).  M = 128 pixels per block,
// N = C, K = 9 taps x C.  Conv1 fills NB1 = ceil((R + 2) P / 128) blocks in TMEM (columns i * C ..),
// the epilogue writes gelu(conv1 + b1) (tanh form on the special-function unit: within 5e-4 of the
// erf form, below the BF16 rounding of the stored value) back to shared memory as BF16 in the same
// layout (zero outside the plane: conv2's padding), and conv2 fills NB2 = ceil(R P / 128) blocks.  The host picks
// (OW, R) per plane size to minimise MMA blocks per output (tall narrow tiles waste least: two
// columns per row instead of a part-empty last block), with enough tiles for every SM.
//
// Persistent warp-specialised CTAs stride over the tiles with two input buffers each: two per SM in
// the BF16 form at C <= 32 (2 loader and 4 epilogue warps and half the TMEM each, so that one CTA's
// GELU and stores overlap the other's MMAs: 1080p conv block 1.51 -> 1.40 ms), one per SM where the
// weights fill the shared memory (the FP32 form's split operands, C = 64; 4 loader and 8 epilogue
// warps):
//   loader warps        normalise tile k into buffer k % 2 once conv2 of tile k - 2 has released it;
//   MMA warp (1 thread) conv1 of tile k into the first half of the CTA's TMEM columns, block by
//                       block, each block once its input is ready and the epilogue has read that
//                       block of tile k - 1; conv2 into the second half, block by block, each once the
//                       GELU of the conv1 blocks its 3x3 window reaches is written and the epilogue
//                       has read that conv2 block of tile k - 1; one commit (mbarrier) per block;
//   epilogue warps      gelu(conv1) -> mid tile (in the input buffer, which conv1 has read), then
//                       the residual and the stores of conv2, each block as soon as its MMAs complete,
// so the loads of one tile, the MMAs of the next and the epilogues of the previous overlap, and
// within a tile the GELU and stores of one block overlap the MMAs of the next (1080p conv block
// 1.40 -> 1.33 ms).  The packed weights are staged once.  mbarriers order the roles; every wait is
// bounded.
//
// FP32 form (SPLIT): the same kernel with every operand x split into two FP16 parts, the rounded
// value x_h = fp16(x) and the scaled remainder x_l = fp16((x - x_h) 2^11), and each product taken
// as x_h w_h + 2^-11 (x_h w_l + x_l w_h) on kind::f16 MMAs (three per K step, into a high and a
// low accumulator per block): each partial product of 11-bit significands is exact in the FP32
// accumulator and the dropped x_l w_l term is 2^-22 of the product, so the convolutions keep FP32
// accuracy at tensor-core rates.  The volume is FP32 in and out, the normalisation, gelu (the erf
// form to FP32 rounding, gelu_fine2) and residual run in FP32, and the two halves of an operand take twice the bytes of a BF16 one
// (smaller tiles).  FP16's range bounds the parts: the launcher takes this path only when the
// weights bound every normalised input and every conv1 output below 2^15 (a check on the host,
// whatever the volume); otherwise the SIMT kernel (k_conv.cu) runs.
#include <cuda_fp16.h>

#include <algorithm>

#include "device_common.cuh"
#include "umma.cuh"

namespace quark {

constexpr int TC_M = 128;
constexpr uint64_t TC_WAIT_NS = 1000000000ull;  // 1 s bound on every wait

// Tile geometry of one launch (host-chosen): pitch P = OW + 4, R output rows, NB1 / NB2 MMA blocks
// of conv1 / conv2.
struct ConvTile {
    int P, R, nb1, nb2, tiles_x, tiles_y;
    FastDiv dP, dtx, dty;  // division by P, tiles_x, tiles_y (set by with_divs)
};
static ConvTile with_divs(ConvTile t) {
    if (t.P > 0) {
        t.dP = make_fastdiv((uint32_t)t.P);
        t.dtx = make_fastdiv((uint32_t)t.tiles_x);
        t.dty = make_fastdiv((uint32_t)t.tiles_y);
    }
    return t;
}

template <int C, bool SPLIT>
struct TcSmem {
    static constexpr int G = C / 8;
    static constexpr int PLANES = SPLIT ? 2 : 1;  // operand parts: BF16, or FP16 high and scaled low
    static constexpr int CTAS = (!SPLIT && C <= 32) ? 2 : 1;  // CTAs per SM
    static constexpr int LOAD_WARPS = CTAS == 2 ? 2 : 4, EPI_WARPS = CTAS == 2 ? 4 : 8;
    static constexpr int MMA_WARP = LOAD_WARPS;  // the warp after the loaders
    static constexpr int THREADS = 32 * (LOAD_WARPS + 1 + EPI_WARPS);
    static constexpr int TMEM_COLS = 512 / CTAS;  // conv1 in the first half, conv2 in the second
    // pixels of an input / mid tile buffer (two buffers and both convs' weights in the CTA's share of
    // the 228 KB; at C = 64 the weights alone take 144 KB)
    static constexpr int NPIX = SPLIT ? (C == 32 ? 600 : 1600) : (C == 64 ? 312 : C == 32 ? 576 : 1152);
    static constexpr int NB_MAX = TMEM_COLS / 2 / (PLANES * C);  // MMA blocks per conv in half the TMEM
    // a tile's mid tile reuses its input buffer: conv1 has finished reading it when the epilogue
    // writes gelu(conv1).  Channel group g of part q at (q G + g) NPIX 16.
    static constexpr int buf_bytes = PLANES * G * NPIX * 16;  // input buffers b = 0, 1 at b * buf_bytes
    static constexpr int wconv_bytes = PLANES * 9 * C * C * 2;  // one conv's packed weights (parts in turn)
    static constexpr int w1_off = 2 * buf_bytes;
    static constexpr int w2_off = w1_off + wconv_bytes;
    static constexpr int misc_off = w2_off + wconv_bytes;
    static constexpr int misc_n = 8 * C + 8;
    // barriers: input full [2], input free [2], drain, then per MMA block: conv1 done, conv2 done,
    // conv1 read and its mid-tile block written, conv2 read [NB_MAX each]
    static constexpr int bar_off = (misc_off + misc_n * 4 + 7) / 8 * 8;
    static constexpr int err_off = bar_off + (5 + 4 * NB_MAX) * 8;
    static constexpr int total = err_off + 16;
    static_assert(CTAS * (total + 1024) <= 233472, "the CTAs of an SM fit its shared memory");
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

// FP32 form: a pixel's channels as the FP16 high parts (groups 0 .. G - 1) and the scaled
// remainders (groups G .. 2G - 1).  x - fp16(x) is exact in FP32, and x 2^11 is exact.
template <int C>
__device__ __forceinline__ void store_pixel_split(uint8_t* base, int npix, int p, const float (&v)[C]) {
#pragma unroll
    for (int g = 0; g < C / 8; ++g) {
        uint4 uh, ul;
        __half2* hh = reinterpret_cast<__half2*>(&uh);
        __half2* hl = reinterpret_cast<__half2*>(&ul);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float x0 = v[8 * g + 2 * j], x1 = v[8 * g + 2 * j + 1];
            const __half2 h = __floats2half2_rn(x0, x1);
            const float2 hf = __half22float2(h);
            hh[j] = h;
            hl[j] = __floats2half2_rn((x0 - hf.x) * 2048.f, (x1 - hf.y) * 2048.f);
        }
        *reinterpret_cast<uint4*>(base + ((size_t)g * npix + p) * 16) = uh;
        *reinterpret_cast<uint4*>(base + ((size_t)(C / 8 + g) * npix + p) * 16) = ul;
    }
}

template <int C>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float (&v)[C]) {
    if constexpr (C == 64) {
        umma::ld_32x32b_x32(taddr, *reinterpret_cast<float(*)[32]>(v));
        umma::ld_32x32b_x32(taddr + 32, *reinterpret_cast<float(*)[32]>(v + 32));
    } else if constexpr (C == 32) {
        umma::ld_32x32b_x32(taddr, v);
    } else {
        umma::ld_32x32b_x16(taddr, v);
    }
}

template <int C, bool SPLIT>
__global__ void __launch_bounds__(TcSmem<C, SPLIT>::THREADS, TcSmem<C, SPLIT>::CTAS)
    conv_block_tc_kernel(const ConvArgs a, const ConvTile tg) {
    using S = TcSmem<C, SPLIT>;
    constexpr int TC_LOAD_WARPS = S::LOAD_WARPS, TC_EPI_WARPS = S::EPI_WARPS, TC_MMA_WARP = S::MMA_WARP;
    constexpr int TC_THREADS = S::THREADS;
    const ConvLayout lay{C};
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* s_w1 = sm + S::w1_off;
    uint8_t* s_w2 = sm + S::w2_off;
    float* misc = reinterpret_cast<float*>(sm + S::misc_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::bar_off);
    uint64_t* full = bars;             // [2] input normalised (loader arrivals)
    uint64_t* freed = bars + 2;        // [2] input buffer free again (conv2 of its tile complete)
    uint64_t* drain = bars + 4;        // every MMA issued has completed
    uint64_t* c1done = bars + 5;       // [NB_MAX] conv1 block complete
    uint64_t* c2done = c1done + S::NB_MAX;  // [NB_MAX] conv2 block complete
    uint64_t* e1done = c2done + S::NB_MAX;  // [NB_MAX] conv1 block read, its mid-tile block written (epilogue arrivals)
    uint64_t* e2done = e1done + S::NB_MAX;  // [NB_MAX] conv2 block read (epilogue arrivals)
    int* s_err = reinterpret_cast<int*>(sm + S::err_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::err_off + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W, L = a.L;
    const int P = tg.P, R = tg.R, OW = P - 4;
    const size_t plane = (size_t)H * W;
    const int ntiles = tg.tiles_x * tg.tiles_y * L;
    constexpr int NLOAD = 32 * TC_LOAD_WARPS;
    constexpr int NACC = S::PLANES * C;  // TMEM columns of one block: the accumulator(s)

    // ---- constants and packed weights (BF16, or the FP16 parts) ----
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
        constexpr int n = S::wconv_bytes / 16;
        for (int i = tid; i < n; i += TC_THREADS) {
            d1[i] = __ldg(src + i);
            d2[i] = __ldg(src + n + i);
        }
    }
    if (warp == 0) umma::tmem_alloc(tslot, S::TMEM_COLS);
    if (tid == 0) {
        umma::mbar_init(full, NLOAD);
        umma::mbar_init(full + 1, NLOAD);
        umma::mbar_init(freed, 1);
        umma::mbar_init(freed + 1, 1);
        // a block's epilogue arrivals come from the four warps (one per TMEM lane quarter) that take it
        for (int i = 0; i < S::NB_MAX; ++i) {
            umma::mbar_init(c1done + i, 1);
            umma::mbar_init(c2done + i, 1);
            umma::mbar_init(e1done + i, 4 * 32);
            umma::mbar_init(e2done + i, 4 * 32);
        }
        umma::mbar_init(drain, 1);
        *s_err = 0;
    }
    umma::fence_smem_to_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = SPLIT ? umma::idesc_f16_f32(TC_M, C) : umma::idesc_bf16_f32(TC_M, C);
    constexpr uint32_t LBO_W = C * 16;        // B: N = C rows of 16 B per core-matrix column
    constexpr uint32_t LBO_A = S::NPIX * 16;  // A: channel-group stride of an input / mid tile
    constexpr uint32_t TB = S::TMEM_COLS / 2;  // TMEM column of conv2's accumulators
    // SPLIT: the low parts, as descriptor start-address offsets (16-byte units)
    constexpr uint32_t A_LO = (S::G * LBO_A) >> 4, W_LO = (9 * C * C * 2) >> 4;

    if (warp < TC_LOAD_WARPS) {
        // ---- loader: normalised input tile k into buffer k % 2 ----
        int k = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
            const int b = k & 1;
            // the buffer's previous tile (k - 2) is complete; the first two waits pass at once
            if (!umma::mbar_wait_suspend(freed + b, ((k >> 1) & 1) ^ 1, TC_WAIT_NS)) {
                atomicOr(s_err, 1);
                break;
            }
            uint8_t* s_in = sm + (size_t)b * S::buf_bytes;
            const int tq = fdiv(tile, tg.dtx), li = fdiv(tq, tg.dty);
            const int x0 = (tile - tq * tg.tiles_x) * OW, y0 = (tq - li * tg.tiles_y) * R;
            // rows y0-2 .. y0+R+1, columns x0-2 .. x0+OW+1 (pitch P); two pixels in flight per thread
            const int NIN = (R + 4) * P;
            for (int p0 = tid; p0 < NIN; p0 += 2 * NLOAD) {
                // a pixel's channels in 256-bit loads (whole sectors), from the clamped address
                constexpr int NV = SPLIT ? C / 4 : C / 8;  // 16-byte words of a pixel
                uint4 raw[2][NV];
                bool in[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int p = p0 + u * NLOAD;
                    const int pr = fdiv(p, tg.dP);
                    const int gy = y0 - 2 + pr, gx = x0 - 2 + (p - pr * P);
                    in[u] = p < NIN && gy >= 0 && gy < H && gx >= 0 && gx < W;
                    const size_t pix = (size_t)li * plane + (size_t)(in[u] ? gy : 0) * W + (in[u] ? gx : 0);
                    const uint8_t* src = reinterpret_cast<const uint8_t*>(a.in) + pix * NV * 16;
#pragma unroll
                    for (int g = 0; g < NV / 2; ++g) ldg256(src + 32 * g, raw[u][2 * g], raw[u][2 * g + 1]);
#pragma unroll
                    for (int g = 0; g < NV; ++g)
                        if (!in[u]) raw[u][g] = make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int p = p0 + u * NLOAD;
                    if (p >= NIN) break;
                    float v[C];
                    if constexpr (SPLIT) {
#pragma unroll
                        for (int g = 0; g < NV; ++g) {
                            v[4 * g] = __uint_as_float(raw[u][g].x);
                            v[4 * g + 1] = __uint_as_float(raw[u][g].y);
                            v[4 * g + 2] = __uint_as_float(raw[u][g].z);
                            v[4 * g + 3] = __uint_as_float(raw[u][g].w);
                        }
                    } else {
#pragma unroll
                        for (int g = 0; g < NV; ++g) {
                            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw[u][g]);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float2 f = __bfloat1622float2(h[j]);
                                v[8 * g + 2 * j] = f.x;
                                v[8 * g + 2 * j + 1] = f.y;
                            }
                        }
                    }
                    float ms = 0.f;
#pragma unroll
                    for (int c = 0; c < C; ++c) ms = fmaf(v[c], v[c], ms);
                    // rsqrt on the special-function unit (2 ulp): the per-pixel chain stays short
                    const float r = in[u] ? rsqrtf(ms / C + 1e-6f) : 0.f;
#pragma unroll
                    for (int c = 0; c < C; ++c) v[c] = v[c] * r * misc[c];
                    if constexpr (SPLIT) store_pixel_split<C>(s_in, S::NPIX, p, v);
                    else store_pixel_bf16<C>(s_in, S::NPIX, p, v);
                }
            }
            umma::fence_smem_to_async();  // these writes, before the MMAs that read them
            umma::mbar_arrive(full + b);
        }
    } else if (warp == TC_MMA_WARP) {
        // ---- MMA issue (one thread) ----
        if (lane == 0) {
            // descriptors built once per conv; each MMA adds its start offset (16-byte units: one
            // pixel) to the start-address field, which stays below 2^14.  BF16: one MMA per K step;
            // SPLIT: x_h w_h into the block's high accumulator, x_h w_l and x_l w_h into its low one.
            auto conv_block = [&](uint64_t ad0, uint64_t bd0, uint32_t d0, int i) {
#pragma unroll
                for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                    for (int kk = 0; kk < C / 16; ++kk) {
                        const int dy = tap / 3, dx = tap % 3;
                        const uint32_t ao = (uint32_t)(i * TC_M + dy * P + dx) + ((2 * kk * LBO_A) >> 4);
                        const uint32_t bo = (tap * C * C * 2 + 2 * kk * LBO_W) >> 4;
                        const uint32_t d = d0 + i * NACC;
                        umma::mma_bf16(d, ad0 + ao, bd0 + bo, idesc, (tap | kk) != 0);
                        if constexpr (SPLIT) {
                            umma::mma_bf16(d + C, ad0 + ao, bd0 + bo + W_LO, idesc, (tap | kk) != 0);
                            umma::mma_bf16(d + C, ad0 + ao + A_LO, bd0 + bo, idesc, 1);
                        }
                    }
            };
            // Block-level pipeline: each conv1 / conv2 block is committed to its own mbarrier, so
            // the epilogue takes block i while the tensor cores run block i + 1; conv1 block i of a
            // tile waits only for the epilogue's read of the previous tile's block i (its TMEM
            // columns), and conv2 block i only for the GELU of the conv1 blocks its 3x3 window
            // reaches (rows up to 2 P + 2 pixels past the block) and for the read of the previous
            // tile's conv2 block i.  Every mbarrier completes once per tile and no role runs a
            // phase ahead of the waits on it, so the waits take the tile's parity.
            int k = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++k) {
                const int b = k & 1;
                uint8_t* s_in = sm + (size_t)b * S::buf_bytes;
                ok = umma::mbar_wait_suspend(full + b, (k >> 1) & 1, TC_WAIT_NS);
                if (!ok) break;
                umma::fence_after_sync();
                const uint64_t ad = umma::desc(umma::smem_u32(s_in), LBO_A, 128);
                const uint64_t bd1 = umma::desc(umma::smem_u32(s_w1), LBO_W, 128);
                const uint64_t bd2 = umma::desc(umma::smem_u32(s_w2), LBO_W, 128);
                for (int i = 0; i < tg.nb1 && ok; ++i) {
                    if (k > 0) {
                        ok = umma::mbar_wait_suspend(e1done + i, (k - 1) & 1, TC_WAIT_NS);
                        if (!ok) break;
                        umma::fence_after_sync();
                    }
                    conv_block(ad, bd1, tmem, i);
                    umma::commit(c1done + i);
                }
                // conv2 on the mid tile, in the input buffer
                int ready = -1;  // the conv1 blocks whose GELU is known complete
                for (int i = 0; i < tg.nb2 && ok; ++i) {
                    const int need = min(tg.nb1 - 1, (i * TC_M + TC_M + 2 * P + 1) / TC_M);
                    while (ok && ready < need) {
                        ++ready;
                        ok = umma::mbar_wait_suspend(e1done + ready, k & 1, TC_WAIT_NS);
                    }
                    if (ok && k > 0) ok = umma::mbar_wait_suspend(e2done + i, (k - 1) & 1, TC_WAIT_NS);
                    if (!ok) break;
                    umma::fence_after_sync();
                    conv_block(ad, bd2, tmem + TB, i);
                    umma::commit(c2done + i);
                }
                if (!ok) break;
                umma::commit(freed + b);  // the buffer is free once conv2 has read the mid tile
            }
            if (!ok) atomicOr(s_err, 2);
            // nothing of ours may still run on the tensor cores when TMEM is released
            umma::commit(drain);
            if (!umma::mbar_wait_suspend(drain, 0, TC_WAIT_NS)) atomicOr(s_err, 2);
        }
    } else {
        // ---- epilogues: TC_EPI_WARPS / 4 warps per TMEM lane quarter ----
        constexpr int NGRP = TC_EPI_WARPS / 4;
        static_assert(TC_EPI_WARPS % 4 == 0, "the epilogue warps cover the four TMEM lane quarters evenly");
        const int q = warp & 3, grp = (warp - TC_MMA_WARP - 1) >> 2;
        const int col = q * 32 + lane;  // the pixel of a block (TMEM lane) this thread reads
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        // a block's accumulated conv output (SPLIT: high + 2^-11 low)
        auto load_acc = [&](uint32_t c0, float (&v)[C]) {
            tmem_load_row<C>(tmem + lanes + c0, v);
            if constexpr (SPLIT) {
                float lo[C];
                tmem_load_row<C>(tmem + lanes + c0 + C, lo);
#pragma unroll
                for (int c = 0; c < C; ++c) v[c] = fmaf(lo[c], 1.0f / 2048.f, v[c]);
            }
        };
        int k = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
            const int b = k & 1;
            uint8_t* s_mid = sm + (size_t)b * S::buf_bytes;
            const int tq = fdiv(tile, tg.dtx), li = fdiv(tq, tg.dty);
            const int x0 = (tile - tq * tg.tiles_x) * OW, y0 = (tq - li * tg.tiles_y) * R;
            bool stop = false;
            // gelu(conv1 + b1) -> mid tile, zero outside the plane and on the discarded pixels, each
            // block as soon as its MMAs complete
            for (int i = grp; i < tg.nb1; i += NGRP) {
                if (!umma::mbar_wait_suspend(c1done + i, k & 1, TC_WAIT_NS)) {
                    atomicOr(s_err, 4);
                    stop = true;
                    break;
                }
                umma::fence_after_sync();
                float v[C];
                load_acc(i * NACC, v);
                const int idx = i * TC_M + col;
                const int row = fdiv(idx, tg.dP), cx = idx - row * P;
                const int gy = y0 - 1 + row, gx = x0 - 1 + cx;
                const bool inside = row < R + 2 && cx < OW + 2 && gy >= 0 && gy < H && gx >= 0 && gx < W;
                if constexpr (SPLIT) {
                    // the FP32 form's gelu: the erf form to FP32 rounding, on packed pairs
#pragma unroll
                    for (int c = 0; c < C; c += 2) {
                        const float2 g = gelu_fine2(__fadd2_rn(make_float2(v[c], v[c + 1]), make_float2(misc[C + c], misc[C + c + 1])));
                        v[c] = inside ? g.x : 0.f;
                        v[c + 1] = inside ? g.y : 0.f;
                    }
                    store_pixel_split<C>(s_mid, S::NPIX, idx, v);
                } else {
#pragma unroll
                    for (int c = 0; c < C; c += 2) {
                        const float2 g =
                            gelu_tanh2(__fadd2_rn(make_float2(v[c], v[c + 1]), make_float2(misc[C + c], misc[C + c + 1])));
                        v[c] = inside ? g.x : 0.f;
                        v[c + 1] = inside ? g.y : 0.f;
                    }
                    store_pixel_bf16<C>(s_mid, S::NPIX, idx, v);
                }
                umma::fence_smem_to_async();
                umma::fence_before_sync();
                umma::mbar_arrive(e1done + i);
            }
            if (stop) break;
            // residual, V_out, decode, each block as soon as its MMAs complete
            for (int i = grp; i < tg.nb2; i += NGRP) {
                if (!umma::mbar_wait_suspend(c2done + i, k & 1, TC_WAIT_NS)) {
                    atomicOr(s_err, 4);
                    stop = true;
                    break;
                }
                umma::fence_after_sync();
                float v[C];
                load_acc(TB + i * NACC, v);
                // the block's accumulators are in registers: conv2 of the next tile may take its columns
                umma::fence_before_sync();
                umma::mbar_arrive(e2done + i);
                const int idx = i * TC_M + col;
                const int row = fdiv(idx, tg.dP), cx = idx - row * P;
                const int gy = y0 + row, gx = x0 + cx;
                if (row >= R || cx >= OW || gy >= H || gx >= W) continue;
                const size_t pix = (size_t)gy * W + gx;
                const size_t el = (size_t)li * plane + pix;
                float t = misc[8 * C + 3], s = misc[8 * C + 4];
                if constexpr (SPLIT) {
                    const float* vin = reinterpret_cast<const float*>(a.in) + el * C;
                    float* out = reinterpret_cast<float*>(a.out) + el * C;
#pragma unroll
                    for (int c0 = 0; c0 < C; c0 += 8) {
                        // eight channels: the residual in one 256-bit load, V' in one 256-bit store
                        uint4 r0, r1;
                        ldg256(vin + c0, r0, r1);
                        const float rr[8] = {__uint_as_float(r0.x), __uint_as_float(r0.y), __uint_as_float(r0.z),
                                             __uint_as_float(r0.w), __uint_as_float(r1.x), __uint_as_float(r1.y),
                                             __uint_as_float(r1.z), __uint_as_float(r1.w)};
                        float o[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int c = c0 + j;
                            o[j] = rr[j] + v[c] + misc[2 * C + c];
                            t = fmaf(o[j], misc[3 * C + c], t);
                            s = fmaf(o[j], misc[4 * C + c], s);
                        }
                        stg256(out + c0, make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]),
                                                    __float_as_uint(o[3])),
                               make_uint4(__float_as_uint(o[4]), __float_as_uint(o[5]), __float_as_uint(o[6]),
                                          __float_as_uint(o[7])));
                    }
                } else {
                    const __nv_bfloat16* vin = reinterpret_cast<const __nv_bfloat16*>(a.in) + (size_t)li * plane * C;
                    __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(a.out) + el * C;
#pragma unroll
                    for (int c0 = 0; c0 < C; c0 += 16) {
                        // the residual's 16 channels in one 256-bit load, V' in one 256-bit store
                        float rr[16];
                        {
                            uint4 r0, r1;
                            ldg256(vin + pix * C + c0, r0, r1);
                            const uint32_t pk[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                rr[2 * j] = __uint_as_float(pk[j] << 16);
                                rr[2 * j + 1] = __uint_as_float(pk[j] & 0xffff0000u);
                            }
                        }
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
                        stg256(out + c0, u[0], u[1]);
                    }
                }
                if (a.t_raw) {
                    a.t_raw[pix * L + li] = t;
                    a.s_raw[pix * L + li] = s;
                }
            }
            if (stop) break;
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (tid == 0 && *s_err) atomicExch(a.err, *s_err & 2 ? 2 : 1);
    if (warp == 0) umma::tmem_dealloc(tmem, S::TMEM_COLS);
}

// Tile geometry for a W x H plane (L planes) that minimises the MMA blocks of the busiest CTA: for
// every column split (OW = ceil(W / tx)) and row count R whose input tile fits a buffer (including
// the reads of the last block, NB1 * 128 + 2 P + 2 pixels) and whose conv1 blocks fit half the
// TMEM, the cost is the tiles per CTA times (NB1 + NB2 + 3), the 3 standing for a tile's load and
// epilogue overheads.  (Weighting the pipeline's fill and drain, which favours more and smaller
// tiles on small planes, measured slower.)
template <int C, bool SPLIT>
static ConvTile choose_tile(int W, int H, int L, int slots) {
    using S = TcSmem<C, SPLIT>;
    ConvTile best{0, 0, 0, 0, 0, 0};
    long best_cost = -1, best_total = -1;
    int last_ow = -1;
    for (int tx = 1; tx <= W; ++tx) {
        const int ow = (W + tx - 1) / tx;
        if (ow == last_ow) continue;
        last_ow = ow;
        const int P = ow + 4;
        for (int R = 1; R <= 64; ++R) {
            const int nb1 = ((R + 2) * P + TC_M - 1) / TC_M, nb2 = (R * P + TC_M - 1) / TC_M;
            if ((R + 4) * P > S::NPIX || nb1 > S::NB_MAX || nb1 * TC_M + 2 * P + 2 > S::NPIX) break;
            const long tiles = (long)tx * ((H + R - 1) / R) * L;
            const long per = nb1 + nb2 + 3;
            const long cost = (tiles + slots - 1) / slots * per, total = tiles * per;
            if (best_cost < 0 || cost < best_cost || (cost == best_cost && total < best_total)) {
                best_cost = cost;
                best_total = total;
                best = ConvTile{P, R, nb1, nb2, tx, (H + R - 1) / R};
            }
        }
        if (ow <= 8) break;
    }
    return with_divs(best);
}

template <int C, bool SPLIT>
static cudaError_t launch_tc(const ConvArgs& a, cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = TcSmem<C, SPLIT>::total;
    auto k = conv_block_tc_kernel<C, SPLIT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // the geometry of the last few plane sizes, per host thread
    struct Entry {
        int W, H, L;
        ConvTile t;
    };
    thread_local Entry cache[8] = {};
    thread_local int next = 0;
    ConvTile tg{};
    for (const Entry& c : cache)
        if (c.t.P && c.W == a.W && c.H == a.H && c.L == a.L) tg = c.t;
    if (!tg.P) {
        tg = choose_tile<C, SPLIT>(a.W, a.H, a.L, TcSmem<C, SPLIT>::CTAS * sms);
        if (!tg.P) return cudaErrorInvalidValue;
        cache[next] = Entry{a.W, a.H, a.L, tg};
        next = (next + 1) % 8;
    }
    const long ntiles = (long)tg.tiles_x * tg.tiles_y * a.L;
    const int grid = (int)std::min<long>(ntiles, (long)TcSmem<C, SPLIT>::CTAS * sms);
    k<<<grid, TcSmem<C, SPLIT>::THREADS, smem, st>>>(a, tg);
    return cudaGetLastError();
}

cudaError_t conv_tc_tile_shape(int C, bool split, int W, int H, int L, int* cols, int* rows) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    ConvTile t{};
    if (split) {
        if (C == 16) t = choose_tile<16, true>(W, H, L, TcSmem<16, true>::CTAS * sms);
        else if (C == 32) t = choose_tile<32, true>(W, H, L, TcSmem<32, true>::CTAS * sms);
    } else {
        if (C == 16) t = choose_tile<16, false>(W, H, L, TcSmem<16, false>::CTAS * sms);
        else if (C == 32) t = choose_tile<32, false>(W, H, L, TcSmem<32, false>::CTAS * sms);
        else if (C == 64) t = choose_tile<64, false>(W, H, L, TcSmem<64, false>::CTAS * sms);
    }
    if (!t.P) return cudaErrorInvalidValue;
    *cols = t.P - 4;
    *rows = t.R;
    return cudaSuccess;
}

cudaError_t launch_conv_block_tc(const ConvArgs& a, int C, bool split, cudaStream_t st) {
    if (!a.wtc || !a.err) return cudaErrorInvalidValue;
    // 256-bit pixel loads and stores
    if (reinterpret_cast<uintptr_t>(a.in) % 32 || reinterpret_cast<uintptr_t>(a.out) % 32) return cudaErrorMisalignedAddress;
    if (split) {
        if (C == 16) return launch_tc<16, true>(a, st);
        if (C == 32) return launch_tc<32, true>(a, st);
        return cudaErrorInvalidValue;
    }
    if (C == 16) return launch_tc<16, false>(a, st);
    if (C == 32) return launch_tc<32, false>(a, st);
    if (C == 64) return launch_tc<64, false>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
