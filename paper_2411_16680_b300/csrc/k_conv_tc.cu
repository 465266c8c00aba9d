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
// columns per row instead of a part-empty last block), with enough tiles for every SM.  Two
// persistent CTAs share an SM and stride over the tiles (the packed weights are staged once per
// CTA), so one CTA's loads and epilogues overlap the other's MMAs.  One thread issues the MMAs;
// completion is signalled through an mbarrier with a bounded wait.
#include <algorithm>

#include "device_common.cuh"
#include "umma.cuh"

namespace quark {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 256;
constexpr uint64_t TC_WAIT_NS = 1000000000ull;  // 1 s bound on every MMA wait

// Tile geometry of one launch (host-chosen): pitch P = OW + 4, R output rows, NB1 / NB2 MMA blocks
// of conv1 / conv2.
struct ConvTile {
    int P, R, nb1, nb2, tiles_x, tiles_y;
};

template <int C>
struct TcSmem {
    static constexpr int G = C / 8;
    static constexpr int NPIX = C == 32 ? 1152 : 2304;  // pixels of the input / mid tile buffer
    static constexpr int NB_MAX = 256 / C;              // conv1 blocks that fit the TMEM allocation
    // the mid tile reuses the input tile's memory: conv1 has finished reading it when the first
    // epilogue writes gelu(conv1)
    static constexpr int in_off = 0;
    static constexpr int w1_off = in_off + G * NPIX * 16;
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
__global__ void __launch_bounds__(TC_THREADS, 2) conv_block_tc_kernel(const ConvArgs a, const ConvTile tg) {
    using S = TcSmem<C>;
    constexpr uint32_t TMEM_COLS = 256;  // NB_MAX blocks of C accumulator columns
    const ConvLayout lay{C};
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* s_in = sm + S::in_off;
    uint8_t* s_mid = sm + S::in_off;
    uint8_t* s_w1 = sm + S::w1_off;
    uint8_t* s_w2 = sm + S::w2_off;
    float* misc = reinterpret_cast<float*>(sm + S::misc_off);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::bar_off + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W, L = a.L;
    const int P = tg.P, R = tg.R, OW = P - 4;
    const size_t plane = (size_t)H * W;
    const int ntiles = tg.tiles_x * tg.tiles_y * L;

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
    constexpr uint32_t LBO_W = C * 16;       // B: N = C rows of 16 B per core-matrix column
    constexpr uint32_t LBO_A = S::NPIX * 16;  // A: channel-group stride of the input / mid tile
    const int q = warp & 3, half = warp >> 2;
    const int col = q * 32 + lane;  // the pixel of a block (TMEM lane) this thread reads
    uint32_t phase = 0;             // parity of the next completion of mbar
    bool failed = false;
    int fail_code = 0;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (tile % tg.tiles_x) * OW, y0 = ((tile / tg.tiles_x) % tg.tiles_y) * R;
        const int li = tile / (tg.tiles_x * tg.tiles_y);
        const __nv_bfloat16* vin = reinterpret_cast<const __nv_bfloat16*>(a.in) + (size_t)li * plane * C;

        // ---- normalised input tile: rows y0-2 .. y0+R+1, columns x0-2 .. x0+OW+1 (pitch P) ----
        // (the mid tile of the previous tile, which shares this memory, was last read by its conv2,
        // complete before that tile's epilogue)
        // two pixels per thread per iteration: both pixels' loads are in flight before either is used
        const int NIN = (R + 4) * P;
        for (int p0 = tid; p0 < NIN; p0 += 2 * TC_THREADS) {
            uint4 raw[2][C / 8];
            bool in[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int p = p0 + u * TC_THREADS;
                const int gy = y0 - 2 + p / P, gx = x0 - 2 + p % P;
                in[u] = p < NIN && gy >= 0 && gy < H && gx >= 0 && gx < W;
                const uint4* src = reinterpret_cast<const uint4*>(vin + ((size_t)(in[u] ? gy : 0) * W + (in[u] ? gx : 0)) * C);
#pragma unroll
                for (int g = 0; g < C / 8; ++g) raw[u][g] = in[u] ? __ldg(src + g) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int p = p0 + u * TC_THREADS;
                if (p >= NIN) break;
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
                store_pixel_bf16<C>(s_in, S::NPIX, p, v);
            }
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();

        // ---- conv1: blocks of 128 mid pixels; tap (dy, dx) starts dy * P + dx pixels later ----
        if (tid == 0) {
            // descriptors built once; each MMA adds its start offset (in 16-byte units, one pixel)
            // to the start-address field, which stays below 2^14 for any shared-memory address
            const uint64_t ad0 = umma::desc(umma::smem_u32(s_in), LBO_A, 128);
            const uint64_t bd0 = umma::desc(umma::smem_u32(s_w1), LBO_W, 128);
            for (int i = 0; i < tg.nb1; ++i) {
#pragma unroll
                for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                    for (int kk = 0; kk < C / 16; ++kk) {
                        const int dy = tap / 3, dx = tap % 3;
                        const uint32_t ao = (uint32_t)(i * TC_M + dy * P + dx) + ((2 * kk * LBO_A) >> 4);
                        const uint32_t bo = (tap * C * C * 2 + 2 * kk * LBO_W) >> 4;
                        umma::mma_bf16(tmem + i * C, ad0 + ao, bd0 + bo, idesc, (tap | kk) != 0);
                    }
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
            // ---- epilogue 1: gelu(conv1 + b1) -> BF16 mid tile, zero outside the plane and on the
            // discarded pixels ----
            for (int i = half; i < tg.nb1; i += 2) {
                float v[C];
                tmem_load_row<C>(tmem + ((uint32_t)(q * 32) << 16) + i * C, v);
                const int idx = i * TC_M + col;
                const int row = idx / P, cx = idx - row * P;
                const int gy = y0 - 1 + row, gx = x0 - 1 + cx;
                const bool inside = row < R + 2 && cx < OW + 2 && gy >= 0 && gy < H && gx >= 0 && gx < W;
#pragma unroll
                for (int c = 0; c < C; c += 2) {
                    const float2 g = gelu_tanh2(__fadd2_rn(make_float2(v[c], v[c + 1]), make_float2(misc[C + c], misc[C + c + 1])));
                    v[c] = inside ? g.x : 0.f;
                    v[c + 1] = inside ? g.y : 0.f;
                }
                store_pixel_bf16<C>(s_mid, S::NPIX, idx, v);
            }
            umma::fence_smem_to_async();
            umma::fence_before_sync();
            __syncthreads();
            umma::fence_after_sync();

            // ---- conv2: blocks of 128 output pixels, reusing TMEM columns ----
            if (tid == 0) {
                const uint64_t ad0 = umma::desc(umma::smem_u32(s_mid), LBO_A, 128);
                const uint64_t bd0 = umma::desc(umma::smem_u32(s_w2), LBO_W, 128);
                for (int i = 0; i < tg.nb2; ++i) {
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                        for (int kk = 0; kk < C / 16; ++kk) {
                            const int dy = tap / 3, dx = tap % 3;
                            const uint32_t ao = (uint32_t)(i * TC_M + dy * P + dx) + ((2 * kk * LBO_A) >> 4);
                            const uint32_t bo = (tap * C * C * 2 + 2 * kk * LBO_W) >> 4;
                            umma::mma_bf16(tmem + i * C, ad0 + ao, bd0 + bo, idesc, (tap | kk) != 0);
                        }
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
                for (int i = half; i < tg.nb2; i += 2) {
                    float v[C];
                    tmem_load_row<C>(tmem + ((uint32_t)(q * 32) << 16) + i * C, v);
                    const int idx = i * TC_M + col;
                    const int row = idx / P, cx = idx - row * P;
                    const int gy = y0 + row, gx = x0 + cx;
                    if (row >= R || cx >= OW || gy >= H || gx >= W) continue;
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

// Tile geometry for a W x H plane (L planes) that minimises the MMA blocks of the slowest CTA: for
// every column split (OW = ceil(W / tx)) and row count R whose input tile fits the buffer (including
// the reads of the last block, NB1 * 128 + 2 P + 2 pixels) and whose conv1 blocks fit TMEM, the
// cost is the tiles per CTA slot times (NB1 + NB2 + 3), the 3 standing for a tile's load and
// epilogue overheads.
template <int C>
static ConvTile choose_tile(int W, int H, int L, int slots) {
    using S = TcSmem<C>;
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
    return best;
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
        tg = choose_tile<C>(a.W, a.H, a.L, 2 * sms);
        if (!tg.P) return cudaErrorInvalidValue;
        cache[next] = Entry{a.W, a.H, a.L, tg};
        next = (next + 1) % 8;
    }
    const long ntiles = (long)tg.tiles_x * tg.tiles_y * a.L;
    const int grid = (int)std::min<long>(ntiles, 2L * sms);
    k<<<grid, TC_THREADS, smem, st>>>(a, tg);
    return cudaGetLastError();
}

cudaError_t launch_conv_block_tc(const ConvArgs& a, int C, cudaStream_t st) {
    if (!a.wtc || !a.err) return cudaErrorInvalidValue;
    if (C == 16) return launch_tc<16>(a, st);
    if (C == 32) return launch_tc<32>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
