// Fused sample-attend step of the BF16 form with the dense contractions on tcgen05 tensor cores
// (Sec. 3.3: MultiHead(N(V), D) = concat_i softmax(N(V) W_i^q D^T / sqrt(C)) D  W^O, plus the
// blend-logit query N(V) W^beta of the last step, Sec. 3.2.3).
//
// A CTA owns 128 LDM elements: a 16 x 8 pixel tile of one layer plane (M = 128), so that the
// bilinear taps of vertically and horizontally neighbouring elements hit the same L1 lines.  The
// layer is the fastest-varying grid index: the CTAs resident at one time cover every layer of a
// band of tiles, so each texel of the (larger than L2) feature level is fetched from DRAM about
// once per step rather than once per layer.
//   1. Volume entering the step (v0, or the previous volume, x2-upsampled on the fly), decoded
//      depth, RMSNorm -> X (BF16) in shared memory as a K-major tcgen05 A operand.
//   2. One MMA chain Q = X [Wq | W^beta] (N = hC (+C), K = C) into TMEM; copied to shared memory.
//   3. Per element, two threads (16 channels each) reproject into every view, bilinearly sample
//      the BF16 level-k features on packed BF16 pairs, and run the online softmax over views
//      (FP32); the last step also writes the blend logits.
//   4. The head outputs O (BF16) go back to shared memory as an A operand; one MMA chain
//      O W^O (N = C, K = hC) into TMEM; residual add in FP32; V_attn stored as BF16.
// Completion of each MMA chain is signalled through an mbarrier; every wait is bounded.
// The same kernel serves the FP32 form (template SPLIT): X, O and the packed weights as FP16
// parts, three MMAs per K step, FP32 features, taps, residual and V_attn (see AtSmem).
#include <cuda_fp16.h>

#include "device_common.cuh"
#include "umma.cuh"

namespace quark {

constexpr int AT_M = 128;
constexpr int AT_TW = 16, AT_TH = 8;  // pixel tile of the 128 elements
constexpr uint64_t AT_WAIT_NS = 1000000000ull;
constexpr float AT_SLACK = 20.f;  // log2 units: a factor of about 1e6
// Leading byte offset of the X and O operand tiles (distance between K-adjacent 8-channel columns of
// core matrices): 128 rows of 16 bytes plus 32, so that the two threads of an element, which write
// columns two apart, and eight consecutive rows fall on distinct banks.
constexpr int AT_LBO = AT_M * 16 + 32;

// Shared memory of one CTA.  Only the query columns in use are copied (the blend query exists
// on the last step only) and the blend logits are staged for the V views present, so that the
// rest of the SM's unified L1 stays free to cache the sampled texels.
//
// FP32 form (SPLIT): the X and O operands and the packed weights come in two FP16 parts, the
// rounded value and the scaled remainder fp16((x - fp16(x)) 2^11), and each projection is
// x_h w_h + 2^-11 (x_h w_l + x_l w_h) on three kind::f16 MMAs per K step into a high and a low
// accumulator (FP32 accuracy: the dropped x_l w_l term is 2^-22 of a product).  The X tile (both
// parts) later holds the FP32 entering volume; the O tile (both parts) takes the Q copy's bytes
// once every thread has left the view loop.  O is scaled per element by a power of two into
// [-1, 1) before the split (any feature magnitude), and the output row scaled back.
template <int C, int NH, bool LAST, bool SPLIT>
struct AtSmem {
    static constexpr int PARTS = SPLIT ? 2 : 1;
    static constexpr int NQ = NH * C + C;        // packed query columns incl. the blend query
    static constexpr int NQ_USED = LAST ? NQ : NH * C;
    static constexpr int QS = NQ_USED + 4;       // padded fp32 row stride of the Q copy
    static constexpr int o_bytes = PARTS * (NH * C / 8) * AT_LBO;
    static constexpr int x_off = 0;                               // A: 128 x C (per part)
    static constexpr int o_sep = x_off + PARTS * (C / 8) * AT_LBO;  // A: 128 x hC (BF16 form)
    static constexpr int wq_off = o_sep + (SPLIT ? 0 : o_bytes);  // B: NQ x C (per part)
    static constexpr int wo_off = wq_off + PARTS * NQ * C * 2;    // B: C x hC (per part)
    static constexpr int q_off = wo_off + PARTS * C * NH * C * 2; // fp32 128 x QS (Q copy, then output copy)
    static constexpr int o_off = SPLIT ? q_off : o_sep;
    static constexpr int misc_off = q_off + AT_M * QS * 4;        // v0, g, w_d, b_d
    static constexpr int bar_off = misc_off + 4 * C * 4;
    static constexpr int oexp_off = bar_off + 16;                 // SPLIT: O's per-element exponent
    static constexpr int beta_off = oexp_off + (SPLIT ? AT_M * 4 : 0);  // fp32 128 x V blend logits (last step)
    static int total(int V) { return beta_off + (LAST ? AT_M * V * 4 : 0); }
    static constexpr int tmem_need = PARTS * NQ;
    static constexpr int tmem_cols = tmem_need <= 32 ? 32 : tmem_need <= 64 ? 64 : tmem_need <= 128 ? 128 : tmem_need <= 256 ? 256 : 512;
    static constexpr uint32_t LO_COL = tmem_cols / 2;            // SPLIT: the low accumulators
    static_assert(!SPLIT || o_bytes <= AT_M * QS * 4, "the O tile fits the Q copy's bytes");
};

// Bilinear interpolation on packed BF16 pairs: each 32-bit word of a tap holds two channels, and
// one fma.rn.bf16x2 adds both channels' weighted taps (BF16 products and sums, one rounding per
// step), so the four taps of 16 channels take 32 instructions on the packed pairs as loaded.  The
// sampled features are BF16 in the precision form; the dot products and the softmax below take
// them to FP32.  One thread's 16 BF16 channels of a texel (32 bytes, 32-byte aligned: a texel is
// C x 2 bytes and a thread's channel group starts at a multiple of 16 channels) come in one
// 256-bit load.
__device__ __forceinline__ uint32_t bf2_mul(uint32_t x, __nv_bfloat162 w) {
    const __nv_bfloat162 r = __hmul2(*reinterpret_cast<const __nv_bfloat162*>(&x), w);
    return *reinterpret_cast<const uint32_t*>(&r);
}
__device__ __forceinline__ uint32_t bf2_fma(uint32_t x, __nv_bfloat162 w, uint32_t c) {
    const __nv_bfloat162 r = __hfma2(*reinterpret_cast<const __nv_bfloat162*>(&x), w,
                                     *reinterpret_cast<const __nv_bfloat162*>(&c));
    return *reinterpret_cast<const uint32_t*>(&r);
}
__device__ __forceinline__ void mul_taps16(const __nv_bfloat16* p, float w, uint32_t (&D)[8]) {
    uint4 a, b;
    ldg256(p, a, b);
    const __nv_bfloat162 w2 = __float2bfloat162_rn(w);
    D[0] = bf2_mul(a.x, w2);
    D[1] = bf2_mul(a.y, w2);
    D[2] = bf2_mul(a.z, w2);
    D[3] = bf2_mul(a.w, w2);
    D[4] = bf2_mul(b.x, w2);
    D[5] = bf2_mul(b.y, w2);
    D[6] = bf2_mul(b.z, w2);
    D[7] = bf2_mul(b.w, w2);
}
__device__ __forceinline__ void fma_taps16(const __nv_bfloat16* p, float w, uint32_t (&D)[8]) {
    uint4 a, b;
    ldg256(p, a, b);
    const __nv_bfloat162 w2 = __float2bfloat162_rn(w);
    D[0] = bf2_fma(a.x, w2, D[0]);
    D[1] = bf2_fma(a.y, w2, D[1]);
    D[2] = bf2_fma(a.z, w2, D[2]);
    D[3] = bf2_fma(a.w, w2, D[3]);
    D[4] = bf2_fma(b.x, w2, D[4]);
    D[5] = bf2_fma(b.y, w2, D[5]);
    D[6] = bf2_fma(b.z, w2, D[6]);
    D[7] = bf2_fma(b.w, w2, D[7]);
}
// the sampled channel pairs as FP32 pairs (a BF16 value is the high half of its FP32 word)
__device__ __forceinline__ void unpack16(const uint32_t (&H)[8], float2 (&D)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) D[j] = make_float2(__uint_as_float(H[j] << 16), __uint_as_float(H[j] & 0xffff0000u));
}
// FP32 form: D += w * texel for 16 FP32 channels at p (32-byte aligned): two 256-bit loads
__device__ __forceinline__ void fma_tap16_f32(const float* p, float w, float2 (&D)[8]) {
    uint4 t[4];
    ldg256(p, t[0], t[1]);
    ldg256(p + 8, t[2], t[3]);
    const float2 w2 = make_float2(w, w);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        D[2 * i] = __ffma2_rn(make_float2(__uint_as_float(t[i].x), __uint_as_float(t[i].y)), w2, D[2 * i]);
        D[2 * i + 1] = __ffma2_rn(make_float2(__uint_as_float(t[i].z), __uint_as_float(t[i].w)), w2, D[2 * i + 1]);
    }
}
// FP32 form: eight channels as their FP16 parts (x - fp16(x) is exact in FP32, x 2^11 exact)
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
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
// A TMEM row chunk of 16 columns of the high (and, SPLIT, the low) accumulator: high + 2^-11 low
template <bool SPLIT, uint32_t LO>
__device__ __forceinline__ void tmem_acc16(uint32_t taddr, float (&v)[16]) {
    umma::ld_32x32b_x16(taddr, v);
    if constexpr (SPLIT) {
        float lo[16];
        umma::ld_32x32b_x16(taddr + LO, lo);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = fmaf(lo[i], 1.0f / 2048.f, v[i]);
    }
}

// The softmax below works in log2 units, so that each weight is one ex2 (ex2_approx); the
// reprojection divides with one reciprocal (reproject_rcp).
template <int C, int NH, int TR, bool LAST, bool SPLIT, int VT>
__global__ void __launch_bounds__(AT_M * (C / 16), (C == 32 && NH <= 2) ? 2 : 1) attend_tc_kernel(const AttendArgs a) {
    constexpr int TPE = C / 16;
    constexpr int NT = AT_M * TPE;
    using S = AtSmem<C, NH, LAST, SPLIT>;
    // views: VT when the launch fixes the count (the view loop then unrolls, each view's map a
    // constant-bank operand), else the argument
    const int NV = VT > 0 ? VT : a.V;
    constexpr int NQ_USED = S::NQ_USED;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* s_x = sm + S::x_off;
    uint8_t* s_o = sm + S::o_off;
    uint8_t* s_wq = sm + S::wq_off;
    uint8_t* s_wo = sm + S::wo_off;
    float* s_q = reinterpret_cast<float*>(sm + S::q_off);
    float* misc = reinterpret_cast<float*>(sm + S::misc_off);
    float* s_beta = reinterpret_cast<float*>(sm + S::beta_off);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::bar_off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::bar_off + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = a.L, H = a.H, W = a.W;
    const int li = blockIdx.x;
    const int e = tid / TPE, sub = tid % TPE, c0 = sub * 16;
    const int x = blockIdx.y * AT_TW + e % AT_TW, y = blockIdx.z * AT_TH + e / AT_TW;
    const bool live = x < W && y < H;
    const int xc = min(x, W - 1), yc = min(y, H - 1);

    // ---- weights: packed BF16 B operands, FP32 misc; in the BF16 form the entering volume's words
    // too.  Every global load of the prologue is issued before the first barrier, so that their
    // latencies overlap instead of adding up. ----
    constexpr int NWQ = S::PARTS * (S::NQ * C * 2 / 16 + C * NH * C * 2 / 16);  // 16-byte words: wq then wo
    constexpr int WPT = (NWQ + NT - 1) / NT;
    uint4 wreg[WPT];
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.wtc);
#pragma unroll
        for (int j = 0; j < WPT; ++j)
            if (tid + j * NT < NWQ) wreg[j] = __ldg(src + tid + j * NT);
    }
    const float mreg = tid < 4 * C ? a.w[tid] : 0.f;  // v0 [C], g [C], w_d [C], b_d (padded); 4C <= NT
    // BF16 form: this element's 16 channels (same resolution), or the four x2-upsample taps' words
    uint4 vraw[TR == TR_UP2 ? 4 : 1][2];
    int ya = 0, yb = 0, xa = 0, xb = 0;
    float wy = 0.f, wx = 0.f;
    if constexpr (!SPLIT && TR == TR_SAME) {
        ldg256(reinterpret_cast<const __nv_bfloat16*>(a.prev) + (((size_t)li * H + yc) * W + xc) * C + c0,
               vraw[0][0], vraw[0][1]);
    } else if constexpr (!SPLIT && TR == TR_UP2) {
        resize_taps(yc, 2, a.Hp, ya, yb, wy);
        resize_taps(xc, 2, a.Wp, xa, xb, wx);
        const __nv_bfloat16* base =
            reinterpret_cast<const __nv_bfloat16*>(a.prev) + (size_t)li * a.Hp * a.Wp * C + c0;
        ldg256(base + ((size_t)ya * a.Wp + xa) * C, vraw[0][0], vraw[0][1]);
        ldg256(base + ((size_t)ya * a.Wp + xb) * C, vraw[1][0], vraw[1][1]);
        ldg256(base + ((size_t)yb * a.Wp + xa) * C, vraw[2][0], vraw[2][1]);
        ldg256(base + ((size_t)yb * a.Wp + xb) * C, vraw[3][0], vraw[3][1]);
    }
    {
        uint4* dq = reinterpret_cast<uint4*>(s_wq);
#pragma unroll
        for (int j = 0; j < WPT; ++j)
            if (tid + j * NT < NWQ) dq[tid + j * NT] = wreg[j];
        if (tid < 4 * C) misc[tid] = mreg;
    }

    // ---- volume entering the step, depth, RMSNorm ----
    // Each thread of an element's group holds its own 16 channels (vres); the depth logit and the
    // mean square are partial sums over those channels, completed with shuffles in the group.
    // Through the view loop the entering volume is held only as BF16 pairs (vpk) for the residual:
    // the stored words when the step keeps the resolution; when it doubles it, the x2-upsampled
    // volume rounded to BF16 (as it would be stored), which the norm and the depth use too.  The
    // first step's constant v0 is read again from shared memory.
    __syncthreads();
    float vres[16];
    uint32_t vpk[8];
    if constexpr (TR == TR_INIT) {
#pragma unroll
        for (int i = 0; i < 16; ++i) vres[i] = misc[c0 + i];
    } else if constexpr (SPLIT && TR == TR_SAME) {
        // FP32 form: the thread's 16 FP32 channels in two 256-bit loads
        uint4 t[4];
        const float* p = reinterpret_cast<const float*>(a.prev) + (((size_t)li * H + yc) * W + xc) * C + c0;
        ldg256(p, t[0], t[1]);
        ldg256(p + 8, t[2], t[3]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            vres[4 * i] = __uint_as_float(t[i].x);
            vres[4 * i + 1] = __uint_as_float(t[i].y);
            vres[4 * i + 2] = __uint_as_float(t[i].z);
            vres[4 * i + 3] = __uint_as_float(t[i].w);
        }
    } else if constexpr (SPLIT) {
        // FP32 form: x2 bilinear upsample in FP32
        int ya, yb, xa, xb;
        float wy, wx;
        resize_taps(yc, 2, a.Hp, ya, yb, wy);
        resize_taps(xc, 2, a.Wp, xa, xb, wx);
        const float* base = reinterpret_cast<const float*>(a.prev) + (size_t)li * a.Hp * a.Wp * C + c0;
        const float* q[4] = {base + ((size_t)ya * a.Wp + xa) * C, base + ((size_t)ya * a.Wp + xb) * C,
                             base + ((size_t)yb * a.Wp + xa) * C, base + ((size_t)yb * a.Wp + xb) * C};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint4 r[4][2];
#pragma unroll
            for (int t = 0; t < 4; ++t) ldg256(q[t] + 8 * h, r[t][0], r[t][1]);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float f[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) f[t] = __uint_as_float((&r[t][i / 4].x)[i % 4]);
                const float top = f[0] + wx * (f[1] - f[0]);
                const float bot = f[2] + wx * (f[3] - f[2]);
                vres[8 * h + i] = top + wy * (bot - top);
            }
        }
    } else if constexpr (TR == TR_SAME) {
        const uint4 u0 = vraw[0][0], u1 = vraw[0][1];  // loaded before the barrier
        vpk[0] = u0.x; vpk[1] = u0.y; vpk[2] = u0.z; vpk[3] = u0.w;
        vpk[4] = u1.x; vpk[5] = u1.y; vpk[6] = u1.z; vpk[7] = u1.w;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            vres[2 * j] = __uint_as_float(vpk[j] << 16);
            vres[2 * j + 1] = __uint_as_float(vpk[j] & 0xffff0000u);
        }
    } else {
        // the four x2-upsample taps, loaded before the barrier (vraw; weights wx, wy)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float t[4][2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t w = (&vraw[q][j / 4].x)[j % 4];
                t[q][0] = __uint_as_float(w << 16);
                t[q][1] = __uint_as_float(w & 0xffff0000u);
            }
            float v2[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float top = t[0][i] + wx * (t[1][i] - t[0][i]);
                const float bot = t[2][i] + wx * (t[3][i] - t[2][i]);
                v2[i] = top + wy * (bot - top);
            }
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v2[0], v2[1]);
            vpk[j] = *reinterpret_cast<const uint32_t*>(&h2);
            vres[2 * j] = __uint_as_float(vpk[j] << 16);
            vres[2 * j + 1] = __uint_as_float(vpk[j] & 0xffff0000u);
        }
    }
    float tpart = 0.f, ms = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        tpart = fmaf(vres[i], misc[2 * C + c0 + i], tpart);
        ms = fmaf(vres[i], vres[i], ms);
    }
#pragma unroll
    for (int off = 1; off < TPE; off <<= 1) {
        tpart += __shfl_xor_sync(0xffffffffu, tpart, off);
        ms += __shfl_xor_sync(0xffffffffu, ms, off);
    }
    float d = TR == TR_INIT ? depth_anchor(li, L, a.dp) : depth_from_logit(misc[3 * C] + tpart, li, L, a.dp);
    {
        // reused depths of an earlier step, or this step's depths kept for a later one
        const size_t de = ((size_t)li * H + yc) * W + xc;
        if (a.depth_in) d = __ldg(a.depth_in + de);
        else if (a.depth_out && live && sub == 0) a.depth_out[de] = d;
    }
    const float rinv = rsqrtf(ms / C + 1e-6f);  // 2 ulp, on the special-function unit
    if constexpr (SPLIT) {
        // this thread's 16 channels of X = N(V_in) as FP16 parts: two 8-channel groups per part,
        // K-major A layout (group g of row m at g * 128 * 16 + m * 16, the low part's groups after
        // the high part's C / 8)
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float xv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) xv[i] = vres[8 * g + i] * rinv * misc[C + c0 + 8 * g + i];
            uint4 hi, lo;
            split8(xv, hi, lo);
            *reinterpret_cast<uint4*>(s_x + (size_t)(c0 / 8 + g) * AT_LBO + e * 16) = hi;
            *reinterpret_cast<uint4*>(s_x + (size_t)(C / 8 + c0 / 8 + g) * AT_LBO + e * 16) = lo;
        }
    } else {
        // this thread's 16 channels of X = N(V_in): two 8-channel groups, K-major A layout
        // (group g of row m at g * 128 * 16 + m * 16)
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            uint4 u;
            __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = 8 * g + 2 * j;
                hh[j] = __floats2bfloat162_rn(vres[i] * rinv * misc[C + c0 + i], vres[i + 1] * rinv * misc[C + c0 + i + 1]);
            }
            *reinterpret_cast<uint4*>(s_x + (size_t)(c0 / 8 + g) * AT_LBO + e * 16) = u;
        }
    }
    if (warp == 0) umma::tmem_alloc(tslot, S::tmem_cols);
    if (tid == 0) umma::mbar_init(mbar, 1);
    umma::fence_smem_to_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;

    // ---- Q = X [Wq | W^beta] ----
    // (a test of the error path leaves the chain unissued: nothing arrives on the mbarrier, the
    // wait below runs out after test_wait_ns, and the drain wait at the end finds nothing in flight)
    const bool test_skip = a.test_wait_ns != 0;
    const uint64_t wait_ns = test_skip ? a.test_wait_ns : AT_WAIT_NS;
    if (tid == 0 && !test_skip) {
        constexpr uint32_t idesc = SPLIT ? umma::idesc_f16_f32(AT_M, NQ_USED) : umma::idesc_bf16_f32(AT_M, NQ_USED);
        const uint32_t a0 = umma::smem_u32(s_x), b0 = umma::smem_u32(s_wq);
        constexpr uint32_t LBO_A = AT_LBO, LBO_B = S::NQ * 16;
        constexpr uint32_t A_LO = (C / 8) * LBO_A, B_LO = S::NQ * C * 2;  // the low parts (bytes)
#pragma unroll
        for (int kk = 0; kk < C / 16; ++kk) {
            const uint32_t ak = a0 + 2 * kk * LBO_A, bk = b0 + 2 * kk * LBO_B;
            umma::mma_bf16(tmem, umma::desc(ak, LBO_A, 128), umma::desc(bk, LBO_B, 128), idesc, kk > 0);
            if constexpr (SPLIT) {
                umma::mma_bf16(tmem + S::LO_COL, umma::desc(ak, LBO_A, 128), umma::desc(bk + B_LO, LBO_B, 128), idesc, kk > 0);
                umma::mma_bf16(tmem + S::LO_COL, umma::desc(ak + A_LO, LBO_A, 128), umma::desc(bk, LBO_B, 128), idesc, 1);
            }
        }
        umma::commit(mbar);
    }
    // ---- the first pair of views' samples, before the wait: their gathers need only the depth, so
    // their latency overlaps the MMA chain, the query copy and the barrier that follow ----
    const float pxc = xc + 0.5f, pyc = yc + 0.5f;
    const __nv_bfloat16* feat0 = reinterpret_cast<const __nv_bfloat16*>(a.feat) + c0;
    const int vstride = a.fh * a.fw * C;  // < 2^31 for every accepted level size
    // Bilinear sample of view m: the four taps are always fetched (clamped into the map, weight
    // zero outside it), with no branch, so all the loads of the view are in flight together.
    // (FP32 form: FP32 features, FP32 taps, the reprojection with an IEEE divide.)
    auto sample = [&](int m, float2 (&D)[8]) {
        float u = 0.f, v = 0.f;
        if constexpr (SPLIT) {
            const bool ok = reproject(a.geo.v[m], pxc, pyc, d, u, v);
            const Taps4 tp = bilinear_taps4(ok, u, v, a.fh, a.fw);
            const float* f = reinterpret_cast<const float*>(a.feat) + c0 + (size_t)m * vstride;
#pragma unroll
            for (int j = 0; j < 8; ++j) D[j] = make_float2(0.f, 0.f);
            fma_tap16_f32(f + tp.i00 * C, tp.w00, D);
            fma_tap16_f32(f + tp.i01 * C, tp.w01, D);
            fma_tap16_f32(f + tp.i10 * C, tp.w10, D);
            fma_tap16_f32(f + tp.i11 * C, tp.w11, D);
        } else {
            const bool ok = reproject_rcp(a.geo.v[m], pxc, pyc, d, u, v);
            const Taps4 tp = bilinear_taps4(ok, u, v, a.fh, a.fw);
            const __nv_bfloat16* f = feat0 + (size_t)m * vstride;
            uint32_t Hs[8];
            mul_taps16(f + tp.i00 * C, tp.w00, Hs);
            fma_taps16(f + tp.i01 * C, tp.w01, Hs);
            fma_taps16(f + tp.i10 * C, tp.w10, Hs);
            fma_taps16(f + tp.i11 * C, tp.w11, Hs);
            unpack16(Hs, D);
        }
    };
    float2 Da[8], Db[8];
    if (NV >= 2) {
        sample(0, Da);
        sample(1, Db);
    }
    bool failed = __syncthreads_or(!umma::mbar_wait(mbar, 0, wait_ns));
    uint32_t failed_phase = 0;
    umma::fence_after_sync();
    if (TR != TR_INIT && !failed) {
        // X has been read by the MMA: its tile now keeps the entering volume for the residual of the
        // output epilogue, in 16-byte columns of the operand layout (8 BF16 channels, BF16 form; 4
        // FP32 channels, FP32 form): column k of element e at k * AT_LBO + e * 16
        if constexpr (TR == TR_INIT) {
            // (not reached: the first step's residual is v0, read from shared memory)
        } else if constexpr (SPLIT) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                *reinterpret_cast<float4*>(s_x + (size_t)(c0 / 4 + i) * AT_LBO + e * 16) =
                    make_float4(vres[4 * i], vres[4 * i + 1], vres[4 * i + 2], vres[4 * i + 3]);
        } else {
            *reinterpret_cast<uint4*>(s_x + (size_t)(c0 / 8) * AT_LBO + e * 16) = make_uint4(vpk[0], vpk[1], vpk[2], vpk[3]);
            *reinterpret_cast<uint4*>(s_x + (size_t)(c0 / 8 + 1) * AT_LBO + e * 16) = make_uint4(vpk[4], vpk[5], vpk[6], vpk[7]);
        }
    }
    if (!failed) {
        // TMEM -> shared: warp w reads lanes 32 (w % 4) .. + 31, column chunks of 16.  The logit
        // scale 1/sqrt(C), and for the attention heads log2(e) (the softmax below runs on ex2), is
        // folded into the packed W^q and W^beta.
        // On the first step every element's queries are those of the constant v0 (identical X rows,
        // so identical Q rows): row 0 alone is copied and read by every element (a shared-memory
        // broadcast in the view loop).
        const int q = warp & 3, grp = warp >> 2;
        if (TR != TR_INIT || q == 0) {
            for (int ch = grp; ch < NQ_USED / 16; ch += TPE) {
                float v[16];
                tmem_acc16<SPLIT, S::LO_COL>(tmem + ((uint32_t)(q * 32) << 16) + ch * 16, v);
                if (TR != TR_INIT || lane == 0) {
                    float4* dst = reinterpret_cast<float4*>(s_q + (size_t)(q * 32 + lane) * S::QS + ch * 16);
#pragma unroll
                    for (int i = 0; i < 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    if (!failed) {
        // the queries stay in shared memory (read once per pair of views) to keep registers for the gathers
        const int qrow = TR == TR_INIT ? 0 : e;  // the first step's queries: one row for all
        const float4* qh4 = reinterpret_cast<const float4*>(s_q + (size_t)qrow * S::QS + c0);
        // the blend query likewise
        const float4* qb4 = reinterpret_cast<const float4*>(s_q + (size_t)qrow * S::QS + NH * C + c0);

        // ---- views: sample, online softmax (log2 units), weighted sum (FP32) ----
        float mx[NH], l[NH];
        float2 o[NH][8];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            mx[h] = -INFINITY;
            l[h] = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) o[h][j] = make_float2(0.f, 0.f);
        }
        // One online-softmax step of head h: logit s (log2 units, this element's full sum), sample D.
        // The softmax is invariant to the reference subtracted from its logits, so the reference
        // moves only when a logit passes it by AT_SLACK (log2 units): taken at the first view and
        // then almost never, the branch stays uniform across the warp.  Weights stay <= 2^AT_SLACK,
        // far from FP32 overflow.
        auto accumulate = [&](int h, float s, const float2 (&D)[8]) {
            if (s > mx[h] + AT_SLACK) {
                const float cs = ex2_approx(mx[h] - s);
                const float2 cs2 = make_float2(cs, cs);
                l[h] *= cs;
#pragma unroll
                for (int j = 0; j < 8; ++j) o[h][j] = __fmul2_rn(o[h][j], cs2);
                mx[h] = s;
            }
            const float p = ex2_approx(s - mx[h]);
            const float2 p2 = make_float2(p, p);
            l[h] += p;
#pragma unroll
            for (int j = 0; j < 8; ++j) o[h][j] = __ffma2_rn(p2, D[j], o[h][j]);
        };
        auto group_sum = [](float s) {
#pragma unroll
            for (int off = 1; off < TPE; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            return s;
        };
        // Views in pairs: each query float4 is read from shared memory once for two samples (the
        // shared-memory reads of the queries were the larger part of the L1 data-pipe traffic).
        // Each view's arithmetic, and the order of the softmax steps, is that of one view at a time.
        int m = 0;
        auto pair_step = [&](int m) {
            if (m > 0) {
                sample(m, Da);
                sample(m + 1, Db);
            }
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 q4 = qh4[h * C / 4 + i];
                    a0 = __ffma2_rn(make_float2(q4.x, q4.y), Da[2 * i], a0);
                    a1 = __ffma2_rn(make_float2(q4.z, q4.w), Da[2 * i + 1], a1);
                    b0 = __ffma2_rn(make_float2(q4.x, q4.y), Db[2 * i], b0);
                    b1 = __ffma2_rn(make_float2(q4.z, q4.w), Db[2 * i + 1], b1);
                }
                const float sa = group_sum((a0.x + a1.x) + (a0.y + a1.y));
                const float sb = group_sum((b0.x + b1.x) + (b0.y + b1.y));
                accumulate(h, sa, Da);
                accumulate(h, sb, Db);
            }
            if constexpr (LAST) {
                float2 ba = make_float2(0.f, 0.f), bb = ba;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 q4 = qb4[i];
                    ba = __ffma2_rn(make_float2(q4.x, q4.y), Da[2 * i], ba);
                    ba = __ffma2_rn(make_float2(q4.z, q4.w), Da[2 * i + 1], ba);
                    bb = __ffma2_rn(make_float2(q4.x, q4.y), Db[2 * i], bb);
                    bb = __ffma2_rn(make_float2(q4.z, q4.w), Db[2 * i + 1], bb);
                }
                const float sa = group_sum(ba.x + ba.y), sb = group_sum(bb.x + bb.y);
                // the element's first and last threads store one each (fewer bank conflicts)
                if (sub == 0) s_beta[e * NV + m] = sa;
                if (sub == TPE - 1) s_beta[e * NV + m + 1] = sb;
            }
        };
        if constexpr (VT > 0) {
#pragma unroll
            for (; m + 1 < VT; m += 2) pair_step(m);
        } else {
            for (; m + 1 < NV; m += 2) pair_step(m);
        }
        if (m < NV) {  // the last view of an odd count
            float2 D[8];
            sample(m, D);
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                float2 a0 = make_float2(0.f, 0.f), a1 = a0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 q4 = qh4[h * C / 4 + i];
                    a0 = __ffma2_rn(make_float2(q4.x, q4.y), D[2 * i], a0);
                    a1 = __ffma2_rn(make_float2(q4.z, q4.w), D[2 * i + 1], a1);
                }
                accumulate(h, group_sum((a0.x + a1.x) + (a0.y + a1.y)), D);
            }
            if constexpr (LAST) {
                float2 ba = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 q4 = qb4[i];
                    ba = __ffma2_rn(make_float2(q4.x, q4.y), D[2 * i], ba);
                    ba = __ffma2_rn(make_float2(q4.z, q4.w), D[2 * i + 1], ba);
                }
                const float sa = group_sum(ba.x + ba.y);
                if (sub == 0) s_beta[e * NV + m] = sa;
            }
        }
        if constexpr (SPLIT) {
            // head outputs -> FP16 parts of the A operand (K = h * C + channel), scaled by 2^-x with
            // x the exponent of the element's largest output (the row is scaled back after W^O).
            // The O tile takes the Q copy's bytes: every thread must be done reading its queries.
            float il[NH], mo = 0.f;
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                il[h] = 1.0f / l[h];
#pragma unroll
                for (int j = 0; j < 8; ++j) mo = fmaxf(mo, fmaxf(fabsf(o[h][j].x), fabsf(o[h][j].y)) * il[h]);
            }
#pragma unroll
            for (int off = 1; off < TPE; off <<= 1) mo = fmaxf(mo, __shfl_xor_sync(0xffffffffu, mo, off));
            int ex = 0;
            frexpf(mo, &ex);
            if (sub == 0) reinterpret_cast<int*>(sm + S::oexp_off)[e] = ex;
            __syncthreads();
#pragma unroll
            for (int h = 0; h < NH; ++h) {
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    float ov[8];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        ov[2 * j] = ldexpf(o[h][4 * g + j].x * il[h], -ex);
                        ov[2 * j + 1] = ldexpf(o[h][4 * g + j].y * il[h], -ex);
                    }
                    uint4 hi, lo;
                    split8(ov, hi, lo);
                    *reinterpret_cast<uint4*>(s_o + (size_t)((h * C + c0) / 8 + g) * AT_LBO + e * 16) = hi;
                    *reinterpret_cast<uint4*>(s_o + (size_t)((NH * C + h * C + c0) / 8 + g) * AT_LBO + e * 16) = lo;
                }
            }
        } else {
            // head outputs -> BF16 A operand (K = h * C + channel)
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                const float il = 1.0f / l[h];
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    uint4 u;
                    __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        hh[j] = __floats2bfloat162_rn(o[h][4 * g + j].x * il, o[h][4 * g + j].y * il);
                    *reinterpret_cast<uint4*>(s_o + (size_t)((h * C + c0) / 8 + g) * AT_LBO + e * 16) = u;
                }
            }
        }
    }
    umma::fence_smem_to_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    if (!failed) {
        // ---- O W^O into TMEM columns [0, C) ----
        if (tid == 0) {
            constexpr uint32_t idesc = SPLIT ? umma::idesc_f16_f32(AT_M, C) : umma::idesc_bf16_f32(AT_M, C);
            const uint32_t a0 = umma::smem_u32(s_o), b0 = umma::smem_u32(s_wo);
            constexpr uint32_t LBO_A = AT_LBO, LBO_B = C * 16;
            constexpr uint32_t A_LO = (NH * C / 8) * LBO_A, B_LO = C * NH * C * 2;  // the low parts (bytes)
#pragma unroll
            for (int kk = 0; kk < NH * C / 16; ++kk) {
                const uint32_t ak = a0 + 2 * kk * LBO_A, bk = b0 + 2 * kk * LBO_B;
                umma::mma_bf16(tmem, umma::desc(ak, LBO_A, 128), umma::desc(bk, LBO_B, 128), idesc, kk > 0);
                if constexpr (SPLIT) {
                    umma::mma_bf16(tmem + S::LO_COL, umma::desc(ak, LBO_A, 128), umma::desc(bk + B_LO, LBO_B, 128), idesc,
                                   kk > 0);
                    umma::mma_bf16(tmem + S::LO_COL, umma::desc(ak + A_LO, LBO_A, 128), umma::desc(bk, LBO_B, 128), idesc, 1);
                }
            }
            umma::commit(mbar);
        }
        failed = __syncthreads_or(!umma::mbar_wait(mbar, 1, AT_WAIT_NS));
        failed_phase = 1;
        umma::fence_after_sync();
        if (!failed) {
            // TMEM lane -> element er, columns ch * 16 .. + 15: residual (the entering volume, from
            // the X tile, or v0 on the first step) added here and V_attn stored as BF16
            const int q = warp & 3, grp = warp >> 2;
            const int er = q * 32 + lane;
            const int ex = blockIdx.y * AT_TW + er % AT_TW, ey = blockIdx.z * AT_TH + er / AT_TW;
            for (int ch = grp; ch < C / 16; ch += TPE) {
                float v[16];
                tmem_acc16<SPLIT, S::LO_COL>(tmem + ((uint32_t)(q * 32) << 16) + ch * 16, v);
                if constexpr (SPLIT) {
                    // FP32 form: the row scaled back (exactly: a power of two), the FP32 residual from
                    // the X tile (or v0), V_attn stored in FP32
                    if (ex < W && ey < H) {
                        const int oe = reinterpret_cast<const int*>(sm + S::oexp_off)[er];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float4 r = make_float4(misc[ch * 16 + 4 * i], misc[ch * 16 + 4 * i + 1],
                                                   misc[ch * 16 + 4 * i + 2], misc[ch * 16 + 4 * i + 3]);
                            if (TR != TR_INIT) r = *reinterpret_cast<const float4*>(s_x + (size_t)(4 * ch + i) * AT_LBO + er * 16);
                            v[4 * i] = ldexpf(v[4 * i], oe) + r.x;
                            v[4 * i + 1] = ldexpf(v[4 * i + 1], oe) + r.y;
                            v[4 * i + 2] = ldexpf(v[4 * i + 2], oe) + r.z;
                            v[4 * i + 3] = ldexpf(v[4 * i + 3], oe) + r.w;
                        }
                        float* dst = reinterpret_cast<float*>(a.out) + (((size_t)li * H + ey) * W + ex) * C + ch * 16;
                        uint4 u[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            u[i] = make_uint4(__float_as_uint(v[4 * i]), __float_as_uint(v[4 * i + 1]),
                                              __float_as_uint(v[4 * i + 2]), __float_as_uint(v[4 * i + 3]));
                        stcs256(dst, u[0], u[1]);
                        stcs256(dst + 8, u[2], u[3]);
                    }
                    continue;
                }
                if (ex < W && ey < H) {
                    if (TR == TR_INIT) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] += misc[ch * 16 + i];
                    } else {
                        const uint4 p0 = *reinterpret_cast<const uint4*>(s_x + (size_t)(2 * ch) * AT_LBO + er * 16);
                        const uint4 p1 = *reinterpret_cast<const uint4*>(s_x + (size_t)(2 * ch + 1) * AT_LBO + er * 16);
                        const uint32_t pk[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            v[2 * j] += __uint_as_float(pk[j] << 16);
                            v[2 * j + 1] += __uint_as_float(pk[j] & 0xffff0000u);
                        }
                    }
                    uint4 u[2];
                    __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(u);
#pragma unroll
                    for (int j = 0; j < 8; ++j) hh[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                    // one 256-bit streaming store: V_attn is read back only by the next kernel
                    stcs256(reinterpret_cast<__nv_bfloat16*>(a.out) + (((size_t)li * H + ey) * W + ex) * C + ch * 16,
                            u[0], u[1]);
                }
            }
        }
        if constexpr (LAST) {
            // blend logits of the element, contiguous [m] in the [H][W][L][V] layout
            if (!failed && live) {
                float* dst = a.beta + (((size_t)y * W + x) * L + li) * NV;
                const float* src = s_beta + e * NV;
                if (NV % (4 * TPE) == 0) {  // 16-byte runs: the element's views split across its lanes
                    for (int m = 4 * sub; m < NV; m += 4 * TPE)
                        __stcs(reinterpret_cast<float4*>(dst + m), *reinterpret_cast<const float4*>(src + m));
                } else {
                    for (int m = sub; m < NV; m += TPE) __stcs(dst + m, src[m]);
                }
            }
        }
    }
    if (failed && tid == 0) atomicExch(a.err, 3 + (int)failed_phase);
    if (failed) umma::mbar_wait(mbar, failed_phase, wait_ns);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(tmem, S::tmem_cols);
}

template <int C, int NH, bool SPLIT>
static cudaError_t launch_tc_nh(const AttendArgs& a, Transition tr, bool last, cudaStream_t st) {
    dim3 grid(a.L, (a.W + AT_TW - 1) / AT_TW, (a.H + AT_TH - 1) / AT_TH);
    const int threads = AT_M * (C / 16);
    // FP32 form, eight views at C = 32 with up to two heads (the 1080p workload): the view count fixed
    // at compile time (measured faster there; the BF16 form's unrolled loop spills at its register cap)
    constexpr bool FIX8 = SPLIT && C == 32 && NH <= 2;
#define QK_TC_LAUNCH_V(TRV, LASTV, VTV)                                                                \
    do {                                                                                               \
        const size_t smem = AtSmem<C, NH, LASTV, SPLIT>::total(a.V);                                   \
        auto k = attend_tc_kernel<C, NH, TRV, LASTV, SPLIT, VTV>;                                      \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                \
        k<<<grid, threads, smem, st>>>(a);                                                             \
    } while (0)
#define QK_TC_LAUNCH(TRV, LASTV)                                                                       \
    do {                                                                                               \
        if (FIX8 && a.V == 8) QK_TC_LAUNCH_V(TRV, LASTV, FIX8 ? 8 : 0);                                \
        else QK_TC_LAUNCH_V(TRV, LASTV, 0);                                                            \
    } while (0)
    if (tr == TR_INIT) {
        if (last) QK_TC_LAUNCH(TR_INIT, true); else QK_TC_LAUNCH(TR_INIT, false);
    } else if (tr == TR_SAME) {
        if (last) QK_TC_LAUNCH(TR_SAME, true); else QK_TC_LAUNCH(TR_SAME, false);
    } else {
        if (last) QK_TC_LAUNCH(TR_UP2, true); else QK_TC_LAUNCH(TR_UP2, false);
    }
#undef QK_TC_LAUNCH
#undef QK_TC_LAUNCH_V
    return cudaGetLastError();
}

template <int C, bool SPLIT>
static cudaError_t launch_tc_c(const AttendArgs& a, int heads, Transition tr, bool last, cudaStream_t st) {
    if (heads == 1) return launch_tc_nh<C, 1, SPLIT>(a, tr, last, st);
    if (heads == 2) return launch_tc_nh<C, 2, SPLIT>(a, tr, last, st);
    // four heads: (4 + 1) C query columns; at C = 64 that is 320, above the 256 columns of one
    // M = 128 MMA (and its shared memory above 227 KB), so that configuration is not built
    if constexpr (C <= 32) {
        if (heads == 4) return launch_tc_nh<C, 4, SPLIT>(a, tr, last, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_attend_tc(const AttendArgs& a, int C, int heads, Transition tr, bool last, bool split, cudaStream_t st) {
    if (!a.wtc || !a.err) return cudaErrorInvalidValue;
    // 256-bit loads of the taps and of the entering volume, 256-bit stores of V_attn
    if (reinterpret_cast<uintptr_t>(a.feat) % 32 || reinterpret_cast<uintptr_t>(a.prev) % 32 ||
        reinterpret_cast<uintptr_t>(a.out) % 32)
        return cudaErrorMisalignedAddress;
    if (split) {
        // FP32 form (C <= 32): the FP16 parts of the operands take twice the shared memory
        if (C == 16) return launch_tc_c<16, true>(a, heads, tr, last, st);
        if (C == 32) return launch_tc_c<32, true>(a, heads, tr, last, st);
        return cudaErrorInvalidValue;
    }
    if (C == 16) return launch_tc_c<16, false>(a, heads, tr, last, st);
    if (C == 32) return launch_tc_c<32, false>(a, heads, tr, last, st);
    if (C == 64) return launch_tc_c<64, false>(a, heads, tr, last, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
