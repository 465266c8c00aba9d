// Templates of the SIMT one-to-many and standard attention kernels and their launchers
// (k_attend.cu describes them); included by the translation units that instantiate them for
// one channel count each (k_attend_c*.cu, k_attend_std_c*.cu), so that the build compiles the
// instantiations in parallel.
#pragma once

#include <algorithm>

#include "device_common.cuh"

namespace quark {

// -------------------------------------------------------------------------------------------
// Sample-attend
// -------------------------------------------------------------------------------------------

constexpr int ATT_THREADS = 128;

// acc[j] += x * (w[2j], w[2j+1]) for 16 weights at w (shared memory): packed FP32x2
__device__ __forceinline__ void fma_row16_x2(const float* w, float x, float2 (&acc)[8]) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
    const float2 x2 = make_float2(x, x);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 t = w4[i];
        acc[2 * i] = __ffma2_rn(x2, make_float2(t.x, t.y), acc[2 * i]);
        acc[2 * i + 1] = __ffma2_rn(x2, make_float2(t.z, t.w), acc[2 * i + 1]);
    }
}
// D[j] += w * texel[2j .. 2j+1] for 16 FP32 channels at p (global memory, 32-byte aligned): two
// 256-bit loads, each a whole 32-byte sector
__device__ __forceinline__ void fma_tap16_x2(const float* p, float w, float2 (&D)[8]) {
    const float2 w2 = make_float2(w, w);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        uint4 a, b;
        ldg256(p + 8 * i, a, b);
        D[4 * i] = __ffma2_rn(make_float2(__uint_as_float(a.x), __uint_as_float(a.y)), w2, D[4 * i]);
        D[4 * i + 1] = __ffma2_rn(make_float2(__uint_as_float(a.z), __uint_as_float(a.w)), w2, D[4 * i + 1]);
        D[4 * i + 2] = __ffma2_rn(make_float2(__uint_as_float(b.x), __uint_as_float(b.y)), w2, D[4 * i + 2]);
        D[4 * i + 3] = __ffma2_rn(make_float2(__uint_as_float(b.z), __uint_as_float(b.w)), w2, D[4 * i + 3]);
    }
}

// Volume entering the step at element e = (layer li, pixel (x, y)) -- v0 (step 0), the previous
// volume at this layer, or its x2 bilinear upsample (Sec. 3.2.2) -- and the depth its views are
// sampled at (anchors at step 0, else Eq. depth_activation of t = V w_d + b_d).
__device__ __forceinline__ void fma_tap16_x2(const __nv_bfloat16* p, float w, float2 (&D)[8]) {
    uint4 u[2];
    ldg256(p, u[0], u[1]);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(u);
    const float2 w2 = make_float2(w, w);
#pragma unroll
    for (int j = 0; j < 8; ++j) D[j] = __ffma2_rn(__bfloat1622float2(h[j]), w2, D[j]);
}

template <typename T, int C, int TR>
__device__ __forceinline__ float volume_in(const AttendArgs& a, const float* sw, const AttendLayout& lay, int li, int y,
                                           int x, size_t e, bool writer, float (&vin)[C]) {
    const int L = a.L;
    if (TR == TR_INIT) {
#pragma unroll
        for (int c = 0; c < C; ++c) vin[c] = sw[lay.v0() + c];
    } else if (TR == TR_SAME) {
        const T* p = reinterpret_cast<const T*>(a.prev) + e * C;
#pragma unroll
        for (int cc = 0; cc < C; cc += 16) {
            float t[16];
            load16(p + cc, t);
#pragma unroll
            for (int i = 0; i < 16; ++i) vin[cc + i] = t[i];
        }
    } else {
        int y0, y1, x0, x1;
        float wy, wx;
        resize_taps(y, 2, a.Hp, y0, y1, wy);
        resize_taps(x, 2, a.Wp, x0, x1, wx);
        const T* base = reinterpret_cast<const T*>(a.prev) + (size_t)li * a.Hp * a.Wp * C;
        const T* p00 = base + ((size_t)y0 * a.Wp + x0) * C;
        const T* p01 = base + ((size_t)y0 * a.Wp + x1) * C;
        const T* p10 = base + ((size_t)y1 * a.Wp + x0) * C;
        const T* p11 = base + ((size_t)y1 * a.Wp + x1) * C;
#pragma unroll
        for (int cc = 0; cc < C; cc += 16) {
            float t00[16], t01[16], t10[16], t11[16];
            load16(p00 + cc, t00);
            load16(p01 + cc, t01);
            load16(p10 + cc, t10);
            load16(p11 + cc, t11);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                float top = t00[i] + wx * (t01[i] - t00[i]);
                float bot = t10[i] + wx * (t11[i] - t10[i]);
                vin[cc + i] = top + wy * (bot - top);
            }
        }
    }

    float d;
    if (TR == TR_INIT) {
        d = depth_anchor(li, L, a.dp);
    } else {
        float t = sw[lay.bd()];
#pragma unroll
        for (int c = 0; c < C; ++c) t = fmaf(vin[c], sw[lay.wd() + c], t);
        d = depth_from_logit(t, li, L, a.dp);
    }
    // reused depths of an earlier step, or this step's depths kept for a later one
    if (a.depth_in) d = __ldg(a.depth_in + e);
    else if (a.depth_out && writer) a.depth_out[e] = d;
    return d;
}

template <typename T, int C, int NH, int TR, bool LAST>
__global__ void __launch_bounds__(ATT_THREADS) attend_kernel(const AttendArgs a) {
    constexpr int TPE = C / 16;  // threads per element
    const AttendLayout lay{C, NH};
    extern __shared__ float4 sw4[];
    float* sw = reinterpret_cast<float*>(sw4);
    for (int i = threadIdx.x; i < lay.total(); i += blockDim.x) sw[i] = a.w[i];
    __syncthreads();

    // Block b covers pixels [(b / L) * EPB, + EPB) of layer b % L: the layer varies fastest, so
    // the blocks resident at one time sample every layer of the same pixels and each texel of the
    // feature level is fetched from DRAM about once per step rather than once per layer.
    constexpr int EPB = ATT_THREADS / TPE;
    const int L = a.L, H = a.H, W = a.W;
    const size_t plane = (size_t)H * W;
    const int li = (int)(blockIdx.x % L);
    const int sub = (int)(threadIdx.x % TPE);
    size_t pix = (size_t)(blockIdx.x / L) * EPB + threadIdx.x / TPE;
    const bool live = pix < plane;
    if (!live) pix = plane - 1;  // keep the group's lanes in the shuffles; no stores
    const size_t e = (size_t)li * plane + pix;
    const int y = (int)(pix / W);
    const int x = (int)(pix % W);
    const int c0 = sub * 16;

    float vin[C];
    const float d = volume_in<T, C, TR>(a, sw, lay, li, y, x, e, live && sub == 0, vin);

    // ---- RMSNorm and query projections ----
    float ms = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) ms = fmaf(vin[c], vin[c], ms);
    const float rinv = 1.0f / sqrtf(ms / C + 1e-6f);
    float xn[C];
#pragma unroll
    for (int c = 0; c < C; ++c) xn[c] = vin[c] * rinv * sw[lay.g() + c];
    float vres[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float s = 0.f;
#pragma unroll
        for (int sb = 0; sb < TPE; ++sb)
            if (sb == sub) s = vin[sb * 16 + i];
        vres[i] = s;
    }
    float2 q[NH][8];
#pragma unroll
    for (int h = 0; h < NH; ++h)
#pragma unroll
        for (int j = 0; j < 8; ++j) q[h][j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < C; ++k) {
#pragma unroll
        for (int h = 0; h < NH; ++h) fma_row16_x2(&sw[lay.wq() + k * NH * C + h * C + c0], xn[k], q[h]);
    }
    float2 qb[8];
    if constexpr (LAST) {
#pragma unroll
        for (int j = 0; j < 8; ++j) qb[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < C; ++k) fma_row16_x2(&sw[lay.wb() + k * C + c0], xn[k], qb);
    }

    // ---- views: sample, online softmax (log2 units, lazy rescale), weighted sum ----
    const float lscale = 1.4426950408889634f / sqrtf((float)C), scale = 1.0f / sqrtf((float)C);
    const float pxc = x + 0.5f, pyc = y + 0.5f;
    float mx[NH], l[NH];
    float2 o[NH][8];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        mx[h] = -INFINITY;
        l[h] = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) o[h][j] = make_float2(0.f, 0.f);
    }
    const T* feat = reinterpret_cast<const T*>(a.feat);
    const size_t vstride = (size_t)a.fh * a.fw * C;
    for (int m = 0; m < a.V; ++m) {
        float2 D[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) D[j] = make_float2(0.f, 0.f);
        float u, v;
        const bool ok = reproject(a.geo.v[m], pxc, pyc, d, u, v);
        const Taps4 tp = bilinear_taps4(ok, u, v, a.fh, a.fw);
        const T* fb = feat + m * vstride + c0;
        fma_tap16_x2(fb + (size_t)tp.i00 * C, tp.w00, D);
        fma_tap16_x2(fb + (size_t)tp.i01 * C, tp.w01, D);
        fma_tap16_x2(fb + (size_t)tp.i10 * C, tp.w10, D);
        fma_tap16_x2(fb + (size_t)tp.i11 * C, tp.w11, D);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc = __ffma2_rn(q[h][j], D[j], acc);
            float s = acc.x + acc.y;
#pragma unroll
            for (int off = 1; off < TPE; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            s *= lscale;
            if (s > mx[h]) {  // the running maximum moves: rescale
                const float cs = exp2f(mx[h] - s);
                const float2 cs2 = make_float2(cs, cs);
                l[h] *= cs;
#pragma unroll
                for (int j = 0; j < 8; ++j) o[h][j] = __fmul2_rn(o[h][j], cs2);
                mx[h] = s;
            }
            const float p = exp2f(s - mx[h]);
            const float2 p2 = make_float2(p, p);
            l[h] += p;
#pragma unroll
            for (int j = 0; j < 8; ++j) o[h][j] = __ffma2_rn(p2, D[j], o[h][j]);
        }
        if constexpr (LAST) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc = __ffma2_rn(qb[j], D[j], acc);
            float s = acc.x + acc.y;
#pragma unroll
            for (int off = 1; off < TPE; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (live && sub == 0) a.beta[(((size_t)y * W + x) * L + li) * a.V + m] = s * scale;
        }
    }

    // ---- output projection and residual ----
    float2 out2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) out2[j] = make_float2(vres[2 * j], vres[2 * j + 1]);
    const int lane = threadIdx.x & 31;
    const int gbase = lane & ~(TPE - 1);
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        const float il = 1.0f / l[h];
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const float2 pr = o[h][(k % 16) / 2];
            float ok = (k & 1) ? pr.y : pr.x;
            if (TPE > 1) ok = __shfl_sync(0xffffffffu, ok, gbase + k / 16);
            fma_row16_x2(&sw[lay.wo() + (h * C + k) * C + c0], ok * il, out2);
        }
    }
    float out[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        out[2 * j] = out2[j].x;
        out[2 * j + 1] = out2[j].y;
    }
    if (live) store16(reinterpret_cast<T*>(a.out) + e * C + c0, out);
}

// -------------------------------------------------------------------------------------------
// Standard multi-head cross attention (attn_mode STANDARD)
// -------------------------------------------------------------------------------------------

// Keys and values in image space: K = F W^k, V = F W^val for every texel of a pyramid level
// (a dense [texels x C] x [C x 2C] product), plus on the last step a copy of F for the blend
// logits.  Sampling the projected maps equals projecting the sampled features, since bilinear
// sampling is linear and the projections have no bias.  Output texel: [K (C) | V (C) (| F (C))].
template <typename T, int C, int NC>
__global__ void __launch_bounds__(128) kv_project_kernel(const T* __restrict__ feat, size_t n,
                                                         const float* __restrict__ wkv, T* __restrict__ out) {
    __shared__ __align__(16) float w[C * 2 * C];
    for (int i = threadIdx.x; i < 2 * C * C; i += blockDim.x) w[i] = wkv[i];
    __syncthreads();
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        float f[C];
#pragma unroll
        for (int c0 = 0; c0 < C; c0 += 16) {
            float v[16];
            load16(feat + t * C + c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) f[c0 + i] = v[i];
        }
        float2 acc[C];  // 2C outputs
#pragma unroll
        for (int j = 0; j < C; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const float4* w4 = reinterpret_cast<const float4*>(w + k * 2 * C);
            const float2 x2 = make_float2(f[k], f[k]);
#pragma unroll
            for (int i = 0; i < C / 2; ++i) {
                const float4 u = w4[i];
                acc[2 * i] = __ffma2_rn(x2, make_float2(u.x, u.y), acc[2 * i]);
                acc[2 * i + 1] = __ffma2_rn(x2, make_float2(u.z, u.w), acc[2 * i + 1]);
            }
        }
        T* o = out + t * NC;
#pragma unroll
        for (int c0 = 0; c0 < 2 * C; c0 += 16) {
            float v[16];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                v[2 * i] = acc[c0 / 2 + i].x;
                v[2 * i + 1] = acc[c0 / 2 + i].y;
            }
            store16(o + c0, v);
        }
        if (NC == 3 * C) {
#pragma unroll
            for (int c0 = 0; c0 < C; c0 += 16) {
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = f[c0 + i];
                store16(o + 2 * C + c0, v);
            }
        }
    }
}

// Standard attention (Sec. 3.3 Eq. MultiHead with Attention(Q, K, V)): per element, q = N(V) W^q;
// per view the key and value rows sampled from the projected maps; head i (channels
// [i C/h, (i+1) C/h)) takes softmax over views of q_i . k_i / sqrt(C/h) and the weighted sum of
// v_i; the heads are concatenated and projected by W^O; residual.  The last step's blend logits
// use the raw features (x W^beta . Delta / sqrt(C)), as in the one-to-many mode.  Same thread
// mapping, block order and online softmax (log2 units) as attend_kernel; a thread's 16 channels
// hold 16 / min(C/h, 16) heads or, with C/h = 32, half of one (its partner lane has the rest).
template <typename T, int C, int NH, int TR, bool LAST>
__global__ void __launch_bounds__(ATT_THREADS) attend_std_kernel(const AttendArgs a) {
    constexpr int TPE = C / 16;
    constexpr int DH = C / NH;              // per-head width
    constexpr int HD = DH < 16 ? DH : 16;   // channels of one head inside a thread's 16
    constexpr int NHT = 16 / HD;            // heads (or head halves) per thread
    constexpr int NC = LAST ? 3 * C : 2 * C;
    const AttendLayout lay{C, NH};
    const StdLayout sl{C};
    extern __shared__ float4 sw4[];
    float* sw = reinterpret_cast<float*>(sw4);
    float* ss = sw + lay.total();
    for (int i = threadIdx.x; i < lay.total(); i += blockDim.x) sw[i] = a.w[i];
    for (int i = threadIdx.x; i < sl.total(); i += blockDim.x) ss[i] = a.w_std[i];
    __syncthreads();

    constexpr int EPB = ATT_THREADS / TPE;
    const int L = a.L, H = a.H, W = a.W;
    const size_t plane = (size_t)H * W;
    const int li = (int)(blockIdx.x % L);
    const int sub = (int)(threadIdx.x % TPE);
    size_t pix = (size_t)(blockIdx.x / L) * EPB + threadIdx.x / TPE;
    const bool live = pix < plane;
    if (!live) pix = plane - 1;  // keep the group's lanes in the shuffles; no stores
    const size_t e = (size_t)li * plane + pix;
    const int y = (int)(pix / W);
    const int x = (int)(pix % W);
    const int c0 = sub * 16;

    float vin[C];
    const float d = volume_in<T, C, TR>(a, sw, lay, li, y, x, e, live && sub == 0, vin);
    float ms = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) ms = fmaf(vin[c], vin[c], ms);
    const float rinv = 1.0f / sqrtf(ms / C + 1e-6f);
    float xn[C];
#pragma unroll
    for (int c = 0; c < C; ++c) xn[c] = vin[c] * rinv * sw[lay.g() + c];
    float vres[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float s = 0.f;
#pragma unroll
        for (int sb = 0; sb < TPE; ++sb)
            if (sb == sub) s = vin[sb * 16 + i];
        vres[i] = s;
    }
    float2 q[8], qb[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) q[j] = qb[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        fma_row16_x2(&ss[sl.wq() + k * C + c0], xn[k], q);
        if constexpr (LAST) fma_row16_x2(&sw[lay.wb() + k * C + c0], xn[k], qb);
    }

    const float lscale = 1.4426950408889634f / sqrtf((float)DH), bscale = 1.0f / sqrtf((float)C);
    const float pxc = x + 0.5f, pyc = y + 0.5f;
    float mx[NHT], l[NHT];
    float2 o[8];
#pragma unroll
    for (int j = 0; j < NHT; ++j) {
        mx[j] = -INFINITY;
        l[j] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = make_float2(0.f, 0.f);
    const T* kv = reinterpret_cast<const T*>(a.feat);
    const size_t vstride = (size_t)a.fh * a.fw * NC;
    for (int m = 0; m < a.V; ++m) {
        float2 K[8], Vv[8], F[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) K[j] = Vv[j] = F[j] = make_float2(0.f, 0.f);
        float u, v;
        const bool ok = reproject(a.geo.v[m], pxc, pyc, d, u, v);
        const Taps4 tp = bilinear_taps4(ok, u, v, a.fh, a.fw);
        const T* fb = kv + m * vstride + c0;
        const int idx[4] = {tp.i00, tp.i01, tp.i10, tp.i11};
        const float wt[4] = {tp.w00, tp.w01, tp.w10, tp.w11};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const T* px = fb + (size_t)idx[t] * NC;
            fma_tap16_x2(px, wt[t], K);
            fma_tap16_x2(px + C, wt[t], Vv);
            if constexpr (LAST) fma_tap16_x2(px + 2 * C, wt[t], F);
        }
#pragma unroll
        for (int j = 0; j < NHT; ++j) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int p = j * HD / 2; p < (j + 1) * HD / 2; ++p) acc = __ffma2_rn(q[p], K[p], acc);
            float s = acc.x + acc.y;
            if (DH > 16) s += __shfl_xor_sync(0xffffffffu, s, 1);  // the other half of the head
            s *= lscale;
            if (s > mx[j]) {  // the running maximum moves: rescale
                const float cs = exp2f(mx[j] - s);
                const float2 cs2 = make_float2(cs, cs);
                l[j] *= cs;
#pragma unroll
                for (int p = j * HD / 2; p < (j + 1) * HD / 2; ++p) o[p] = __fmul2_rn(o[p], cs2);
                mx[j] = s;
            }
            const float pw = exp2f(s - mx[j]);
            const float2 p2 = make_float2(pw, pw);
            l[j] += pw;
#pragma unroll
            for (int p = j * HD / 2; p < (j + 1) * HD / 2; ++p) o[p] = __ffma2_rn(p2, Vv[p], o[p]);
        }
        if constexpr (LAST) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc = __ffma2_rn(qb[j], F[j], acc);
            float s = acc.x + acc.y;
#pragma unroll
            for (int off = 1; off < TPE; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (live && sub == 0) a.beta[(((size_t)y * W + x) * L + li) * a.V + m] = s * bscale;
        }
    }

    // ---- concat heads, W^O, residual ----
#pragma unroll
    for (int j = 0; j < NHT; ++j) {
        const float il = 1.0f / l[j];
        const float2 il2 = make_float2(il, il);
#pragma unroll
        for (int p = j * HD / 2; p < (j + 1) * HD / 2; ++p) o[p] = __fmul2_rn(o[p], il2);
    }
    float2 out2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) out2[j] = make_float2(vres[2 * j], vres[2 * j + 1]);
    const int lane = threadIdx.x & 31;
    const int gbase = lane & ~(TPE - 1);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const float2 pr = o[(k % 16) / 2];
        float ok = (k & 1) ? pr.y : pr.x;
        if (TPE > 1) ok = __shfl_sync(0xffffffffu, ok, gbase + k / 16);
        fma_row16_x2(&ss[sl.wo() + k * C + c0], ok, out2);
    }
    float out[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        out[2 * j] = out2[j].x;
        out[2 * j + 1] = out2[j].y;
    }
    if (live) store16(reinterpret_cast<T*>(a.out) + e * C + c0, out);
}

template <typename T, int C>
static cudaError_t launch_kv_t(const void* feat, size_t n, const float* wkv, void* out, bool with_f, cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const unsigned grid = (unsigned)std::min<size_t>((n + 127) / 128, (size_t)sms * 16);
    if (with_f)
        kv_project_kernel<T, C, 3 * C><<<grid, 128, 0, st>>>((const T*)feat, n, wkv, (T*)out);
    else
        kv_project_kernel<T, C, 2 * C><<<grid, 128, 0, st>>>((const T*)feat, n, wkv, (T*)out);
    return cudaGetLastError();
}

template <typename T, int C, int NH>
static cudaError_t launch_std_nh(const AttendArgs& a, Transition tr, bool last, cudaStream_t st) {
    const AttendLayout lay{C, NH};
    const StdLayout sl{C};
    const size_t smem = (size_t)(lay.total() + sl.total()) * sizeof(float);
    constexpr int EPB = ATT_THREADS / (C / 16);
    const size_t plane = (size_t)a.H * a.W;
    const unsigned grid = (unsigned)(((plane + EPB - 1) / EPB) * a.L);
#define QK_STD_LAUNCH(TRV, LASTV)                                                                      \
    do {                                                                                               \
        auto k = attend_std_kernel<T, C, NH, TRV, LASTV>;                                              \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                \
        k<<<grid, ATT_THREADS, smem, st>>>(a);                                                         \
    } while (0)
    if (tr == TR_INIT) {
        if (last) QK_STD_LAUNCH(TR_INIT, true); else QK_STD_LAUNCH(TR_INIT, false);
    } else if (tr == TR_SAME) {
        if (last) QK_STD_LAUNCH(TR_SAME, true); else QK_STD_LAUNCH(TR_SAME, false);
    } else {
        if (last) QK_STD_LAUNCH(TR_UP2, true); else QK_STD_LAUNCH(TR_UP2, false);
    }
#undef QK_STD_LAUNCH
    return cudaGetLastError();
}

template <typename T, int C>
static cudaError_t launch_std_c(const AttendArgs& a, int heads, Transition tr, bool last, cudaStream_t st) {
    if (heads == 1) return launch_std_nh<T, C, 1>(a, tr, last, st);
    if (heads == 2) return launch_std_nh<T, C, 2>(a, tr, last, st);
    if (heads == 4) return launch_std_nh<T, C, 4>(a, tr, last, st);
    return cudaErrorInvalidValue;
}

template <typename T, int C, int NH>
static cudaError_t launch_nh(const AttendArgs& a, Transition tr, bool last, cudaStream_t st) {
    const AttendLayout lay{C, NH};
    const size_t smem = (size_t)lay.total() * sizeof(float);
    constexpr int EPB = ATT_THREADS / (C / 16);
    const size_t plane = (size_t)a.H * a.W;
    const unsigned grid = (unsigned)(((plane + EPB - 1) / EPB) * a.L);
#define QK_LAUNCH(TRV, LASTV)                                                                          \
    do {                                                                                               \
        auto k = attend_kernel<T, C, NH, TRV, LASTV>;                                                  \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                \
        k<<<grid, ATT_THREADS, smem, st>>>(a);                                                         \
    } while (0)
    if (tr == TR_INIT) {
        if (last) QK_LAUNCH(TR_INIT, true); else QK_LAUNCH(TR_INIT, false);
    } else if (tr == TR_SAME) {
        if (last) QK_LAUNCH(TR_SAME, true); else QK_LAUNCH(TR_SAME, false);
    } else {
        if (last) QK_LAUNCH(TR_UP2, true); else QK_LAUNCH(TR_UP2, false);
    }
#undef QK_LAUNCH
    return cudaGetLastError();
}

template <typename T, int C>
static cudaError_t launch_c(const AttendArgs& a, int heads, Transition tr, bool last, cudaStream_t st) {
    if (heads == 1) return launch_nh<T, C, 1>(a, tr, last, st);
    if (heads == 2) return launch_nh<T, C, 2>(a, tr, last, st);
    if (heads == 4) return launch_nh<T, C, 4>(a, tr, last, st);
    return cudaErrorInvalidValue;
}

// Per-channel-count entry points (one translation unit each).
cudaError_t attend_fp32_c16(const AttendArgs& a, int heads, Transition tr, bool last, cudaStream_t st);
cudaError_t attend_fp32_c32(const AttendArgs& a, int heads, Transition tr, bool last, cudaStream_t st);
cudaError_t attend_fp32_c64(const AttendArgs& a, int heads, Transition tr, bool last, cudaStream_t st);
cudaError_t attend_std_c16(const AttendArgs& a, int heads, Transition tr, bool last, bool bf16, cudaStream_t st);
cudaError_t attend_std_c32(const AttendArgs& a, int heads, Transition tr, bool last, bool bf16, cudaStream_t st);
cudaError_t attend_std_c64(const AttendArgs& a, int heads, Transition tr, bool last, bool bf16, cudaStream_t st);

}  // namespace quark
