// Hand-written adjoint of the differentiable stage (FP32 form): the last Update & Fuse step and
// the final render as a function of the volume entering the step, the step's pyramid level and
// the step's weights.  Loss gradients arrive as dL/dRGB per output pixel.
//
//   render_bwd_kernel   over operator (reverse scan with the colour behind each layer), blend
//                       softmax Jacobian, image bilinear sampling -> sample coordinates -> depth
//                       (Eq. depth_activation) -> raw logits; upsample adjoint as a scatter.
//   decode_bwd_kernel   t = V w_d + b_d and s = V w_sigma + b_sigma.
//   conv3x3_kernel      3x3 convolution per layer plane, or its transpose (the adjoint of the
//                       conv block's convolutions), with an optional gelu' epilogue.
//   rmsnorm / rmsnorm_bwd_kernel   N(V) and its adjoint (+ the residual path).
//   attend_bwd_kernel   one-to-many attention with sampling: recomputes the sampled features
//                       (nothing is stored by the forward), softmax Jacobian, query / output
//                       projections, scatter of the feature gradient into the pyramid level
//                       (atomics), coordinate gradient through the decoded depth.
//   xty_kernel + reduce_kernel     deterministic weight-gradient reductions sum_e X^T Y (with
//                       3x3 tap shifts for the conv weights).
#include "device_common.cuh"
#include "bwd_internal.cuh"

namespace quark {

constexpr int BW_THREADS = 128;
constexpr int L_MAX = 64;

// d/dt of Eq. (depth_activation) at depth d: d = 1/D, D = (delta + 0.5/L tanh t) span + 1/far.
__device__ __forceinline__ float ddepth_dt(float t, float d, int L, DepthParams dp) {
    const float th = tanhf(t);
    return -d * d * dp.span * (0.5f / L) * (1.0f - th * th);
}

// Bilinear sample of an RGBA image with the derivatives w.r.t. the sample coordinates.
__device__ __forceinline__ void sample_rgb_grad(const float4* __restrict__ img, int h, int w, float u, float v,
                                                float (&c)[3], float (&cu)[3], float (&cv)[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] = cu[i] = cv[i] = 0.f;
    Taps t;
    if (!bilinear_taps(u, v, h, w, t)) return;
    const int xs[2] = {t.x0, t.x0 + 1}, ys[2] = {t.y0, t.y0 + 1};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int yy = ys[a], xx = xs[b];
            if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
            const float4 p = __ldg(img + (size_t)yy * w + xx);
            const float wy = a ? t.fy : 1.f - t.fy, wx = b ? t.fx : 1.f - t.fx;
            const float dwx = b ? 1.f : -1.f, dwy = a ? 1.f : -1.f;  // d(wx)/du, d(wy)/dv
            const float pv[3] = {p.x, p.y, p.z};
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                c[i] = fmaf(wy * wx, pv[i], c[i]);
                cu[i] = fmaf(wy * dwx, pv[i], cu[i]);
                cv[i] = fmaf(dwy * wx, pv[i], cv[i]);
            }
        }
}

// Reprojection with du/dd and dv/dd (X = d a + b, u = X / Z).
__device__ __forceinline__ bool reproject_grad(const ViewMap& m, float px, float py, float d, float& u, float& v,
                                               float& du, float& dv) {
    const float ax = fmaf(m.A[0], px, fmaf(m.A[1], py, m.A[2]));
    const float ay = fmaf(m.A[3], px, fmaf(m.A[4], py, m.A[5]));
    const float az = fmaf(m.A[6], px, fmaf(m.A[7], py, m.A[8]));
    const float X = fmaf(d, ax, m.b[0]), Y = fmaf(d, ay, m.b[1]), Z = fmaf(d, az, m.b[2]);
    if (!(Z > 1e-6f)) return false;
    const float iz = 1.0f / Z;
    u = X * iz;
    v = Y * iz;
    du = (ax - u * az) * iz;
    dv = (ay - v * az) * iz;
    return true;
}

__global__ void __launch_bounds__(BW_THREADS) render_bwd_kernel(const RenderArgs a, const float* __restrict__ dl,
                                                                float* dt_raw, float* ds_raw, float* dbeta_raw) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)a.Hout * a.Wout) return;
    const int X = (int)(idx % a.Wout), Y = (int)(idx / a.Wout);
    const int L = a.L, V = a.V;
    int y0, y1, x0, x1;
    float wy, wx;
    resize_taps(Y, a.sy, a.Hl, y0, y1, wy);
    resize_taps(X, a.sx, a.Wl, x0, x1, wx);
    const size_t q[4] = {(size_t)y0 * a.Wl + x0, (size_t)y0 * a.Wl + x1, (size_t)y1 * a.Wl + x0,
                         (size_t)y1 * a.Wl + x1};
    const float qw[4] = {(1 - wy) * (1 - wx), (1 - wy) * wx, wy * (1 - wx), wy * wx};
    auto up = [&](const float* f, size_t stride, size_t off) {
        float top = f[q[0] * stride + off] * (1 - wx) + f[q[1] * stride + off] * wx;
        float bot = f[q[2] * stride + off] * (1 - wx) + f[q[3] * stride + off] * wx;
        return top * (1 - wy) + bot * wy;
    };
    auto scatter = [&](float* f, size_t stride, size_t off, float g) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (qw[i] != 0.f) atomicAdd(f + q[i] * stride + off, qw[i] * g);
    };
    const float pxc = X + 0.5f, pyc = Y + 0.5f;
    const size_t img_stride = (size_t)a.Hi * a.Wi;
    const float w3[3] = {dl[3 * idx], dl[3 * idx + 1], dl[3 * idx + 2]};
    float al[L_MAX], Tl[L_MAX], cl[L_MAX][3];
    float T = 1.f;
    for (int li = L - 1; li >= 0; --li) {  // forward, front to back
        const float d = depth_from_logit(up(a.t_raw, L, li), li, L, a.dp);
        const float alpha = sigmoidf_(up(a.s_raw, L, li));
        const size_t bs = (size_t)L * V, bo = (size_t)li * V;
        float bmax = -INFINITY;
        for (int m = 0; m < V; ++m) bmax = fmaxf(bmax, up(a.beta, bs, bo + m));
        float sum = 0.f, c[3] = {0.f, 0.f, 0.f};
        for (int m = 0; m < V; ++m) {
            const float p = expf(up(a.beta, bs, bo + m) - bmax);
            sum += p;
            float u, v;
            if (reproject(a.geo.v[m], pxc, pyc, d, u, v)) {
                float cm[3], cu[3], cv[3];
                sample_rgb_grad(a.rgba + m * img_stride, a.Hi, a.Wi, u, v, cm, cu, cv);
#pragma unroll
                for (int i = 0; i < 3; ++i) c[i] = fmaf(p, cm[i], c[i]);
            }
        }
        al[li] = alpha;
        Tl[li] = T;
#pragma unroll
        for (int i = 0; i < 3; ++i) cl[li][i] = c[i] / sum;
        T *= 1.f - alpha;
    }
    float cb[3] = {0.f, 0.f, 0.f};  // colour composited behind the current layer
    for (int li = 0; li < L; ++li) {  // adjoint, back to front
        const float alpha = al[li], Tli = Tl[li];
        float dal = 0.f, dc[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dal = fmaf(w3[i], cl[li][i] - cb[i], dal);
            dc[i] = Tli * alpha * w3[i];
        }
        dal *= Tli;
#pragma unroll
        for (int i = 0; i < 3; ++i) cb[i] = alpha * cl[li][i] + (1.f - alpha) * cb[i];
        scatter(ds_raw, L, li, dal * alpha * (1.f - alpha));
        // blend weights and sampled colours of the layer, recomputed
        const float t_up = up(a.t_raw, L, li);
        const float d = depth_from_logit(t_up, li, L, a.dp);
        const size_t bs = (size_t)L * V, bo = (size_t)li * V;
        float bmax = -INFINITY;
        for (int m = 0; m < V; ++m) bmax = fmaxf(bmax, up(a.beta, bs, bo + m));
        float sum = 0.f;
        for (int m = 0; m < V; ++m) sum += expf(up(a.beta, bs, bo + m) - bmax);
        float sbd = 0.f;  // sum_m beta_m dbeta_m with dbeta_m = dc . col_m
        for (int m = 0; m < V; ++m) {
            const float beta = expf(up(a.beta, bs, bo + m) - bmax) / sum;
            float u, v, du, dv;
            float cm[3] = {0.f, 0.f, 0.f}, cu[3] = {0.f, 0.f, 0.f}, cv[3] = {0.f, 0.f, 0.f};
            if (reproject_grad(a.geo.v[m], pxc, pyc, d, u, v, du, dv))
                sample_rgb_grad(a.rgba + m * img_stride, a.Hi, a.Wi, u, v, cm, cu, cv);
            sbd += beta * (dc[0] * cm[0] + dc[1] * cm[1] + dc[2] * cm[2]);
        }
        float dd = 0.f;
        for (int m = 0; m < V; ++m) {
            const float beta = expf(up(a.beta, bs, bo + m) - bmax) / sum;
            float u, v, du = 0.f, dv = 0.f;
            float cm[3] = {0.f, 0.f, 0.f}, cu[3] = {0.f, 0.f, 0.f}, cv[3] = {0.f, 0.f, 0.f};
            if (reproject_grad(a.geo.v[m], pxc, pyc, d, u, v, du, dv))
                sample_rgb_grad(a.rgba + m * img_stride, a.Hi, a.Wi, u, v, cm, cu, cv);
            const float dbm = dc[0] * cm[0] + dc[1] * cm[1] + dc[2] * cm[2];
            scatter(dbeta_raw, bs, bo + m, beta * (dbm - sbd));
            // colour of view m enters with weight beta: d(loss)/d(col_m) = beta dc
            dd += beta * ((dc[0] * cu[0] + dc[1] * cu[1] + dc[2] * cu[2]) * du +
                          (dc[0] * cv[0] + dc[1] * cv[1] + dc[2] * cv[2]) * dv);
        }
        scatter(dt_raw, L, li, dd * ddepth_dt(t_up, d, L, a.dp));
    }
}

// dV_out = dt w_d + ds w_sigma per element of [L][H][W]; (dt, ds) kept per element for the
// decoder-weight reductions.
__global__ void decode_bwd_kernel(const float* __restrict__ dt_raw, const float* __restrict__ ds_raw, int L, int H,
                                  int W, int C, const float* __restrict__ w_d, const float* __restrict__ w_s,
                                  float* dv_out, float* dts) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t plane = (size_t)H * W;
    if (e >= (size_t)L * plane) return;
    const int li = (int)(e / plane);
    const size_t pix = e % plane;
    const float dt = dt_raw[pix * L + li], ds = ds_raw[pix * L + li];
    for (int c = 0; c < C; ++c) dv_out[e * C + c] = dt * w_d[c] + ds * w_s[c];
    dts[2 * e] = dt;
    dts[2 * e + 1] = ds;
}

// out[p][co] = bias + sum_tap sum_ci in[p + off][ci] W[tap][ci][co]          (transpose = 0)
// out[p][ci] = sum_tap sum_co W[tap][ci][co] in[p - off][co]                  (transpose = 1)
// per layer plane, zero padding; optional epilogue out *= gelu'(aux[p]).
template <int C>
__global__ void __launch_bounds__(BW_THREADS) conv3x3_kernel(const float* __restrict__ in, const float* __restrict__ w,
                                                             const float* __restrict__ bias, float* out, int L, int H,
                                                             int W, int transpose, const float* __restrict__ gelu_aux) {
    __shared__ float sw[9 * C * C];
    for (int i = threadIdx.x; i < 9 * C * C; i += blockDim.x) sw[i] = w[i];
    __syncthreads();
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t plane = (size_t)H * W;
    if (e >= (size_t)L * plane) return;
    const int li = (int)(e / plane);
    const int y = (int)((e % plane) / W), x = (int)(e % W);
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = (!transpose && bias) ? bias[c] : 0.f;
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const int yy = transpose ? y - dy : y + dy, xx = transpose ? x - dx : x + dx;
        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
        const float* src = in + ((size_t)li * plane + (size_t)yy * W + xx) * C;
        const float* wt = sw + tap * C * C;
        if (!transpose) {
            for (int ci = 0; ci < C; ++ci) {
                const float v = src[ci];
#pragma unroll
                for (int co = 0; co < C; ++co) acc[co] = fmaf(v, wt[ci * C + co], acc[co]);
            }
        } else {
            for (int co = 0; co < C; ++co) {
                const float v = src[co];
#pragma unroll
                for (int ci = 0; ci < C; ++ci) acc[ci] = fmaf(v, wt[ci * C + co], acc[ci]);
            }
        }
    }
    if (gelu_aux) {
        const float* h = gelu_aux + e * C;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float z = h[c];
            const float cdf = 0.5f * (1.f + erff(z * 0.70710678118654752f));
            const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
            acc[c] *= cdf + z * pdf;
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) out[e * C + c] = acc[c];
}

// n = g v / rms(v) per element
template <int C>
__global__ void rmsnorm_kernel(const float* __restrict__ v, const float* __restrict__ g, float* n, size_t E) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    float ms = 0.f;
    for (int c = 0; c < C; ++c) ms = fmaf(v[e * C + c], v[e * C + c], ms);
    const float r = 1.0f / sqrtf(ms / C + 1e-6f);
    for (int c = 0; c < C; ++c) n[e * C + c] = g[c] * v[e * C + c] * r;
}

// dv = resid + adjoint of n = g v r at v given dn; dgterm = dn * v * r (column sums give dg)
template <int C>
__global__ void rmsnorm_bwd_kernel(const float* __restrict__ v, const float* __restrict__ g,
                                   const float* __restrict__ dn, const float* __restrict__ resid, float* dv,
                                   float* dgterm, size_t E) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    float ms = 0.f, dot = 0.f;
    for (int c = 0; c < C; ++c) {
        const float x = v[e * C + c];
        ms = fmaf(x, x, ms);
        dot = fmaf(g[c] * dn[e * C + c], x, dot);
    }
    const float r = 1.0f / sqrtf(ms / C + 1e-6f);
    const float k = r * r * r * dot / C;
    for (int c = 0; c < C; ++c) {
        const float x = v[e * C + c], dy = g[c] * dn[e * C + c];
        dv[e * C + c] = (resid ? resid[e * C + c] : 0.f) + r * dy - k * x;
        dgterm[e * C + c] = dn[e * C + c] * x * r;
    }
}

// ---------------------------------------------------------------------------------------------
// Attention with sampling
// ---------------------------------------------------------------------------------------------

template <int C, int NH>
__global__ void __launch_bounds__(BW_THREADS) attend_bwd_kernel(const AttendBwdArgs a) {
    constexpr int HC = NH * C;
    extern __shared__ float4 sw4[];
    float* sw = reinterpret_cast<float*>(sw4);  // g, w_d, b_d, Wq [C][HC], Wo [HC][C], Wb [C][C]
    float* sg = sw;
    float* swd = sw + C;
    float* swq = sw + 2 * C + 4;
    float* swo = swq + C * HC;
    float* swb = swo + HC * C;
    for (int i = threadIdx.x; i < C; i += blockDim.x) {
        sg[i] = a.g[i];
        swd[i] = a.w_d[i];
    }
    if (threadIdx.x == 0) sw[2 * C] = a.b_d;
    for (int i = threadIdx.x; i < C * HC; i += blockDim.x) {
        swq[i] = a.Wq[i];
        swo[i] = a.Wo[i];
    }
    for (int i = threadIdx.x; i < C * C; i += blockDim.x) swb[i] = a.Wb[i];
    __syncthreads();
    const size_t plane = (size_t)a.H * a.W;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)a.L * plane) return;
    const int li = (int)(e / plane);
    const int y = (int)((e % plane) / a.W), x = (int)(e % a.W);
    const int L = a.L, V = a.V;

    float vin[C], xn[C];
    for (int c = 0; c < C; ++c) vin[c] = a.v0 ? a.v0[c] : a.v_in[e * C + c];
    float t = sw[2 * C];
    float ms = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        t = fmaf(vin[c], swd[c], t);
        ms = fmaf(vin[c], vin[c], ms);
    }
    const float r = 1.0f / sqrtf(ms / C + 1e-6f);
#pragma unroll
    for (int c = 0; c < C; ++c) xn[c] = sg[c] * vin[c] * r;
    // the initialisation samples at the depth anchors, which no weight moves
    const float d = a.v0 ? depth_anchor(li, L, a.dp) : depth_from_logit(t, li, L, a.dp);
    const float scale = 1.0f / sqrtf((float)C);

    float q[NH][C], qb[C];
#pragma unroll
    for (int h = 0; h < NH; ++h)
#pragma unroll
        for (int c = 0; c < C; ++c) q[h][c] = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) qb[c] = 0.f;
    for (int k = 0; k < C; ++k) {
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
            for (int c = 0; c < C; ++c) q[h][c] = fmaf(xn[k], swq[k * HC + h * C + c], q[h][c]);
        if (a.last)
#pragma unroll
            for (int c = 0; c < C; ++c) qb[c] = fmaf(xn[k], swb[k * C + c], qb[c]);
    }

    const float px = x + 0.5f, py = y + 0.5f;
    const size_t vstride = (size_t)a.fh * a.fw * C;
    // sample view m: Delta and its derivative along the depth direction
    auto sample = [&](int m, float (&D)[C], float (&Dd)[C], Taps& tp, bool& ok) {
#pragma unroll
        for (int c = 0; c < C; ++c) D[c] = Dd[c] = 0.f;
        float u, v, du, dv;
        ok = reproject_grad(a.geo.v[m], px, py, d, u, v, du, dv) && bilinear_taps(u, v, a.fh, a.fw, tp);
        if (!ok) return;
        const float* fb = a.feat + m * vstride;
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            const int yy = tp.y0 + (ab >> 1), xx = tp.x0 + (ab & 1);
            if (yy < 0 || yy >= a.fh || xx < 0 || xx >= a.fw) continue;
            const float wy = (ab >> 1) ? tp.fy : 1.f - tp.fy, wx = (ab & 1) ? tp.fx : 1.f - tp.fx;
            const float dwx = (ab & 1) ? 1.f : -1.f, dwy = (ab >> 1) ? 1.f : -1.f;
            const float wd = wy * dwx * du + dwy * wx * dv;  // d(weight)/dd
            const float* src = fb + ((size_t)yy * a.fw + xx) * C;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                D[c] = fmaf(wy * wx, src[c], D[c]);
                Dd[c] = fmaf(wd, src[c], Dd[c]);
            }
        }
    };

    // pass 1: softmax normalisers and head outputs
    float mx[NH], lsum[NH], o[NH][C];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        mx[h] = -INFINITY;
        lsum[h] = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) o[h][c] = 0.f;
    }
    for (int m = 0; m < V; ++m) {
        float D[C], Dd[C];
        Taps tp;
        bool ok;
        sample(m, D, Dd, tp, ok);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) s = fmaf(q[h][c], D[c], s);
            s *= scale;
            const float mn = fmaxf(mx[h], s);
            const float cs = expf(mx[h] - mn), p = expf(s - mn);
            lsum[h] = fmaf(lsum[h], cs, p);
#pragma unroll
            for (int c = 0; c < C; ++c) o[h][c] = fmaf(o[h][c], cs, p * D[c]);
            mx[h] = mn;
        }
    }
#pragma unroll
    for (int h = 0; h < NH; ++h)
#pragma unroll
        for (int c = 0; c < C; ++c) o[h][c] /= lsum[h];

    // do_h = dV_attn Wo_h^T
    float dov[NH][C];
    {
        float dva[C];
        for (int c = 0; c < C; ++c) dva[c] = a.dv_attn[e * C + c];
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < C; ++k) s = fmaf(dva[k], swo[(h * C + c) * C + k], s);
                dov[h][c] = s;
            }
    }
    // pass 2: S_h = sum_m p_hm dp_hm, dp_hm = do_h . Delta_m
    float S[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) S[h] = 0.f;
    for (int m = 0; m < V; ++m) {
        float D[C], Dd[C];
        Taps tp;
        bool ok;
        sample(m, D, Dd, tp, ok);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            float s = 0.f, dp = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                s = fmaf(q[h][c], D[c], s);
                dp = fmaf(dov[h][c], D[c], dp);
            }
            S[h] = fmaf(expf(s * scale - mx[h]) / lsum[h], dp, S[h]);
        }
    }
    // pass 3: score gradients, query gradients, feature scatter, coordinate gradient
    float dq[NH][C], dqb[C];
#pragma unroll
    for (int h = 0; h < NH; ++h)
#pragma unroll
        for (int c = 0; c < C; ++c) dq[h][c] = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) dqb[c] = 0.f;
    float dd = 0.f;
    const size_t pix = (size_t)y * a.W + x;
    for (int m = 0; m < V; ++m) {
        float D[C], Dd[C];
        Taps tp;
        bool ok;
        sample(m, D, Dd, tp, ok);
        float dD[C];
        const float db = a.last ? a.dbeta[(pix * L + li) * V + m] * scale : 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            dD[c] = db * qb[c];
            dqb[c] = fmaf(db, D[c], dqb[c]);
        }
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            float s = 0.f, dp = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                s = fmaf(q[h][c], D[c], s);
                dp = fmaf(dov[h][c], D[c], dp);
            }
            const float p = expf(s * scale - mx[h]) / lsum[h];
            const float ds = p * (dp - S[h]) * scale;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                dD[c] = fmaf(p, dov[h][c], fmaf(ds, q[h][c], dD[c]));
                dq[h][c] = fmaf(ds, D[c], dq[h][c]);
            }
        }
        if (!ok) continue;
        float g = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) g = fmaf(dD[c], Dd[c], g);
        dd += g;
        float* fb = a.dfeat + m * vstride;
#pragma unroll
        for (int ab = 0; ab < 4; ++ab) {
            const int yy = tp.y0 + (ab >> 1), xx = tp.x0 + (ab & 1);
            if (yy < 0 || yy >= a.fh || xx < 0 || xx >= a.fw) continue;
            const float wt = ((ab >> 1) ? tp.fy : 1.f - tp.fy) * ((ab & 1) ? tp.fx : 1.f - tp.fx);
            float* dst = fb + ((size_t)yy * a.fw + xx) * C;
#pragma unroll
            for (int c = 0; c < C; ++c) atomicAdd(dst + c, wt * dD[c]);
        }
    }
    // dx = sum_h dq_h Wq_h^T + dqb Wb^T; rmsnorm adjoint; depth adjoint
    float dx[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
        float s = 0.f;
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
            for (int c = 0; c < C; ++c) s = fmaf(dq[h][c], swq[k * HC + h * C + c], s);
        if (a.last)
#pragma unroll
            for (int c = 0; c < C; ++c) s = fmaf(dqb[c], swb[k * C + c], s);
        dx[k] = s;
    }
    const float dt = a.v0 ? 0.f : dd * ddepth_dt(t, d, L, a.dp);
    float dot = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) dot = fmaf(sg[c] * dx[c], vin[c], dot);
    const float kk = r * r * r * dot / C;
    for (int c = 0; c < C; ++c) {
        a.dv_in[e * C + c] = a.dv_attn[e * C + c] + r * sg[c] * dx[c] - kk * vin[c] + dt * swd[c];
        a.x_out[e * C + c] = xn[c];
        a.dgterm[e * C + c] = dx[c] * vin[c] * r;
        a.dqb_out[e * C + c] = dqb[c];
    }
#pragma unroll
    for (int h = 0; h < NH; ++h)
        for (int c = 0; c < C; ++c) {
            a.dq_out[e * HC + h * C + c] = dq[h][c];
            a.o_out[e * HC + h * C + c] = o[h][c];
        }
    a.dt_in[e] = dt;
}

// ---------------------------------------------------------------------------------------------
// Weight-gradient reductions: partial[b][tap][i][j] = sum_{e in block b} X[shift_tap(e)][i] Y[e][j]
// (X[.] = 1 when X is NULL; gelu applied to X when x_gelu), then out = sum_b partial[b].
// ---------------------------------------------------------------------------------------------

constexpr int XTY_THREADS = 256;
constexpr int XTY_MAX_PER_THREAD = 40;

__global__ void __launch_bounds__(XTY_THREADS) xty_kernel(const XtyArgs a) {
    const int n_out = a.taps * a.cx * a.cy;
    const size_t E = (size_t)a.L * a.H * a.W;
    const size_t per = (E + gridDim.x - 1) / gridDim.x;
    const size_t e0 = (size_t)blockIdx.x * per, e1 = min(E, e0 + per);
    float acc[XTY_MAX_PER_THREAD];
#pragma unroll
    for (int i = 0; i < XTY_MAX_PER_THREAD; ++i) acc[i] = 0.f;
    const size_t plane = (size_t)a.H * a.W;
    for (size_t e = e0; e < e1; ++e) {
        const int y = (int)((e % plane) / a.W), x = (int)(e % a.W);
        const size_t lbase = e - (e % plane);
#pragma unroll 4
        for (int i = 0; i < XTY_MAX_PER_THREAD; ++i) {
            const int o = threadIdx.x + i * XTY_THREADS;
            if (o >= n_out) break;
            const int j = o % a.cy, ii = (o / a.cy) % a.cx, tap = o / (a.cy * a.cx);
            float xv = 1.f;
            if (a.X) {
                int yy = y, xx = x;
                if (a.taps == 9) {
                    yy += tap / 3 - 1;
                    xx += tap % 3 - 1;
                    if (yy < 0 || yy >= a.H || xx < 0 || xx >= a.W) continue;
                }
                xv = a.X[(lbase + (size_t)yy * a.W + xx) * a.ldx + ii];
                if (a.x_gelu) xv = gelu_erf(xv);
            }
            acc[i] = fmaf(xv, a.Y[e * a.ldy + j], acc[i]);
        }
    }
    for (int i = 0; i < XTY_MAX_PER_THREAD; ++i) {
        const int o = threadIdx.x + i * XTY_THREADS;
        if (o >= n_out) break;
        a.partial[(size_t)blockIdx.x * n_out + o] = acc[i];
    }
}

__global__ void reduce_partials_kernel(const float* __restrict__ partial, int nb, int n_out, float* out, int accumulate) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += partial[(size_t)b * n_out + o];
    out[o] = accumulate ? out[o] + s : s;
}

// x2 bilinear upsample (edge clamp, pixel centres aligned) of [L][Hp][Wp][C] to [L][2Hp][2Wp][C]:
// the transition of a step whose pyramid factor halves, materialised for the differentiable stage.
__global__ void upsample2_kernel(const float* __restrict__ in, float* out, int L, int Hp, int Wp, int C) {
    const size_t H = 2 * (size_t)Hp, W = 2 * (size_t)Wp;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)L * H * W * C) return;
    const int c = (int)(i % C);
    const size_t e = i / C;
    const int x = (int)(e % W), y = (int)((e / W) % H), li = (int)(e / (W * H));
    int y0, y1, x0, x1;
    float wy, wx;
    resize_taps(y, 2, Hp, y0, y1, wy);
    resize_taps(x, 2, Wp, x0, x1, wx);
    const float* b = in + (size_t)li * Hp * Wp * C + c;
    const float top = b[((size_t)y0 * Wp + x0) * C] + wx * (b[((size_t)y0 * Wp + x1) * C] - b[((size_t)y0 * Wp + x0) * C]);
    const float bot = b[((size_t)y1 * Wp + x0) * C] + wx * (b[((size_t)y1 * Wp + x1) * C] - b[((size_t)y1 * Wp + x0) * C]);
    out[i] = top + wy * (bot - top);
}

cudaError_t launch_upsample2(const float* in, float* out, int L, int Hp, int Wp, int C, cudaStream_t st) {
    const size_t n = (size_t)L * 4 * Hp * Wp * C;
    upsample2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, L, Hp, Wp, C);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------------

static unsigned blocks(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_render_bwd(const RenderArgs& a, const float* dl, float* dt_raw, float* ds_raw, float* dbeta_raw,
                              cudaStream_t st) {
    if (a.L > L_MAX) return cudaErrorInvalidValue;
    render_bwd_kernel<<<blocks((size_t)a.Hout * a.Wout, BW_THREADS), BW_THREADS, 0, st>>>(a, dl, dt_raw, ds_raw,
                                                                                            dbeta_raw);
    return cudaGetLastError();
}

cudaError_t launch_decode_bwd(const float* dt_raw, const float* ds_raw, int L, int H, int W, int C, const float* w_d,
                              const float* w_s, float* dv_out, float* dts, cudaStream_t st) {
    decode_bwd_kernel<<<blocks((size_t)L * H * W, 256), 256, 0, st>>>(dt_raw, ds_raw, L, H, W, C, w_d, w_s, dv_out, dts);
    return cudaGetLastError();
}

cudaError_t launch_conv3x3(const float* in, const float* w, const float* bias, float* out, int L, int H, int W, int C,
                           int transpose, const float* gelu_aux, cudaStream_t st) {
    const unsigned g = blocks((size_t)L * H * W, BW_THREADS);
    if (C == 16) conv3x3_kernel<16><<<g, BW_THREADS, 0, st>>>(in, w, bias, out, L, H, W, transpose, gelu_aux);
    else if (C == 32) conv3x3_kernel<32><<<g, BW_THREADS, 0, st>>>(in, w, bias, out, L, H, W, transpose, gelu_aux);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_rmsnorm(const float* v, const float* g, float* n, size_t E, int C, cudaStream_t st) {
    if (C == 16) rmsnorm_kernel<16><<<blocks(E, 256), 256, 0, st>>>(v, g, n, E);
    else if (C == 32) rmsnorm_kernel<32><<<blocks(E, 256), 256, 0, st>>>(v, g, n, E);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_rmsnorm_bwd(const float* v, const float* g, const float* dn, const float* resid, float* dv,
                               float* dgterm, size_t E, int C, cudaStream_t st) {
    if (C == 16) rmsnorm_bwd_kernel<16><<<blocks(E, 256), 256, 0, st>>>(v, g, dn, resid, dv, dgterm, E);
    else if (C == 32) rmsnorm_bwd_kernel<32><<<blocks(E, 256), 256, 0, st>>>(v, g, dn, resid, dv, dgterm, E);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <int C, int NH>
static cudaError_t launch_ab(const AttendBwdArgs& a, cudaStream_t st) {
    const size_t smem = (size_t)(2 * C + 4 + 2 * C * NH * C + C * C) * sizeof(float);
    auto k = attend_bwd_kernel<C, NH>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<blocks((size_t)a.L * a.H * a.W, BW_THREADS), BW_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_attend_bwd(const AttendBwdArgs& a, int C, int heads, cudaStream_t st) {
    if (C == 16 && heads == 1) return launch_ab<16, 1>(a, st);
    if (C == 16 && heads == 2) return launch_ab<16, 2>(a, st);
    if (C == 16 && heads == 4) return launch_ab<16, 4>(a, st);
    if (C == 32 && heads == 1) return launch_ab<32, 1>(a, st);
    if (C == 32 && heads == 2) return launch_ab<32, 2>(a, st);
    if (C == 32 && heads == 4) return launch_ab<32, 4>(a, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_xty(const XtyArgs& a, float* out, int accumulate, cudaStream_t st) {
    const int n_out = a.taps * a.cx * a.cy;
    if (n_out > XTY_THREADS * XTY_MAX_PER_THREAD) return cudaErrorInvalidValue;
    const int nb = a.n_blocks;
    xty_kernel<<<nb, XTY_THREADS, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_partials_kernel<<<blocks(n_out, 256), 256, 0, st>>>(a.partial, nb, n_out, out, accumulate);
    return cudaGetLastError();
}

}  // namespace quark
