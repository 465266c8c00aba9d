// Differentiation form: the last Update & Fuse step and the render as a differentiable stage
// (quark_step_input, quark_stage_forward, quark_stage_backward).  FP32 form only.
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "bwd_internal.cuh"

using namespace quark;

#define QK_CU(ctx, call)                                                                          \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return qk_fail(ctx, QUARK_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static quark_status check_stage(quark_ctx* ctx, const quark_pyramid* pyr, const quark_ldm* ldm) {
    if (!ctx || !pyr || !ldm) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (ctx->cfg.precision != QUARK_FP32) return qk_fail(ctx, QUARK_EINVAL, "the differentiable stage is FP32 only");
    if (ctx->cfg.attn_mode != QUARK_ATTN_ONE_TO_MANY)
        return qk_fail(ctx, QUARK_EINVAL, "the differentiable stage covers one-to-many attention");
    if (ctx->cfg.ray_encoding) return qk_fail(ctx, QUARK_EINVAL, "the differentiable stage runs without the ray encoding");
    if (!qk_uniform(ctx->cfg)) return qk_fail(ctx, QUARK_EINVAL, "the differentiable stage takes the uniform schedule only");
    if (ctx->cfg.render_refine) return qk_fail(ctx, QUARK_EINVAL, "the differentiable stage runs without render-and-refine");
    if (pyr->ctx != ctx || ldm->ctx != ctx) return qk_fail(ctx, QUARK_EINVAL, "handle from another context");
    if (!ctx->weights_loaded) return qk_fail(ctx, QUARK_EINVAL, "weights not loaded");
    return QUARK_OK;
}

extern "C" quark_status quark_step_input(quark_ctx* ctx, quark_ldm* ldm, int scale, float* v_in, void* stream) {
    if (!ctx || !ldm || !v_in) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    const quark_config& c = ctx->cfg;
    if (c.precision != QUARK_FP32) return qk_fail(ctx, QUARK_EINVAL, "FP32 form only");
    if (c.attn_mode != QUARK_ATTN_ONE_TO_MANY) return qk_fail(ctx, QUARK_EINVAL, "one-to-many attention only");
    if (c.ray_encoding) return qk_fail(ctx, QUARK_EINVAL, "no ray encoding in the differentiable stage");
    if (!qk_uniform(c) || c.render_refine)
        return qk_fail(ctx, QUARK_EINVAL, "the differentiable stage takes the uniform schedule without render-and-refine");
    if (scale < 1 || scale >= c.n_scales || ldm->done != scale - 1)
        return qk_fail(ctx, QUARK_EINVAL, "step %d's input needs step %d done (latest: %d)", scale, scale - 1, ldm->done);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int kp = c.k[scale - 1], Lp = c.L[scale - 1], L = c.L[scale], k = c.k[scale];
    const int Hp = ldm->target.height / kp, Wp = ldm->target.width / kp;
    const float* src = (const float*)ldm->vol[ldm->cur];
    if (Lp == 2 * L) {
        CollapseArgs ca{};
        ca.in = src;
        ca.out = ldm->collapsed;
        ca.L = L;
        ca.H = Hp;
        ca.W = Wp;
        ca.w = ctx->wdev + ctx->off_collapse[scale];
        quark_status s = qk_launch(ctx, st, KF_COLLAPSE, [&] { return launch_collapse(ca, c.C, false, st); });
        if (s != QUARK_OK) return s;
        src = (const float*)ldm->collapsed;
    }
    const size_t bytes = (size_t)L * (ldm->target.height / k) * (ldm->target.width / k) * c.C * sizeof(float);
    if (kp == 2 * k)
        return qk_launch(ctx, st, KF_BACKWARD, [&] { return launch_upsample2(src, v_in, L, Hp, Wp, c.C, st); });
    QK_CU(ctx, cudaMemcpyAsync(v_in, src, bytes, cudaMemcpyDeviceToDevice, st));
    return QUARK_OK;
}

extern "C" quark_status quark_stage_forward(quark_ctx* ctx, const quark_pyramid* pyr, const float* feat,
                                            const float* v_in, quark_ldm* ldm, float* rgba, void* stream) {
    quark_status s = check_stage(ctx, pyr, ldm);
    if (s != QUARK_OK) return s;
    if (!feat || !v_in || !rgba) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (reinterpret_cast<uintptr_t>(feat) % 32) return qk_fail(ctx, QUARK_EINVAL, "feat must be 32-byte aligned");
    const int last = ctx->cfg.n_scales - 1;
    s = qk_update_fuse(ctx, pyr, pyr->V, last, ldm, (cudaStream_t)stream, v_in, feat);
    if (s != QUARK_OK) return s;
    return qk_render(ctx, ldm, pyr, pyr->V, rgba, 0, (cudaStream_t)stream);
}

extern "C" quark_status quark_stage_backward(quark_ctx* ctx, const quark_pyramid* pyr, const float* feat,
                                             const float* v_in, quark_ldm* ldm, const float* dl_drgb, float* dv_in,
                                             float* dfeat, const quark_stage_grads* g, void* stream) {
    quark_status s = check_stage(ctx, pyr, ldm);
    if (s != QUARK_OK) return s;
    if (!feat || !v_in || !dl_drgb || !dv_in || !dfeat || !g) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    const quark_config& c = ctx->cfg;
    const int n = c.n_scales - 1;
    if (ldm->done != n) return qk_fail(ctx, QUARK_EINVAL, "run quark_stage_forward first");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int C = c.C, h = c.heads, L = c.L[n], k = c.k[n], V = pyr->V;
    const int H = ldm->target.height / k, W = ldm->target.width / k;
    const size_t E = (size_t)L * H * W;
    const int HC = h * C;
    const int NB = 296;

    // workspace: dt, ds, dbeta (LDM grid), G, N, H1, dH1, dN, dVattn, dgterm, X, dQ, O, dQb, dt_in, dts, partials
    const size_t f_dt = E, f_dbeta = E * V, f_EC = E * C, f_EHC = E * HC, f_part = (size_t)NB * 9 * C * C;
    const size_t parts[] = {f_dt, f_dt, f_dbeta, f_EC, f_EC, f_EC, f_EC, f_EC, f_EC, f_EC, f_EC,
                            f_EHC, f_EHC, f_EC, E, 2 * E, f_part};
    size_t floats = 0;
    for (size_t nf : parts) floats += (nf + 31) & ~(size_t)31;  // each part starts 128-byte aligned
    if (ctx->bwd_ws_bytes < floats * sizeof(float)) {
        qk_free(ctx, ctx->bwd_ws, ctx->bwd_ws_bytes);
        ctx->bwd_ws = nullptr;
        ctx->bwd_ws_bytes = 0;
        s = qk_alloc(ctx, &ctx->bwd_ws, floats * sizeof(float));
        if (s != QUARK_OK) return s;
        ctx->bwd_ws_bytes = floats * sizeof(float);
    }
    float* p = (float*)ctx->bwd_ws;
    auto take = [&](size_t nf) {
        float* r = p;
        p += (nf + 31) & ~(size_t)31;
        return r;
    };
    float* dt_raw = take(f_dt);
    float* ds_raw = take(f_dt);
    float* dbeta = take(f_dbeta);
    float* G = take(f_EC);
    float* Nn = take(f_EC);
    float* H1 = take(f_EC);
    float* dH1 = take(f_EC);
    float* dN = take(f_EC);
    float* dVa = take(f_EC);
    float* dgt = take(f_EC);
    float* Xn = take(f_EC);
    float* dQ = take(f_EHC);
    float* Oo = take(f_EHC);
    float* dQb = take(f_EC);
    float* dt_in = take(E);
    float* dts = take(2 * E);
    float* part = take(f_part);

    const ConvLayout cl{C};
    const AttendLayout al{C, h};
    const float* wc = ctx->wdev + ctx->off_conv[n];
    const float* wa = ctx->wdev + ctx->off_attend[n];
    DepthParams dp{(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
    const float* V_attn = (const float*)ldm->vattn;
    const float* V_out = (const float*)ldm->vol[ldm->cur];

    QK_CU(ctx, cudaMemsetAsync(dt_raw, 0, 2 * ((f_dt + 31) & ~(size_t)31) * sizeof(float) + f_dbeta * sizeof(float), st));
    QK_CU(ctx, cudaMemsetAsync(dfeat, 0, (size_t)V * (pyr->H / k) * (pyr->W / k) * C * sizeof(float), st));

    // render adjoint
    RenderArgs ra{};
    ra.t_raw = ldm->t_raw;
    ra.s_raw = ldm->s_raw;
    ra.beta = ldm->beta;
    ra.rgba = (const float4*)pyr->rgba;
    ra.L = L;
    ra.V = V;
    ra.Hl = H;
    ra.Wl = W;
    ra.sx = ra.sy = (float)k;
    ra.Hout = ldm->target.height;
    ra.Wout = ldm->target.width;
    ra.Hi = pyr->H;
    ra.Wi = pyr->W;
    ra.dp = dp;
    for (int m = 0; m < V; ++m) ra.geo.v[m] = qk_view_map(ldm->target, 1.0, 1.0, pyr->cams[m], 1.0);
    auto L_ = [&](auto fn) { return qk_launch(ctx, st, KF_BACKWARD, fn); };
    if ((s = L_([&] { return launch_render_bwd(ra, dl_drgb, dt_raw, ds_raw, dbeta, st); })) != QUARK_OK) return s;
    // decode adjoint -> G = dL/dV_out
    if ((s = L_([&] { return launch_decode_bwd(dt_raw, ds_raw, L, H, W, C, wc + cl.wd(), wc + cl.ws(), G, dts, st); })) != QUARK_OK)
        return s;
    // conv block adjoint (forward intermediates recomputed)
    if ((s = L_([&] { return launch_rmsnorm(V_attn, wc + cl.g(), Nn, E, C, st); })) != QUARK_OK) return s;
    if ((s = L_([&] { return launch_conv3x3(Nn, wc + cl.w1(), wc + cl.b1(), H1, L, H, W, C, 0, nullptr, st); })) != QUARK_OK)
        return s;
    if ((s = L_([&] { return launch_conv3x3(G, wc + cl.w2(), nullptr, dH1, L, H, W, C, 1, H1, st); })) != QUARK_OK)
        return s;
    if ((s = L_([&] { return launch_conv3x3(dH1, wc + cl.w1(), nullptr, dN, L, H, W, C, 1, nullptr, st); })) != QUARK_OK)
        return s;
    if ((s = L_([&] { return launch_rmsnorm_bwd(V_attn, wc + cl.g(), dN, G, dVa, dgt, E, C, st); })) != QUARK_OK)
        return s;

    auto xty = [&](const float* X, int ldx, const float* Y, int ldy, int cx, int cy, int taps, int x_gelu, float* out,
                   int acc) {
        XtyArgs xa{};
        xa.X = X;
        xa.ldx = ldx;
        xa.Y = Y;
        xa.ldy = ldy;
        xa.L = L;
        xa.H = H;
        xa.W = W;
        xa.cx = cx;
        xa.cy = cy;
        xa.taps = taps;
        xa.x_gelu = x_gelu;
        xa.partial = part;
        xa.n_blocks = NB;
        return L_([&] { return launch_xty(xa, out, acc, st); });
    };
    // conv block and decoder weight gradients
    if ((s = xty(H1, C, G, C, C, C, 9, 1, g->conv2_w, 0)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, G, C, 1, C, 1, 0, g->conv2_b, 0)) != QUARK_OK) return s;
    if ((s = xty(Nn, C, dH1, C, C, C, 9, 0, g->conv1_w, 0)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dH1, C, 1, C, 1, 0, g->conv1_b, 0)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dgt, C, 1, C, 1, 0, g->conv_g, 0)) != QUARK_OK) return s;
    if ((s = xty(V_out, C, dts, 2, C, 1, 1, 0, g->w_d, 0)) != QUARK_OK) return s;
    if ((s = xty(V_out, C, dts + 1, 2, C, 1, 1, 0, g->w_sigma, 0)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dts, 2, 1, 1, 1, 0, g->b_d, 0)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dts + 1, 2, 1, 1, 1, 0, g->b_sigma, 0)) != QUARK_OK) return s;

    // attention-with-sampling adjoint
    AttendBwdArgs ab{};
    ab.v_in = v_in;
    ab.feat = feat;
    ab.dv_attn = dVa;
    ab.dbeta = dbeta;
    ab.L = L;
    ab.H = H;
    ab.W = W;
    ab.V = V;
    ab.fh = pyr->H / k;
    ab.fw = pyr->W / k;
    ab.last = 1;
    ab.dp = dp;
    ab.g = wa + al.g();
    ab.w_d = wa + al.wd();
    std::vector<float> bd(1);
    QK_CU(ctx, cudaMemcpy(bd.data(), wa + al.bd(), sizeof(float), cudaMemcpyDeviceToHost));
    ab.b_d = bd[0];
    ab.Wq = wa + al.wq();
    ab.Wo = wa + al.wo();
    ab.Wb = wa + al.wb();
    for (int m = 0; m < V; ++m) ab.geo.v[m] = qk_view_map(ldm->target, k, k, pyr->cams[m], k);
    ab.dv_in = dv_in;
    ab.dfeat = dfeat;
    ab.x_out = Xn;
    ab.dq_out = dQ;
    ab.o_out = Oo;
    ab.dqb_out = dQb;
    ab.dgterm = dgt;
    ab.dt_in = dt_in;
    if ((s = L_([&] { return launch_attend_bwd(ab, C, h, st); })) != QUARK_OK) return s;
    if ((s = xty(Xn, C, dQ, HC, C, HC, 1, 0, g->Wq, 0)) != QUARK_OK) return s;
    if ((s = xty(Oo, HC, dVa, C, HC, C, 1, 0, g->Wo, 0)) != QUARK_OK) return s;
    if ((s = xty(Xn, C, dQb, C, C, C, 1, 0, g->W_beta, 0)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dgt, C, 1, C, 1, 0, g->attn_g, 0)) != QUARK_OK) return s;
    if ((s = xty(v_in, C, dt_in, 1, C, 1, 1, 0, g->w_d, 1)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dt_in, 1, 1, 1, 1, 0, g->b_d, 1)) != QUARK_OK) return s;
    return QUARK_OK;
}
