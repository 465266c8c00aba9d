// Differentiation form (FP32 form only):
//   - the last Update & Fuse step and the render as a differentiable stage (quark_step_input,
//     quark_stage_forward, quark_stage_backward);
//   - the backward pass through the whole network, one call per forward call
//     (quark_render_ldm_bwd, quark_update_fuse_bwd, quark_encode_pyramid_bwd), on an LDM that
//     kept every step's volumes (quark_ldm_keep_steps).
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
    if (ctx->cfg.C > 32) return qk_fail(ctx, QUARK_EINVAL, "the backward pass covers C = 16, 32");
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
    // 1x1 fusion-block convolutions sit at the centre tap of the 3x3 layout (exact in the 3x3
    // adjoints); their weight gradient is the unshifted product
    const int ctaps = c.conv_kernel == 1 ? 1 : 9;
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
    if ((s = xty(H1, C, G, C, C, C, ctaps, 1, g->conv2_w, 0)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, G, C, 1, C, 1, 0, g->conv2_b, 0)) != QUARK_OK) return s;
    if ((s = xty(Nn, C, dH1, C, C, C, ctaps, 0, g->conv1_w, 0)) != QUARK_OK) return s;
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

// ---------------------------------------------------------------------------------------------
// Backward pass through the whole network
// ---------------------------------------------------------------------------------------------

extern "C" quark_status quark_ldm_keep_steps(quark_ldm* ldm, int keep) {
    if (!ldm) return qk_fail(nullptr, QUARK_EINVAL, "NULL LDM");
    ldm->keep = keep != 0;
    return QUARK_OK;
}

static quark_status check_network(quark_ctx* ctx, const quark_pyramid* pyr, const quark_ldm* ldm) {
    quark_status s = check_stage(ctx, pyr, ldm);
    if (s != QUARK_OK) return s;
    if (ctx->cfg.C != 16 && ctx->cfg.C != 32) return qk_fail(ctx, QUARK_EINVAL, "the backward pass covers C = 16, 32");
    return QUARK_OK;
}

// Workspace of the backward calls: floats carved from the context's grown-on-demand buffer, each
// part 128-byte aligned.
namespace {
struct Carve {
    float* p;
    float* take(size_t nf) {
        float* r = p;
        p += (nf + 31) & ~(size_t)31;
        return r;
    }
};
size_t carved(std::initializer_list<size_t> parts) {
    size_t f = 0;
    for (size_t n : parts) f += (n + 31) & ~(size_t)31;
    return f;
}
quark_status grow_ws(quark_ctx* ctx, size_t floats) {
    if (ctx->bwd_ws_bytes >= floats * sizeof(float)) return QUARK_OK;
    qk_free(ctx, ctx->bwd_ws, ctx->bwd_ws_bytes);
    ctx->bwd_ws = nullptr;
    ctx->bwd_ws_bytes = 0;
    quark_status s = qk_alloc(ctx, &ctx->bwd_ws, floats * sizeof(float));
    if (s == QUARK_OK) ctx->bwd_ws_bytes = floats * sizeof(float);
    return s;
}
constexpr int kRedBlocks = 296;  // blocks of the weight-gradient reductions (2 per SM)
}  // namespace

extern "C" quark_status quark_render_ldm_bwd(quark_ctx* ctx, const quark_ldm* ldm, const quark_pyramid* pyr,
                                             const float* dl_drgb, float* dv_out, float* dbeta,
                                             const quark_grads* g, void* stream) {
    quark_status s = check_network(ctx, pyr, ldm);
    if (s != QUARK_OK) return s;
    if (!dl_drgb || !dv_out || !dbeta || !g || !g->w_d || !g->b_d || !g->w_sigma || !g->b_sigma)
        return qk_fail(ctx, QUARK_EINVAL, "NULL argument (dl_drgb, dv_out, dbeta and the decoder gradients are needed)");
    const quark_config& c = ctx->cfg;
    const int n = c.n_scales - 1;
    if (ldm->done != n) return qk_fail(ctx, QUARK_EINVAL, "the render's backward needs every Update & Fuse step done");
    if (ldm->V != pyr->V) return qk_fail(ctx, QUARK_EINVAL, "the LDM's last step used %d views, the pyramid has %d", ldm->V, pyr->V);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int C = c.C, L = c.L[n], k = c.k[n], V = pyr->V;
    const int H = ldm->target.height / k, W = ldm->target.width / k;
    const size_t E = (size_t)L * H * W;
    const size_t part = (size_t)kRedBlocks * 2 * C;
    s = grow_ws(ctx, carved({E, E, 2 * E, part}));
    if (s != QUARK_OK) return s;
    Carve cv{(float*)ctx->bwd_ws};
    float* dt_raw = cv.take(E);
    float* ds_raw = cv.take(E);
    float* dts = cv.take(2 * E);
    float* partial = cv.take(part);
    QK_CU(ctx, cudaMemsetAsync(dt_raw, 0, E * sizeof(float), st));
    QK_CU(ctx, cudaMemsetAsync(ds_raw, 0, E * sizeof(float), st));
    QK_CU(ctx, cudaMemsetAsync(dbeta, 0, E * V * sizeof(float), st));
    const DepthParams dp{(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
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
    const ConvLayout cl{C};
    const float* wc = ctx->wdev + ctx->off_conv[n];
    if ((s = L_([&] { return launch_decode_bwd(dt_raw, ds_raw, L, H, W, C, wc + cl.wd(), wc + cl.ws(), dv_out, dts, st); })) !=
        QUARK_OK)
        return s;
    const float* V_out = (const float*)ldm->vol[ldm->cur];
    auto xty = [&](const float* X, int ldx, const float* Y, int ldy, int cx, float* out) {
        XtyArgs xa{};
        xa.X = X;
        xa.ldx = ldx;
        xa.Y = Y;
        xa.ldy = ldy;
        xa.L = L;
        xa.H = H;
        xa.W = W;
        xa.cx = cx;
        xa.cy = 1;
        xa.taps = 1;
        xa.partial = partial;
        xa.n_blocks = kRedBlocks;
        return L_([&] { return launch_xty(xa, out, 1, st); });
    };
    if ((s = xty(V_out, C, dts, 2, C, g->w_d)) != QUARK_OK) return s;
    if ((s = xty(V_out, C, dts + 1, 2, C, g->w_sigma)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dts, 2, 1, g->b_d)) != QUARK_OK) return s;
    return xty(nullptr, 0, dts + 1, 2, 1, g->b_sigma);
}

extern "C" quark_status quark_update_fuse_bwd(quark_ctx* ctx, const quark_pyramid* pyr, int scale, quark_ldm* ldm,
                                              const float* dv_out, const float* dbeta, float* dv_prev, float* dfeat,
                                              const quark_grads* g, void* stream) {
    quark_status s = check_network(ctx, pyr, ldm);
    if (s != QUARK_OK) return s;
    const quark_config& c = ctx->cfg;
    if (scale < 0 || scale >= c.n_scales) return qk_fail(ctx, QUARK_EINVAL, "scale %d out of range", scale);
    const bool last = scale == c.n_scales - 1;
    if (!dv_out || !dfeat || !g) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (last && !dbeta) return qk_fail(ctx, QUARK_EINVAL, "the last step needs the blend-logit gradient dbeta");
    if (scale > 0 && !dv_prev) return qk_fail(ctx, QUARK_EINVAL, "step %d writes dv_prev: NULL", scale);
    if (!g->attn_g[scale] || !g->Wq[scale] || !g->Wo[scale] || !g->conv_g[scale] || !g->conv1_w[scale] ||
        !g->conv1_b[scale] || !g->conv2_w[scale] || !g->conv2_b[scale] || (last && !g->W_beta) ||
        (scale == 0 && !g->v0) || (scale > 0 && (!g->w_d || !g->b_d)))
        return qk_fail(ctx, QUARK_EINVAL, "a gradient buffer step %d accumulates into is NULL", scale);
    if (!ldm->keep || !ldm->hist_out[scale] || ldm->done < scale || (scale > 0 && !ldm->hist_out[scale - 1]))
        return qk_fail(ctx, QUARK_EINVAL, "step %d's backward needs its forward run on an LDM that keeps its steps "
                       "(quark_ldm_keep_steps)", scale);
    if (last && ldm->V != pyr->V)
        return qk_fail(ctx, QUARK_EINVAL, "the LDM's last step used %d views, the pyramid has %d", ldm->V, pyr->V);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int C = c.C, h = c.heads, L = c.L[scale], k = c.k[scale], V = pyr->V, HC = h * C;
    const int H = ldm->target.height / k, W = ldm->target.width / k;
    const size_t E = (size_t)L * H * W;
    int Lp = 0, Hp = 0, Wp = 0;
    bool collapse = false, up = false;
    if (scale > 0) {
        Lp = c.L[scale - 1];
        Hp = ldm->target.height / c.k[scale - 1];
        Wp = ldm->target.width / c.k[scale - 1];
        collapse = Lp == 2 * L;
        up = Hp != H;
    }
    const size_t Ec = (size_t)L * Hp * Wp;  // the collapsed (or carried) volume, before the upsample
    const size_t part = (size_t)kRedBlocks * 9 * C * C;
    s = grow_ws(ctx, carved({E * C, E * C, E * C, E * C, E * C, E * C, E * C, E * C, E * C, E * HC, E * HC, E,
                             E * C, Ec * C, Ec * C, Ec * C, Ec * C, 2 * Ec * C, part}));
    if (s != QUARK_OK) return s;
    Carve cv{(float*)ctx->bwd_ws};
    float* Vin = cv.take(E * C);
    float* Nn = cv.take(E * C);
    float* H1 = cv.take(E * C);
    float* dH1 = cv.take(E * C);
    float* dN = cv.take(E * C);
    float* dVa = cv.take(E * C);
    float* dgt = cv.take(E * C);
    float* Xn = cv.take(E * C);
    float* dQb = cv.take(E * C);
    float* dQ = cv.take(E * HC);
    float* Oo = cv.take(E * HC);
    float* dt_in = cv.take(E);
    float* dVin = cv.take(E * C);
    float* col = cv.take(Ec * C);    // forward: the collapsed volume
    float* dcol = cv.take(Ec * C);   // its gradient (the upsample's adjoint)
    float* colG = cv.take(Ec * C);   // collapse MLP: gelu output, pre-activation gradient, input
    float* colDH = cv.take(Ec * C);
    float* colCat = cv.take(2 * Ec * C);
    float* partial = cv.take(part);

    auto L_ = [&](auto fn) { return qk_launch(ctx, st, KF_BACKWARD, fn); };
    const DepthParams dp{(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
    const float* vprev = scale > 0 ? (const float*)ldm->hist_out[scale - 1] : nullptr;

    // ---- the volume entering the step, recomputed: layer collapse, then x2 upsample ----
    if (scale > 0) {
        const float* src = vprev;
        if (collapse) {
            CollapseArgs ca{};
            ca.in = vprev;
            ca.out = col;
            ca.L = L;
            ca.H = Hp;
            ca.W = Wp;
            ca.w = ctx->wdev + ctx->off_collapse[scale];
            if ((s = qk_launch(ctx, st, KF_COLLAPSE, [&] { return launch_collapse(ca, C, false, st); })) != QUARK_OK)
                return s;
            src = col;
        }
        if (up) {
            if ((s = L_([&] { return launch_upsample2(src, Vin, L, Hp, Wp, C, st); })) != QUARK_OK) return s;
        } else {
            QK_CU(ctx, cudaMemcpyAsync(Vin, src, E * C * sizeof(float), cudaMemcpyDeviceToDevice, st));
        }
    }

    const ConvLayout cl{C};
    const AttendLayout al{C, h};
    // 1x1 fusion-block convolutions sit at the centre tap of the 3x3 layout (exact in the 3x3
    // adjoints); their weight gradient is the unshifted product
    const int ctaps = c.conv_kernel == 1 ? 1 : 9;
    const float* wc = ctx->wdev + ctx->off_conv[scale];
    const float* wa = ctx->wdev + ctx->off_attend[scale];
    const float* V_attn = (const float*)ldm->hist_attn[scale];

    auto xty = [&](const float* X, int ldx, const float* Y, int ldy, int cx, int cy, int taps, int x_gelu, int l,
                   int hh, int ww, float* out) {
        XtyArgs xa{};
        xa.X = X;
        xa.ldx = ldx;
        xa.Y = Y;
        xa.ldy = ldy;
        xa.L = l;
        xa.H = hh;
        xa.W = ww;
        xa.cx = cx;
        xa.cy = cy;
        xa.taps = taps;
        xa.x_gelu = x_gelu;
        xa.partial = partial;
        xa.n_blocks = kRedBlocks;
        return L_([&] { return launch_xty(xa, out, 1, st); });
    };

    // ---- conv block adjoint (forward intermediates recomputed from V_attn) ----
    if ((s = L_([&] { return launch_rmsnorm(V_attn, wc + cl.g(), Nn, E, C, st); })) != QUARK_OK) return s;
    if ((s = L_([&] { return launch_conv3x3(Nn, wc + cl.w1(), wc + cl.b1(), H1, L, H, W, C, 0, nullptr, st); })) != QUARK_OK)
        return s;
    if ((s = L_([&] { return launch_conv3x3(dv_out, wc + cl.w2(), nullptr, dH1, L, H, W, C, 1, H1, st); })) != QUARK_OK)
        return s;
    if ((s = L_([&] { return launch_conv3x3(dH1, wc + cl.w1(), nullptr, dN, L, H, W, C, 1, nullptr, st); })) != QUARK_OK)
        return s;
    if ((s = L_([&] { return launch_rmsnorm_bwd(V_attn, wc + cl.g(), dN, dv_out, dVa, dgt, E, C, st); })) != QUARK_OK)
        return s;
    if ((s = xty(H1, C, dv_out, C, C, C, ctaps, 1, L, H, W, g->conv2_w[scale])) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dv_out, C, 1, C, 1, 0, L, H, W, g->conv2_b[scale])) != QUARK_OK) return s;
    if ((s = xty(Nn, C, dH1, C, C, C, ctaps, 0, L, H, W, g->conv1_w[scale])) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dH1, C, 1, C, 1, 0, L, H, W, g->conv1_b[scale])) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dgt, C, 1, C, 1, 0, L, H, W, g->conv_g[scale])) != QUARK_OK) return s;

    // ---- attention-with-sampling adjoint ----
    AttendBwdArgs ab{};
    ab.v_in = Vin;
    ab.v0 = scale == 0 ? wa + al.v0() : nullptr;
    ab.feat = (const float*)pyr->level[k == 1 ? 0 : k == 2 ? 1 : k == 4 ? 2 : 3];
    ab.dv_attn = dVa;
    ab.dbeta = last ? dbeta : nullptr;
    ab.L = L;
    ab.H = H;
    ab.W = W;
    ab.V = V;
    ab.fh = pyr->H / k;
    ab.fw = pyr->W / k;
    ab.last = last ? 1 : 0;
    ab.dp = dp;
    ab.g = wa + al.g();
    ab.w_d = wa + al.wd();
    float bd = 0.f;
    QK_CU(ctx, cudaMemcpy(&bd, wa + al.bd(), sizeof(float), cudaMemcpyDeviceToHost));
    ab.b_d = bd;
    ab.Wq = wa + al.wq();
    ab.Wo = wa + al.wo();
    ab.Wb = wa + al.wb();
    for (int m = 0; m < V; ++m) ab.geo.v[m] = qk_view_map(ldm->target, k, k, pyr->cams[m], k);
    ab.dv_in = dVin;
    ab.dfeat = dfeat;
    ab.x_out = Xn;
    ab.dq_out = dQ;
    ab.o_out = Oo;
    ab.dqb_out = dQb;
    ab.dgterm = dgt;
    ab.dt_in = dt_in;
    if ((s = L_([&] { return launch_attend_bwd(ab, C, h, st); })) != QUARK_OK) return s;
    if ((s = xty(Xn, C, dQ, HC, C, HC, 1, 0, L, H, W, g->Wq[scale])) != QUARK_OK) return s;
    if ((s = xty(Oo, HC, dVa, C, HC, C, 1, 0, L, H, W, g->Wo[scale])) != QUARK_OK) return s;
    if (last && (s = xty(Xn, C, dQb, C, C, C, 1, 0, L, H, W, g->W_beta)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dgt, C, 1, C, 1, 0, L, H, W, g->attn_g[scale])) != QUARK_OK) return s;

    if (scale == 0)  // every element entered as v0
        return xty(nullptr, 0, dVin, C, 1, C, 1, 0, L, H, W, g->v0);

    // depth decoded from V_in (the sample coordinates' gradient)
    if ((s = xty(Vin, C, dt_in, 1, C, 1, 1, 0, L, H, W, g->w_d)) != QUARK_OK) return s;
    if ((s = xty(nullptr, 0, dt_in, 1, 1, 1, 1, 0, L, H, W, g->b_d)) != QUARK_OK) return s;

    // ---- transition adjoint: x2 upsample, then layer collapse ----
    float* dsrc = dVin;
    if (up) {
        float* dst = collapse ? dcol : dv_prev;
        if ((s = L_([&] { return launch_upsample2_bwd(dVin, dst, L, Hp, Wp, C, st); })) != QUARK_OK) return s;
        dsrc = dst;
    }
    if (collapse) {
        if (!g->col_w1[scale] || !g->col_b1[scale] || !g->col_w2[scale] || !g->col_b2[scale])
            return qk_fail(ctx, QUARK_EINVAL, "step %d collapses layers: its collapse gradient buffers are NULL", scale);
        const float* w = ctx->wdev + ctx->off_collapse[scale];
        if ((s = L_([&] { return launch_collapse_bwd(vprev, dsrc, L, Hp, Wp, C, w, dv_prev, colG, colDH, colCat, st); })) !=
            QUARK_OK)
            return s;
        if ((s = xty(colG, C, dsrc, C, C, C, 1, 0, L, Hp, Wp, g->col_w2[scale])) != QUARK_OK) return s;
        if ((s = xty(nullptr, 0, dsrc, C, 1, C, 1, 0, L, Hp, Wp, g->col_b2[scale])) != QUARK_OK) return s;
        if ((s = xty(colCat, 2 * C, colDH, C, 2 * C, C, 1, 0, L, Hp, Wp, g->col_w1[scale])) != QUARK_OK) return s;
        if ((s = xty(nullptr, 0, colDH, C, 1, C, 1, 0, L, Hp, Wp, g->col_b1[scale])) != QUARK_OK) return s;
    } else if (!up) {
        QK_CU(ctx, cudaMemcpyAsync(dv_prev, dVin, E * C * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    return QUARK_OK;
}

extern "C" quark_status quark_encode_pyramid_bwd(quark_ctx* ctx, const quark_pyramid* pyr, const float* const* dfeat,
                                                 const quark_grads* g, void* stream) {
    if (!ctx || !pyr || !dfeat || !g || !g->enc_w || !g->enc_b) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (pyr->ctx != ctx) return qk_fail(ctx, QUARK_EINVAL, "pyramid from another context");
    if (ctx->cfg.precision != QUARK_FP32) return qk_fail(ctx, QUARK_EINVAL, "the backward pass is FP32 only");
    if (ctx->cfg.ray_encoding) return qk_fail(ctx, QUARK_EINVAL, "the backward pass runs without the ray encoding");
    const float* lev[4] = {dfeat[0], dfeat[1], dfeat[2], dfeat[3]};
    for (int i = 0; i < 4; ++i)
        if (lev[i] && !pyr->level[i])
            return qk_fail(ctx, QUARK_EINVAL, "gradient given for pyramid level %d, which this pyramid does not hold", 1 << i);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int C = ctx->cfg.C, V = pyr->V, H = pyr->H, W = pyr->W;
    const size_t P = (size_t)V * H * W;
    const size_t part = (size_t)kRedBlocks * 27 * C;
    quark_status s = grow_ws(ctx, carved({P * C, part}));
    if (s != QUARK_OK) return s;
    Carve cv{(float*)ctx->bwd_ws};
    float* d1 = cv.take(P * C);
    float* partial = cv.take(part);
    auto L_ = [&](auto fn) { return qk_launch(ctx, st, KF_BACKWARD, fn); };
    // the mean-pool chain's adjoint: the full-resolution conv output's gradient
    if ((s = L_([&] { return launch_pool_chain_bwd(lev, V, H, W, C, d1, st); })) != QUARK_OK) return s;
    // conv weights: sum over views and pixels of the image patch times that gradient (the images are
    // the pyramid's RGBA copy, read as 3 of 4 channels); bias: the gradient's sum
    XtyArgs xa{};
    xa.X = (const float*)pyr->rgba;
    xa.ldx = 4;
    xa.Y = d1;
    xa.ldy = C;
    xa.L = V;
    xa.H = H;
    xa.W = W;
    xa.cx = 3;
    xa.cy = C;
    xa.taps = 9;
    xa.partial = partial;
    xa.n_blocks = kRedBlocks;
    if ((s = L_([&] { return launch_xty(xa, g->enc_w, 1, st); })) != QUARK_OK) return s;
    xa.X = nullptr;
    xa.cx = 1;
    xa.taps = 1;
    return L_([&] { return launch_xty(xa, g->enc_b, 1, st); });
}
