// Internal interfaces of the differentiable stage's adjoint kernels (k_backward.cu).
#pragma once

#include "quark_internal.cuh"

namespace quark {

struct AttendBwdArgs {
    const float* v_in;     // [L][H][W][C] volume entering the step
    const float* feat;     // pyramid level [V][fh][fw][C]
    const float* dv_attn;  // [L][H][W][C] gradient of the attention block's output
    const float* dbeta;    // [H][W][L][V] gradient of the blend logits
    const float* v0;       // step 0 (initialisation): V_in = v0 [C] everywhere and the depths are the
                           // anchors (no depth gradient); v_in is then unused.  NULL otherwise
    int L, H, W, V, fh, fw, last;
    DepthParams dp;
    const float* g;        // attention RMSNorm gain [C]
    const float* w_d;      // [C]
    float b_d;
    const float* Wq;       // [C][h C]
    const float* Wo;       // [h C][C]
    const float* Wb;       // [C][C]
    Geometry geo;
    float* dv_in;          // [L][H][W][C]
    float* dfeat;          // [V][fh][fw][C], accumulated with atomics
    float* x_out;          // [E][C]   N(V_in)
    float* dq_out;         // [E][hC]  query gradients
    float* o_out;          // [E][hC]  head outputs
    float* dqb_out;        // [E][C]   blend-query gradient
    float* dgterm;         // [E][C]   per-element terms of the gain gradient
    float* dt_in;          // [E]      gradient of the depth logit of V_in
};

struct XtyArgs {
    const float* X;  // [E][ldx] (NULL: ones)
    int ldx;
    const float* Y;  // [E][ldy]
    int ldy;
    int L, H, W;     // element grid (for the 3x3 tap shifts)
    int cx, cy, taps;
    int x_gelu;
    float* partial;  // [n_blocks][taps * cx * cy]
    int n_blocks;
};

cudaError_t launch_render_bwd(const RenderArgs& a, const float* dl, float* dt_raw, float* ds_raw, float* dbeta_raw,
                              cudaStream_t st);
cudaError_t launch_decode_bwd(const float* dt_raw, const float* ds_raw, int L, int H, int W, int C, const float* w_d,
                              const float* w_s, float* dv_out, float* dts, cudaStream_t st);
cudaError_t launch_conv3x3(const float* in, const float* w, const float* bias, float* out, int L, int H, int W, int C,
                           int transpose, const float* gelu_aux, cudaStream_t st);
cudaError_t launch_rmsnorm(const float* v, const float* g, float* n, size_t E, int C, cudaStream_t st);
cudaError_t launch_rmsnorm_bwd(const float* v, const float* g, const float* dn, const float* resid, float* dv,
                               float* dgterm, size_t E, int C, cudaStream_t st);
cudaError_t launch_attend_bwd(const AttendBwdArgs& a, int C, int heads, cudaStream_t st);
cudaError_t launch_xty(const XtyArgs& a, float* out, int accumulate, cudaStream_t st);
cudaError_t launch_upsample2(const float* in, float* out, int L, int Hp, int Wp, int C, cudaStream_t st);
// Adjoints of the step transitions and of the encoder's pooling (k_network_bwd.cu).
cudaError_t launch_upsample2_bwd(const float* dout, float* din, int L, int Hp, int Wp, int C, cudaStream_t st);
cudaError_t launch_collapse_bwd(const float* vprev, const float* dcol, int L, int H, int W, int C, const float* w,
                                float* dvprev, float* g_out, float* dh_out, float* cat_out, cudaStream_t st);
cudaError_t launch_pool_chain_bwd(const float* const dlev[4], int V, int H, int W, int C, float* out, cudaStream_t st);

}  // namespace quark
