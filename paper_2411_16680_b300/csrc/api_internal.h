// Host-side state behind the opaque handles of quark.h.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "quark.h"
#include "quark_internal.cuh"

enum KernelFamily { KF_ENCODE = 0, KF_COLLAPSE, KF_ATTEND, KF_CONV, KF_RENDER, KF_BACKWARD, KF_REFINE, KF_COUNT };

struct PendingTiming {
    KernelFamily fam;
    cudaEvent_t e0, e1;
};

struct quark_ctx {
    quark_config cfg{};
    int device = 0;
    std::string last_error;
    // packed weights (device) and the offsets (floats) of each block
    float* wdev = nullptr;
    size_t wbytes = 0;
    bool weights_loaded = false;
    size_t off_enc = 0;
    size_t off_attend[QUARK_MAX_SCALES] = {};  // or (size_t)-1 for a block without attention
    size_t off_conv[QUARK_MAX_SCALES] = {};
    size_t off_collapse[QUARK_MAX_SCALES] = {};
    size_t off_std[QUARK_MAX_SCALES] = {};  // standard attention weights (StdLayout), or (size_t)-1
    size_t off_ray[4] = {};                   // ray encoding projection per level index, or (size_t)-1
    size_t off_upd[QUARK_MAX_SCALES] = {};    // Update Block (ConvLayout, then W_r, b_r), or (size_t)-1
    void* wupd = nullptr;                     // Update Block convs packed as tcgen05 B operands (FP32 form: split)
    size_t wupd_bytes = 0;
    // BF16 form: conv weights packed as tcgen05 B operands, per step W1 then W2
    void* wtc = nullptr;
    size_t wtc_bytes = 0;
    size_t wtc_step_bytes = 0;
    // BF16 form: [Wq | W_beta] and W^O (then the layer collapse's W1, W2) packed as tcgen05 B
    // operands, per step at byte offset off_wat[j]
    void* wat = nullptr;
    size_t wat_bytes = 0;
    // FP32 form: the layer collapses' MLP as split FP16 B operands, per step at byte offset off_wcol[j]
    void* wcol = nullptr;
    size_t wcol_bytes = 0;
    size_t off_wcol[QUARK_MAX_SCALES] = {};
    size_t off_wat[QUARK_MAX_SCALES] = {};
    // BF16 form: the encoder conv packed as a tcgen05 B operand (C x 32)
    void* wenc = nullptr;
    size_t wenc_bytes = 0;
    // device error word written by kernels whose bounded waits run out
    int* dev_err = nullptr;
    // quark_test_wait_timeout: the next tensor-core sampling launch leaves its query MMA unissued
    bool test_wait_armed = false;
    // device memory accounting against cfg.hbm_cap_bytes
    std::mutex mem_mu;
    size_t bytes = 0;
    // launch accounting / profiling
    uint64_t launches = 0;
    bool profiling = false;
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> event_pool;
    double fam_ms[KF_COUNT] = {};
    uint64_t fam_n[KF_COUNT] = {};
    // pyramids and LDMs of this context not yet released (quark_destroy refuses while any remain)
    std::atomic<int> live_handles{0};
    // differentiable stage: backward workspace (grown on demand)
    void* bwd_ws = nullptr;
    size_t bwd_ws_bytes = 0;
};

struct quark_pyramid {
    quark_ctx* ctx = nullptr;
    int V = 0, H = 0, W = 0;
    std::vector<quark_camera> cams;
    void* level[4] = {};  // k = 1, 2, 4, 8
    size_t level_bytes[4] = {};
    void* rgba = nullptr;  // float4 [V][H][W]
    size_t rgba_bytes = 0;
    void* staging = nullptr;  // device copy of host images
    size_t staging_bytes = 0;
};

struct DevBuf {
    void* p;
    size_t bytes;
};

struct quark_ldm {
    quark_ctx* ctx = nullptr;
    quark_camera target{};
    std::vector<DevBuf> bufs;
    void* vol[2] = {};
    int cur = 0;
    void* vattn = nullptr;
    void* collapsed = nullptr;
    float* colour = nullptr;
    float* alpha = nullptr;
    float* depth = nullptr;
    float* t_raw = nullptr;
    float* s_raw = nullptr;
    float* beta = nullptr;
    size_t beta_bytes = 0;
    float* dsamp = nullptr;  // [L][H][W] depths of the latest sampling step, kept for reuse_depth
    // render-and-refine scratch: splat sums, rendered views, Update Block input and output
    void* splat = nullptr;
    size_t splat_bytes = 0;
    void* upd_in = nullptr;
    size_t upd_in_bytes = 0;
    void* delta = nullptr;  // [V][h][w][C] update features of the current Update & Fuse step
    size_t delta_bytes = 0;
    bool delta_ok = false;  // delta holds the current Update & Fuse step's features
    int Hs[QUARK_MAX_SCALES] = {}, Ws[QUARK_MAX_SCALES] = {};  // LDM grid of each step
    void* kv = nullptr;  // standard attention: the projected keys / values of the step's level
    size_t kv_bytes = 0;
    float* ray_g = nullptr;  // ray encoding: the projected coarse encoding of the step's level
    size_t ray_g_bytes = 0;
    void* ray_feat = nullptr;  // ray encoding: the step's level plus gamma_k
    size_t ray_feat_bytes = 0;
    void* out = nullptr;  // device staging of a host render target
    size_t out_bytes = 0;
    size_t last_e = 0;
    int V = 0;
    int done = -1;     // latest Update & Fuse step completed
    int decoded = -1;  // step whose decoded attributes (colour, alpha, depth, logits) are current
    bool async = false;            // buffers from the stream-ordered allocator on `stream`
    cudaStream_t stream = nullptr;
    // quark_ldm_keep_steps: every step's output volume and attention-block output, kept for the
    // backward pass (allocated on first use)
    bool keep = false;
    void* hist_out[QUARK_MAX_SCALES] = {};
    void* hist_attn[QUARK_MAX_SCALES] = {};
};

quark_status qk_fail(const quark_ctx* ctx, quark_status st, const char* fmt, ...);
quark_status qk_alloc(quark_ctx* ctx, void** p, size_t bytes);
void qk_free(quark_ctx* ctx, void* p, size_t bytes);
quark_status qk_launch(quark_ctx* ctx, cudaStream_t st, KernelFamily fam, const std::function<cudaError_t()>& fn);
quark_status qk_validate_config(const quark_config* c);
// Per-step schedule of a config (zero-filled fields = the uniform schedule).
int qk_heads(const quark_config& c, int j);     // attention heads of step j, 0 = no attention
double qk_f(const quark_config& c, int j);      // LDM grid factor of step j
bool qk_uniform(const quark_config& c);         // no per-step heads, grid factors or reuse
bool qk_refines(const quark_config& c, int j);  // step j renders the views and runs the Update Block
bool qk_grid(const quark_config& c, int j, int width, int height, int& H, int& W);  // false: not divisible
quark_status qk_validate_camera(const quark_ctx* ctx, const quark_camera& c, const char* what);
// View map from a target grid with factors (k_tx, k_ty) (target pixels per grid pixel along x, y)
// to view `view`'s level-k_m grid.
quark::ViewMap qk_view_map(const quark_camera& tgt, double k_tx, double k_ty, const quark_camera& view, double k_m);
quark::ViewMap qk_ray_map(const quark_camera& tgt, const quark_camera& view, double k0);
size_t qk_ldm_bytes(const quark_config& c, int width, int height, int V, bool host_out);
quark_status qk_ldm_create(quark_ctx* ctx, const quark_camera* target, int V_beta, cudaStream_t async_stream,
                           quark_ldm** out);
void qk_ldm_free(quark_ldm* l);
quark_status qk_update_fuse(quark_ctx* ctx, const quark_pyramid* pyr, int V_use, int scale, quark_ldm* ldm,
                            cudaStream_t stream, const void* prev_override = nullptr,
                            const void* feat_override = nullptr);
quark_status qk_ldm_scratch(quark_ldm* l, void** p, size_t bytes);
quark_status qk_decode(quark_ctx* ctx, int scale, const void* vol, int L, int H, int W, float* colour, float* alpha,
                       float* depth, float* t_raw, float* s_raw, cudaStream_t st);
const void* qk_collapse_wtc(const quark_ctx* ctx, int scale);
quark_status qk_render(quark_ctx* ctx, const quark_ldm* ldm, const quark_pyramid* pyr, int V_use, float* rgba,
                       int host_out, cudaStream_t stream);
quark_status qk_encode_pyramid_sync(quark_ctx* ctx, const float* images, const quark_camera* cams, int V,
                                    quark_pyramid** out);
