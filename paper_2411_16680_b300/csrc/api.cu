// C ABI of the library (include/quark.h): contexts, validation, weight packing, handles and
// the per-step launch sequence.  Host code only; the compute is in the k_*.cu kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "quark_internal.cuh"
#include "api_internal.h"

using namespace quark;

// -------------------------------------------------------------------------------------------
// Errors
// -------------------------------------------------------------------------------------------

static thread_local std::string g_thread_error;

quark_status qk_fail(const quark_ctx* ctx, quark_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) const_cast<quark_ctx*>(ctx)->last_error = buf;
    g_thread_error = buf;
    return st;
}

#define QK_CUDA(ctx, call)                                                                       \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return qk_fail(ctx, QUARK_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char* quark_last_error(const quark_ctx* ctx) {
    if (ctx) return ctx->last_error.c_str();
    return g_thread_error.c_str();
}

// -------------------------------------------------------------------------------------------
// Device memory with the context's cap
// -------------------------------------------------------------------------------------------

quark_status qk_alloc(quark_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return QUARK_OK;
    {
        std::lock_guard<std::mutex> g(ctx->mem_mu);
        if (ctx->cfg.hbm_cap_bytes && ctx->bytes + bytes > ctx->cfg.hbm_cap_bytes)
            return qk_fail(ctx, QUARK_ENOMEM, "allocation of %zu bytes exceeds the HBM cap (%zu of %zu in use)",
                           bytes, ctx->bytes, ctx->cfg.hbm_cap_bytes);
        ctx->bytes += bytes;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> g(ctx->mem_mu);
        ctx->bytes -= bytes;
        *p = nullptr;
        cudaGetLastError();
        return qk_fail(ctx, QUARK_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    return QUARK_OK;
}

void qk_free(quark_ctx* ctx, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    std::lock_guard<std::mutex> g(ctx->mem_mu);
    ctx->bytes -= bytes;
}

// -------------------------------------------------------------------------------------------
// Launch accounting
// -------------------------------------------------------------------------------------------

static const char* kFamilyNames[KF_COUNT] = {"encode", "collapse", "attend", "conv_block", "render", "backward",
                                              "refine"};

static cudaEvent_t get_event(quark_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

quark_status qk_launch(quark_ctx* ctx, cudaStream_t st, KernelFamily fam, const std::function<cudaError_t()>& fn) {
    cudaEvent_t e0 = nullptr;
    if (ctx->profiling) {
        e0 = get_event(ctx);
        cudaEventRecord(e0, st);
    }
    cudaError_t err = fn();
    ctx->launches++;
    if (ctx->profiling) {
        cudaEvent_t e1 = get_event(ctx);
        cudaEventRecord(e1, st);
        ctx->pending.push_back({fam, e0, e1});
    }
    if (err != cudaSuccess)
        return qk_fail(ctx, QUARK_ECUDA, "launch of %s kernel failed: %s", kFamilyNames[fam], cudaGetErrorString(err));
    return QUARK_OK;
}

extern "C" uint64_t quark_launch_count(const quark_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" void quark_reset_counters(quark_ctx* ctx) {
    if (!ctx) return;
    ctx->launches = 0;
    for (auto& p : ctx->pending) {
        cudaEventSynchronize(p.e1);
        ctx->event_pool.push_back(p.e0);
        ctx->event_pool.push_back(p.e1);
    }
    ctx->pending.clear();
    for (int i = 0; i < KF_COUNT; ++i) {
        ctx->fam_ms[i] = 0.0;
        ctx->fam_n[i] = 0;
    }
}

extern "C" quark_status quark_set_profiling(quark_ctx* ctx, int enable) {
    if (!ctx) return qk_fail(nullptr, QUARK_EINVAL, "NULL context");
    ctx->profiling = enable != 0;
    return QUARK_OK;
}

extern "C" int quark_kernel_times(quark_ctx* ctx, const char** names, double* ms, uint64_t* launches, int cap) {
    if (!ctx) return 0;
    for (auto& p : ctx->pending) {
        cudaEventSynchronize(p.e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, p.e0, p.e1);
        ctx->fam_ms[p.fam] += t;
        ctx->fam_n[p.fam] += 1;
        ctx->event_pool.push_back(p.e0);
        ctx->event_pool.push_back(p.e1);
    }
    ctx->pending.clear();
    for (int i = 0; i < KF_COUNT && i < cap; ++i) {
        if (names) names[i] = kFamilyNames[i];
        if (ms) ms[i] = ctx->fam_ms[i];
        if (launches) launches[i] = ctx->fam_n[i];
    }
    return KF_COUNT;
}

// -------------------------------------------------------------------------------------------
// Context
// -------------------------------------------------------------------------------------------

static bool is_pow2_factor(int k) { return k == 1 || k == 2 || k == 4 || k == 8; }

int qk_heads(const quark_config& c, int j) {
    const int h = c.scale_heads[j];
    return h == 0 ? c.heads : h < 0 ? 0 : h;
}

double qk_f(const quark_config& c, int j) { return c.ldm_f[j] > 0.f ? (double)c.ldm_f[j] : (double)c.k[j]; }

bool qk_uniform(const quark_config& c) {
    if (c.model_width || c.model_height) return false;
    for (int j = 0; j < QUARK_MAX_SCALES; ++j)
        if (c.scale_heads[j] != 0 || c.ldm_f[j] != 0.f || c.reuse_depth[j] != 0) return false;
    return true;
}

bool qk_grid(const quark_config& c, int j, int width, int height, int& H, int& W) {
    if (c.model_width > 0) {
        // aspect-adaptive: the model's step-0 grid area at the output's aspect, then x2 multiples
        const double f0 = qk_f(c, 0);
        const double area = (c.model_height / f0) * (c.model_width / f0);
        const double aspect = (double)width / height;
        const int h0 = std::max(1, (int)std::floor(std::sqrt(area / aspect) + 0.5));
        const int w0 = std::max(1, (int)std::floor(h0 * aspect + 0.5));
        const int m = (int)std::lround(f0 / qk_f(c, j));
        H = h0 * m;
        W = w0 * m;
        return true;
    }
    const double f = qk_f(c, j);
    H = (int)std::lround(height / f);
    W = (int)std::lround(width / f);
    return H >= 1 && W >= 1 && std::fabs(H * f - height) < 1e-3 && std::fabs(W * f - width) < 1e-3;
}

// a == 2 b (x2 upsample) or a == b, for grid factors given as float
static bool same_f(double a, double b) { return std::fabs(a - b) <= 1e-6 * b; }

quark_status qk_validate_config(const quark_config* c) {
    if (!c) return qk_fail(nullptr, QUARK_EINVAL, "NULL config");
    if (c->C != 16 && c->C != 32 && c->C != 64)
        return qk_fail(nullptr, QUARK_EINVAL, "C must be 16, 32 or 64 (got %d)", c->C);
    if (c->heads != 1 && c->heads != 2 && c->heads != 4)
        return qk_fail(nullptr, QUARK_EINVAL, "heads must be 1, 2 or 4 (got %d)", c->heads);
    if (c->n_scales < 1 || c->n_scales > QUARK_MAX_SCALES)
        return qk_fail(nullptr, QUARK_EINVAL, "n_scales must be 1..%d", QUARK_MAX_SCALES);
    for (int j = 0; j < QUARK_MAX_SCALES; ++j) {
        const int h = c->scale_heads[j];
        if (h != 0 && h != -1 && h != 1 && h != 2 && h != 4)
            return qk_fail(nullptr, QUARK_EINVAL, "scale_heads[%d] must be 0, -1, 1, 2 or 4 (got %d)", j, h);
        if (!(c->ldm_f[j] >= 0.f) || !std::isfinite(c->ldm_f[j]))
            return qk_fail(nullptr, QUARK_EINVAL, "ldm_f[%d] must be finite and >= 0", j);
        if (c->reuse_depth[j] != 0 && c->reuse_depth[j] != 1)
            return qk_fail(nullptr, QUARK_EINVAL, "reuse_depth[%d] must be 0 or 1", j);
        if (j >= c->n_scales && (h != 0 || c->ldm_f[j] != 0.f || c->reuse_depth[j] != 0))
            return qk_fail(nullptr, QUARK_EINVAL, "schedule fields set beyond n_scales (step %d)", j);
    }
    int sampled = -1;  // latest step that sampled the views
    for (int j = 0; j < c->n_scales; ++j) {
        if (!is_pow2_factor(c->k[j])) return qk_fail(nullptr, QUARK_EINVAL, "k[%d] must be 1, 2, 4 or 8", j);
        if (c->L[j] < 1 || c->L[j] > 64) return qk_fail(nullptr, QUARK_EINVAL, "L[%d] must be 1..64", j);
        const int h = qk_heads(*c, j);
        if (j > 0) {
            if (c->k[j - 1] != c->k[j] && c->k[j - 1] != 2 * c->k[j])
                return qk_fail(nullptr, QUARK_EINVAL, "k[%d]/k[%d] must be 1 or 2", j - 1, j);
            if (c->L[j - 1] != c->L[j] && c->L[j - 1] != 2 * c->L[j])
                return qk_fail(nullptr, QUARK_EINVAL, "L[%d]/L[%d] must be 1 or 2", j - 1, j);
            const double fp = qk_f(*c, j - 1), f = qk_f(*c, j);
            if (!same_f(fp, f) && !same_f(fp, 2 * f))
                return qk_fail(nullptr, QUARK_EINVAL, "grid factor ratio f[%d]/f[%d] must be 1 or 2", j - 1, j);
            if ((h == 0 || c->reuse_depth[j]) && (!same_f(fp, f) || c->L[j - 1] != c->L[j]))
                return qk_fail(nullptr, QUARK_EINVAL,
                               "step %d (no attention or reused depths) needs the grid and layers of step %d", j, j - 1);
        } else if (h == 0 || c->reuse_depth[0]) {
            return qk_fail(nullptr, QUARK_EINVAL, "step 0 must attend and decode its depths");
        }
        if (c->reuse_depth[j] && sampled < 0)
            return qk_fail(nullptr, QUARK_EINVAL, "step %d reuses depths but no step sampled before it", j);
        if (h > 0) sampled = j;
        if (c->attn_mode == QUARK_ATTN_STANDARD && h > 0 && c->C % h)
            return qk_fail(nullptr, QUARK_EINVAL, "standard attention needs C divisible by heads (step %d)", j);
        if (c->precision == QUARK_BF16 && c->attn_mode == QUARK_ATTN_ONE_TO_MANY && c->C == 64 && h == 4)
            return qk_fail(nullptr, QUARK_EINVAL,
                           "the BF16 form runs one-to-many attention with C = 64 for 1 or 2 heads (step %d has 4: "
                           "its 5C = 320 query columns exceed one tensor-core MMA's 256)", j);
    }
    if (qk_heads(*c, c->n_scales - 1) == 0)
        return qk_fail(nullptr, QUARK_EINVAL, "the last step must attend (its attention gives the blend logits)");
    if (!(c->near_m > 0.f) || !(c->far_m > c->near_m) || !std::isfinite(c->far_m))
        return qk_fail(nullptr, QUARK_EINVAL, "need 0 < near < far < inf");
    if (c->precision != QUARK_FP32 && c->precision != QUARK_BF16)
        return qk_fail(nullptr, QUARK_EINVAL, "unknown precision %d", c->precision);
    if (c->attn_mode != QUARK_ATTN_ONE_TO_MANY && c->attn_mode != QUARK_ATTN_STANDARD)
        return qk_fail(nullptr, QUARK_EINVAL, "unknown attention mode %d", c->attn_mode);
    if (c->ray_encoding != 0 && c->ray_encoding != 1) return qk_fail(nullptr, QUARK_EINVAL, "ray_encoding must be 0 or 1");
    if (c->render_refine != 0 && c->render_refine != 1)
        return qk_fail(nullptr, QUARK_EINVAL, "render_refine must be 0 or 1");
    if (c->model_width < 0 || c->model_height < 0 || (c->model_width > 0) != (c->model_height > 0))
        return qk_fail(nullptr, QUARK_EINVAL, "model_width and model_height must both be 0 or both positive");
    if (c->conv_kernel != 0 && c->conv_kernel != 1 && c->conv_kernel != 3)
        return qk_fail(nullptr, QUARK_EINVAL, "conv_kernel must be 3 or 1 (0 = 3; got %d)", c->conv_kernel);
    return QUARK_OK;
}

bool qk_refines(const quark_config& c, int j) {
    return c.render_refine && j > 0 && qk_heads(c, j) > 0 && !c.reuse_depth[j];
}

extern "C" quark_status quark_create(const quark_config* cfg, int device, quark_ctx** out) {
    if (!out) return qk_fail(nullptr, QUARK_EINVAL, "NULL out");
    *out = nullptr;
    quark_status s = qk_validate_config(cfg);
    if (s != QUARK_OK) return s;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return qk_fail(nullptr, QUARK_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    if (device < 0 || device >= n) return qk_fail(nullptr, QUARK_EINVAL, "device %d out of range", device);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return qk_fail(nullptr, QUARK_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    quark_ctx* ctx = new quark_ctx();
    ctx->cfg = *cfg;
    ctx->device = device;
    *out = ctx;
    return QUARK_OK;
}

extern "C" quark_status quark_destroy(quark_ctx* ctx) {
    if (!ctx) return QUARK_OK;
    // a pyramid or LDM keeps a pointer to its context: destroying the context under it would
    // leave its release with freed state
    if (const int n = ctx->live_handles.load())
        return qk_fail(ctx, QUARK_EBUSY, "%d pyramid / LDM handle(s) of this context are still alive: release them first", n);
    cudaSetDevice(ctx->device);
    for (auto& p : ctx->pending) {
        cudaEventSynchronize(p.e1);
        ctx->event_pool.push_back(p.e0);
        ctx->event_pool.push_back(p.e1);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    qk_free(ctx, ctx->wdev, ctx->wbytes);
    qk_free(ctx, ctx->wtc, ctx->wtc_bytes);
    qk_free(ctx, ctx->wat, ctx->wat_bytes);
    qk_free(ctx, ctx->wcol, ctx->wcol_bytes);
    qk_free(ctx, ctx->wupd, ctx->wupd_bytes);
    qk_free(ctx, ctx->wenc, ctx->wenc_bytes);
    qk_free(ctx, ctx->dev_err, sizeof(int));
    qk_free(ctx, ctx->bwd_ws, ctx->bwd_ws_bytes);
    delete ctx;
    return QUARK_OK;
}

// -------------------------------------------------------------------------------------------
// Weights: packed into one device blob per context
// -------------------------------------------------------------------------------------------

// float -> bf16 bits, round to nearest even (weights are finite)
static uint16_t to_bf16_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// 3x3 conv weights [dy][dx][ci][co] (fp32) -> per tap a K-major tcgen05 B operand (N = co rows,
// K = ci): element (co, ci) at (ci / 8) * C * 8 + co * 8 + ci % 8 (bf16 elements).
static void pack_conv_weights_bf16(const float* w, int C, uint16_t* dst) {
    for (int tap = 0; tap < 9; ++tap)
        for (int ci = 0; ci < C; ++ci)
            for (int co = 0; co < C; ++co)
                dst[(size_t)tap * C * C + (ci / 8) * C * 8 + co * 8 + ci % 8] =
                    to_bf16_bits(w[((size_t)tap * C + ci) * C + co]);
}

// FP32 form on the tensor cores: a value as its FP16 parts, the rounded value hi[i] = fp16(x) and the
// scaled remainder lo[i] = fp16((x - hi) 2^11) (x - hi is exact in FP32, the scaling too).  The
// parts stay finite while |x| < kSplitMax; the kernels take x_h w_h + 2^-11 (x_h w_l + x_l w_h).
constexpr double kSplitMax = 32768.0;
static void put_f16split(uint16_t* hi, uint16_t* lo, size_t i, float x) {
    const __half h = __float2half_rn(x);
    hi[i] = __half_as_ushort(h);
    lo[i] = __half_as_ushort(__float2half_rn((x - __half2float(h)) * 2048.f));
}
static bool in_split_range(double v) { return std::fabs(v) < kSplitMax; }

// The same B layout as pack_conv_weights_bf16 in FP16 parts: the rounded weights (hi), then the
// scaled remainders (lo), 9 C C elements each.
static void pack_conv_weights_f16split(const float* w, int C, uint16_t* hi, uint16_t* lo) {
    for (int tap = 0; tap < 9; ++tap)
        for (int ci = 0; ci < C; ++ci)
            for (int co = 0; co < C; ++co)
                put_f16split(hi, lo, (size_t)tap * C * C + (ci / 8) * C * 8 + co * 8 + ci % 8,
                             w[((size_t)tap * C + ci) * C + co]);
}

// Whether every FP16 part the split conv block forms stays below 2^15, for any volume: the
// normalised input is at most sqrt(C) max|g| per channel (RMSNorm), conv1's output at most
// sum |w1| times that plus |b1| (and gelu(y) <= max(|y|, 0.17)), the weights themselves; the
// remainders are 2^-11 of their values, scaled by 2^11.
static bool conv_split_in_range(const float* g, const float* w1, const float* b1, const float* w2, int C) {
    double gmax = 0.0;
    for (int c = 0; c < C; ++c) gmax = std::max(gmax, (double)std::fabs(g[c]));
    const double xmax = std::sqrt((double)C) * gmax;
    if (!in_split_range(xmax)) return false;
    for (int co = 0; co < C; ++co) {
        double s = std::fabs((double)b1[co]);
        for (int tap = 0; tap < 9; ++tap)
            for (int ci = 0; ci < C; ++ci) s += std::fabs((double)w1[((size_t)tap * C + ci) * C + co]) * xmax;
        if (!in_split_range(s)) return false;
    }
    for (size_t i = 0; i < 9 * (size_t)C * C; ++i)
        if (!in_split_range(w1[i]) || !in_split_range(w2[i])) return false;
    return true;
}

static int level_index(int k) { return k == 1 ? 0 : k == 2 ? 1 : k == 4 ? 2 : 3; }

extern "C" quark_status quark_load_weights(quark_ctx* ctx, const quark_weights* w) {
    if (!ctx || !w) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    cudaSetDevice(ctx->device);
    const quark_config& c = ctx->cfg;
    const int C = c.C;
    auto need = [&](const void* p, const char* name) -> bool {
        if (!p) {
            qk_fail(ctx, QUARK_EINVAL, "weight %s is NULL", name);
            return false;
        }
        return true;
    };
    if (!need(w->enc_w, "enc_w") || !need(w->enc_b, "enc_b") || !need(w->v0, "v0") || !need(w->w_d, "w_d") ||
        !need(w->w_sigma, "w_sigma") || !need(w->W_a, "W_a") || !need(w->b_a, "b_a") || !need(w->W_beta, "W_beta"))
        return QUARK_EINVAL;
    // the fusion blocks' conv weights as 3x3 kernels: 1x1 weights (conv_kernel 1) sit at the centre
    // tap, zeros elsewhere, so every kernel, the decode and the backward share one layout
    std::vector<std::vector<float>> tap9(2 * (size_t)c.n_scales);
    const float* cw1[QUARK_MAX_SCALES] = {};
    const float* cw2[QUARK_MAX_SCALES] = {};
    for (int j = 0; j < c.n_scales; ++j) {
        cw1[j] = w->conv1_w[j];
        cw2[j] = w->conv2_w[j];
        if (c.conv_kernel == 1 && w->conv1_w[j] && w->conv2_w[j]) {
            for (int q = 0; q < 2; ++q) {
                std::vector<float>& t = tap9[2 * j + q];
                t.assign(9 * (size_t)C * C, 0.f);
                std::memcpy(t.data() + 4 * (size_t)C * C, q ? w->conv2_w[j] : w->conv1_w[j], (size_t)C * C * 4);
            }
            cw1[j] = tap9[2 * j].data();
            cw2[j] = tap9[2 * j + 1].data();
        }
    }
    std::vector<float> blob;
    auto put = [&](const float* p, size_t n) {
        size_t off = blob.size();
        blob.insert(blob.end(), p, p + n);
        return off;
    };
    auto pad4 = [&]() {
        while (blob.size() % 4) blob.push_back(0.f);
    };
    ctx->off_enc = put(w->enc_w, 27 * (size_t)C);
    put(w->enc_b, C);
    pad4();
    for (int j = 0; j < c.n_scales; ++j) {
        const int h = qk_heads(c, j);
        if (!need(w->conv_g[j], "conv_g") || !need(w->conv1_w[j], "conv1_w") || !need(w->conv1_b[j], "conv1_b") ||
            !need(w->conv2_w[j], "conv2_w") || !need(w->conv2_b[j], "conv2_b"))
            return QUARK_EINVAL;
        ctx->off_attend[j] = (size_t)-1;
        if (h > 0) {
            if (!need(w->attn_g[j], "attn_g") || !need(w->Wq[j], "Wq") || !need(w->Wo[j], "Wo")) return QUARK_EINVAL;
            // attend block: v0, g, w_d, b_d (padded to C), Wq, Wo, W_beta
            const AttendLayout al{C, h};
            ctx->off_attend[j] = blob.size();
            put(w->v0, C);
            put(w->attn_g[j], C);
            put(w->w_d, C);
            blob.push_back(w->b_d);
            for (int i = 1; i < C; ++i) blob.push_back(0.f);
            put(w->Wq[j], (size_t)C * h * C);
            put(w->Wo[j], (size_t)h * C * C);
            put(w->W_beta, (size_t)C * C);
            if (blob.size() - ctx->off_attend[j] != (size_t)al.total())
                return qk_fail(ctx, QUARK_EINTERNAL, "attend layout");
            pad4();
        }
        // conv block: g, W1, b1, W2, b2, w_d, w_s, W_a, b_a, b_d, b_s (+3 pad)
        const ConvLayout cl{C};
        ctx->off_conv[j] = blob.size();
        put(w->conv_g[j], C);
        put(cw1[j], 9 * (size_t)C * C);
        put(w->conv1_b[j], C);
        put(cw2[j], 9 * (size_t)C * C);
        put(w->conv2_b[j], C);
        put(w->w_d, C);
        put(w->w_sigma, C);
        put(w->W_a, 3 * (size_t)C);
        put(w->b_a, 3);
        blob.push_back(w->b_d);
        blob.push_back(w->b_sigma);
        blob.push_back(0.f);
        blob.push_back(0.f);
        blob.push_back(0.f);
        if (blob.size() - ctx->off_conv[j] != (size_t)cl.total()) return qk_fail(ctx, QUARK_EINTERNAL, "conv layout");
        pad4();
        ctx->off_std[j] = (size_t)-1;
        if (c.attn_mode == QUARK_ATTN_STANDARD && h > 0) {
            if (!need(w->Wq_std[j], "Wq_std") || !need(w->Wk_std[j], "Wk_std") || !need(w->Wv_std[j], "Wv_std") ||
                !need(w->Wo_std[j], "Wo_std"))
                return QUARK_EINVAL;
            // StdLayout: W^q, W^O, then rows k of [W^k | W^val]
            ctx->off_std[j] = blob.size();
            put(w->Wq_std[j], (size_t)C * C);
            put(w->Wo_std[j], (size_t)C * C);
            for (int k = 0; k < C; ++k) {
                for (int n = 0; n < C; ++n) blob.push_back(w->Wk_std[j][(size_t)k * C + n]);
                for (int n = 0; n < C; ++n) blob.push_back(w->Wv_std[j][(size_t)k * C + n]);
            }
            if (blob.size() - ctx->off_std[j] != (size_t)StdLayout{C}.total())
                return qk_fail(ctx, QUARK_EINTERNAL, "standard attention layout");
            pad4();
        }
        ctx->off_collapse[j] = (size_t)-1;
        if (j > 0 && c.L[j - 1] == 2 * c.L[j]) {
            if (!need(w->col_w1[j], "col_w1") || !need(w->col_b1[j], "col_b1") || !need(w->col_w2[j], "col_w2") ||
                !need(w->col_b2[j], "col_b2"))
                return QUARK_EINVAL;
            ctx->off_collapse[j] = blob.size();
            put(w->col_w1[j], 2 * (size_t)C * C);
            put(w->col_b1[j], C);
            put(w->col_w2[j], (size_t)C * C);
            put(w->col_b2[j], C);
            pad4();
        }
    }
    // Update Blocks of the steps that render (ConvLayout with the decode fields copied, then W_r, b_r)
    for (int j = 0; j < c.n_scales; ++j) {
        ctx->off_upd[j] = (size_t)-1;
        if (!qk_refines(c, j)) continue;
        if (!need(w->upd_Wr[j], "upd_Wr") || !need(w->upd_br[j], "upd_br") || !need(w->upd_g[j], "upd_g") ||
            !need(w->upd1_w[j], "upd1_w") || !need(w->upd1_b[j], "upd1_b") || !need(w->upd2_w[j], "upd2_w") ||
            !need(w->upd2_b[j], "upd2_b"))
            return QUARK_EINVAL;
        ctx->off_upd[j] = blob.size();
        put(w->upd_g[j], C);
        put(w->upd1_w[j], 9 * (size_t)C * C);
        put(w->upd1_b[j], C);
        put(w->upd2_w[j], 9 * (size_t)C * C);
        put(w->upd2_b[j], C);
        put(w->w_d, C);
        put(w->w_sigma, C);
        put(w->W_a, 3 * (size_t)C);
        put(w->b_a, 3);
        blob.push_back(w->b_d);
        blob.push_back(w->b_sigma);
        blob.push_back(0.f);
        blob.push_back(0.f);
        blob.push_back(0.f);
        if (blob.size() - ctx->off_upd[j] != (size_t)ConvLayout{C}.total())
            return qk_fail(ctx, QUARK_EINTERNAL, "update block layout");
        put(w->upd_Wr[j], 4 * (size_t)C);
        put(w->upd_br[j], C);
        pad4();
    }
    for (int i = 0; i < 4; ++i) ctx->off_ray[i] = (size_t)-1;
    if (c.ray_encoding) {
        for (int j = 0; j < c.n_scales; ++j) {
            const int li = level_index(c.k[j]);
            if (qk_heads(c, j) == 0 || ctx->off_ray[li] != (size_t)-1) continue;
            if (!need(w->W_ray[li], "W_ray")) return QUARK_EINVAL;
            ctx->off_ray[li] = blob.size();
            put(w->W_ray[li], 32 * (size_t)C);
            pad4();
        }
    }
    for (float f : blob)
        if (!std::isfinite(f)) return qk_fail(ctx, QUARK_EINVAL, "non-finite weight");
    qk_free(ctx, ctx->wdev, ctx->wbytes);
    ctx->wdev = nullptr;
    ctx->wbytes = blob.size() * sizeof(float);
    quark_status s = qk_alloc(ctx, (void**)&ctx->wdev, ctx->wbytes);
    if (s != QUARK_OK) return s;
    QK_CUDA(ctx, cudaMemcpy(ctx->wdev, blob.data(), ctx->wbytes, cudaMemcpyHostToDevice));
    if (c.precision != QUARK_BF16) {
        // FP32 form: the conv blocks on the tensor cores through split FP16 operands (C <= 32, 3 x 3
        // kernels, every step's weights in the split's range), else the SIMT kernel (wtc stays NULL)
        qk_free(ctx, ctx->wtc, ctx->wtc_bytes);
        ctx->wtc = nullptr;
        ctx->wtc_bytes = 0;
        ctx->wtc_step_bytes = 4 * 9 * (size_t)C * C * sizeof(uint16_t);
        bool split = C <= 32 && c.conv_kernel != 1;
        for (int j = 0; j < c.n_scales && split; ++j)
            split = conv_split_in_range(w->conv_g[j], cw1[j], w->conv1_b[j], cw2[j], C);
        if (split) {
            std::vector<uint16_t> tc(ctx->wtc_step_bytes / sizeof(uint16_t) * c.n_scales);
            const size_t n = 9 * (size_t)C * C;
            for (int j = 0; j < c.n_scales; ++j) {
                uint16_t* d = tc.data() + (size_t)j * 4 * n;
                pack_conv_weights_f16split(cw1[j], C, d, d + n);
                pack_conv_weights_f16split(cw2[j], C, d + 2 * n, d + 3 * n);
            }
            ctx->wtc_bytes = tc.size() * sizeof(uint16_t);
            s = qk_alloc(ctx, &ctx->wtc, ctx->wtc_bytes);
            if (s != QUARK_OK) return s;
            QK_CUDA(ctx, cudaMemcpy(ctx->wtc, tc.data(), ctx->wtc_bytes, cudaMemcpyHostToDevice));
        }
        // the layer collapses' MLP likewise (C <= 32): W1 (N = C, K = 2C) and W2 (K = C) in the BF16
        // form's element order, FP16 high parts then scaled remainders; the kernel scales each
        // element's activations by a power of two, so only the weights bound the parts
        qk_free(ctx, ctx->wcol, ctx->wcol_bytes);
        ctx->wcol = nullptr;
        ctx->wcol_bytes = 0;
        {
            bool csplit = C <= 32, any = false;
            for (int j = 0; j < c.n_scales && csplit; ++j) {
                if (ctx->off_collapse[j] == (size_t)-1) continue;
                any = true;
                for (size_t i = 0; i < 2 * (size_t)C * C && csplit; ++i) csplit = in_split_range(w->col_w1[j][i]);
                for (size_t i = 0; i < (size_t)C * C && csplit; ++i) csplit = in_split_range(w->col_w2[j][i]);
            }
            if (csplit && any) {
                size_t total = 0;
                for (int j = 0; j < c.n_scales; ++j) {
                    ctx->off_wcol[j] = total * sizeof(uint16_t);
                    if (ctx->off_collapse[j] != (size_t)-1) total += 2 * 3 * (size_t)C * C;
                }
                std::vector<uint16_t> cb(total);
                for (int j = 0; j < c.n_scales; ++j) {
                    if (ctx->off_collapse[j] == (size_t)-1) continue;
                    uint16_t* b1 = cb.data() + ctx->off_wcol[j] / sizeof(uint16_t);
                    uint16_t* b1l = b1 + 2 * (size_t)C * C;
                    uint16_t* b2 = b1l + 2 * (size_t)C * C;
                    uint16_t* b2l = b2 + (size_t)C * C;
                    for (int n = 0; n < C; ++n) {
                        for (int k = 0; k < 2 * C; ++k)
                            put_f16split(b1, b1l, (size_t)(k / 8) * C * 8 + n * 8 + k % 8, w->col_w1[j][(size_t)k * C + n]);
                        for (int k = 0; k < C; ++k)
                            put_f16split(b2, b2l, (size_t)(k / 8) * C * 8 + n * 8 + k % 8, w->col_w2[j][(size_t)k * C + n]);
                    }
                }
                ctx->wcol_bytes = cb.size() * sizeof(uint16_t);
                s = qk_alloc(ctx, &ctx->wcol, ctx->wcol_bytes);
                if (s != QUARK_OK) return s;
                QK_CUDA(ctx, cudaMemcpy(ctx->wcol, cb.data(), ctx->wcol_bytes, cudaMemcpyHostToDevice));
            }
        }
        // render-and-refine: the Update Blocks' residual CNN likewise, per step at j * wtc_step_bytes
        qk_free(ctx, ctx->wupd, ctx->wupd_bytes);
        ctx->wupd = nullptr;
        ctx->wupd_bytes = 0;
        bool usplit = C <= 32 && c.render_refine;
        for (int j = 0; j < c.n_scales && usplit; ++j)
            if (qk_refines(c, j)) usplit = conv_split_in_range(w->upd_g[j], w->upd1_w[j], w->upd1_b[j], w->upd2_w[j], C);
        if (usplit) {
            std::vector<uint16_t> up(ctx->wtc_step_bytes / sizeof(uint16_t) * c.n_scales);
            const size_t n = 9 * (size_t)C * C;
            for (int j = 0; j < c.n_scales; ++j) {
                if (!qk_refines(c, j)) continue;
                uint16_t* d = up.data() + (size_t)j * 4 * n;
                pack_conv_weights_f16split(w->upd1_w[j], C, d, d + n);
                pack_conv_weights_f16split(w->upd2_w[j], C, d + 2 * n, d + 3 * n);
            }
            ctx->wupd_bytes = up.size() * sizeof(uint16_t);
            s = qk_alloc(ctx, &ctx->wupd, ctx->wupd_bytes);
            if (s != QUARK_OK) return s;
            QK_CUDA(ctx, cudaMemcpy(ctx->wupd, up.data(), ctx->wupd_bytes, cudaMemcpyHostToDevice));
        }
        // the one-to-many attention's projections likewise (C <= 32): [W^q | W^beta] and W^O in the
        // BF16 form's element order and logit-scale folding, as FP16 high parts then scaled
        // remainders.  Range: the normalised input is at most sqrt(C) max|g| per channel, the
        // weights are the weights; the head outputs are scaled per element in the kernel.
        qk_free(ctx, ctx->wat, ctx->wat_bytes);
        ctx->wat = nullptr;
        ctx->wat_bytes = 0;
        const double qs = 1.0 / std::sqrt((double)C), log2e = 1.4426950408889634;
        bool asplit = C <= 32 && c.attn_mode == QUARK_ATTN_ONE_TO_MANY;
        for (int j = 0; j < c.n_scales && asplit; ++j) {
            const int h = qk_heads(c, j);
            if (h == 0) continue;
            double gmax = 0.0;
            for (int i = 0; i < C; ++i) gmax = std::max(gmax, (double)std::fabs(w->attn_g[j][i]));
            asplit = in_split_range(std::sqrt((double)C) * gmax);
            for (size_t i = 0; i < (size_t)C * h * C && asplit; ++i)
                asplit = in_split_range(w->Wq[j][i] * qs * log2e) && in_split_range(w->Wo[j][i]);
            for (size_t i = 0; i < (size_t)C * C && asplit; ++i) asplit = in_split_range(w->W_beta[i] * qs);
        }
        if (asplit) {
            size_t total = 0;
            for (int j = 0; j < c.n_scales; ++j) {
                const int h = qk_heads(c, j);
                ctx->off_wat[j] = total * sizeof(uint16_t);
                total += h > 0 ? 2 * ((size_t)(h * C + C) * C + (size_t)C * h * C) : 0;
            }
            std::vector<uint16_t> at(std::max<size_t>(total, 8));
            for (int j = 0; j < c.n_scales; ++j) {
                const int h = qk_heads(c, j), NQ = h * C + C;
                if (h == 0) continue;
                uint16_t* bq = at.data() + ctx->off_wat[j] / sizeof(uint16_t);
                uint16_t* bq_lo = bq + (size_t)NQ * C;
                uint16_t* bo = bq_lo + (size_t)NQ * C;
                uint16_t* bo_lo = bo + (size_t)C * h * C;
                for (int n = 0; n < NQ; ++n)
                    for (int k = 0; k < C; ++k)
                        put_f16split(bq, bq_lo, (size_t)(k / 8) * NQ * 8 + n * 8 + k % 8,
                                  n < h * C ? w->Wq[j][(size_t)k * h * C + n] * qs * log2e
                                            : w->W_beta[(size_t)k * C + (n - h * C)] * qs);
                for (int n = 0; n < C; ++n)
                    for (int k = 0; k < h * C; ++k)
                        put_f16split(bo, bo_lo, (size_t)(k / 8) * C * 8 + n * 8 + k % 8, w->Wo[j][(size_t)k * C + n]);
            }
            ctx->wat_bytes = at.size() * sizeof(uint16_t);
            s = qk_alloc(ctx, &ctx->wat, ctx->wat_bytes);
            if (s != QUARK_OK) return s;
            QK_CUDA(ctx, cudaMemcpy(ctx->wat, at.data(), ctx->wat_bytes, cudaMemcpyHostToDevice));
        }
    } else {
        ctx->wtc_step_bytes = 2 * 9 * (size_t)C * C * sizeof(uint16_t);
        std::vector<uint16_t> tc(ctx->wtc_step_bytes / sizeof(uint16_t) * c.n_scales);
        for (int j = 0; j < c.n_scales; ++j) {
            uint16_t* d = tc.data() + (size_t)j * 2 * 9 * C * C;
            pack_conv_weights_bf16(cw1[j], C, d);
            pack_conv_weights_bf16(cw2[j], C, d + 9 * (size_t)C * C);
        }
        // attention: B_q rows n < hC from Wq[k][n], rows hC.. from W_beta[k][n - hC] (K = C);
        // B_o rows n < C from Wo[k][n] (K = hC); element (n, k) at (k / 8) * N * 8 + n * 8 + k % 8
        // layer collapse of the step (when it has one), after B_o: B_1 rows n < C from col_w1[k][n]
        // (K = 2C), then B_2 from col_w2[k][n] (K = C), same element order.  Every step's block
        // is a multiple of 16 bytes (C is 16 or 32).
        size_t total = 0;
        for (int j = 0; j < c.n_scales; ++j) {
            const int h = qk_heads(c, j);
            ctx->off_wat[j] = total;
            total += (h > 0 ? (size_t)(h * C + C) * C + (size_t)C * h * C : 0) +
                     (ctx->off_collapse[j] != (size_t)-1 ? 3 * (size_t)C * C : 0);
        }
        std::vector<uint16_t> at(std::max<size_t>(total, 8));
        for (int j = 0; j < c.n_scales; ++j) {
            const int h = qk_heads(c, j), NQ = h * C + C;
            uint16_t* bq = at.data() + ctx->off_wat[j];
            uint16_t* bo = bq + (size_t)NQ * C;
            const size_t att_elems = h > 0 ? (size_t)NQ * C + (size_t)C * h * C : 0;
            if (h > 0) {
                // the logit scale 1/sqrt(C) is folded into W^q and W^beta, and for the attention
                // heads also log2(e) (their softmax runs on exp2)
                const double qs = 1.0 / std::sqrt((double)C), log2e = 1.4426950408889634;
                for (int n = 0; n < NQ; ++n)
                    for (int k = 0; k < C; ++k) {
                        const double v = n < h * C ? w->Wq[j][(size_t)k * h * C + n] * qs * log2e
                                                   : w->W_beta[(size_t)k * C + (n - h * C)] * qs;
                        bq[(size_t)(k / 8) * NQ * 8 + n * 8 + k % 8] = to_bf16_bits((float)v);
                    }
                for (int n = 0; n < C; ++n)
                    for (int k = 0; k < h * C; ++k)
                        bo[(size_t)(k / 8) * C * 8 + n * 8 + k % 8] = to_bf16_bits(w->Wo[j][(size_t)k * C + n]);
            }
            if (ctx->off_collapse[j] != (size_t)-1) {
                uint16_t* b1 = bq + att_elems;
                uint16_t* b2 = b1 + 2 * (size_t)C * C;
                for (int n = 0; n < C; ++n) {
                    for (int k = 0; k < 2 * C; ++k)
                        b1[(size_t)(k / 8) * C * 8 + n * 8 + k % 8] = to_bf16_bits(w->col_w1[j][(size_t)k * C + n]);
                    for (int k = 0; k < C; ++k)
                        b2[(size_t)(k / 8) * C * 8 + n * 8 + k % 8] = to_bf16_bits(w->col_w2[j][(size_t)k * C + n]);
                }
            }
        }
        for (int j = 0; j < c.n_scales; ++j) ctx->off_wat[j] *= sizeof(uint16_t);
        qk_free(ctx, ctx->wat, ctx->wat_bytes);
        ctx->wat = nullptr;
        ctx->wat_bytes = at.size() * sizeof(uint16_t);
        s = qk_alloc(ctx, &ctx->wat, ctx->wat_bytes);
        if (s != QUARK_OK) return s;
        QK_CUDA(ctx, cudaMemcpy(ctx->wat, at.data(), ctx->wat_bytes, cudaMemcpyHostToDevice));
        {
            // encoder conv as a tcgen05 B operand: N = C output channels x K = 32 (the 27 taps x
            // input channels in (dy, dx, c_in) order, then zeros), element (n, k) at
            // (k / 8) * C * 8 + n * 8 + k % 8
            std::vector<uint16_t> be((size_t)32 * C, 0);
            for (int n = 0; n < C; ++n)
                for (int k = 0; k < 27; ++k) be[(size_t)(k / 8) * C * 8 + n * 8 + k % 8] = to_bf16_bits(w->enc_w[(size_t)k * C + n]);
            qk_free(ctx, ctx->wenc, ctx->wenc_bytes);
            ctx->wenc = nullptr;
            ctx->wenc_bytes = be.size() * sizeof(uint16_t);
            s = qk_alloc(ctx, &ctx->wenc, ctx->wenc_bytes);
            if (s != QUARK_OK) return s;
            QK_CUDA(ctx, cudaMemcpy(ctx->wenc, be.data(), ctx->wenc_bytes, cudaMemcpyHostToDevice));
        }
        if (c.render_refine) {
            // Update Block convs, per step at j * wtc_step_bytes (steps that render)
            std::vector<uint16_t> up(ctx->wtc_step_bytes / sizeof(uint16_t) * c.n_scales);
            for (int j = 0; j < c.n_scales; ++j) {
                if (!qk_refines(c, j)) continue;
                uint16_t* d = up.data() + (size_t)j * 2 * 9 * C * C;
                pack_conv_weights_bf16(w->upd1_w[j], C, d);
                pack_conv_weights_bf16(w->upd2_w[j], C, d + 9 * (size_t)C * C);
            }
            qk_free(ctx, ctx->wupd, ctx->wupd_bytes);
            ctx->wupd = nullptr;
            ctx->wupd_bytes = up.size() * sizeof(uint16_t);
            s = qk_alloc(ctx, &ctx->wupd, ctx->wupd_bytes);
            if (s != QUARK_OK) return s;
            QK_CUDA(ctx, cudaMemcpy(ctx->wupd, up.data(), ctx->wupd_bytes, cudaMemcpyHostToDevice));
        }
        qk_free(ctx, ctx->wtc, ctx->wtc_bytes);
        ctx->wtc = nullptr;
        ctx->wtc_bytes = tc.size() * sizeof(uint16_t);
        s = qk_alloc(ctx, &ctx->wtc, ctx->wtc_bytes);
        if (s != QUARK_OK) return s;
        QK_CUDA(ctx, cudaMemcpy(ctx->wtc, tc.data(), ctx->wtc_bytes, cudaMemcpyHostToDevice));
    }
    if (!ctx->dev_err) {
        s = qk_alloc(ctx, (void**)&ctx->dev_err, sizeof(int));
        if (s != QUARK_OK) return s;
        QK_CUDA(ctx, cudaMemset(ctx->dev_err, 0, sizeof(int)));
    }
    ctx->weights_loaded = true;
    return QUARK_OK;
}

extern "C" quark_status quark_test_wait_timeout(quark_ctx* ctx) {
    if (!ctx) return qk_fail(nullptr, QUARK_EINVAL, "NULL context");
    if (ctx->cfg.precision != QUARK_BF16 || ctx->cfg.attn_mode != QUARK_ATTN_ONE_TO_MANY)
        return qk_fail(ctx, QUARK_EINVAL, "the wait-timeout test needs the BF16 form with one-to-many attention");
    ctx->test_wait_armed = true;
    return QUARK_OK;
}

extern "C" quark_status quark_check_device(quark_ctx* ctx) {
    if (!ctx) return qk_fail(nullptr, QUARK_EINVAL, "NULL context");
    cudaSetDevice(ctx->device);
    QK_CUDA(ctx, cudaDeviceSynchronize());
    if (!ctx->dev_err) return QUARK_OK;
    int e = 0;
    QK_CUDA(ctx, cudaMemcpy(&e, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        QK_CUDA(ctx, cudaMemset(ctx->dev_err, 0, sizeof(int)));
        return qk_fail(ctx, QUARK_ETIMEDOUT, "a kernel's bounded wait ran out (code %d); its outputs are invalid", e);
    }
    return QUARK_OK;
}

// -------------------------------------------------------------------------------------------
// Cameras and geometry
// -------------------------------------------------------------------------------------------

quark_status qk_validate_camera(const quark_ctx* ctx, const quark_camera& c, const char* what) {
    bool ok = c.width > 0 && c.height > 0 && std::isfinite(c.fx) && std::isfinite(c.fy) && c.fx > 0 && c.fy > 0 &&
              std::isfinite(c.cx) && std::isfinite(c.cy);
    for (int i = 0; i < 9; ++i) ok = ok && std::isfinite(c.R[i]);
    for (int i = 0; i < 3; ++i) ok = ok && std::isfinite(c.t[i]);
    if (!ok) return qk_fail(ctx, QUARK_EINVAL, "%s camera is not a finite pinhole camera", what);
    // R must be a rotation (orthonormal, det +1) to 1e-6
    double rrt[9] = {0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) rrt[3 * i + j] += c.R[3 * i + k] * c.R[3 * j + k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (std::fabs(rrt[3 * i + j] - (i == j ? 1.0 : 0.0)) > 1e-6)
                return qk_fail(ctx, QUARK_EINVAL, "%s camera R is not orthonormal", what);
    return QUARK_OK;
}

// A = K_m R_m R_t^T K_t^-1 and b = K_m (t_m - R_m R_t^T t_t), both grids scaled by 1/k.
// Ray of view pixel (x + 0.5, y + 0.5) on the view's k0-coarser grid in target-camera coordinates:
// direction A p with A = R_t R_m^T K_{m,k0}^-1, origin b = R_t c_m + t_t (c_m = -R_m^T t_m).
ViewMap qk_ray_map(const quark_camera& tgt, const quark_camera& view, double k0) {
    const double Kinv[9] = {k0 / view.fx, 0, -view.cx / view.fx, 0, k0 / view.fy, -view.cy / view.fy, 0, 0, 1};
    double Rrel[9] = {0}, A[9] = {0}, cm[3] = {0}, b[3] = {0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int q = 0; q < 3; ++q) Rrel[3 * i + j] += tgt.R[3 * i + q] * view.R[3 * j + q];  // R_t R_m^T
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int q = 0; q < 3; ++q) A[3 * i + j] += Rrel[3 * i + q] * Kinv[3 * q + j];
    for (int i = 0; i < 3; ++i)
        for (int q = 0; q < 3; ++q) cm[i] -= view.R[3 * q + i] * view.t[q];  // -R_m^T t_m
    for (int i = 0; i < 3; ++i) {
        b[i] = tgt.t[i];
        for (int q = 0; q < 3; ++q) b[i] += tgt.R[3 * i + q] * cm[q];
    }
    ViewMap m;
    for (int i = 0; i < 9; ++i) m.A[i] = (float)A[i];
    for (int i = 0; i < 3; ++i) m.b[i] = (float)b[i];
    return m;
}

ViewMap qk_view_map(const quark_camera& tgt, double k_tx, double k_ty, const quark_camera& view, double k_m) {
    double Kt_inv[9] = {k_tx / tgt.fx, 0, -tgt.cx / tgt.fx, 0, k_ty / tgt.fy, -tgt.cy / tgt.fy, 0, 0, 1};
    double Km[9] = {view.fx / k_m, 0, view.cx / k_m, 0, view.fy / k_m, view.cy / k_m, 0, 0, 1};
    double Rrel[9] = {0};  // R_m R_t^T
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) Rrel[3 * i + j] += view.R[3 * i + k] * tgt.R[3 * j + k];
    double M[9] = {0}, A[9] = {0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) M[3 * i + j] += Km[3 * i + k] * Rrel[3 * k + j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) A[3 * i + j] += M[3 * i + k] * Kt_inv[3 * k + j];
    double tr[3];
    for (int i = 0; i < 3; ++i) {
        tr[i] = view.t[i];
        for (int k = 0; k < 3; ++k) tr[i] -= Rrel[3 * i + k] * tgt.t[k];
    }
    ViewMap vm;
    for (int i = 0; i < 9; ++i) vm.A[i] = (float)A[i];
    for (int i = 0; i < 3; ++i) {
        double b = 0;
        for (int k = 0; k < 3; ++k) b += Km[3 * i + k] * tr[k];
        vm.b[i] = (float)b;
    }
    return vm;
}

// -------------------------------------------------------------------------------------------
// Pyramid
// -------------------------------------------------------------------------------------------

static bool is_device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static void pyramid_free(quark_pyramid* p) {
    quark_ctx* ctx = p->ctx;
    for (int i = 0; i < 4; ++i) qk_free(ctx, p->level[i], p->level_bytes[i]);
    qk_free(ctx, p->rgba, p->rgba_bytes);
    qk_free(ctx, p->staging, p->staging_bytes);
    ctx->live_handles.fetch_sub(1);
    delete p;
}

extern "C" quark_status quark_release_pyramid(quark_pyramid* pyr) {
    if (!pyr) return QUARK_OK;
    cudaSetDevice(pyr->ctx->device);
    pyramid_free(pyr);
    return QUARK_OK;
}


extern "C" quark_status quark_pyramid_read(const quark_pyramid* pyr, int k, void* dst, size_t bytes) {
    if (!pyr || !dst) return qk_fail(nullptr, QUARK_EINVAL, "NULL argument");
    if (k != 1 && k != 2 && k != 4 && k != 8) return qk_fail(pyr->ctx, QUARK_EINVAL, "k must be 1, 2, 4 or 8");
    const int li = level_index(k);
    if (!pyr->level[li]) return qk_fail(pyr->ctx, QUARK_EINVAL, "level %d is not part of this pyramid", k);
    if (bytes != pyr->level_bytes[li])
        return qk_fail(pyr->ctx, QUARK_EINVAL, "level %d holds %zu bytes, %zu given", k, pyr->level_bytes[li], bytes);
    cudaSetDevice(pyr->ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(dst, pyr->level[li], bytes, cudaMemcpyDefault);
    if (e != cudaSuccess) return qk_fail(pyr->ctx, QUARK_ECUDA, "level copy: %s", cudaGetErrorString(e));
    return QUARK_OK;
}

extern "C" quark_status quark_encode_pyramid(quark_ctx* ctx, const float* images, const quark_camera* cams, int V,
                                             void* stream, quark_pyramid** out) {
    if (!ctx || !images || !cams || !out) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (!ctx->weights_loaded) return qk_fail(ctx, QUARK_EINVAL, "weights not loaded");
    if (V < 1 || V > QUARK_MAX_VIEWS) return qk_fail(ctx, QUARK_EINVAL, "V must be 1..%d (got %d)", QUARK_MAX_VIEWS, V);
    for (int m = 0; m < V; ++m) {
        quark_status s = qk_validate_camera(ctx, cams[m], "input");
        if (s != QUARK_OK) return s;
        if (cams[m].width != cams[0].width || cams[m].height != cams[0].height)
            return qk_fail(ctx, QUARK_EINVAL, "all views must share one resolution");
    }
    const int H = cams[0].height, W = cams[0].width;
    const quark_config& c = ctx->cfg;
    for (int j = 0; j < c.n_scales; ++j)
        if (H % c.k[j] || W % c.k[j])
            return qk_fail(ctx, QUARK_EINVAL, "image %dx%d not divisible by k=%d", W, H, c.k[j]);
    quark_pyramid* p = *out;
    if (p && (p->ctx != ctx || p->V != V || p->H != H || p->W != W))
        return qk_fail(ctx, QUARK_EINVAL, "existing pyramid has another context, view count or resolution");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool fresh = p == nullptr;
    quark_status s = QUARK_OK;
    if (fresh) {
        p = new quark_pyramid();
        p->ctx = ctx;
        ctx->live_handles.fetch_add(1);
        p->V = V;
        p->H = H;
        p->W = W;
        const size_t elt = c.precision == QUARK_BF16 ? 2 : 4;
        for (int j = 0; j < c.n_scales && s == QUARK_OK; ++j) {
            int li = level_index(c.k[j]);
            if (p->level[li]) continue;
            p->level_bytes[li] = (size_t)V * (H / c.k[j]) * (W / c.k[j]) * c.C * elt;
            s = qk_alloc(ctx, &p->level[li], p->level_bytes[li]);
        }
        if (s == QUARK_OK) {
            p->rgba_bytes = (size_t)V * H * W * sizeof(float4);
            s = qk_alloc(ctx, &p->rgba, p->rgba_bytes);
        }
    }
    p->cams.assign(cams, cams + V);
    const float* src = images;
    if (s == QUARK_OK && !is_device_pointer(images)) {
        if (!p->staging) {
            p->staging_bytes = (size_t)V * H * W * 3 * sizeof(float);
            s = qk_alloc(ctx, &p->staging, p->staging_bytes);
        }
        if (s == QUARK_OK) {
            cudaError_t e = cudaMemcpyAsync(p->staging, images, p->staging_bytes, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) s = qk_fail(ctx, QUARK_ECUDA, "image upload: %s", cudaGetErrorString(e));
            src = (const float*)p->staging;
        }
    }
    if (s == QUARK_OK) {
        EncodeArgs a{};
        a.images = src;
        a.V = V;
        a.H = H;
        a.W = W;
        a.w = ctx->wdev + ctx->off_enc;
        a.rgba = (float4*)p->rgba;
        for (int i = 0; i < 4; ++i) a.level[i] = p->level[i];
        if (c.precision == QUARK_BF16) {
            // BF16 form: the encoder conv on tcgen05 (BF16 operands, FP32 accumulation)
            bool aligned = true;
            for (int i = 0; i < 4; ++i) aligned = aligned && reinterpret_cast<uintptr_t>(a.level[i]) % 32 == 0;
            s = aligned ? qk_launch(ctx, st, KF_ENCODE,
                                    [&] { return launch_encode_tc(a, c.C, ctx->wenc, ctx->dev_err, st); })
                        : qk_fail(ctx, QUARK_EINTERNAL, "pyramid level not 32-byte aligned");
        } else {
            s = qk_launch(ctx, st, KF_ENCODE, [&] { return launch_encode(a, c.C, false, st); });
        }
    }
    if (s != QUARK_OK) {
        if (fresh) pyramid_free(p);
        return s;
    }
    *out = p;
    return QUARK_OK;
}

// -------------------------------------------------------------------------------------------
// LDM
// -------------------------------------------------------------------------------------------

static void ldm_free(quark_ldm* l) {
    quark_ctx* ctx = l->ctx;
    for (auto& b : l->bufs) {
        if (l->async) cudaFreeAsync(b.p, l->stream);
        else qk_free(ctx, b.p, b.bytes);
    }
    ctx->live_handles.fetch_sub(1);
    delete l;
}

void qk_ldm_free(quark_ldm* l) { ldm_free(l); }

extern "C" quark_status quark_release_ldm(quark_ldm* ldm) {
    if (!ldm) return QUARK_OK;
    cudaSetDevice(ldm->ctx->device);
    ldm_free(ldm);
    return QUARK_OK;
}

static quark_status ldm_buf(quark_ldm* l, void** p, size_t bytes);

// A scratch buffer of the LDM that grows on demand (the superseded one is freed with the LDM).
quark_status qk_ldm_scratch(quark_ldm* l, void** p, size_t bytes) { return ldm_buf(l, p, bytes); }

static quark_status ldm_buf(quark_ldm* l, void** p, size_t bytes) {
    quark_status s;
    if (l->async) {
        *p = nullptr;
        cudaError_t e = cudaMallocAsync(p, bytes, l->stream);
        s = e == cudaSuccess ? QUARK_OK
                             : qk_fail(l->ctx, QUARK_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
        if (e != cudaSuccess) cudaGetLastError();
    } else {
        s = qk_alloc(l->ctx, p, bytes);
    }
    if (s == QUARK_OK) l->bufs.push_back({*p, bytes});
    return s;
}

// Buffer sizes of an LDM for a width x height target: the largest volume, collapse input and
// element count over the steps, the last step's element count, and whether a step reuses depths.
struct LdmSizes {
    size_t vmax = 0, cmax = 0, emax = 0, last_e = 0;
    bool reuse = false;
};
static LdmSizes ldm_sizes(const quark_config& c, int width, int height) {
    const size_t elt = c.precision == QUARK_BF16 ? 2 : 4;
    LdmSizes z;
    for (int j = 0; j < c.n_scales; ++j) {
        int H, W;
        qk_grid(c, j, width, height, H, W);
        const size_t e = (size_t)c.L[j] * H * W;
        z.emax = std::max(z.emax, e);
        z.vmax = std::max(z.vmax, e * c.C * elt);
        if (j > 0 && c.L[j - 1] == 2 * c.L[j]) {
            int Hp, Wp;
            qk_grid(c, j - 1, width, height, Hp, Wp);
            z.cmax = std::max(z.cmax, (size_t)c.L[j] * Hp * Wp * c.C * elt);
        }
        z.reuse = z.reuse || c.reuse_depth[j];
        z.last_e = e;
    }
    return z;
}

// Bytes an LDM for `target` holds (three volumes, collapse buffer, decoded attributes, reused
// depths, blend logits for V views, and a host-output staging buffer when host_out).
size_t qk_ldm_bytes(const quark_config& c, int width, int height, int V, bool host_out) {
    const LdmSizes z = ldm_sizes(c, width, height);
    return 3 * z.vmax + z.cmax + z.emax * (z.reuse ? 8 : 7) * sizeof(float) + z.last_e * V * sizeof(float) +
           (host_out ? (size_t)width * height * 16 : 0);
}

extern "C" quark_status quark_ldm_create(quark_ctx* ctx, const quark_camera* target, quark_ldm** out) {
    return qk_ldm_create(ctx, target, 0, nullptr, out);
}

// LDM for `target`.  With a non-NULL `async_stream` every buffer comes from the stream-ordered
// allocator on that stream (no device-wide synchronisation) and the blend logits are sized for
// V_beta views up front.
quark_status qk_ldm_create(quark_ctx* ctx, const quark_camera* target, int V_beta, cudaStream_t async_stream,
                           quark_ldm** out) {
    if (!ctx || !target || !out) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    *out = nullptr;
    quark_status s = qk_validate_camera(ctx, *target, "target");
    if (s != QUARK_OK) return s;
    const quark_config& c = ctx->cfg;
    int Hs[QUARK_MAX_SCALES], Ws[QUARK_MAX_SCALES];
    for (int j = 0; j < c.n_scales; ++j)
        if (!qk_grid(c, j, target->width, target->height, Hs[j], Ws[j]))
            return qk_fail(ctx, QUARK_EINVAL, "output %dx%d not divisible by the grid factor %g of step %d", target->width,
                           target->height, qk_f(c, j), j);
    cudaSetDevice(ctx->device);
    quark_ldm* l = new quark_ldm();
    l->ctx = ctx;
    ctx->live_handles.fetch_add(1);
    l->target = *target;
    l->async = async_stream != nullptr;
    l->stream = async_stream;
    for (int j = 0; j < c.n_scales; ++j) {
        l->Hs[j] = Hs[j];
        l->Ws[j] = Ws[j];
    }
    const LdmSizes z = ldm_sizes(c, target->width, target->height);
    const size_t vmax = z.vmax, cmax = z.cmax, emax = z.emax, last_e = z.last_e;
    s = ldm_buf(l, &l->vol[0], vmax);
    if (s == QUARK_OK) s = ldm_buf(l, &l->vol[1], vmax);
    if (s == QUARK_OK) s = ldm_buf(l, &l->vattn, vmax);
    if (s == QUARK_OK && cmax) s = ldm_buf(l, &l->collapsed, cmax);
    if (s == QUARK_OK) s = ldm_buf(l, (void**)&l->colour, emax * 3 * sizeof(float));
    if (s == QUARK_OK) s = ldm_buf(l, (void**)&l->alpha, emax * sizeof(float));
    if (s == QUARK_OK) s = ldm_buf(l, (void**)&l->depth, emax * sizeof(float));
    if (s == QUARK_OK) s = ldm_buf(l, (void**)&l->t_raw, emax * sizeof(float));
    if (s == QUARK_OK) s = ldm_buf(l, (void**)&l->s_raw, emax * sizeof(float));
    if (s == QUARK_OK && z.reuse) s = ldm_buf(l, (void**)&l->dsamp, emax * sizeof(float));
    l->last_e = last_e;
    if (s == QUARK_OK && V_beta > 0) {
        s = ldm_buf(l, (void**)&l->beta, last_e * V_beta * sizeof(float));
        l->beta_bytes = last_e * V_beta * sizeof(float);
    }
    if (s != QUARK_OK) {
        ldm_free(l);
        return s;
    }
    *out = l;
    return QUARK_OK;
}

static void step_dims(const quark_ldm* l, int j, int& L, int& H, int& W) {
    L = l->ctx->cfg.L[j];
    H = l->Hs[j];
    W = l->Ws[j];
}

extern "C" quark_status quark_update_fuse(quark_ctx* ctx, const quark_pyramid* pyr, int scale, quark_ldm* ldm,
                                          void* stream) {
    if (!pyr) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    return qk_update_fuse(ctx, pyr, pyr->V, scale, ldm, (cudaStream_t)stream);
}

// Grow an LDM scratch buffer to at least `bytes`.
static quark_status grow_scratch(quark_ldm* l, void** p, size_t& have, size_t bytes) {
    if (have >= bytes) return QUARK_OK;
    for (auto it = l->bufs.begin(); it != l->bufs.end(); ++it)
        if (it->p == *p) {
            qk_free(l->ctx, it->p, it->bytes);
            l->bufs.erase(it);
            break;
        }
    *p = nullptr;
    have = 0;
    quark_status s = qk_ldm_scratch(l, p, bytes);
    if (s == QUARK_OK) have = bytes;
    return s;
}

// Render-and-refine of step `scale` (Sec. 3.2.2, Eq. overcomposite-result, the Update Block): the
// volume entering the step (`prev`, on step scale-1's Hp x Wp grid, already collapsed) decoded,
// splatted into the first V views at step scale-1's level and over-composited there; then
// Delta = F' + Conv(gelu(Conv(N(F')))), F' = F + up(I~) W_r + b_r, from the level-k features
// `feat`, into ldm->delta.
static quark_status refine_step(quark_ctx* ctx, const quark_pyramid* pyr, int V, int scale, quark_ldm* ldm,
                                const void* prev, int Hp, int Wp, const void* feat, cudaStream_t st) {
    const quark_config& c = ctx->cfg;
    const bool bf16 = c.precision == QUARK_BF16;
    const int C = c.C, L = c.L[scale], kp = c.k[scale - 1], k = c.k[scale];
    const int hr = pyr->H / kp, wr = pyr->W / kp, h = pyr->H / k, w = pyr->W / k;
    const DepthParams dp{(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
    // scratch: splat sums (float4) and weights, the rendered views, the Update Block's input and output
    const size_t ns = (size_t)V * L * hr * wr;
    const size_t off_w = ns * sizeof(float4);
    const size_t off_r = (off_w + ns * sizeof(float) + 255) & ~(size_t)255;
    const size_t splat_bytes = off_r + (size_t)V * hr * wr * sizeof(float4);
    const size_t feat_bytes = (size_t)V * h * w * C * (bf16 ? 2 : 4);
    quark_status s = grow_scratch(ldm, &ldm->splat, ldm->splat_bytes, splat_bytes);
    if (s == QUARK_OK) s = grow_scratch(ldm, &ldm->upd_in, ldm->upd_in_bytes, feat_bytes);
    if (s == QUARK_OK) s = grow_scratch(ldm, &ldm->delta, ldm->delta_bytes, feat_bytes);
    if (s != QUARK_OK) return s;
    // intermediate LDM, activated (the LDM's decoded-attribute buffers; recomputed when read)
    DecodeArgs da{};
    da.vol = prev;
    da.L = L;
    da.H = Hp;
    da.W = Wp;
    da.dp = dp;
    da.w = ctx->wdev + ctx->off_conv[scale];
    da.colour = ldm->colour;
    da.alpha = ldm->alpha;
    da.depth = ldm->depth;
    ldm->decoded = -1;
    s = qk_launch(ctx, st, KF_REFINE, [&] { return launch_decode(da, C, bf16, st); });
    if (s != QUARK_OK) return s;
    SplatArgs sa{};
    sa.colour = ldm->colour;
    sa.alpha = ldm->alpha;
    sa.depth = ldm->depth;
    sa.L = L;
    sa.H = Hp;
    sa.W = Wp;
    sa.V = V;
    sa.h = hr;
    sa.w = wr;
    sa.acc = (float4*)ldm->splat;
    sa.wsum = (float*)((uint8_t*)ldm->splat + off_w);
    sa.out = (float4*)((uint8_t*)ldm->splat + off_r);
    for (int m = 0; m < V; ++m)
        sa.geo.v[m] = qk_view_map(ldm->target, (double)ldm->target.width / Wp, (double)ldm->target.height / Hp,
                                  pyr->cams[m], kp);
    QK_CUDA(ctx, cudaMemsetAsync(ldm->splat, 0, off_w + ns * sizeof(float), st));
    s = qk_launch(ctx, st, KF_REFINE, [&] { return launch_splat(sa, st); });
    if (s == QUARK_OK) s = qk_launch(ctx, st, KF_REFINE, [&] { return launch_composite_views(sa, st); });
    if (s != QUARK_OK) return s;
    RefineArgs ra{};
    ra.feat = feat;
    ra.rend = sa.out;
    ra.V = V;
    ra.C = C;
    ra.h = h;
    ra.w = w;
    ra.hr = hr;
    ra.wr = wr;
    ra.ratio = kp / k;
    ra.wr_b = ctx->wdev + ctx->off_upd[scale] + ConvLayout{C}.total();
    ra.out = ldm->upd_in;
    s = qk_launch(ctx, st, KF_REFINE, [&] { return launch_refine_add(ra, bf16, st); });
    if (s != QUARK_OK) return s;
    // the Update Block's residual CNN block on the V view planes
    ConvArgs cv{};
    cv.in = ldm->upd_in;
    cv.out = ldm->delta;
    cv.L = V;
    cv.H = h;
    cv.W = w;
    cv.dp = dp;
    cv.w = ctx->wdev + ctx->off_upd[scale];
    cv.wtc = ctx->wupd ? (const uint8_t*)ctx->wupd + scale * ctx->wtc_step_bytes : nullptr;
    cv.err = ctx->dev_err;
    s = qk_launch(ctx, st, KF_REFINE, [&] { return launch_conv_block(cv, C, bf16, st); });
    if (s != QUARK_OK) return s;
    ldm->delta_ok = true;
    return QUARK_OK;
}

// Whether the next step after `j` that samples the views reuses the depths step j samples at.
static bool next_reuses(const quark_config& c, int j) {
    for (int i = j + 1; i < c.n_scales; ++i)
        if (qk_heads(c, i) > 0) return c.reuse_depth[i] != 0;
    return false;
}

// One Update & Fuse step using the first V_use views of the pyramid.
quark_status qk_update_fuse(quark_ctx* ctx, const quark_pyramid* pyr, int V_use, int scale, quark_ldm* ldm,
                            cudaStream_t stream, const void* prev_override, const void* feat_override) {
    if (!ctx || !pyr || !ldm) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (V_use < 1 || V_use > pyr->V) return qk_fail(ctx, QUARK_EINVAL, "view count %d outside 1..%d", V_use, pyr->V);
    if (pyr->ctx != ctx || ldm->ctx != ctx) return qk_fail(ctx, QUARK_EINVAL, "handle from another context");
    const quark_config& c = ctx->cfg;
    if (scale < 0 || scale >= c.n_scales) return qk_fail(ctx, QUARK_EINVAL, "scale %d out of range", scale);
    if (scale != 0 && ldm->done != scale - 1 && !prev_override)
        return qk_fail(ctx, QUARK_EINVAL, "step %d needs step %d first (latest done: %d)", scale, scale - 1, ldm->done);
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream;
    const bool bf16 = c.precision == QUARK_BF16;
    const bool last = scale == c.n_scales - 1;
    int L, H, W;
    step_dims(ldm, scale, L, H, W);
    const int k = c.k[scale];
    const int heads = qk_heads(c, scale);
    quark_status s;

    if (last) {
        size_t need = ldm->last_e * V_use * sizeof(float);
        if (ldm->beta_bytes < need) {
            for (auto it = ldm->bufs.begin(); it != ldm->bufs.end(); ++it)
                if (it->p == ldm->beta) {
                    qk_free(ctx, it->p, it->bytes);
                    ldm->bufs.erase(it);
                    break;
                }
            ldm->beta = nullptr;
            s = ldm_buf(ldm, (void**)&ldm->beta, need);
            if (s != QUARK_OK) return s;
            ldm->beta_bytes = need;
        }
        ldm->V = V_use;
    }

    // ---- transition ----
    const void* prev = nullptr;
    int Hp = 0, Wp = 0;
    Transition tr = TR_INIT;
    if (prev_override) {
        prev = prev_override;  // the volume entering the step, given on the step's own grid
        Hp = H;
        Wp = W;
        tr = TR_SAME;
    } else if (scale > 0) {
        int Lp;
        step_dims(ldm, scale - 1, Lp, Hp, Wp);
        prev = ldm->vol[ldm->cur];
        if (Lp == 2 * L) {
            CollapseArgs ca{};
            ca.in = prev;
            ca.out = ldm->collapsed;
            ca.L = L;
            ca.H = Hp;
            ca.W = Wp;
            ca.w = ctx->wdev + ctx->off_collapse[scale];
            ca.wtc = qk_collapse_wtc(ctx, scale);
            ca.err = ctx->dev_err;
            s = qk_launch(ctx, st, KF_COLLAPSE, [&] { return launch_collapse(ca, c.C, bf16, st); });
            if (s != QUARK_OK) return s;
            prev = ldm->collapsed;
        }
        tr = ldm->Hs[scale] == Hp ? TR_SAME : TR_UP2;  // the grid keeps its size or doubles
    }

    // ---- sample-attend ----
    if (heads > 0) {
        AttendArgs aa{};
        aa.prev = prev;
        aa.Hp = Hp;
        aa.Wp = Wp;
        aa.feat = feat_override ? feat_override : pyr->level[level_index(k)];
        aa.fh = pyr->H / k;
        aa.fw = pyr->W / k;
        aa.L = L;
        aa.H = H;
        aa.W = W;
        aa.V = V_use;
        aa.dp = {(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
        aa.w = ctx->wdev + ctx->off_attend[scale];
        aa.out = ldm->vattn;
        aa.beta = last ? ldm->beta : nullptr;
        aa.wtc = ctx->wat ? (const uint8_t*)ctx->wat + ctx->off_wat[scale] : nullptr;
        aa.err = ctx->dev_err;
        for (int m = 0; m < V_use; ++m)
            aa.geo.v[m] = qk_view_map(ldm->target, (double)ldm->target.width / W, (double)ldm->target.height / H,
                                      pyr->cams[m], k);
        // reused depths (Update & Fuse steps with several fusion blocks sample once)
        aa.depth_in = c.reuse_depth[scale] ? ldm->dsamp : nullptr;
        aa.depth_out = !c.reuse_depth[scale] && next_reuses(c, scale) ? ldm->dsamp : nullptr;
        // render-and-refine: this step renders the views and forms new update features, or it
        // reuses those of its Update & Fuse step
        const bool refining = qk_refines(c, scale) && !prev_override;
        if (!c.reuse_depth[scale] && !refining) ldm->delta_ok = false;
        const bool from_delta = c.render_refine && (refining || ldm->delta_ok);
        if (c.ray_encoding && !(from_delta && !refining)) {
            // gamma_k (Sec. 3.2.1) added to this level of the first V_use views, into LDM scratch
            int k0 = 1;
            for (int j = 0; j < c.n_scales; ++j) k0 = std::max(k0, c.k[j]);
            RayArgs ra{};
            ra.V = V_use;
            ra.C = c.C;
            ra.h0 = pyr->H / k0;
            ra.w0 = pyr->W / k0;
            ra.h = aa.fh;
            ra.w = aa.fw;
            ra.ratio = k0 / k;
            ra.span = (float)(1.0 / c.near_m - 1.0 / c.far_m);
            ra.w_ray = ctx->wdev + ctx->off_ray[level_index(k)];
            for (int m = 0; m < V_use; ++m) ra.geo.v[m] = qk_ray_map(ldm->target, pyr->cams[m], k0);
            const size_t gbytes = (size_t)V_use * ra.h0 * ra.w0 * c.C * sizeof(float);
            const size_t fbytes = (size_t)V_use * ra.h * ra.w * c.C * (bf16 ? 2 : 4);
            if (ldm->ray_g_bytes < gbytes) {
                s = qk_ldm_scratch(ldm, (void**)&ldm->ray_g, gbytes);
                if (s != QUARK_OK) return s;
                ldm->ray_g_bytes = gbytes;
            }
            if (ldm->ray_feat_bytes < fbytes) {
                s = qk_ldm_scratch(ldm, &ldm->ray_feat, fbytes);
                if (s != QUARK_OK) return s;
                ldm->ray_feat_bytes = fbytes;
            }
            ra.g = ldm->ray_g;
            const void* level = aa.feat;
            s = qk_launch(ctx, st, KF_ATTEND, [&] { return launch_ray_coarse(ra, st); });
            if (s == QUARK_OK)
                s = qk_launch(ctx, st, KF_ATTEND, [&] { return launch_ray_add(ra, level, ldm->ray_feat, bf16, st); });
            if (s != QUARK_OK) return s;
            aa.feat = ldm->ray_feat;
        }
        if (refining) {
            s = refine_step(ctx, pyr, V_use, scale, ldm, prev, Hp, Wp, aa.feat, st);
            if (s != QUARK_OK) return s;
        }
        if (from_delta) aa.feat = ldm->delta;
        if (c.attn_mode == QUARK_ATTN_STANDARD) {
            // keys and values (and on the last step the features) projected in image space, then sampled
            const size_t texels = (size_t)V_use * aa.fh * aa.fw;
            const size_t need = texels * (size_t)(last ? 3 : 2) * c.C * (bf16 ? 2 : 4);
            if (ldm->kv_bytes < need) {
                s = qk_ldm_scratch(ldm, &ldm->kv, need);
                if (s != QUARK_OK) return s;
                ldm->kv_bytes = need;
            }
            const float* wkv = ctx->wdev + ctx->off_std[scale] + StdLayout{c.C}.wkv();
            const void* level = aa.feat;
            s = qk_launch(ctx, st, KF_ATTEND,
                          [&] { return launch_kv_project(level, texels, c.C, wkv, ldm->kv, last, bf16, st); });
            if (s != QUARK_OK) return s;
            aa.feat = ldm->kv;
            aa.w_std = ctx->wdev + ctx->off_std[scale];
            s = qk_launch(ctx, st, KF_ATTEND, [&] { return launch_attend_std(aa, c.C, heads, tr, last, bf16, st); });
        } else {
            if (ctx->test_wait_armed && bf16) {
                aa.test_wait_ns = 1000000;  // 1 ms: the test's wait runs out at once, not after 1 s
                ctx->test_wait_armed = false;
            }
            s = qk_launch(ctx, st, KF_ATTEND, [&] { return launch_attend(aa, c.C, heads, tr, last, bf16, st); });
        }
        if (s != QUARK_OK) return s;
    }

    // ---- conv block + decode ----
    ConvArgs ca{};
    ca.in = heads > 0 ? ldm->vattn : prev;  // a block without attention: the conv block on V_in
    ca.out = ldm->vol[1 - ldm->cur];
    ca.L = L;
    ca.H = H;
    ca.W = W;
    ca.dp = {(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
    ca.w = ctx->wdev + ctx->off_conv[scale];
    // the raw depth / density logits are written here for the step that is rendered; every other
    // decoded attribute is produced on demand (qk_decode) when it is read
    ca.t_raw = last ? ldm->t_raw : nullptr;
    ca.s_raw = last ? ldm->s_raw : nullptr;
    ca.wtc = ctx->wtc ? (const uint8_t*)ctx->wtc + scale * ctx->wtc_step_bytes : nullptr;
    ca.err = ctx->dev_err;
    ca.ks = c.conv_kernel == 1 ? 1 : 3;
    s = qk_launch(ctx, st, KF_CONV, [&] { return launch_conv_block(ca, c.C, bf16, st); });
    if (s != QUARK_OK) return s;
    if (ldm->keep) {
        // the step's volumes, kept for quark_update_fuse_bwd
        const size_t bytes = (size_t)L * H * W * c.C * (bf16 ? 2 : 4);
        if (!ldm->hist_out[scale] && (s = ldm_buf(ldm, &ldm->hist_out[scale], bytes)) != QUARK_OK) return s;
        if (!ldm->hist_attn[scale] && (s = ldm_buf(ldm, &ldm->hist_attn[scale], bytes)) != QUARK_OK) return s;
        cudaError_t e = cudaMemcpyAsync(ldm->hist_out[scale], ca.out, bytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ldm->hist_attn[scale], ca.in, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return qk_fail(ctx, QUARK_ECUDA, "keeping step %d's volumes: %s", scale, cudaGetErrorString(e));
    }
    ldm->cur = 1 - ldm->cur;
    ldm->done = scale;
    ldm->decoded = -1;
    return QUARK_OK;
}

// Decoded attributes (colour, alpha, depth, raw logits) of step `scale` from its stored volume.
quark_status qk_decode(quark_ctx* ctx, int scale, const void* vol, int L, int H, int W, float* colour, float* alpha,
                       float* depth, float* t_raw, float* s_raw, cudaStream_t st) {
    const quark_config& c = ctx->cfg;
    DecodeArgs da{};
    da.vol = vol;
    da.L = L;
    da.H = H;
    da.W = W;
    da.dp = {(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
    da.w = ctx->wdev + ctx->off_conv[scale];
    da.colour = colour;
    da.alpha = alpha;
    da.depth = depth;
    da.t_raw = t_raw;
    da.s_raw = s_raw;
    return qk_launch(ctx, st, KF_CONV, [&] { return launch_decode(da, c.C, c.precision == QUARK_BF16, st); });
}

// Packed collapse weights of step `scale`: BF16 (after the step's attention packs), or the FP32
// form's split parts; NULL where the step has none (or the FP32 form keeps the SIMT kernel).
const void* qk_collapse_wtc(const quark_ctx* ctx, int scale) {
    if (ctx->cfg.precision != QUARK_BF16)
        return ctx->wcol && ctx->off_collapse[scale] != (size_t)-1 ? (const uint8_t*)ctx->wcol + ctx->off_wcol[scale]
                                                                    : nullptr;
    if (!ctx->wat) return nullptr;
    const quark_config& c = ctx->cfg;
    const int h = qk_heads(c, scale);
    const size_t att_bytes = h > 0 ? ((size_t)(h * c.C + c.C) * c.C + (size_t)c.C * h * c.C) * 2 : 0;
    return (const uint8_t*)ctx->wat + ctx->off_wat[scale] + att_bytes;
}

extern "C" quark_status quark_render_ldm(quark_ctx* ctx, const quark_ldm* ldm, const quark_pyramid* pyr, float* rgba,
                                         void* stream) {
    if (!ldm || !pyr) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    return qk_render(ctx, ldm, pyr, ldm->V, rgba, is_device_pointer(rgba) ? 0 : 1, (cudaStream_t)stream);
}

// Final render from the first V_use views; host_out: rgba is host memory (copied out on the stream).
quark_status qk_render(quark_ctx* ctx, const quark_ldm* ldm, const quark_pyramid* pyr, int V_use, float* rgba,
                       int host_out, cudaStream_t stream) {
    if (!ctx || !ldm || !pyr || !rgba) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    const quark_config& c = ctx->cfg;
    if (ldm->done != c.n_scales - 1) return qk_fail(ctx, QUARK_EINVAL, "render needs every Update & Fuse step first");
    if (ldm->V != V_use || V_use > pyr->V)
        return qk_fail(ctx, QUARK_EINVAL, "render uses %d views; the LDM was solved with %d", V_use, ldm->V);
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream;
    quark_ldm* l = const_cast<quark_ldm*>(ldm);
    const int n = c.n_scales - 1;
    RenderArgs ra{};
    ra.t_raw = l->t_raw;
    ra.s_raw = l->s_raw;
    ra.beta = l->beta;
    ra.rgba = (const float4*)pyr->rgba;
    ra.L = c.L[n];
    ra.V = V_use;
    ra.Hl = l->Hs[n];
    ra.Wl = l->Ws[n];
    ra.sx = (float)((double)l->target.width / l->Ws[n]);
    ra.sy = (float)((double)l->target.height / l->Hs[n]);
    ra.Hout = l->target.height;
    ra.Wout = l->target.width;
    ra.Hi = pyr->H;
    ra.Wi = pyr->W;
    ra.dp = {(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
    for (int m = 0; m < V_use; ++m) ra.geo.v[m] = qk_view_map(l->target, 1.0, 1.0, pyr->cams[m], 1.0);
    const size_t out_bytes = (size_t)ra.Hout * ra.Wout * sizeof(float4);
    if (host_out && l->out_bytes < out_bytes) {
        for (auto it = l->bufs.begin(); it != l->bufs.end(); ++it)
            if (it->p == l->out) {
                qk_free(ctx, it->p, it->bytes);
                l->bufs.erase(it);
                break;
            }
        l->out = nullptr;
        quark_status s = ldm_buf(l, &l->out, out_bytes);
        if (s != QUARK_OK) return s;
        l->out_bytes = out_bytes;
    }
    ra.out = host_out ? (float4*)l->out : (float4*)rgba;
    quark_status s = qk_launch(ctx, st, KF_RENDER, [&] { return launch_render(ra, st); });
    if (s != QUARK_OK) return s;
    if (host_out) QK_CUDA(ctx, cudaMemcpyAsync(rgba, l->out, out_bytes, cudaMemcpyDeviceToHost, st));
    return QUARK_OK;
}

extern "C" quark_status quark_render_depth(quark_ctx* ctx, const quark_ldm* ldm, float* depth, void* stream) {
    if (!ctx || !ldm || !depth) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (ldm->ctx != ctx) return qk_fail(ctx, QUARK_EINVAL, "LDM from another context");
    const quark_config& c = ctx->cfg;
    if (ldm->done != c.n_scales - 1) return qk_fail(ctx, QUARK_EINVAL, "the depth map needs every Update & Fuse step first");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    quark_ldm* l = const_cast<quark_ldm*>(ldm);
    const int n = c.n_scales - 1;
    RenderArgs ra{};
    ra.t_raw = l->t_raw;
    ra.s_raw = l->s_raw;
    ra.L = c.L[n];
    ra.Hl = l->Hs[n];
    ra.Wl = l->Ws[n];
    ra.sx = (float)((double)l->target.width / l->Ws[n]);
    ra.sy = (float)((double)l->target.height / l->Hs[n]);
    ra.Hout = l->target.height;
    ra.Wout = l->target.width;
    ra.dp = {(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
    const bool host_out = !is_device_pointer(depth);
    const size_t bytes = (size_t)ra.Hout * ra.Wout * sizeof(float);
    float* dst = depth;
    if (host_out) {
        // the render's host-output staging buffer (RGBA-sized, so large enough)
        const size_t need = (size_t)ra.Hout * ra.Wout * sizeof(float4);
        if (l->out_bytes < need) {
            for (auto it = l->bufs.begin(); it != l->bufs.end(); ++it)
                if (it->p == l->out) {
                    qk_free(ctx, it->p, it->bytes);
                    l->bufs.erase(it);
                    break;
                }
            l->out = nullptr;
            quark_status s = ldm_buf(l, &l->out, need);
            if (s != QUARK_OK) return s;
            l->out_bytes = need;
        }
        dst = (float*)l->out;
    }
    quark_status s = qk_launch(ctx, st, KF_RENDER, [&] { return launch_render_depth(ra, dst, st); });
    if (s != QUARK_OK) return s;
    if (host_out) QK_CUDA(ctx, cudaMemcpyAsync(depth, dst, bytes, cudaMemcpyDeviceToHost, st));
    return QUARK_OK;
}

extern "C" quark_status quark_render_novel_view(quark_ctx* ctx, const quark_pyramid* pyr, quark_ldm* ldm, float* rgba,
                                                void* stream) {
    if (!ctx) return qk_fail(nullptr, QUARK_EINVAL, "NULL context");
    for (int j = 0; j < ctx->cfg.n_scales; ++j) {
        quark_status s = quark_update_fuse(ctx, pyr, j, ldm, stream);
        if (s != QUARK_OK) return s;
    }
    return quark_render_ldm(ctx, ldm, pyr, rgba, stream);
}

// -------------------------------------------------------------------------------------------
// Inspection
// -------------------------------------------------------------------------------------------

extern "C" size_t quark_ldm_field_bytes(const quark_ldm* l, int field) {
    if (!l || l->done < 0) return 0;
    int L, H, W;
    step_dims(l, l->done, L, H, W);
    const size_t e = (size_t)L * H * W;
    switch (field) {
        case QUARK_FIELD_VOLUME:
        case QUARK_FIELD_VOLUME_ATTN: return e * l->ctx->cfg.C * sizeof(float);
        case QUARK_FIELD_COLOUR: return e * 3 * sizeof(float);
        case QUARK_FIELD_ALPHA:
        case QUARK_FIELD_DEPTH:
        case QUARK_FIELD_DEPTH_LOGIT:
        case QUARK_FIELD_DENSITY_LOGIT: return e * sizeof(float);
        case QUARK_FIELD_BETA_LOGITS: return l->done == l->ctx->cfg.n_scales - 1 ? e * l->V * sizeof(float) : 0;
        default: return 0;
    }
}

extern "C" quark_status quark_ldm_read(quark_ldm* l, int field, void* dst, size_t bytes) {
    if (!l || !dst) return qk_fail(l ? l->ctx : nullptr, QUARK_EINVAL, "NULL argument");
    quark_ctx* ctx = l->ctx;
    size_t need = quark_ldm_field_bytes(l, field);
    if (need == 0 || need != bytes) return qk_fail(ctx, QUARK_EINVAL, "field %d: %zu bytes expected, %zu given", field, need, bytes);
    cudaSetDevice(ctx->device);
    QK_CUDA(ctx, cudaDeviceSynchronize());
    const bool decoded_field = field == QUARK_FIELD_COLOUR || field == QUARK_FIELD_ALPHA || field == QUARK_FIELD_DEPTH ||
                               field == QUARK_FIELD_DEPTH_LOGIT || field == QUARK_FIELD_DENSITY_LOGIT;
    if (decoded_field && l->decoded != l->done) {
        int L, H, W;
        step_dims(l, l->done, L, H, W);
        quark_status s = qk_decode(ctx, l->done, l->vol[l->cur], L, H, W, l->colour, l->alpha, l->depth, l->t_raw,
                                   l->s_raw, nullptr);
        if (s != QUARK_OK) return s;
        QK_CUDA(ctx, cudaDeviceSynchronize());
        l->decoded = l->done;
    }
    const void* src = nullptr;
    switch (field) {
        case QUARK_FIELD_VOLUME: src = l->vol[l->cur]; break;
        case QUARK_FIELD_VOLUME_ATTN:
            // a block without attention leaves V_attn = V_in: the step's input, still in the other buffer
            src = qk_heads(ctx->cfg, l->done) > 0 ? l->vattn : l->vol[1 - l->cur];
            break;
        case QUARK_FIELD_COLOUR: src = l->colour; break;
        case QUARK_FIELD_ALPHA: src = l->alpha; break;
        case QUARK_FIELD_DEPTH: src = l->depth; break;
        case QUARK_FIELD_BETA_LOGITS: src = l->beta; break;
        case QUARK_FIELD_DEPTH_LOGIT: src = l->t_raw; break;
        case QUARK_FIELD_DENSITY_LOGIT: src = l->s_raw; break;
    }
    const bool vol = field == QUARK_FIELD_VOLUME || field == QUARK_FIELD_VOLUME_ATTN;
    if (vol && ctx->cfg.precision == QUARK_BF16) {
        const size_t n = bytes / sizeof(float);
        std::vector<uint16_t> tmp(n);
        QK_CUDA(ctx, cudaMemcpy(tmp.data(), src, n * 2, cudaMemcpyDeviceToHost));
        float* f = (float*)dst;
        for (size_t i = 0; i < n; ++i) {
            uint32_t u = (uint32_t)tmp[i] << 16;
            std::memcpy(&f[i], &u, 4);
        }
    } else {
        QK_CUDA(ctx, cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    }
    return QUARK_OK;
}
