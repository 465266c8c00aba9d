// quark_update_fuse_noalloc: one Update & Fuse step that allocates no device memory.
//
// The regular step (quark_update_fuse) keeps its intermediate buffers -- the volume after the
// attention block and, where the layer count halves, the collapsed volume -- in memory the
// library allocates for the LDM handle.  This variant takes every input and output from the
// caller and keeps those two intermediates in one fixed, file-scope device array instead, so
// the call itself never allocates.  It launches the same kernels as the regular step, and the
// attribute decode that the regular step runs when its decoded attributes are read.
#include <cmath>
#include <mutex>

#include "quark_internal.cuh"
#include "api_internal.h"

using namespace quark;

// The shared scratch.  Every GPU that loads this library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QUARK_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The array's name is only a
// host-side stand-in for the symbol, so its device address is looked up once per device with
// that device current, and the looked-up pointer is what the kernels receive.
quark_status scratch_address(const quark_ctx* ctx, int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return qk_fail(ctx, QUARK_EINVAL, "device %d beyond the scratch table", dev);
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return qk_fail(ctx, QUARK_ECUDA, "cudaGetSymbolAddress(static scratch) on device %d: %s", dev,
                           cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return QUARK_OK;
}

size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }

// A caller buffer must be device (or managed) memory of the context's device: the kernels
// dereference it.  cudaPointerGetAttributes allocates nothing; host memory (pageable or pinned)
// and memory of another device are refused before any launch.
quark_status check_device_buffer(const quark_ctx* ctx, const void* p, const char* what) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return qk_fail(ctx, QUARK_EINVAL, "%s is not a device pointer", what);
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return qk_fail(ctx, QUARK_EINVAL, "%s must be device memory (got host memory)", what);
    if (at.device != ctx->device)
        return qk_fail(ctx, QUARK_EINVAL, "%s is memory of device %d, the context runs on device %d", what, at.device,
                       ctx->device);
    return QUARK_OK;
}
}  // namespace

extern "C" quark_status quark_update_fuse_noalloc(quark_ctx* ctx, const quark_pyramid* pyr, int scale,
                                                  const quark_camera* target, const void* v_prev, void* v_out,
                                                  float* colour, float* alpha, float* depth, float* t_raw,
                                                  float* s_raw, float* beta, void* stream) {
    if (!ctx || !pyr || !target || !v_out || !colour || !alpha || !depth || !t_raw || !s_raw)
        return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (pyr->ctx != ctx) return qk_fail(ctx, QUARK_EINVAL, "pyramid from another context");
    if (ctx->cfg.attn_mode != QUARK_ATTN_ONE_TO_MANY)
        return qk_fail(ctx, QUARK_EINVAL, "the no-alloc step runs one-to-many attention only (use quark_update_fuse)");
    if (ctx->cfg.ray_encoding)
        return qk_fail(ctx, QUARK_EINVAL, "the no-alloc step runs without the ray encoding (use quark_update_fuse)");
    if (ctx->cfg.render_refine)
        return qk_fail(ctx, QUARK_EINVAL, "the no-alloc step runs without render-and-refine (use quark_update_fuse)");
    if (!qk_uniform(ctx->cfg))
        return qk_fail(ctx, QUARK_EINVAL, "the no-alloc step takes the uniform schedule only (use quark_update_fuse)");
    if (!ctx->weights_loaded) return qk_fail(ctx, QUARK_EINVAL, "weights not loaded");
    const quark_config& c = ctx->cfg;
    if (scale < 0 || scale >= c.n_scales) return qk_fail(ctx, QUARK_EINVAL, "scale %d out of range", scale);
    if (scale > 0 && !v_prev) return qk_fail(ctx, QUARK_EINVAL, "step %d needs the previous step's volume", scale);
    const bool last = scale == c.n_scales - 1;
    if (last && !beta) return qk_fail(ctx, QUARK_EINVAL, "the last step writes blend logits: beta is NULL");
    if (reinterpret_cast<uintptr_t>(v_out) % 32 || (scale > 0 && reinterpret_cast<uintptr_t>(v_prev) % 32) ||
        (last && reinterpret_cast<uintptr_t>(beta) % 32))
        return qk_fail(ctx, QUARK_EINVAL, "v_prev, v_out and beta must be 32-byte aligned");
    quark_status s = qk_validate_camera(ctx, *target, "target");
    if (s != QUARK_OK) return s;
    {
        const void* bufs[] = {scale > 0 ? v_prev : nullptr, v_out, colour, alpha, depth, t_raw, s_raw,
                              last ? beta : nullptr};
        const char* names[] = {"v_prev", "v_out", "colour", "alpha", "depth", "t_raw", "s_raw", "beta"};
        for (int i = 0; i < 8; ++i)
            if (bufs[i] && (s = check_device_buffer(ctx, bufs[i], names[i])) != QUARK_OK) return s;
    }
    for (int j = 0; j < c.n_scales; ++j)
        if (target->height % c.k[j] || target->width % c.k[j])
            return qk_fail(ctx, QUARK_EINVAL, "output %dx%d not divisible by k=%d", target->width, target->height,
                           c.k[j]);

    const bool bf16 = c.precision == QUARK_BF16;
    const size_t elt = bf16 ? 2 : 4;
    const int k = c.k[scale], L = c.L[scale];
    const int H = target->height / k, W = target->width / k;
    int Lp = 0, Hp = 0, Wp = 0;
    bool collapse = false;
    if (scale > 0) {
        Lp = c.L[scale - 1];
        Hp = target->height / c.k[scale - 1];
        Wp = target->width / c.k[scale - 1];
        collapse = Lp == 2 * L;
    }
    const size_t attn_bytes = round256((size_t)L * H * W * c.C * elt);
    const size_t col_bytes = collapse ? round256((size_t)L * Hp * Wp * c.C * elt) : 0;
    if (attn_bytes + col_bytes > QUARK_NOALLOC_SCRATCH_BYTES)
        return qk_fail(ctx, QUARK_EINVAL,
                       "step %d needs %zu bytes of scratch; the static scratch holds %zu (use quark_update_fuse)",
                       scale, attn_bytes + col_bytes, (size_t)QUARK_NOALLOC_SCRATCH_BYTES);

    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return qk_fail(ctx, QUARK_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    unsigned char* scratch = nullptr;
    s = scratch_address(ctx, ctx->device, &scratch);
    if (s != QUARK_OK) return s;
    void* vattn = scratch;
    void* collapsed = scratch + attn_bytes;
    cudaStream_t st = (cudaStream_t)stream;

    const void* prev = v_prev;
    Transition tr = TR_INIT;
    if (scale > 0) {
        if (collapse) {
            CollapseArgs ca{};
            ca.in = v_prev;
            ca.out = collapsed;
            ca.L = L;
            ca.H = Hp;
            ca.W = Wp;
            ca.w = ctx->wdev + ctx->off_collapse[scale];
            ca.wtc = qk_collapse_wtc(ctx, scale);
            ca.err = ctx->dev_err;
            s = qk_launch(ctx, st, KF_COLLAPSE, [&] { return launch_collapse(ca, c.C, bf16, st); });
            if (s != QUARK_OK) return s;
            prev = collapsed;
        }
        tr = (c.k[scale - 1] == 2 * k) ? TR_UP2 : TR_SAME;
    }

    AttendArgs aa{};
    aa.prev = prev;
    aa.Hp = Hp;
    aa.Wp = Wp;
    const int li = k == 1 ? 0 : k == 2 ? 1 : k == 4 ? 2 : 3;
    aa.feat = pyr->level[li];
    aa.fh = pyr->H / k;
    aa.fw = pyr->W / k;
    aa.L = L;
    aa.H = H;
    aa.W = W;
    aa.V = pyr->V;
    aa.dp = {(float)(1.0 / c.near_m - 1.0 / c.far_m), (float)(1.0 / c.far_m)};
    aa.w = ctx->wdev + ctx->off_attend[scale];
    aa.out = vattn;
    aa.beta = last ? beta : nullptr;
    aa.wtc = ctx->wat ? (const uint8_t*)ctx->wat + ctx->off_wat[scale] : nullptr;
    aa.err = ctx->dev_err;
    for (int m = 0; m < pyr->V; ++m) aa.geo.v[m] = qk_view_map(*target, k, k, pyr->cams[m], k);
    s = qk_launch(ctx, st, KF_ATTEND, [&] { return launch_attend(aa, c.C, c.heads, tr, last, bf16, st); });
    if (s != QUARK_OK) return s;

    ConvArgs cv{};
    cv.in = vattn;
    cv.out = v_out;
    cv.L = L;
    cv.H = H;
    cv.W = W;
    cv.dp = aa.dp;
    cv.w = ctx->wdev + ctx->off_conv[scale];
    cv.wtc = ctx->wtc ? (const uint8_t*)ctx->wtc + scale * ctx->wtc_step_bytes : nullptr;
    cv.err = ctx->dev_err;
    cv.ks = c.conv_kernel == 1 ? 1 : 3;
    s = qk_launch(ctx, st, KF_CONV, [&] { return launch_conv_block(cv, c.C, bf16, st); });
    if (s != QUARK_OK) return s;
    // the decoded attributes, from the volume just written (the regular step makes them on demand)
    return qk_decode(ctx, scale, v_out, L, H, W, colour, alpha, depth, t_raw, s_raw, st);
}
