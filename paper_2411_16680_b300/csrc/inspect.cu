// Inspection of the sampling geometry (quark_sample_coords): the reprojection and the bilinear tap
// origin of given target pixels at given depths, with exactly the device functions the Update &
// Fuse kernels use in the context's precision form, so that the integer tap decisions can be
// compared with an FP64 reference.
#include <vector>

#include "api_internal.h"
#include "device_common.cuh"

using namespace quark;

namespace {

__global__ void sample_coords_kernel(ViewMap m, int n, const float* px, const float* py, const float* d, bool rcp,
                                     float2* uv, int2* taps, int* valid) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float u = 0.f, v = 0.f;
    const bool ok = rcp ? reproject_rcp(m, px[i], py[i], d[i], u, v) : reproject(m, px[i], py[i], d[i], u, v);
    uv[i] = ok ? make_float2(u, v) : make_float2(0.f, 0.f);
    // the tap origin as bilinear_taps computes it
    taps[i] = ok ? make_int2((int)floorf(u - 0.5f), (int)floorf(v - 0.5f)) : make_int2(0, 0);
    valid[i] = ok ? 1 : 0;
}

}  // namespace

extern "C" quark_status quark_sample_coords(quark_ctx* ctx, const quark_camera* target, double k_tx, double k_ty,
                                            const quark_camera* view, double k_m, int n, const float* px,
                                            const float* py, const float* depth, float* uv, int* taps, int* valid) {
    if (!ctx || !target || !view || !px || !py || !depth || !uv || !taps || !valid || n < 0)
        return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (!(k_tx > 0) || !(k_ty > 0) || !(k_m > 0)) return qk_fail(ctx, QUARK_EINVAL, "grid factors must be positive");
    quark_status s = qk_validate_camera(ctx, *target, "target");
    if (s == QUARK_OK) s = qk_validate_camera(ctx, *view, "view");
    if (s != QUARK_OK || n == 0) return s;
    cudaSetDevice(ctx->device);
    const ViewMap m = qk_view_map(*target, k_tx, k_ty, *view, k_m);
    const size_t fb = (size_t)n * sizeof(float);
    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };  // every array 16-byte aligned
    const size_t o_py = up16(fb), o_d = o_py + up16(fb), o_uv = o_d + up16(fb);
    const size_t o_t = o_uv + up16((size_t)n * sizeof(float2)), o_v = o_t + up16((size_t)n * sizeof(int2));
    const size_t bytes = o_v + up16((size_t)n * sizeof(int));
    void* buf = nullptr;
    s = qk_alloc(ctx, &buf, bytes);
    if (s != QUARK_OK) return s;
    uint8_t* base = (uint8_t*)buf;
    float* dpx = (float*)base;
    float* dpy = (float*)(base + o_py);
    float* dd = (float*)(base + o_d);
    float2* duv = (float2*)(base + o_uv);
    int2* dt = (int2*)(base + o_t);
    int* dv = (int*)(base + o_v);
    cudaError_t e = cudaMemcpy(dpx, px, fb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dpy, py, fb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dd, depth, fb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        sample_coords_kernel<<<(n + 255) / 256, 256>>>(m, n, dpx, dpy, dd, ctx->cfg.precision == QUARK_BF16, duv, dt, dv);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(uv, duv, (size_t)n * sizeof(float2), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(taps, dt, (size_t)n * sizeof(int2), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(valid, dv, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost);
    qk_free(ctx, buf, bytes);
    if (e != cudaSuccess) return qk_fail(ctx, QUARK_ECUDA, "sample coordinates: %s", cudaGetErrorString(e));
    return QUARK_OK;
}

extern "C" quark_status quark_conv_tiles(quark_ctx* ctx, int L, int H, int W, int* tile_cols, int* tile_rows) {
    if (!ctx || !tile_cols || !tile_rows) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (L <= 0 || H <= 0 || W <= 0) return qk_fail(ctx, QUARK_EINVAL, "non-positive volume size");
    const bool split = ctx->cfg.precision != QUARK_BF16;
    if (split && !ctx->wtc) {
        *tile_cols = 16;  // the FP32 SIMT conv block's fixed 16 x 8 pixel tile
        *tile_rows = 8;
        return QUARK_OK;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = conv_tc_tile_shape(ctx->cfg.C, split, W, H, L, tile_cols, tile_rows);
    if (e != cudaSuccess) return qk_fail(ctx, QUARK_ECUDA, "conv tile geometry: %s", cudaGetErrorString(e));
    return QUARK_OK;
}

extern "C" quark_status quark_tensor_core_paths(quark_ctx* ctx, int* attend, int* conv) {
    if (!ctx || !attend || !conv) return qk_fail(ctx, QUARK_EINVAL, "NULL argument");
    if (!ctx->weights_loaded) return qk_fail(ctx, QUARK_EINVAL, "weights not loaded");
    const quark_config& c = ctx->cfg;
    const bool bf16 = c.precision == QUARK_BF16;
    // the dispatch rules of launch_attend and launch_conv_block for this context's packed weights
    *attend = c.attn_mode == QUARK_ATTN_ONE_TO_MANY && (bf16 || (ctx->wat != nullptr && c.C <= 32));
    *conv = bf16 || (c.conv_kernel != 1 && ctx->wtc != nullptr && c.C <= 32);
    return QUARK_OK;
}
