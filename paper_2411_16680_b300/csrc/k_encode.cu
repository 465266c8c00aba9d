// Encode Input Images (Sec. 3.2.1): F_1 = conv3x3(I) (3 -> C, zero pad, bias, no activation),
// F_2k = 2x2 mean pool of F_k.  One CTA per 16x16 pixel tile of one view.  A thread owns a 2x2
// pixel quad and 16 of the C channels, so level 2 is its own quad mean; levels 4 and 8 are means
// of neighbouring quads, taken with warp shuffles (a warp covers 8 x 4 quads = 16 x 8 pixels).
// Level 1 is never read back from HBM.  Also writes the RGBA-padded copy of the images used by
// the render.  The conv runs on packed FP32x2 arithmetic, two channels per instruction.
//
// The CTAs are persistent (a few per SM, striding over the tiles): the weights are staged once,
// and the image patch of the next tile is fetched with cp.async into the second of two patch
// buffers while the current tile is computed.
#include <algorithm>

#include "device_common.cuh"

namespace quark {

constexpr int ENC_T = 16;  // tile edge (pixels)
constexpr int ENC_P = ENC_T + 2;

// 4-byte asynchronous copy global -> shared; zero-fills when `valid` is false (no bytes read)
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// 16 channels of one texel of a level at p (T = float or bf16)
// (256-bit stores: a whole 32-byte sector per store; the levels are 32-byte aligned)
__device__ __forceinline__ void store16x2(float* p, const float2 (&v)[8]) {
    uint4 u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        u[i] = make_uint4(__float_as_uint(v[2 * i].x), __float_as_uint(v[2 * i].y), __float_as_uint(v[2 * i + 1].x),
                          __float_as_uint(v[2 * i + 1].y));
    stg256(p, u[0], u[1]);
    stg256(p + 8, u[2], u[3]);
}
__device__ __forceinline__ void store16x2(__nv_bfloat16* p, const float2 (&v)[8]) {
    uint4 u[2];
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(u);
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[j].x, v[j].y);
    stg256(p, u[0], u[1]);
}

// 2x2 mean of the 16-channel texels held by this lane and its partners at lane ^ dx and ^ dy
__device__ __forceinline__ void quad_mean(float2 (&t)[8], int dx, int dy) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float2 s = t[j];
        s.x += __shfl_xor_sync(0xffffffffu, s.x, dx);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, dx);
        s.x += __shfl_xor_sync(0xffffffffu, s.x, dy);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, dy);
        t[j] = make_float2(0.25f * s.x, 0.25f * s.y);
    }
}

// the view and pixel origin of a tile (divisions by the launch's tile counts: FastDiv)
__device__ __forceinline__ void tile_origin(int tile, const FastDiv& per_view, const FastDiv& tiles_x, int& v, int& X0, int& Y0) {
    v = fdiv(tile, per_view);
    const int r = tile - v * (int)per_view.d, ty = fdiv(r, tiles_x);
    X0 = (r - ty * (int)tiles_x.d) * ENC_T;
    Y0 = ty * ENC_T;
}

template <int NT>
__device__ __forceinline__ void fetch_patch(const EncodeArgs& a, int tile, const FastDiv& per_view, const FastDiv& tiles_x,
                                            float (*patch)[ENC_P][3]) {
    int v, X0, Y0;
    tile_origin(tile, per_view, tiles_x, v, X0, Y0);
    const float* img = a.images + (size_t)v * a.H * a.W * 3;
    for (int i = threadIdx.x; i < ENC_P * ENC_P * 3; i += NT) {
        const int c = i % 3, px = (i / 3) % ENC_P, py = i / (3 * ENC_P);
        const int gy = Y0 - 1 + py, gx = X0 - 1 + px;
        const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
        cp_async4(&patch[py][px][c], in ? img + ((size_t)gy * a.W + gx) * 3 + c : img, in);
    }
}

template <typename T, int C>
__global__ void __launch_bounds__(64 * (C / 16), C == 64 ? 2 : 4) encode_kernel(EncodeArgs a, FastDiv per_view, FastDiv tiles_x) {
    constexpr int NT = 64 * (C / 16);
    __shared__ float patch_buf[2][ENC_P][ENC_P][3];
    __shared__ __align__(16) float w[28 * C];  // [tap = (dy * 3 + dx) * 3 + ci][C], then bias [C]

    const int tid = threadIdx.x, lane = tid & 31;
    const int H = a.H, W = a.W;
    const int ntiles = (int)per_view.d * a.V;
    for (int i = tid; i < 28 * C; i += NT) w[i] = a.w[i];

    // quad (qx, qy) of the 8 x 8 quads of the tile; warp w % 4 holds quad rows 4 (w % 4) .. + 3
    const int cg = tid / 64, c0 = cg * 16;
    const int qx = lane & 7, qy = ((tid & 63) >> 5) * 4 + (lane >> 3);
    const int px0 = 2 * qx, py0 = 2 * qy;

    int tile = blockIdx.x;
    if (tile < ntiles) fetch_patch<NT>(a, tile, per_view, tiles_x, patch_buf[0]);
    cp_async_commit();
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        if (tile + (int)gridDim.x < ntiles) fetch_patch<NT>(a, tile + gridDim.x, per_view, tiles_x, patch_buf[(it + 1) & 1]);
        cp_async_commit();
        cp_async_wait_prior();  // this tile's patch has landed
        __syncthreads();
        float (*patch)[ENC_P][3] = patch_buf[it & 1];
        int v, X0, Y0;
        tile_origin(tile, per_view, tiles_x, v, X0, Y0);

        // RGBA copy of the tile
        for (int i = tid; i < ENC_T * ENC_T; i += NT) {
            const int px = i % ENC_T, py = i / ENC_T, X = X0 + px, Y = Y0 + py;
            if (X < W && Y < H)
                a.rgba[((size_t)v * H + Y) * W + X] =
                    make_float4(patch[py + 1][px + 1][0], patch[py + 1][px + 1][1], patch[py + 1][px + 1][2], 0.f);
        }

        float2 acc[4][8];
        {
            const float4* b4 = reinterpret_cast<const float4*>(&w[27 * C + c0]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 b = b4[i];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    acc[p][2 * i] = make_float2(b.x, b.y);
                    acc[p][2 * i + 1] = make_float2(b.z, b.w);
                }
            }
        }
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                for (int ci = 0; ci < 3; ++ci) {
                    const float4* w4 = reinterpret_cast<const float4*>(&w[((dy * 3 + dx) * 3 + ci) * C + c0]);
                    float2 wr[8];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 t = w4[i];
                        wr[2 * i] = make_float2(t.x, t.y);
                        wr[2 * i + 1] = make_float2(t.z, t.w);
                    }
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const float x = patch[py0 + (p >> 1) + dy][px0 + (p & 1) + dx][ci];
                        const float2 x2 = make_float2(x, x);
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[p][j] = __ffma2_rn(x2, wr[j], acc[p][j]);
                    }
                }

        // level 1: the four pixels of the quad
        if (a.level[0]) {
            T* l1 = reinterpret_cast<T*>(a.level[0]) + (size_t)v * H * W * C + c0;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int X = X0 + px0 + (p & 1), Y = Y0 + py0 + (p >> 1);
                if (X < W && Y < H) store16x2(l1 + ((size_t)Y * W + X) * C, acc[p]);
            }
        }
        // level 2: the quad mean
        float2 t[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 s01 = make_float2(acc[0][j].x + acc[1][j].x, acc[0][j].y + acc[1][j].y);
            const float2 s23 = make_float2(acc[2][j].x + acc[3][j].x, acc[2][j].y + acc[3][j].y);
            t[j] = make_float2(0.25f * (s01.x + s23.x), 0.25f * (s01.y + s23.y));
        }
        {
            const int H2 = H / 2, W2 = W / 2, X = X0 / 2 + qx, Y = Y0 / 2 + qy;
            if (a.level[1] && X < W2 && Y < H2)
                store16x2(reinterpret_cast<T*>(a.level[1]) + (((size_t)v * H2 + Y) * W2 + X) * C + c0, t);
        }
        // level 4: quads (qx ^ 1, qy ^ 1) are lanes ^ 1 and ^ 8
        quad_mean(t, 1, 8);
        {
            const int H4 = H / 4, W4 = W / 4, X = X0 / 4 + qx / 2, Y = Y0 / 4 + qy / 2;
            if (a.level[2] && !(qx & 1) && !(qy & 1) && X < W4 && Y < H4)
                store16x2(reinterpret_cast<T*>(a.level[2]) + (((size_t)v * H4 + Y) * W4 + X) * C + c0, t);
        }
        // level 8: level-4 texels at lanes ^ 2 and ^ 16
        quad_mean(t, 2, 16);
        {
            const int H8 = H / 8, W8 = W / 8, X = X0 / 8 + qx / 4, Y = Y0 / 8 + qy / 4;
            if (a.level[3] && !(qx & 3) && !(qy & 3) && X < W8 && Y < H8)
                store16x2(reinterpret_cast<T*>(a.level[3]) + (((size_t)v * H8 + Y) * W8 + X) * C + c0, t);
        }
        __syncthreads();  // the patch buffer is refilled by the next iteration's prefetch
    }
}

template <typename T, int C>
static cudaError_t launch_t(const EncodeArgs& a, cudaStream_t st) {
    static int ctas_per_sm = 0, sms = 0;
    if (!ctas_per_sm) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm, encode_kernel<T, C>, 64 * (C / 16), 0);
        if (e != cudaSuccess) return e;
        if (ctas_per_sm < 1) ctas_per_sm = 1;
    }
    const int tiles_x = (a.W + ENC_T - 1) / ENC_T, tiles_y = (a.H + ENC_T - 1) / ENC_T;
    const long ntiles = (long)tiles_x * tiles_y * a.V;
    const int grid = (int)std::min<long>(ntiles, (long)sms * ctas_per_sm);
    encode_kernel<T, C><<<grid, 64 * (C / 16), 0, st>>>(a, make_fastdiv((uint32_t)(tiles_x * tiles_y)), make_fastdiv((uint32_t)tiles_x));
    return cudaGetLastError();
}

cudaError_t launch_encode(const EncodeArgs& a, int C, bool bf16, cudaStream_t st) {
    for (int i = 0; i < 4; ++i)  // 256-bit stores of the levels
        if (reinterpret_cast<uintptr_t>(a.level[i]) % 32) return cudaErrorMisalignedAddress;
    if (C == 16) return bf16 ? launch_t<__nv_bfloat16, 16>(a, st) : launch_t<float, 16>(a, st);
    if (C == 32) return bf16 ? launch_t<__nv_bfloat16, 32>(a, st) : launch_t<float, 32>(a, st);
    if (C == 64) return bf16 ? launch_t<__nv_bfloat16, 64>(a, st) : launch_t<float, 64>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
