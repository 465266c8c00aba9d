// Encode Input Images (Sec. 3.2.1): F_1 = conv3x3(I) (3 -> C, zero pad, bias, no activation),
// F_2k = 2x2 mean pool of F_k.  One CTA per 8x8 pixel tile of one view: the conv output of the
// tile stays in shared memory and is pooled to levels 2, 4 and 8 there, so level 1 is never
// read back from HBM.  Also writes the RGBA-padded copy of the images used by the render.
#include "device_common.cuh"

namespace quark {

constexpr int ENC_T = 8;  // tile edge (pixels); the largest pyramid factor is 8

template <typename T, int C>
__device__ __forceinline__ void store_level(void* base, int v, int hk, int wk, int Y, int X, int c, float val) {
    T* p = reinterpret_cast<T*>(base);
    from_f(p[(((size_t)v * hk + Y) * wk + X) * C + c], val);
}

template <typename T, int C>
__global__ void __launch_bounds__(64) encode_kernel(EncodeArgs a) {
    __shared__ float patch[ENC_T + 2][ENC_T + 2][3];
    __shared__ float w[28 * C];
    __shared__ float f1[ENC_T * ENC_T][C + 1];
    __shared__ float f2[16][C + 1];
    __shared__ float f4[4][C + 1];

    const int tid = threadIdx.x;
    const int v = blockIdx.z;
    const int X0 = blockIdx.x * ENC_T, Y0 = blockIdx.y * ENC_T;
    const int H = a.H, W = a.W;

    for (int i = tid; i < 28 * C; i += 64) w[i] = a.w[i];
    for (int i = tid; i < (ENC_T + 2) * (ENC_T + 2) * 3; i += 64) {
        int c = i % 3, px = (i / 3) % (ENC_T + 2), py = i / (3 * (ENC_T + 2));
        int gy = Y0 - 1 + py, gx = X0 - 1 + px;
        float val = 0.f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) val = a.images[(((size_t)v * H + gy) * W + gx) * 3 + c];
        patch[py][px][c] = val;
    }
    __syncthreads();

    const int px = tid % ENC_T, py = tid / ENC_T;
    const int X = X0 + px, Y = Y0 + py;
    const bool inside = (X < W) && (Y < H);
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = w[27 * C + c];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int ci = 0; ci < 3; ++ci) {
                float x = patch[py + dy][px + dx][ci];
                const float* wr = &w[((dy * 3 + dx) * 3 + ci) * C];
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] = fmaf(x, wr[c], acc[c]);
            }
    if (inside) {
        a.rgba[((size_t)v * H + Y) * W + X] =
            make_float4(patch[py + 1][px + 1][0], patch[py + 1][px + 1][1], patch[py + 1][px + 1][2], 0.f);
        if (a.level[0]) {
            T* p = reinterpret_cast<T*>(a.level[0]) + (((size_t)v * H + Y) * W + X) * C;
#pragma unroll
            for (int c0 = 0; c0 < C; c0 += 16) {
                float t[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) t[i] = acc[c0 + i];
                store16(p + c0, t);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) f1[tid][c] = acc[c];
    __syncthreads();

    // 2x2 mean-pool chain; image sizes are divisible by every level used, so a level-k texel
    // inside the image always has its whole k x k block inside this tile.
    for (int i = tid; i < 16 * C; i += 64) {
        int c = i % C, t = i / C, ty = t / 4, tx = t % 4;
        float s = f1[(2 * ty) * ENC_T + 2 * tx][c] + f1[(2 * ty) * ENC_T + 2 * tx + 1][c] +
                  f1[(2 * ty + 1) * ENC_T + 2 * tx][c] + f1[(2 * ty + 1) * ENC_T + 2 * tx + 1][c];
        s *= 0.25f;
        f2[t][c] = s;
        int Yk = Y0 / 2 + ty, Xk = X0 / 2 + tx;
        if (a.level[1] && Yk < H / 2 && Xk < W / 2) store_level<T, C>(a.level[1], v, H / 2, W / 2, Yk, Xk, c, s);
    }
    __syncthreads();
    for (int i = tid; i < 4 * C; i += 64) {
        int c = i % C, t = i / C, ty = t / 2, tx = t % 2;
        float s = f2[(2 * ty) * 4 + 2 * tx][c] + f2[(2 * ty) * 4 + 2 * tx + 1][c] + f2[(2 * ty + 1) * 4 + 2 * tx][c] +
                  f2[(2 * ty + 1) * 4 + 2 * tx + 1][c];
        s *= 0.25f;
        f4[t][c] = s;
        int Yk = Y0 / 4 + ty, Xk = X0 / 4 + tx;
        if (a.level[2] && Yk < H / 4 && Xk < W / 4) store_level<T, C>(a.level[2], v, H / 4, W / 4, Yk, Xk, c, s);
    }
    __syncthreads();
    if (a.level[3]) {
        for (int c = tid; c < C; c += 64) {
            float s = 0.25f * (f4[0][c] + f4[1][c] + f4[2][c] + f4[3][c]);
            int Yk = Y0 / 8, Xk = X0 / 8;
            if (Yk < H / 8 && Xk < W / 8) store_level<T, C>(a.level[3], v, H / 8, W / 8, Yk, Xk, c, s);
        }
    }
}

template <typename T, int C>
static cudaError_t launch_t(const EncodeArgs& a, cudaStream_t st) {
    dim3 grid((a.W + ENC_T - 1) / ENC_T, (a.H + ENC_T - 1) / ENC_T, a.V);
    encode_kernel<T, C><<<grid, 64, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_encode(const EncodeArgs& a, int C, bool bf16, cudaStream_t st) {
    if (C == 16) return bf16 ? launch_t<__nv_bfloat16, 16>(a, st) : launch_t<float, 16>(a, st);
    if (C == 32) return bf16 ? launch_t<__nv_bfloat16, 32>(a, st) : launch_t<float, 32>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
