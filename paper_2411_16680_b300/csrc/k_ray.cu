// Ray directional encoding gamma_k (Sec. 3.2.1) added to a pyramid level before it is sampled.
//
// ray_coarse_kernel  one thread per pixel of view m's coarsest-level grid (factor k0): the pixel
//                    ray A + lam B in target-camera coordinates (A = the view's centre, B = its
//                    direction, both from the host in FP64), the difference of its intersections
//                    with the target-depth planes near and far in the target's normalised image
//                    plane -- eliminating lam, (1/near - 1/far) (A_z B_xy / B_z - A_xy) -- tanh,
//                    8 octaves of sin / cos (32 values), projected to C by the level's W_ray.
//                    Projecting before the upsample is exact: both are linear.
// ray_add_kernel     one thread per 16 channels of a level-k texel: F' = F + the bilinear x(k0/k)
//                    upsample (pixel centres aligned, edge clamp) of the projected coarse map.
#include "device_common.cuh"

namespace quark {

constexpr int RAY_PE = 32;  // 8 octaves x 2 axes x (sin, cos)

__global__ void __launch_bounds__(128) ray_coarse_kernel(const RayArgs a) {
    extern __shared__ float w[];  // W_ray [32][C]
    const int C = a.C;
    for (int i = threadIdx.x; i < RAY_PE * C; i += blockDim.x) w[i] = a.w_ray[i];
    __syncthreads();
    const size_t n = (size_t)a.V * a.h0 * a.w0;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int m = (int)(idx / ((size_t)a.h0 * a.w0));
    const int r = (int)(idx % ((size_t)a.h0 * a.w0));
    const float px = (r % a.w0) + 0.5f, py = (r / a.w0) + 0.5f;
    const ViewMap& vm = a.geo.v[m];  // A[9] = ray direction map, b[3] = view centre (target coords)
    const float Bx = fmaf(vm.A[0], px, fmaf(vm.A[1], py, vm.A[2]));
    const float By = fmaf(vm.A[3], px, fmaf(vm.A[4], py, vm.A[5]));
    float Bz = fmaf(vm.A[6], px, fmaf(vm.A[7], py, vm.A[8]));
    if (fabsf(Bz) < 1e-30f) Bz = Bz < 0.f ? -1e-30f : 1e-30f;  // a ray parallel to the image plane
    const float ex = tanhf(a.span * (vm.b[2] * (Bx / Bz) - vm.b[0]));
    const float ey = tanhf(a.span * (vm.b[2] * (By / Bz) - vm.b[1]));
    float pe[RAY_PE];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float f = (float)(1 << i) * 3.14159265358979323846f;
        sincosf(f * ex, &pe[4 * i], &pe[4 * i + 1]);
        sincosf(f * ey, &pe[4 * i + 2], &pe[4 * i + 3]);
    }
    float* out = a.g + idx * C;
    for (int c = 0; c < C; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < RAY_PE; ++i) acc = fmaf(pe[i], w[i * C + c], acc);
        out[c] = acc;
    }
}

template <typename T, int C>
__global__ void __launch_bounds__(256) ray_add_kernel(const RayArgs a, const T* __restrict__ feat, T* __restrict__ out) {
    constexpr int G = C / 16;
    const size_t n = (size_t)a.V * a.h * a.w * G;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int c0 = (int)(idx % G) * 16;
    const size_t t = idx / G;  // texel of the level
    const int m = (int)(t / ((size_t)a.h * a.w));
    const int r = (int)(t % ((size_t)a.h * a.w));
    const int y = r / a.w, x = r % a.w;
    int y0, y1, x0, x1;
    float wy, wx;
    resize_taps(y, a.ratio, a.h0, y0, y1, wy);
    resize_taps(x, a.ratio, a.w0, x0, x1, wx);
    const float* g = a.g + (size_t)m * a.h0 * a.w0 * C + c0;
    const float* g00 = g + ((size_t)y0 * a.w0 + x0) * C;
    const float* g01 = g + ((size_t)y0 * a.w0 + x1) * C;
    const float* g10 = g + ((size_t)y1 * a.w0 + x0) * C;
    const float* g11 = g + ((size_t)y1 * a.w0 + x1) * C;
    float f[16];
    load16(feat + t * C + c0, f);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float top = g00[i] * (1 - wx) + g01[i] * wx;
        const float bot = g10[i] * (1 - wx) + g11[i] * wx;
        f[i] += top * (1 - wy) + bot * wy;
    }
    store16(out + t * C + c0, f);
}

cudaError_t launch_ray_coarse(const RayArgs& a, cudaStream_t st) {
    const size_t n = (size_t)a.V * a.h0 * a.w0;
    if (n == 0) return cudaSuccess;
    ray_coarse_kernel<<<(unsigned)((n + 127) / 128), 128, RAY_PE * a.C * sizeof(float), st>>>(a);
    return cudaGetLastError();
}

template <typename T, int C>
static cudaError_t launch_add_t(const RayArgs& a, const void* feat, void* out, cudaStream_t st) {
    const size_t n = (size_t)a.V * a.h * a.w * (C / 16);
    ray_add_kernel<T, C><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, (const T*)feat, (T*)out);
    return cudaGetLastError();
}

cudaError_t launch_ray_add(const RayArgs& a, const void* feat, void* out, bool bf16, cudaStream_t st) {
    if ((size_t)a.V * a.h * a.w == 0) return cudaSuccess;
    if (a.C == 16) return bf16 ? launch_add_t<__nv_bfloat16, 16>(a, feat, out, st) : launch_add_t<float, 16>(a, feat, out, st);
    if (a.C == 32) return bf16 ? launch_add_t<__nv_bfloat16, 32>(a, feat, out, st) : launch_add_t<float, 32>(a, feat, out, st);
    if (a.C == 64) return bf16 ? launch_add_t<__nv_bfloat16, 64>(a, feat, out, st) : launch_add_t<float, 64>(a, feat, out, st);
    return cudaErrorInvalidValue;
}

}  // namespace quark
