// Internal interfaces between the C ABI (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "quark.h"

namespace quark {

// Plane-induced mapping of one view for a given target grid and view grid:
// X = d * (A p) + b with p = (x + 0.5, y + 0.5, 1) on the target grid, and
// (u, v) = (X.x / X.z, X.y / X.z) on the view's grid.  A = K_m R_m R_t^T K_t^-1,
// b = K_m (t_m - R_m R_t^T t_t); composed on the host in float64, stored as float32.
struct ViewMap {
    float A[9];
    float b[3];
};
struct Geometry {
    ViewMap v[QUARK_MAX_VIEWS];
};

// Reciprocal-depth parameters of Eq. (depth_activation).
struct DepthParams {
    float span;     // 1/near - 1/far
    float inv_far;  // 1/far
};

struct EncodeArgs {
    const float* images;  // [V][H][W][3]
    int V, H, W;
    const float* w;       // [27][C] then bias [C]
    float4* rgba;         // [V][H][W] padded copy of the images
    void* level[4];       // levels 1, 2, 4, 8 ([V][H/k][W/k][C]); NULL where unused
};

struct CollapseArgs {
    const void* in;   // [2L][H][W][C]
    void* out;        // [L][H][W][C]
    int L, H, W;
    const float* w;   // W1 [2C][C], b1 [C], W2 [C][C], b2 [C]
    const void* wtc;  // BF16 form: packed B operands of W1 (C x 2C) then W2 (C x C); else NULL
    int* err;         // BF16 form: set when a bounded wait of the tensor-core kernel runs out
};

enum Transition { TR_INIT = 0, TR_SAME = 1, TR_UP2 = 2 };

struct AttendArgs {
    const void* prev;  // [L][Hp][Wp][C] volume entering the step (already collapsed); NULL at step 0
    int Hp, Wp;
    const void* feat;  // pyramid level [V][fh][fw][C]
    int fh, fw;
    int L, H, W, V;
    DepthParams dp;
    const float* w;    // v0 [C], g [C], w_d [C], b_d (padded to C), Wq [C][h*C], Wo [h*C][C], W_beta [C][C]
    void* out;         // V_attn [L][H][W][C]
    float* beta;       // [H][W][L][V] blend logits (last step), else NULL
    const void* wtc;   // BF16 form: [Wq | W_beta] and W^O packed as tcgen05 B operands
    int* err;          // device error word (bounded waits)
    const float* w_std;  // standard mode: StdLayout (W^q, W^O); else NULL
    const float* depth_in;  // [L][H][W] depths to sample at (reused from an earlier step), or NULL
    float* depth_out;       // [L][H][W] the depths sampled at, kept for a later step, or NULL
    // Test of the bounded-wait error path (quark_test_wait_timeout), tensor-core kernel only: when
    // set, the query MMA chain is not issued, so the wait on its completion runs out after
    // test_wait_ns; 0 in normal launches
    uint64_t test_wait_ns;
    Geometry geo;
};

struct ConvArgs {
    const void* in;    // V_attn [L][H][W][C]
    void* out;         // V_out [L][H][W][C]
    int L, H, W;
    DepthParams dp;
    const float* w;    // g [C], W1 [9][C][C], b1 [C], W2 [9][C][C], b2 [C], dec: w_d [C], w_s [C], W_a [C][3], b_a[3], b_d, b_s
    float* t_raw;      // [H][W][L] raw depth logits, or NULL (not written)
    float* s_raw;      // [H][W][L] raw density logits, or NULL (not written)
    const void* wtc;   // BF16 form: W1 then W2 packed as tcgen05 B operands (see pack_conv_weights_bf16)
    int* err;          // device error word: set when a bounded wait inside the kernel runs out
    int ks;            // kernel size: 3, or 1 (the weights at the centre tap; k_mlp.cu); 0 = 3
};

// Decode of the LDM attributes from a stored volume (Sec. 3.2.2 "Decoding", Eq. depth_activation).
struct DecodeArgs {
    const void* vol;   // V [L][H][W][C] as stored (FP32 or BF16)
    int L, H, W;
    DepthParams dp;
    const float* w;    // the step's conv-block weights (ConvLayout: w_d, w_s, W_a, b_a, b_d, b_s)
    float* colour;     // [L][H][W][3]
    float* alpha;      // [L][H][W]
    float* depth;      // [L][H][W]
    float* t_raw;      // [H][W][L], or NULL (not written)
    float* s_raw;      // [H][W][L], or NULL (not written)
};

// Render-and-refine (Sec. 3.2.2 "Decoding and rendering the intermediate LDM", Eq.
// overcomposite-result; the Update Block): the intermediate LDM decoded from the volume entering
// a step, splatted into every input view and over-composited there.
struct SplatArgs {
    const float* colour;  // [L][H][W][3] appearance of the intermediate LDM
    const float* alpha;   // [L][H][W] density
    const float* depth;   // [L][H][W]
    int L, H, W, V;       // the LDM grid (previous step's) and the views
    int h, w;             // the views' grid at the rendering level
    float4* acc;          // [V][L][h][w] bilinear-weighted sums of (colour, density)
    float* wsum;          // [V][L][h][w] weight sums
    float4* out;          // [V][h][w] rendered views: RGB and accumulated alpha
    Geometry geo;         // per view: LDM grid -> the view's grid at the rendering level
};
struct RefineArgs {
    const void* feat;     // [V][h][w][C] level-k features (plus the ray encoding when on)
    const float4* rend;   // [V][hr][wr] rendered views at the previous step's level
    int V, C, h, w, hr, wr, ratio;  // ratio = h / hr (1 or 2)
    const float* wr_b;    // W_r [4][C] then b_r [C]
    void* out;            // [V][h][w][C] F' = F + up(I~) W_r + b_r (the Update Block's CNN input)
};

// Ray directional encoding of one step's pyramid level (Sec. 3.2.1).
struct RayArgs {
    int V, C;
    int h0, w0;          // the coarsest level's grid (factor k0)
    int h, w, ratio;     // this level's grid and k0 / k
    float span;          // 1/near - 1/far
    const float* w_ray;  // [32][C] projection of this level
    float* g;            // [V][h0][w0][C] projected coarse encoding
    Geometry geo;        // per view: A = R_t R_m^T K_{m,k0}^-1 (ray direction map), b = centre (target coords)
};

struct RenderArgs {
    const float* t_raw;  // [Hl][Wl][L]
    const float* s_raw;  // [Hl][Wl][L]
    const float* beta;   // [Hl][Wl][L][V]
    const float4* rgba;  // [V][Hi][Wi]
    int L, V, Hl, Wl, Hout, Wout, Hi, Wi;
    float sx, sy;        // upsampling factors of the last LDM grid to the output (e.g. 3.75)
    DepthParams dp;
    float4* out;         // [Hout][Wout]
    Geometry geo;
};

// Offsets (in floats) of the packed per-step weight blocks.
struct AttendLayout {
    int C, h;
    __host__ __device__ constexpr int v0() const { return 0; }
    __host__ __device__ constexpr int g() const { return C; }
    __host__ __device__ constexpr int wd() const { return 2 * C; }
    __host__ __device__ constexpr int bd() const { return 3 * C; }
    __host__ __device__ constexpr int wq() const { return 4 * C; }
    __host__ __device__ constexpr int wo() const { return 4 * C + C * h * C; }
    __host__ __device__ constexpr int wb() const { return 4 * C + 2 * C * h * C; }
    __host__ __device__ constexpr int total() const { return 4 * C + 2 * C * h * C + C * C; }
};
// Standard-mode weights of one step: W^q [C][C], W^O [C][C], then [W^k | W^val] [C][2C].
struct StdLayout {
    int C;
    __host__ __device__ constexpr int wq() const { return 0; }
    __host__ __device__ constexpr int wo() const { return C * C; }
    __host__ __device__ constexpr int wkv() const { return 2 * C * C; }
    __host__ __device__ constexpr int total() const { return 4 * C * C; }
};
struct ConvLayout {
    int C;
    __host__ __device__ constexpr int g() const { return 0; }
    __host__ __device__ constexpr int w1() const { return C; }
    __host__ __device__ constexpr int b1() const { return C + 9 * C * C; }
    __host__ __device__ constexpr int w2() const { return 2 * C + 9 * C * C; }
    __host__ __device__ constexpr int b2() const { return 2 * C + 18 * C * C; }
    __host__ __device__ constexpr int wd() const { return 3 * C + 18 * C * C; }
    __host__ __device__ constexpr int ws() const { return 4 * C + 18 * C * C; }
    __host__ __device__ constexpr int wa() const { return 5 * C + 18 * C * C; }
    __host__ __device__ constexpr int ba() const { return 8 * C + 18 * C * C; }
    __host__ __device__ constexpr int bd() const { return 8 * C + 18 * C * C + 3; }
    __host__ __device__ constexpr int bs() const { return 8 * C + 18 * C * C + 4; }
    __host__ __device__ constexpr int total() const { return 8 * C + 18 * C * C + 8; }
};
struct CollapseLayout {
    int C;
    __host__ __device__ constexpr int w1() const { return 0; }
    __host__ __device__ constexpr int b1() const { return 2 * C * C; }
    __host__ __device__ constexpr int w2() const { return 2 * C * C + C; }
    __host__ __device__ constexpr int b2() const { return 3 * C * C + C; }
    __host__ __device__ constexpr int total() const { return 3 * C * C + 2 * C; }
};

// Launchers (k_*.cu).  Each returns the launch's cudaError_t.
cudaError_t launch_encode(const EncodeArgs& a, int C, bool bf16, cudaStream_t st);
cudaError_t launch_encode_tc(const EncodeArgs& a, int C, const void* wtc, int* err, cudaStream_t st);
cudaError_t launch_collapse(const CollapseArgs& a, int C, bool bf16, cudaStream_t st);
// split: the FP32 form on FP16 operand parts (CollapseArgs.wtc from the context's split packs)
cudaError_t launch_collapse_tc(const CollapseArgs& a, int C, bool split, cudaStream_t st);
cudaError_t launch_attend(const AttendArgs& a, int C, int heads, Transition tr, bool last, bool bf16,
                          cudaStream_t st);
cudaError_t launch_conv_block(const ConvArgs& a, int C, bool bf16, cudaStream_t st);
// split: the FP32 form on FP16 operand parts (ConvArgs.wtc from pack_conv_weights_f16split)
cudaError_t launch_conv_block_tc(const ConvArgs& a, int C, bool split, cudaStream_t st);
cudaError_t launch_mlp_block(const ConvArgs& a, int C, bool bf16, cudaStream_t st);
// Output tile (columns, rows) the tensor-core conv block uses for an L x H x W volume.
cudaError_t conv_tc_tile_shape(int C, bool split, int W, int H, int L, int* cols, int* rows);
cudaError_t launch_decode(const DecodeArgs& a, int C, bool bf16, cudaStream_t st);
// split: the FP32 form on FP16 operand parts (AttendArgs.wtc packed by pack_attention_f16split)
cudaError_t launch_attend_tc(const AttendArgs& a, int C, int heads, Transition tr, bool last, bool split,
                             cudaStream_t st);
cudaError_t launch_kv_project(const void* feat, size_t texels, int C, const float* wkv, void* out, bool with_f, bool bf16,
                              cudaStream_t st);
cudaError_t launch_attend_std(const AttendArgs& a, int C, int heads, Transition tr, bool last, bool bf16,
                              cudaStream_t st);
cudaError_t launch_render(const RenderArgs& a, cudaStream_t st);
cudaError_t launch_ray_coarse(const RayArgs& a, cudaStream_t st);
cudaError_t launch_ray_add(const RayArgs& a, const void* feat, void* out, bool bf16, cudaStream_t st);
cudaError_t launch_render_depth(const RenderArgs& a, float* depth, cudaStream_t st);
cudaError_t launch_splat(const SplatArgs& a, cudaStream_t st);
cudaError_t launch_composite_views(const SplatArgs& a, cudaStream_t st);
cudaError_t launch_refine_add(const RefineArgs& a, bool bf16, cudaStream_t st);

}  // namespace quark
