/*
 * quark.h -- C ABI of the B300 (sm_103a) implementation of Quark's Update & Fuse steps and
 * final LDM render (Flynn et al., "Quark: Real-time, High-resolution, and General Neural
 * View Synthesis", 2024).
 *
 * Problem statement (Sec. 2 and Sec. 3): posed input images with intrinsics/extrinsics in,
 * novel-view RGB out.  Network weights are passed in (random-init tensors; no checkpoint
 * exists).  All compute runs in this library's CUDA kernels on one GPU; there is no CPU
 * fallback.
 *
 * Conventions shared by every entry point:
 *   - Pixel centres sit at (x + 0.5, y + 0.5).  Camera frame: x right, y down, z forward.
 *     Extrinsics are world->camera, X_c = R X_w + t (R row-major).  Depth is camera z.
 *   - A pyramid level k has intrinsics diag(1/k, 1/k, 1) K.  Scale j of an LDM uses pyramid
 *     level k_j and a grid of (target.height / k_j, target.width / k_j) pixels.
 *   - Layer l = 1..L, l = 1 farthest, l = L nearest (Sec. 3.2.3, depth anchors).
 *   - Device arrays are dense, row-major, channel-last; element types are float32 unless
 *     stated.  Every GPU call is asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream).
 *   - Errors are return codes; nothing aborts and nothing throws across the ABI.  A failing
 *     call leaves its outputs unspecified and stores a message readable with quark_last_error.
 *   - A context and its handles are used from one host thread at a time, except the
 *     quark_serve_* calls, which are thread-safe.
 */
#ifndef QUARK_H
#define QUARK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QUARK_OK = 0,
    QUARK_EINVAL = 1,     /* bad argument: sizes, shapes, non-finite camera, NULL pointer */
    QUARK_ENOMEM = 2,     /* device allocation failed or the HBM cap would be exceeded */
    QUARK_ECUDA = 3,      /* a CUDA runtime call failed (message names it) */
    QUARK_EAGAIN = 4,     /* result not ready yet (serve poll) */
    QUARK_ETIMEDOUT = 5,  /* a bounded wait ran out */
    QUARK_ENOTFOUND = 6,  /* unknown ticket / time step */
    QUARK_EBUSY = 7,      /* queue full or handle in use */
    QUARK_EINTERNAL = 8
} quark_status;

#define QUARK_MAX_SCALES 32
#define QUARK_MAX_VIEWS 64

enum { QUARK_FP32 = 0, QUARK_BF16 = 1 };             /* storage / tensor-core precision form */
enum { QUARK_ATTN_ONE_TO_MANY = 0,                    /* Sec. 3.3 "Optimized Attention" */
       QUARK_ATTN_STANDARD = 1 };                     /* Sec. 3.3 Eq. MultiHead with K/V projections */

/* Pinhole camera (Sec. 3.1: camera parameters theta).  R row-major, world->camera. */
typedef struct {
    int width, height;
    double fx, fy, cx, cy;
    double R[9];
    double t[3];
} quark_camera;

/* Network shape (Sec. 3.2; tables "Model description for Quark / Quark+").
 *   C          channels of features, pyramid and feature volume: 16, 32 or 64 (the paper's models
 *              use 32; the BF16 form takes C = 64 with 1 or 2 heads per step; the backward pass
 *              and the differentiable stage take 16 or 32)
 *   heads      attention heads h: 1, 2 or 4 (one-to-many: per-head width C, appendix A;
 *              standard: per-head width C/h)
 *   n_scales   number of fusion steps j, 1..32 (one per fusion block of the model tables)
 *   k[j], L[j] pyramid factor and LDM layer count of step j, coarse to fine.  k in {1,2,4,8};
 *              k[j-1]/k[j] in {1,2}; L[j-1]/L[j] in {1,2} (layer collapse, Sec. 3.2.2);
 *              L <= 64.  Step j's LDM grid is (target height / f_j, target width / f_j) with
 *              f_j = ldm_f[j], or k[j] where ldm_f[j] is 0; f[j-1]/f[j] in {1,2} (x2 spatial
 *              upsample).  The final render upsamples by s = f of the last step (e.g. 3.75).
 *   near_m, far_m  near and far planes eta and f of Eq. (depth_activation), 0 < near < far
 *   precision  QUARK_FP32 (all storage FP32, arithmetic to FP32 accuracy: the conv blocks, the
 *              sampling kernel's projections, the layer collapse and the Update Block run on
 *              tensor cores with each operand split into two FP16 parts and three products per
 *              FP32 product -- error at FP32 rounding -- where the weights keep every part in
 *              FP16 range (C <= 32), on SIMT kernels otherwise; see quark_tensor_core_paths) or
 *              QUARK_BF16 (pyramid and feature volume stored in BF16, contractions on tensor
 *              cores with BF16 operands and FP32 accumulation; geometry, softmax and
 *              transmittance stay FP32)
 *   attn_mode  QUARK_ATTN_ONE_TO_MANY (the paper's optimized attention: no K/V projections)
 *              or QUARK_ATTN_STANDARD (textbook multi-head cross attention, Sec. 3.3 Eq.
 *              MultiHead: keys and values are the sampled features times W^k and W^val, here
 *              projected once per pyramid texel -- exact, since bilinear sampling is linear and
 *              the projections have no bias -- and sampled from the projected maps).  The
 *              standard mode runs on SIMT kernels in both precisions and needs the *_std
 *              weights; quark_update_fuse_noalloc accepts one-to-many only.
 *   ray_encoding  1: the ray directional encoding gamma_k of Sec. 3.2.1 is added to each view's
 *              level-k features before they are sampled -- per input pixel, the difference of
 *              its ray's intersections with the near and far planes of the target (LDM)
 *              frustum in the target's normalised image plane, tanh, 8 octaves of sinusoids
 *              (32 values) on the coarsest level, bilinearly upsampled to level k and projected
 *              to C channels by W_ray of that level.  Needs the W_ray weights; not with
 *              quark_update_fuse_noalloc nor the differentiable stage.  0: off.
 *   render_refine  1: render-and-refine (Sec. 3.2.2 "Decoding and rendering the intermediate
 *              LDM", Eq. overcomposite-result, the Update Block): every Update & Fuse step after
 *              the first (a step j > 0 that attends and does not reuse depths) decodes the volume
 *              entering it, bilinearly splats its appearance and density into every input view at
 *              step j-1's pyramid level (normalised by max(weight sum, 1e-2)), over-composites
 *              them front to back into the rendered views I~ (RGB, alpha), and forms the update
 *              features Delta = F' + Conv(gelu(Conv(N(F')))), F' = F + up(I~) W_r + b_r, from the
 *              level-k features F (plus the ray encoding when on; up = x2 bilinear when the level
 *              changes).  The step and the steps reusing its depths sample Delta instead of F.
 *              Needs the upd_* weights.  0: off (Delta = F).
 *   hbm_cap_bytes  cap on this context's device allocations (0 = no cap)
 * Full model schedule (Sec. 3.2; tables "Model description for Quark / Quark+": an Update &
 * Fuse step back-projects its update features once and runs several fusion blocks, each an
 * attention block A_h followed by residual CNN blocks C).  Each fusion step j here is one
 * A_h + C pair or one further C; zero-filled arrays give the uniform schedule above.
 *   scale_heads[j]  0: `heads`; 1, 2 or 4: this step's heads; -1: a block without attention
 *              (the conv block only: same grid and layers as step j-1, j > 0)
 *   ldm_f[j]   LDM grid factor relative to the target (0: k[j]); the target's width and height
 *              must be multiples of it (e.g. 30, 15, 7.5, 3.75 for 1920 x 1080)
 *   model_width, model_height  aspect-adaptive LDM dimensions (Sec. 4): 0, 0 = off; else the
 *              output size the grid factors are given for (e.g. 1920 x 1080).  An LDM for any other
 *              output keeps the model's area per layer at the output's own aspect: step 0's grid is
 *              h0 = floor(sqrt(A / a) + 0.5), w0 = floor(h0 a + 0.5) (A = the model's step-0 grid
 *              area, a = output width / height), step j's grid is (h0, w0) x f_0 / f_j, and the
 *              target maps onto a grid with the factors width / W_j and height / H_j, which may
 *              differ (the final upsample too).  The output need not be divisible by anything.
 *   conv_kernel  kernel size of the fusion blocks' residual convolutions (Sec. 3.3): 3 (0 = 3), or 1,
 *              the position-wise MLP block of a Transformer that the residual convolution block
 *              mirrors (V + W2 gelu(W1 N(V) + b1) + b2 per element; conv1_w / conv2_w are then
 *              [1][1][C][C]).  The Update Block of render-and-refine keeps 3x3 convolutions.
 *   reuse_depth[j]  1: sample the views at the depths the latest sampling step used instead of
 *              the depths decoded from this step's input (one set of update features per Update
 *              & Fuse step); needs the same grid and layers back to that step.  0: decode.
 * quark_update_fuse_noalloc and the differentiable stage take the uniform schedule only, without
 * render-and-refine.                                                                         */
typedef struct {
    int C, heads, n_scales;
    int k[QUARK_MAX_SCALES];
    int L[QUARK_MAX_SCALES];
    float near_m, far_m;
    int precision;
    int attn_mode;
    int ray_encoding;
    int render_refine;
    int scale_heads[QUARK_MAX_SCALES];
    float ldm_f[QUARK_MAX_SCALES];
    int reuse_depth[QUARK_MAX_SCALES];
    int model_width, model_height;
    int conv_kernel;
    size_t hbm_cap_bytes;
} quark_config;

/* Host FP32 weights, row-vector convention y = x W + b.  Copied (and packed) by
 * quark_load_weights; the caller keeps ownership.  Shapes for C channels and h heads:
 *   enc_w [3][3][3][C] (dy, dx, c_in, c_out), enc_b [C]   encoder conv (Sec. 3.2.1)
 *   v0 [C]                                              learned initial feature (Sec. 3.2.2)
 *   per step j (h = that step's heads):
 *     attn_g[j] [C], Wq[j] [C][h*C], Wo[j] [h*C][C]      RMSNorm gain, one-to-many attention
 *                                                       (NULL for a block without attention)
 *     conv_g[j] [C], conv1_w[j], conv2_w[j] [k][k][C][C] (k = conv_kernel), conv1_b[j], conv2_b[j] [C]
 *                                                       residual conv block (Sec. 3.3)
 *     col_w1[j] [2C][C], col_b1[j] [C], col_w2[j] [C][C], col_b2[j] [C]
 *                                                       layer collapse into step j (Sec. 3.2.2);
 *                                                       may be NULL where L does not halve
 *   w_d [C], b_d; w_sigma [C], b_sigma; W_a [C][3], b_a [3]   depth, density, appearance
 *   W_beta [C][C]                                       blend-logit query of the last step   */
typedef struct {
    const float* enc_w;
    const float* enc_b;
    const float* v0;
    const float* attn_g[QUARK_MAX_SCALES];
    const float* Wq[QUARK_MAX_SCALES];
    const float* Wo[QUARK_MAX_SCALES];
    const float* conv_g[QUARK_MAX_SCALES];
    const float* conv1_w[QUARK_MAX_SCALES];
    const float* conv1_b[QUARK_MAX_SCALES];
    const float* conv2_w[QUARK_MAX_SCALES];
    const float* conv2_b[QUARK_MAX_SCALES];
    const float* col_w1[QUARK_MAX_SCALES];
    const float* col_b1[QUARK_MAX_SCALES];
    const float* col_w2[QUARK_MAX_SCALES];
    const float* col_b2[QUARK_MAX_SCALES];
    const float* w_d;
    float b_d;
    const float* w_sigma;
    float b_sigma;
    const float* W_a;
    const float* b_a;
    const float* W_beta;
    /* attn_mode QUARK_ATTN_STANDARD only (else may be NULL), per step j: [C][C] each */
    const float* Wq_std[QUARK_MAX_SCALES];
    const float* Wk_std[QUARK_MAX_SCALES];
    const float* Wv_std[QUARK_MAX_SCALES];
    const float* Wo_std[QUARK_MAX_SCALES];
    /* ray_encoding only (else may be NULL): [32][C] projection of the encoding for pyramid level
     * k = 1, 2, 4, 8 (index 0..3), for every level some step uses */
    const float* W_ray[4];
    /* render_refine only (else may be NULL), per step j that renders (see render_refine): the
     * Update Block, W_r [4][C], b_r [C], RMSNorm gain g [C], then the residual CNN block's
     * conv1_w, conv2_w [3][3][C][C], conv1_b, conv2_b [C] */
    const float* upd_Wr[QUARK_MAX_SCALES];
    const float* upd_br[QUARK_MAX_SCALES];
    const float* upd_g[QUARK_MAX_SCALES];
    const float* upd1_w[QUARK_MAX_SCALES];
    const float* upd1_b[QUARK_MAX_SCALES];
    const float* upd2_w[QUARK_MAX_SCALES];
    const float* upd2_b[QUARK_MAX_SCALES];
} quark_weights;

typedef struct quark_ctx quark_ctx;
typedef struct quark_pyramid quark_pyramid;
typedef struct quark_ldm quark_ldm;

/* Create a context on CUDA device `device` (made current for the call).  Validates the
 * config (EINVAL).  No device memory is allocated until weights or handles are made. */
quark_status quark_create(const quark_config* cfg, int device, quark_ctx** out);

/* Free a context and every device buffer it owns.  Handles made from it must be released
 * first: while any pyramid or LDM of the context is alive the call returns QUARK_EBUSY and frees
 * nothing.  NULL is accepted. */
quark_status quark_destroy(quark_ctx* ctx);

/* Copy (and pack for the kernels) the network weights.  Synchronous. */
quark_status quark_load_weights(quark_ctx* ctx, const quark_weights* w);

/* Encode Input Images (Sec. 3.2.1): F_1 = conv3x3(I) (3 -> C, zero pad, bias, no
 * activation), F_2k = 2x2 mean pool of F_k, for every level some step uses.  Also keeps a
 * padded RGBA copy of the images for the final render (Eq. 1 samples the input images).
 *   images  [V][H][W][3] float32 in [0, 1]; device memory, or host memory (pinned for an
 *           asynchronous copy), which is then copied in on `stream`
 *   cams    V host cameras; all views share one resolution W x H, divisible by every k
 *   V       1..64
 * If *out is NULL on entry, a new pyramid is allocated ([V][H/k][W/k][C] per level, FP32 or
 * BF16 by the precision form) and returned in *out; free it with quark_release_pyramid.  If
 * *out holds a pyramid of this context with the same V and resolution, it is re-encoded in
 * place (new images and cameras, e.g. the next video frame) without allocating; its previous
 * contents must no longer be in use on another stream.  `images` may be reused once the
 * stream has passed this call. */
quark_status quark_encode_pyramid(quark_ctx* ctx, const float* images, const quark_camera* cams, int V,
                                  void* stream, quark_pyramid** out);

/* Allocate an LDM (feature volume, decoded attributes and blend logits for every step)
 * in the frustum of the novel view `target` (Sec. 3.1).  target->width/height is the
 * output resolution and must be divisible by every step's grid factor f. */
quark_status quark_ldm_create(quark_ctx* ctx, const quark_camera* target, quark_ldm** out);

/* One Update & Fuse step (Sec. 3.2.2, Fig. "Update & Fuse Step"; Sec. 3.3), step `scale`
 * (steps run in order 0..n_scales-1 on one LDM):
 *   transition   step 0: broadcast v0, layers flat at the depth anchors; step j > 0: layer
 *                collapse when L halves, then x2 bilinear upsample when f halves
 *   back-project decode depth (Eq. depth_activation; or the reused depths), unproject each LDM
 *                pixel x layer, reproject into every view, bilinearly sample its level-k
 *                features (zero pad); skipped with the attention by a block without attention
 *   fusion block V += MultiHead(N(V), Delta) (one-to-many, Sec. 3.3), then
 *                V += Conv(gelu(Conv(N(V)))) (3x3 per layer plane)
 *   decode       colour = sigmoid(V W_a + b_a), alpha = sigmoid(V w_sigma + b_sigma),
 *                depth (Eq. depth_activation); the last step also writes the blend logits
 *                (Sec. 3.2.3) and the raw depth / density logits for the render. */
quark_status quark_update_fuse(quark_ctx* ctx, const quark_pyramid* pyr, int scale, quark_ldm* ldm,
                               void* stream);

/* Final render (Sec. 3.1 Eq. 1; Sec. 3.2.3 "Upsampling & Activation"): bilinear upsample by
 * s of the raw depth, density and blend logits, activation, back-projection of the input
 * images onto the layers, blend with softmax(beta), over-composite front to back.
 *   rgba  [H_out][W_out][4] float32: RGB and accumulated alpha (black background); device
 *         memory, or host memory (copied out on `stream`; synchronise before reading). */
quark_status quark_render_ldm(quark_ctx* ctx, const quark_ldm* ldm, const quark_pyramid* pyr, float* rgba,
                              void* stream);

/* Depth map of the novel view (Sec. 3.1: "a depth map can optionally be produced by
 * over-compositing the decoded depth instead of the blended input views"): the last LDM's raw
 * depth and density logits are upsampled and activated as for quark_render_ldm, and, front to
 * back, D += T alpha_l d_l, T *= 1 - alpha_l (0 behind the last layer; not normalised by the
 * accumulated alpha).  depth: [target height][target width] float, device or host memory (a
 * host target is copied out on the stream).  Needs every Update & Fuse step run (EINVAL). */
quark_status quark_render_depth(quark_ctx* ctx, const quark_ldm* ldm, float* depth, void* stream);

/* Convenience: every Update & Fuse step then the render, for one novel view. */
quark_status quark_render_novel_view(quark_ctx* ctx, const quark_pyramid* pyr, quark_ldm* ldm, float* rgba,
                                     void* stream);

/* One Update & Fuse step that allocates no device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while they run, e.g. a
 * frame loop with a fixed memory budget reserved up front (cudaMalloc can fail at run time and
 * synchronises the device, stalling the frame), a process whose device memory is owned by
 * another allocator, or code that must not make allocating CUDA calls at that point.
 *
 * It computes exactly what quark_update_fuse computes for step `scale`, launching the same
 * kernels, but takes the LDM buffers from the caller instead of an LDM handle:
 *   target    the novel view (as for quark_ldm_create)
 *   v_prev    step scale-1's output volume [L'][H'][W'][C] (FP32, or BF16 in the BF16 form);
 *             ignored at scale 0
 *   v_out     this step's output volume [L][H][W][C], same element type
 *   colour [L][H][W][3], alpha / depth [L][H][W], t_raw / s_raw [H][W][L] (float32)
 *   beta      blend logits [H][W][L][V] (float32), required on the last step, else ignored
 * All buffers are device memory of the context's device, owned by the caller (host memory, or
 * memory of another device, is refused with QUARK_EINVAL before any launch; the check allocates
 * nothing); v_prev, v_out and beta must start on a 32-byte boundary (the kernels move them in 16- and 32-byte vectors; cudaMalloc and PyTorch's
 * allocator give 256), else QUARK_EINVAL.  The two intermediates (the volume after
 * the attention block and, where L halves, the collapsed volume) live in one static device
 * array of QUARK_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library holds until the
 * process exits; a step whose intermediates need more returns QUARK_EINVAL (use
 * quark_update_fuse for it).  Every call shares that array and it keeps the last call's
 * contents (each call overwrites what it reads), so calls whose work overlaps on the GPU --
 * on different streams, or from different contexts on one device -- race; serialise them.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current and keeps it for the life of the process; make that first call
 * before any stream capture.  A device reset (cudaDeviceReset) invalidates that address, as it
 * does every context and handle of this library on the device: do not use the library on a
 * device after resetting it. */
#define QUARK_NOALLOC_SCRATCH_BYTES (32u << 20)
quark_status quark_update_fuse_noalloc(quark_ctx* ctx, const quark_pyramid* pyr, int scale,
                                       const quark_camera* target, const void* v_prev, void* v_out,
                                       float* colour, float* alpha, float* depth, float* t_raw, float* s_raw,
                                       float* beta, void* stream);

/* Fields of an LDM readable for inspection (state after the latest quark_update_fuse). */
enum {
    QUARK_FIELD_VOLUME = 0,       /* [L][H][W][C] feature volume after the step (FP32 out)    */
    QUARK_FIELD_VOLUME_ATTN = 1,  /* [L][H][W][C] after the attention block, before the conv  */
    QUARK_FIELD_COLOUR = 2,       /* [L][H][W][3] appearance c                                 */
    QUARK_FIELD_ALPHA = 3,        /* [L][H][W] density (alpha)                                  */
    QUARK_FIELD_DEPTH = 4,        /* [L][H][W] depth in metres                                 */
    QUARK_FIELD_BETA_LOGITS = 5,  /* [H][W][L][V] blend logits (last step only)                 */
    QUARK_FIELD_DEPTH_LOGIT = 6,  /* [H][W][L] raw depth logit t = V w_d + b_d                  */
    QUARK_FIELD_DENSITY_LOGIT = 7 /* [H][W][L] raw density logit                                */
};

/* Copy one field of the LDM's latest step into host memory `dst` of `bytes` bytes
 * (synchronous; EINVAL if `bytes` differs from the field's size, which
 * quark_ldm_field_bytes returns). */
quark_status quark_ldm_read(quark_ldm* ldm, int field, void* dst, size_t bytes);
size_t quark_ldm_field_bytes(const quark_ldm* ldm, int field);

/* Copy pyramid level k ([V][H/k][W/k][C], the precision form's element type) to dst (host or
 * device; synchronous).  `bytes` must equal the level's size. */
quark_status quark_pyramid_read(const quark_pyramid* pyr, int k, void* dst, size_t bytes);

/* Sampling geometry as the Update & Fuse kernels compute it (inspection; Sec. 3.1 operator P^T and
 * the bilinear tap rule): for n target-grid pixel centres (px[i], py[i]) of a grid with factors
 * (k_tx, k_ty) relative to `target` (target pixels per grid pixel along x and y), at depths
 * depth[i] (metres), the continuous coordinates uv[i] = (u, v) in `view`'s level-k_m grid and the
 * origin of the four bilinear taps taps[i] = (floor(u - 0.5), floor(v - 0.5)), with the device
 * arithmetic of the context's precision form (FP32: IEEE divide; BF16: one reciprocal).
 * valid[i] = 0 where the point is behind the view (camera z <= 1e-6; uv and taps then 0).  All
 * arrays are host memory, [n] (px, py, depth, valid) or [n][2] (uv, taps); synchronous. */
quark_status quark_sample_coords(quark_ctx* ctx, const quark_camera* target, double k_tx, double k_ty,
                                 const quark_camera* view, double k_m, int n, const float* px, const float* py,
                                 const float* depth, float* uv, int* taps, int* valid);

/* Output tile of the conv-block kernel of the context's precision form for an L x H x W volume
 * (inspection, so that tests can place windows on its tile seams; Sec. 3.3 conv block): tiles of
 * *tile_rows rows by *tile_cols columns start at multiples of those in y and x (the last ones
 * ragged).  The tile the tensor-core kernel chooses for this plane size on the context's device
 * (BF16 form, and the FP32 form's split-operand kernel); the fixed 16 x 8 tile where the FP32
 * form runs the SIMT kernel (C = 64, or weights outside the split's range).  Call after
 * quark_load_weights. */
quark_status quark_conv_tiles(quark_ctx* ctx, int L, int H, int W, int* tile_cols, int* tile_rows);

/* Which kernels the context runs on the 5th-generation tensor cores (inspection): *attend = 1 when
 * the one-to-many sampling kernel's query and output projections do (BF16 form; FP32 form with
 * C <= 32 through split FP16 operands, when the weights bound the normalised input and the
 * weights below 2^15), *conv = 1 when the conv block's convolutions do (BF16 form; FP32 form with
 * C <= 32 and 3 x 3 kernels through split FP16 operands, when the weights bound every operand part
 * below 2^15).  0 where the SIMT kernels run.  EINVAL before quark_load_weights. */
quark_status quark_tensor_core_paths(quark_ctx* ctx, int* attend, int* conv);

quark_status quark_release_pyramid(quark_pyramid* pyr);
quark_status quark_release_ldm(quark_ldm* ldm);

/* Last error message of a context (or of the calling thread when ctx is NULL). */
const char* quark_last_error(const quark_ctx* ctx);

/* ---- Serving (spec form 5; the paper serves one novel view per frame, Sec. 1) ----------
 * A server owns the context while it runs: one scheduler thread makes every launch.  Time steps
 * (sets of posed input images) are encoded once and kept resident; requests name a time step,
 * a target camera (whose width x height is the output resolution) and how many of the time
 * step's views to use (the first n_views).  Requests queue FIFO and are admitted as soon as a
 * slot (its own CUDA stream) is free and the request's device footprint fits under
 * hbm_cap_bytes next to the resident pyramids; admitted requests run concurrently.  A result is
 * identical whether the request ran alone or among others. */
typedef struct quark_server quark_server;

typedef struct {
    int n_slots;           /* requests in flight on the device at once, 1..64 */
    int queue_capacity;    /* pending requests beyond which submit returns QUARK_EBUSY */
    size_t hbm_cap_bytes;  /* admission cap: resident pyramids + in-flight LDMs (0 = none) */
} quark_serve_config;

typedef struct {
    int timestep;          /* resident time step (quark_serve_set_timestep) */
    quark_camera target;   /* novel view; width x height = output resolution */
    int n_views;           /* use the first n_views views of the time step */
    float* rgba;           /* [height][width][4] float32 output: device memory or host memory
                              (pinned); owned by the caller, valid until the result is polled */
    uint64_t user_tag;
} quark_request;

typedef struct {
    quark_status status;   /* QUARK_OK, or why the request failed (QUARK_EINVAL when cancelled) */
    int cancelled;
    uint64_t user_tag;
    double queue_ms;       /* submit -> admission */
    double gpu_ms;         /* admission -> completion seen by the scheduler */
    double total_ms;       /* submit -> completion */
} quark_result;

typedef struct {
    uint64_t submitted, completed, failed, cancelled, rejected;
    int in_flight, queued;
    double p50_ms, p99_ms, mean_ms;  /* submit -> completion of completed requests */
    double fps;                      /* completed requests per second since start */
    size_t hbm_in_use, hbm_high_water;
} quark_stats;

/* Start the scheduler thread.  The context's weights must be loaded. */
quark_status quark_serve_start(quark_ctx* ctx, const quark_serve_config* cfg, quark_server** out);
/* Encode (or re-encode) time step `timestep` from V posed images (as quark_encode_pyramid) and
 * keep it resident.  Synchronous.  QUARK_EBUSY while requests for that step are queued/running. */
quark_status quark_serve_set_timestep(quark_server* srv, int timestep, const float* images,
                                      const quark_camera* cams, int V);
/* Queue a request (thread-safe).  QUARK_EINVAL: bad camera / view count / NULL output;
 * QUARK_ENOTFOUND: time step not resident; QUARK_ENOMEM: footprint can never fit the cap;
 * QUARK_EBUSY: queue full. */
quark_status quark_serve_submit(quark_server* srv, const quark_request* req, uint64_t* ticket);
/* Wait up to timeout_us for a ticket (0: do not wait).  QUARK_OK consumes the ticket and fills
 * *out; QUARK_EAGAIN (timeout_us == 0) / QUARK_ETIMEDOUT if not done; QUARK_ENOTFOUND if the
 * ticket is unknown or already consumed. */
quark_status quark_serve_poll(quark_server* srv, uint64_t ticket, int timeout_us, quark_result* out);
/* Cancel a request that has not been admitted (QUARK_EBUSY once it runs). */
quark_status quark_serve_cancel(quark_server* srv, uint64_t ticket);
/* Hold (1) or resume (0) admissions; queued requests wait while held. */
quark_status quark_serve_pause(quark_server* srv, int paused);
quark_status quark_serve_stats(quark_server* srv, quark_stats* out);
/* Cancel queued requests, wait for running ones, stop the thread, free the resident pyramids. */
quark_status quark_serve_stop(quark_server* srv);

/* ---- Differentiation (spec form 3; the paper trains with differentiable rendering,
 * Sec. 3.1 and Sec. 3.4) -------------------------------------------------------------------------
 * The differentiable stage is the last Update & Fuse step and the final render, as a function
 * of the volume entering the step (V_in), the step's pyramid level (F) and the step's weights.
 * FP32 form only.  The backward pass is hand written: the over operator's reverse scan, the
 * blend softmax, the image sampling and its coordinates, the decode, the conv block, and the
 * one-to-many attention with its sampling (feature gradient scattered into F with atomics,
 * coordinate gradient through the decoded depth).  The sampled features are recomputed in the
 * backward pass, not stored by the forward. */

/* Volume entering step `scale` (collapse and x2 upsample of step scale-1's output), written to
 * v_in [L][H][W][C] (device, float32).  Needs steps 0..scale-1 done on `ldm`. */
quark_status quark_step_input(quark_ctx* ctx, quark_ldm* ldm, int scale, float* v_in, void* stream);

/* Forward of the stage: last step from v_in [L][H][W][C] with level features feat [V][h][w][C]
 * (device float32, e.g. a copy of the pyramid's level; 32-byte aligned, as cudaMalloc and
 * PyTorch's allocator give, since the sampling reads it in 256-bit loads, else QUARK_EINVAL), then
 * the render into rgba [H][W][4] (device).  `pyr` provides the cameras and the images the render
 * samples. */
quark_status quark_stage_forward(quark_ctx* ctx, const quark_pyramid* pyr, const float* feat, const float* v_in,
                                 quark_ldm* ldm, float* rgba, void* stream);

/* Weight gradients of the stage (device float32, caller-owned, every field overwritten); shapes
 * as in quark_weights for the last step. */
typedef struct {
    float* attn_g;   /* [C] */
    float* Wq;       /* [C][h C] */
    float* Wo;       /* [h C][C] */
    float* W_beta;   /* [C][C] */
    float* conv_g;   /* [C] */
    float* conv1_w;  /* [3][3][C][C] */
    float* conv1_b;  /* [C] */
    float* conv2_w;  /* [3][3][C][C] */
    float* conv2_b;  /* [C] */
    float* w_d;      /* [C] */
    float* b_d;      /* [1] */
    float* w_sigma;  /* [C] */
    float* b_sigma;  /* [1] */
} quark_stage_grads;

/* Backward of the stage after quark_stage_forward on the same ldm / v_in / feat: from
 * dl_drgb [H][W][3] (gradient of the loss w.r.t. the output RGB) writes dv_in [L][H][W][C],
 * dfeat [V][h][w][C] and the weight gradients.  The feature gradient is accumulated with
 * atomics, so its last bits depend on scheduling; every other output is deterministic. */
quark_status quark_stage_backward(quark_ctx* ctx, const quark_pyramid* pyr, const float* feat, const float* v_in,
                                  quark_ldm* ldm, const float* dl_drgb, float* dv_in, float* dfeat,
                                  const quark_stage_grads* grads, void* stream);

/* ---- Backward pass through the whole network (spec form 3; the paper trains the whole
 * network end to end through its differentiable render, Sec. 3.1 and Sec. 3.4) ---------------
 * One backward call mirrors each forward call, in reverse order:
 *     quark_render_ldm_bwd                       (Sec. 3.1 Eq. 1, Sec. 3.2.3)
 *     quark_update_fuse_bwd(scale = n-1 .. 0)    (Sec. 3.2.2, Sec. 3.3)
 *     quark_encode_pyramid_bwd                   (Sec. 3.2.1)
 * FP32 form, uniform schedule, one-to-many attention, C = 16 or 32, without the ray encoding or
 * render-and-refine (EINVAL otherwise).  The forward must have run with quark_ldm_keep_steps on
 * the LDM and with every view of the pyramid.  The backward recomputes what it needs (the
 * volume entering each step, the normalised inputs and the first convolution of each conv block,
 * the sampled features -- nothing sampled is stored by the forward); the loss may depend on the
 * output RGB (not on its alpha channel).  All gradient buffers are device float32, caller-owned.
 * Weight gradients and the feature gradients are ACCUMULATED into (+=), so that the
 * contributions of every step and of several scenes sum in one set of buffers: zero them before
 * the first call.  The feature gradients are summed with atomics, so their last bits depend on
 * scheduling; everything else is deterministic. */

/* Weight gradients, shaped as the quark_weights fields.  A call needs the fields of the weights it
 * differentiates (EINVAL if NULL); the others may be NULL.  The appearance decoder W_a, b_a does
 * not reach the render (its colours are the input images', blended by beta), so it has no field. */
typedef struct {
    float* enc_w;   /* [3][3][3][C] */
    float* enc_b;   /* [C] */
    float* v0;      /* [C] */
    float* attn_g[QUARK_MAX_SCALES];
    float* Wq[QUARK_MAX_SCALES];
    float* Wo[QUARK_MAX_SCALES];
    float* conv_g[QUARK_MAX_SCALES];
    float* conv1_w[QUARK_MAX_SCALES];
    float* conv1_b[QUARK_MAX_SCALES];
    float* conv2_w[QUARK_MAX_SCALES];
    float* conv2_b[QUARK_MAX_SCALES];
    float* col_w1[QUARK_MAX_SCALES];  /* only where L halves into step j */
    float* col_b1[QUARK_MAX_SCALES];
    float* col_w2[QUARK_MAX_SCALES];
    float* col_b2[QUARK_MAX_SCALES];
    float* w_d;     /* [C] */
    float* b_d;     /* [1] */
    float* w_sigma; /* [C] */
    float* b_sigma; /* [1] */
    float* W_beta;  /* [C][C] */
} quark_grads;

/* keep = 1: every later quark_update_fuse on this LDM also copies its step's output volume and
 * the attention block's output ([L][H][W][C] each) into per-step buffers of the LDM, allocated on
 * first use and freed with the LDM; the backward pass reads them.  keep = 0: no copies. */
quark_status quark_ldm_keep_steps(quark_ldm* ldm, int keep);

/* Backward of quark_render_ldm (after every step ran on `ldm` with pyramid `pyr`):
 *   dl_drgb  [H_out][W_out][3] gradient of the loss w.r.t. the output RGB (device)
 *   dv_out   [L][H][W][C] gradient w.r.t. the last step's output volume (written), through the
 *            raw depth and density logits (the depth moves the image samples, Eq. depth_activation)
 *   dbeta    [H][W][L][V] gradient w.r.t. the last step's blend logits (written)
 *   g        w_d, b_d, w_sigma, b_sigma accumulated */
quark_status quark_render_ldm_bwd(quark_ctx* ctx, const quark_ldm* ldm, const quark_pyramid* pyr,
                                  const float* dl_drgb, float* dv_out, float* dbeta, const quark_grads* g,
                                  void* stream);

/* Backward of quark_update_fuse step `scale`:
 *   dv_out   [L][H][W][C] gradient w.r.t. the step's output volume (from the next step's
 *            backward, or from quark_render_ldm_bwd for the last step); read only
 *   dbeta    last step: the blend-logit gradient from quark_render_ldm_bwd; else ignored
 *   dv_prev  [L'][H'][W'][C] gradient w.r.t. step scale-1's output volume, through the x2
 *            upsample and the layer collapse (written); step 0: ignored (its input is v0)
 *   dfeat    [V][H_img/k][W_img/k][C] gradient w.r.t. pyramid level k = k[scale] (accumulated)
 *   g        the step's attention, conv-block and layer-collapse weights, W_beta (last step), v0
 *            (step 0), w_d and b_d (steps > 0: their depths are decoded from the entering volume)
 *            accumulated */
quark_status quark_update_fuse_bwd(quark_ctx* ctx, const quark_pyramid* pyr, int scale, quark_ldm* ldm,
                                   const float* dv_out, const float* dbeta, float* dv_prev, float* dfeat,
                                   const quark_grads* g, void* stream);

/* Backward of quark_encode_pyramid: from the gradients of the pyramid levels k = 1, 2, 4, 8
 * (dfeat[0..3], [V][H/k][W/k][C] each, NULL where no step used the level) through the 2x2
 * mean-pool chain and the 3x3 conv, accumulates g->enc_w and g->enc_b. */
quark_status quark_encode_pyramid_bwd(quark_ctx* ctx, const quark_pyramid* pyr, const float* const* dfeat,
                                      const quark_grads* g, void* stream);

/* Synchronise the context's device and report device-side failures: QUARK_ETIMEDOUT if a
 * kernel's bounded wait (on tensor-core completion) ran out since the last check, in which case
 * that launch's outputs are invalid; the error word is then cleared. */
quark_status quark_check_device(quark_ctx* ctx);

/* Test of the error path of the bounded waits (the context stays usable; nothing faults): the
 * next BF16 one-to-many sampling launch of this context (a quark_update_fuse step with attention)
 * leaves its query MMA chain unissued, so that its wait on the chain's completion -- an mbarrier
 * nothing arrives at -- runs out after 1 ms.  The kernel then records the timeout in the error
 * word, skips its outputs, frees its tensor memory and returns; quark_check_device reports
 * QUARK_ETIMEDOUT and clears the word, and later launches run normally.  The outputs of that one
 * step (and of anything computed from them) are invalid.  EINVAL for the FP32 form or standard
 * attention. */
quark_status quark_test_wait_timeout(quark_ctx* ctx);

/* Measured FP32 SIMT peak of CUDA device `device` (synchronous; allocates and frees a small
 * buffer): the FLOP rate of kernels that keep every FP32 lane busy with independent fused
 * multiply-add chains, as scalar FMAs (*fma_tflops) and as packed FP32x2 FMAs (*ffma2_tflops), in
 * TFLOP/s (2 FLOP per lane-FMA), best of three timed launches.  The denominator of the FP32
 * roofline fractions of the benchmark.  No counterpart in the paper. */
quark_status quark_measure_fp32_peak(int device, double* fma_tflops, double* ffma2_tflops);

/* Kernel accounting.  quark_launch_count returns the number of kernels this context has
 * launched since creation or the last reset.  With profiling on, every launch is bracketed
 * by CUDA events on its own stream and quark_kernel_times (which synchronises) returns, per
 * kernel family, the number of launches and the summed device time in ms.  names receives
 * at most `cap` entries; returns the number of families. */
uint64_t quark_launch_count(const quark_ctx* ctx);
void quark_reset_counters(quark_ctx* ctx);
quark_status quark_set_profiling(quark_ctx* ctx, int enable);
int quark_kernel_times(quark_ctx* ctx, const char** names, double* ms, uint64_t* launches, int cap);

#ifdef __cplusplus
}
#endif
#endif /* QUARK_H */
