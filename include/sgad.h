/*
 * sgad.h - C ABI of the GB300 (sm_103a) splatting library for pixel-aligned Gaussians
 * at adjusted depth (SGAD-SLAM mapping, CVPR 2026).
 *
 * The library renders keyframes of pixel-aligned Gaussians into camera views and
 * back-propagates image-space gradients into the Gaussians' parameters:
 *
 *   Sec. 3.1  each Gaussian carries a colour (3), one isotropic variance ("radius"), an
 *             opacity and a depth offset delta;
 *   Sec. 3.2  Gaussian j of keyframe i lies on the ray of pixel j at the adjusted depth
 *             |D_i(j) + delta_i(j)|, and (V'_k, D'_k) = splat(G_i, p_k) renders colour
 *             and depth into view k; Eq. 1 fits them to the observations, with only the
 *             current keyframe learnable (neighbours fixed);
 *   Supp. A   radius initialised to D/F; Adam learning rates per attribute.
 *
 * The splatting itself follows the 3DGS conventions the paper builds on (the paper
 * prints no formulas): EWA projection of the isotropic 3D Gaussian with a 0.3 px
 * dilation, square bounds of ceil(3 sqrt(lambda_max)) px, tiles of tile_w x tile_h
 * pixels, per-tile lists sorted front to back by (view-space depth rounded to f32,
 * global Gaussian index), alpha = min(0.99, sigmoid(logit) e^power), entries with
 * alpha < 1/255 skipped, the walk stopped before transmittance drops below 1e-4. Pixel
 * (u, v) has its centre at integer coordinates; the ray through it is
 * ((u - cx)/fx, (v - cy)/fy, 1); depth maps hold z-depth; Gaussians with view depth
 * <= 0.2 are culled. Depth is composited without normalisation: D' = sum_i w_i z_i.
 *
 * Conventions of this ABI
 *   - Every buffer argument is a DEVICE pointer owned by the caller unless stated. The
 *     library allocates no device memory: the caller passes one workspace buffer sized
 *     by sgad_workspace_size().
 *   - Float data is FP32. Images and per-keyframe planes are row-major [H][W]; colour is
 *     planar [3][H][W].
 *   - Poses are row-major 3x4 [R | t]: keyframes cam->world, views world->cam.
 *   - Global Gaussian index: keyframe-major (keyframe 0's pixels first), then the pixel
 *     index y * W + x inside the keyframe.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as void*, NULL =
 *     the legacy default stream) and never synchronise, except where stated
 *     (sgad_count_keys, sgad_check).
 *   - Inputs are validated on the host; a bad argument returns SGAD_ERR_INVALID_ARG and
 *     launches nothing. Failures found on the device (more keys than the workspace holds,
 *     a bounded wait that gave up) are recorded in the workspace and reported by
 *     sgad_check(). No call traps or aborts; sgad_last_error() gives a message for the
 *     last failing call on the calling thread.
 */
#ifndef SGAD_H
#define SGAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sgad_status;

#define SGAD_OK 0
#define SGAD_ERR_INVALID_ARG (-1)          /* a host-side argument check failed */
#define SGAD_ERR_CUDA (-2)                 /* a CUDA runtime call or launch failed */
#define SGAD_ERR_WORKSPACE_TOO_SMALL (-3)  /* ws_bytes below sgad_workspace_size() */
#define SGAD_ERR_KEY_OVERFLOW (-4)         /* device: more (tile, Gaussian) keys than key_capacity */
#define SGAD_ERR_TIMEOUT (-5)              /* device: a bounded wait gave up */
#define SGAD_ERR_UNSUPPORTED (-6)          /* option combination not supported */
#define SGAD_ERR_NO_FORWARD (-7)           /* backward on a workspace without a forward */

#define SGAD_MAX_KEYFRAMES 32
#define SGAD_MAX_VIEWS 64

/* Pinhole camera. pose: row-major 3x4 [R | t]. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float pose[12];
} sgad_camera;

/* One keyframe's Gaussians, one per pixel (Sec. 3.1, 3.2). All planes [H][W] device
 * FP32 (rgb [3][H][W]); cam.pose is cam->world. learnable = 0 marks a fixed neighbour
 * keyframe (Sec. 3.2: only the current frame's Gaussians are optimised): it is rendered
 * but receives no gradient.
 * world_transform (optional, device, 12 floats row-major 3x4 [R | t]): when not NULL,
 * every centre mu of this keyframe is rendered at R mu + t, read from device memory by
 * the projection kernels at launch time (so a transform a kernel updates takes effect
 * without the host; rendering-based camera initialisation moves fixed Gaussians by
 * W0^-1 E W0 instead of moving the view W0 by E). Only for fixed keyframes
 * (learnable = 0; SGAD_ERR_INVALID_ARG otherwise). */
typedef struct {
    const float *depth;          /* D: observed z-depth */
    const float *offset;         /* delta: learnable depth offset */
    const float *rgb;            /* colour, planar */
    const float *opacity_logit;  /* opacity = sigmoid(logit) */
    const float *scale;          /* s: isotropic standard deviation in metres */
    sgad_camera cam;
    int32_t learnable;
    const float *world_transform;
} sgad_keyframe;

/* Rendered images of one view (device, caller-owned, fully overwritten). */
typedef struct {
    float *rgb;                  /* [3][H][W] V' */
    float *depth;                /* [H][W] D' = sum_i w_i z_i */
    float *alpha;                /* [H][W] A = sum_i w_i */
} sgad_images;

/* d loss / d (rgb, depth, alpha) of one view (device). A NULL plane means zero.
 * d_pose (device, 12 floats, optional): when not NULL, sgad_backward writes
 * d loss / d W of this view's world->cam matrix W = [R | t] (row-major 3x4, the layout of
 * sgad_camera.pose), through t = R mu + t of every Gaussian's view-space centre (the 2D
 * covariance of an isotropic Gaussian does not involve R). This is the gradient the
 * rendering-based camera initialisation of tracking descends (Sec. 3.3,
 * "Initialization"). */
typedef struct {
    const float *d_rgb;
    const float *d_depth;
    const float *d_alpha;
    float *d_pose;
} sgad_image_grads;

/* Gradients of one keyframe's parameters (device, caller-owned). For learnable
 * keyframes every element is overwritten; fixed keyframes' pointers may be NULL and
 * are never touched. */
typedef struct {
    float *d_offset;
    float *d_rgb;                /* [3][H][W] */
    float *d_opacity_logit;
    float *d_scale;
} sgad_keyframe_grads;

/* Work split of a compositing pass (forward or backward) over the tiles of all views.
 * Every schedule computes the same images bit for bit and the same gradients up to the
 * order of floating-point additions. */
#define SGAD_SCHEDULE_TILES 0       /* one launch; one thread block per tile, in view order */
#define SGAD_SCHEDULE_PERSISTENT 1  /* one launch of as many blocks as are resident on the
                                       GPU; each block takes tiles from a queue ordered by
                                       list length, longest first */
#define SGAD_SCHEDULE_PER_VIEW 2    /* one launch per view (one block per tile) */

/* Backward compositing algorithm (default WARP_LOCAL). All give the same gradients up
 * to the order of floating-point additions.
 *   WARP_LOCAL: every warp independently takes (tile, 8x4 pixel block) units from a queue
 *     (heaviest tile first under the persistent schedule) and walks only the entries the
 *     forward's per-warp masks mark for its block, 32 per round with no block-wide
 *     barrier; per (entry, pixel) pair it keeps two numbers in shared memory, and one lane
 *     per entry sums them (bwd_batch does not apply).
 *   WARP_REDUCE: thread blocks walk the masked entries of a tile in batches of bwd_batch
 *     staged entries per block-wide barrier, evaluate each at all 32 pixels of a warp's
 *     block and reduce the per-pair moments over the warp.
 *   PAIRS: the forward records, per pixel and list chunk, which entries contributed
 *     (4 bytes per pixel per 32 entries walked); the backward walks only those pairs, one
 *     pixel per thread, and sums the per-pair moments per Gaussian with shared-memory
 *     atomics. */
#define SGAD_BWD_WARP_REDUCE 0
#define SGAD_BWD_PAIRS 1
#define SGAD_BWD_WARP_LOCAL 2

/* Options fixed at sgad_create() (sgad_autotune() may change tile shape, batches,
 * schedules and the backward algorithm). */
typedef struct {
    int32_t tile_w, tile_h;      /* 16x16 (default), 8x32 or 32x8 */
    float bg[3];                 /* background colour (default black) */
    int32_t sort_smem_cap;       /* tiles with more entries than this are sorted through
                                    global memory; 0 = default (6144); >= 64 */
    int32_t freeze_offset;       /* 1: delta is held fixed (Table 9 "Mode3"): d_offset is
                                    written as zeros */
    int32_t fwd_batch;           /* list entries staged per thread-block barrier in forward
                                    compositing: 128, 192, 256, 384, 512, 768 or 1024;
                                    0 = default (512) */
    int32_t bwd_batch;           /* the same for the warp-reduced backward; 0 = default (256) */
    int32_t fwd_schedule;        /* SGAD_SCHEDULE_* of forward compositing (default TILES) */
    int32_t bwd_schedule;        /* SGAD_SCHEDULE_* of backward compositing (default TILES) */
    int32_t bwd_algorithm;       /* SGAD_BWD_* (default WARP_LOCAL) */
    int32_t max_blocks;          /* persistent schedules: launch at most this many blocks
                                    (0 = as many as are resident on the GPU, the default);
                                    a small cap makes every block take many tiles, for
                                    tests of the queue on small problems */
    int32_t reserved[2];         /* must be zero */
} sgad_options;

typedef struct sgad_ctx sgad_ctx;

/* Fill *opt with the defaults above. */
sgad_status sgad_default_options(sgad_options *opt);

/* Create a context (host memory only). opt == NULL selects the defaults. */
sgad_status sgad_create(sgad_ctx **out, const sgad_options *opt);
void sgad_destroy(sgad_ctx *ctx);

/* Message describing the last failing call on this thread ("" if none). */
const char *sgad_last_error(void);

/* Bytes of workspace needed for a problem of this shape holding up to key_capacity
 * (tile, Gaussian) keys. Host arithmetic only. The workspace holds the per-Gaussian
 * world records and gradient accumulators (64 B per Gaussian), the tile rectangle of
 * every (Gaussian, view) pair (8 B each), per-tile offsets, counters, heavy-first order and the list of tiles sorted exactly (16 B per tile), the
 * per-pixel state kept for the backward pass (8 B per view pixel), two key arrays
 * (16 B per key), the per-pixel
 * contribution words of the pair-parallel backward (32 B per key + 1 KB per tile) and
 * the per-warp contribution masks the forward leaves for the warp-local and
 * warp-reduced backwards (1 B per key + 64 B per tile). */
sgad_status sgad_workspace_size(const sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                                const sgad_camera *views, int32_t n_views, int64_t key_capacity,
                                size_t *bytes);

/* Exact number of (tile, Gaussian) keys the forward pass will emit for these inputs.
 * Runs the projection and binning on `stream`, then SYNCHRONISES the stream. The
 * workspace must be at least sgad_workspace_size(..., key_capacity = 0). Not capturable
 * in a CUDA graph. */
sgad_status sgad_count_keys(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                            const sgad_camera *views, int32_t n_views, void *workspace,
                            size_t ws_bytes, int64_t *n_keys, void *stream);

/* Forward splatting (Sec. 3.2, splat(G, p_k)) of all keyframes into all views:
 * projection and tile binning of every (Gaussian, view) pair, a per-tile sort by
 * (depth, index), and front-to-back compositing of colour, depth and alpha.
 * out[k] receives view k. The per-pixel final transmittance and contributor count, the
 * sorted tile lists and, per warp of 8x4 pixels and chunk of 32 list entries, the mask
 * of entries that reached one of those pixels are kept in the workspace for
 * sgad_backward(). If the keys do
 * not fit in key_capacity the outputs are left untouched and sgad_check() reports
 * SGAD_ERR_KEY_OVERFLOW together with the count needed. */
sgad_status sgad_forward(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                         const sgad_camera *views, int32_t n_views, sgad_images *out,
                         void *workspace, size_t ws_bytes, int64_t key_capacity, void *stream);

/* Adjoint of the last sgad_forward() on this workspace (same kfs, views and options):
 * walks every pixel's list back to front over the entries the forward's masks mark,
 * recomputing transmittance by division from the saved final value, and accumulates
 * d loss / d (offset, colour, opacity logit, scale) of every learnable keyframe, summed
 * over views. */
sgad_status sgad_backward(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                          const sgad_camera *views, int32_t n_views,
                          const sgad_image_grads *grad_in, sgad_keyframe_grads *grads_out,
                          void *workspace, size_t ws_bytes, int64_t key_capacity, void *stream);

/* Project-written autotuner for one problem shape (synchronous; not capturable).
 * Sweeps the tile shapes {16x16, 8x32, 32x8}, the batch sizes {128, 192, 256, 384, 512}
 * (forward also 768 and 1024)
 * and the schedules {TILES, PERSISTENT} of both compositing passes (and, for the
 * backward, the warp-local algorithm, reported with batch -1, and the pair-parallel
 * algorithm, reported with batch 0 and charged with the cost of the contribution words
 * its forward writes), timing each candidate
 * with CUDA events on `stream` (median of `reps` runs after one warm-up), and stores the
 * fastest combination in ctx's options: per tile shape, binning + emission + sort is
 * timed once, then each (batch, schedule) of forward compositing, then of backward
 * compositing (including the clearing of the gradient accumulators) on the gradients
 * grad_in; the shape with the smallest sum of the three best times wins.
 *
 * kfs, views, out, grad_in and grads_out are as for sgad_forward() / sgad_backward();
 * the workspace must hold the keys of every tile shape tried (a shape whose keys do not
 * fit is skipped and reported with ms = -1). The contents of out, grads_out and the
 * workspace are unspecified afterwards, and the key count depends on the tile shape:
 * size the workspace again (sgad_count_keys) before the next sgad_forward().
 * entries (host memory, up to max_entries) receives one row per timed candidate;
 * *n_entries the number of rows written (both may be NULL / 0). */
#define SGAD_TUNE_PREP 0         /* binning + emission + sort; batch and schedule are 0 */
#define SGAD_TUNE_FWD 1          /* forward compositing */
#define SGAD_TUNE_BWD 2          /* backward compositing */
typedef struct {
    int32_t tile_w, tile_h, stage, batch, schedule;
    float ms;
} sgad_tune_entry;

sgad_status sgad_autotune(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                          const sgad_camera *views, int32_t n_views, sgad_images *out,
                          const sgad_image_grads *grad_in, sgad_keyframe_grads *grads_out,
                          void *workspace, size_t ws_bytes, int32_t reps,
                          sgad_tune_entry *entries, int32_t max_entries, int32_t *n_entries,
                          void *stream);

/* The options ctx currently uses (after sgad_autotune(), its choice). */
sgad_status sgad_get_options(const sgad_ctx *ctx, sgad_options *opt);

/* Synchronise `stream`, then read the device-side status of the workspace: the first
 * error recorded by any forward since the previous sgad_check() (SGAD_OK,
 * SGAD_ERR_KEY_OVERFLOW or SGAD_ERR_TIMEOUT), and clear it. *keys_needed receives the
 * largest key count a forward needed since then, *n_keys the key count of the last
 * forward (both may be NULL). The status block is the first 256 bytes of the workspace:
 * sgad_count_keys() zeroes it; a workspace used without it must start with those bytes
 * zeroed. */
sgad_status sgad_check(sgad_ctx *ctx, void *workspace, size_t ws_bytes, int64_t *n_keys,
                       int64_t *keys_needed, void *stream);

/* Device views into the workspace after a forward, for inspection and tests. All
 * pointers are device pointers inside the workspace; lengths follow from the problem
 * shape: tile_offsets has n_tiles + 1 uint32 entries (tile t's sorted list is
 * entries[tile_offsets[t] .. tile_offsets[t+1])); each entry is
 * (f32 bits of the view depth << 32) | global Gaussian index; t_final and n_contrib
 * hold one value per view pixel, views concatenated. */
typedef struct {
    const uint32_t *tile_offsets;
    const uint64_t *entries;
    const float *t_final;
    const uint32_t *n_contrib;
    int32_t n_tiles;
    int64_t n_pixels;
} sgad_state_view;

sgad_status sgad_state(const sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                       const sgad_camera *views, int32_t n_views, void *workspace,
                       size_t ws_bytes, int64_t key_capacity, sgad_state_view *out);

/* Work counters of the last forward on this workspace (synchronises `stream`): keys
 * emitted, keys needed, (pixel, entry) pairs composited (the contributors: alpha >= 1/255
 * before the stop), pairs whose alpha was evaluated, and tiles the one-pass bucket sort
 * handed to the exact radix sort (a bucket of many near-equal depths, or a long list).
 * Host memory out. */
typedef struct {
    int64_t n_keys;
    int64_t keys_needed;
    int64_t n_pairs;
    int64_t n_evals;
    int64_t n_sort_exact;
} sgad_stats;

sgad_status sgad_read_stats(sgad_ctx *ctx, void *workspace, size_t ws_bytes, sgad_stats *out,
                            void *stream);

/* Per-stage timing. When enabled, sgad_forward / sgad_backward record CUDA events on
 * their stream between stages; sgad_profile_read waits for them and returns the last
 * call's stage times in milliseconds, in this order:
 *   0 projection + binning count + scan   1 key emission   2 per-tile sort
 *   3 forward compositing                 4 backward compositing (incl. clearing the
 *                                           gradient accumulators)
 *   5 gradient finalisation (d delta, d logit)
 * A stage of a call that was not made reads 0. */
#define SGAD_NUM_STAGES 6
sgad_status sgad_profile_enable(sgad_ctx *ctx, int32_t enable);
sgad_status sgad_profile_read(sgad_ctx *ctx, float *ms /* [SGAD_NUM_STAGES] */);

/* L1 terms of the mapping loss Eq. 1 (the SSIM term is not included), per view:
 *   rgb_weight   * mean over pixels and channels |V' - V|
 * + depth_weight * mean over pixels with target depth > 0 of |D' - D|,
 * summed over views. Writes d loss / d V' into d_rgb[k] ([3][H][W]) and d loss / d D'
 * into d_depth[k] ([H][W]) with sign(0) = 0, and adds the loss value to *loss_accum (one
 * device float, zeroed by the caller; may be NULL). target_depth and d_depth may be NULL
 * when depth_weight == 0. valid_count is caller-owned device scratch of n_views uint32
 * (the valid-depth pixel count U_k per view; overwritten), required when depth_weight
 * != 0. min_alpha: pixels whose rendered alpha (rendered[k].alpha) is at most min_alpha
 * add no loss and get zero gradients (the silhouette mask of rendering-based tracking,
 * Sec. 3.3 "Initialization"; the means keep their denominators); a negative value keeps
 * every pixel and does not read the alpha images. */
sgad_status sgad_l1_loss_grad(int32_t n_views, const sgad_camera *views,
                              const sgad_images *rendered, const float *const *target_rgb,
                              const float *const *target_depth, float rgb_weight,
                              float depth_weight, float min_alpha, float *const *d_rgb, float *const *d_depth,
                              float *loss_accum, uint32_t *valid_count, void *stream);

/* SSIM term of the mapping loss Eq. 1 (tau L_S, L_S the SSIM loss between the observed
 * colour V_k and the rendering V'_k; Sec. 3.2). The paper cites the SSIM of Wang et
 * al. 2004 without window details; this library reads it as: per colour channel, an
 * 11 x 11 Gaussian window of standard deviation 1.5 (weights normalised to sum 1), zero
 * padding outside the image, C1 = 0.01^2, C2 = 0.03^2, and
 *   L_S = 1 - mean over pixels and channels of SSIM(V', V).
 *
 * sgad_ssim_workspace_size: bytes of device scratch sgad_ssim_loss_grad needs for these
 * views (9 floats per pixel per view, each view's block 256-byte aligned).
 *
 * sgad_ssim_loss_grad: for every view k (device pointers, [3][H][W] FP32 planar, W and H
 * from views[k]) adds weight * L_S(rendered[k].rgb, target_rgb[k]) to *loss_accum (one
 * device float; may be NULL) and ADDS weight * d L_S / d V'_k into d_rgb[k], so it runs
 * after sgad_l1_loss_grad, which overwrites d_rgb. Only rendered[k].rgb is read.
 * workspace: caller-owned device memory of at least the size above, 256-byte aligned,
 * overwritten. Two kernel launches on `stream`, no host synchronisation.
 * Errors: SGAD_ERR_INVALID_ARG for a NULL pointer, a view count outside
 * [1, SGAD_MAX_VIEWS], a view size outside [1, 16384], a misaligned workspace or a
 * non-finite weight; SGAD_ERR_WORKSPACE_TOO_SMALL; SGAD_ERR_CUDA when a launch fails. */
sgad_status sgad_ssim_workspace_size(int32_t n_views, const sgad_camera *views, size_t *bytes);
sgad_status sgad_ssim_loss_grad(int32_t n_views, const sgad_camera *views,
                                const sgad_images *rendered, const float *const *target_rgb,
                                float weight, float *const *d_rgb, float *loss_accum,
                                void *workspace, size_t ws_bytes, void *stream);

/* FP32 FMA throughput probe: launches `blocks` blocks of 256 threads, each thread running
 * 8 independent chains of 16 * iters dependent FMAs, on `stream`, and sets *flops (host)
 * to the floating-point operations the launch performs (2 per FMA). Timing it with events
 * on the stream gives the device's measured FP32 peak, the denominator of the
 * compositing kernels' roofline. sink: device float [blocks * 256], written only in a
 * case that does not occur (it keeps the arithmetic from being removed). */
sgad_status sgad_fma_burn(int32_t blocks, int32_t iters, float *sink, double *flops, void *stream);

/* One bias-corrected Adam step (PyTorch convention) on `n` FP32 parameters in place:
 *   m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
 *   p <- p - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * Supp. A gives the learning rates: colour 0.0025, radius 0.005, opacity 0.05,
 * offset 0.01. With mode SGAD_ADAM_LOG the array holds s = exp(p) > 0 (the scale): the
 * step is taken on p = log s with gradient s * d/ds, and s = exp(p) is written back,
 * which is the parameterisation the radius learning rate refers to. */
#define SGAD_ADAM_PLAIN 0
#define SGAD_ADAM_LOG 1
sgad_status sgad_adam_step(int64_t n, float *param, const float *grad, float *m, float *v,
                           float lr, float beta1, float beta2, float eps, int32_t step,
                           int32_t mode, void *stream);

/* One tensor of a multi-tensor Adam step (device pointers, n elements each). */
typedef struct {
    float *param;
    const float *grad;
    float *m;
    float *v;
    int64_t n;
    float lr;
    int32_t mode;                /* SGAD_ADAM_PLAIN or SGAD_ADAM_LOG */
} sgad_adam_tensor;

#define SGAD_ADAM_MAX_TENSORS 256

/* The Adam step above over up to SGAD_ADAM_MAX_TENSORS tensors in one launch. The step
 * number lives in device memory: *step_counter (a device int32, 0 before the first step)
 * counts the steps taken; this call uses step = *step_counter + 1 and then increments
 * it, so the call can be captured once in a CUDA graph and replayed. */
sgad_status sgad_adam_step_multi(int32_t n_tensors, const sgad_adam_tensor *tensors, float beta1,
                                 float beta2, float eps, int32_t *step_counter, void *stream);

/* One step of the rendering-based camera initialisation of tracking (Sec. 3.3,
 * "Initialization") on the device, with no host round trip. The view stays at its
 * world->cam pose W0 (view_pose, host, row-major 3x4) and the fixed Gaussians move by
 * M = W0^-1 E W0, where E is the camera correction accumulated so far: rendering
 * M mu into W0 equals rendering mu into E W0. state (device, SGAD_POSE_STATE_FLOATS
 * floats, caller-owned; set E and M to the identity [I | 0] and the rest to zero before
 * the first step) holds E (state[0..11]), M (state[12..23], the keyframes'
 * world_transform), the Adam moments m (24..29) and v (30..35), the step count (36) and
 * the current pose E W0 (37..48). From d_pose (device, 12 floats: d loss / d W0 of the
 * last sgad_backward), the gradient of a left twist xi = (omega, v) of the pose is
 * d/d v = the translation column c of d_pose and d/d omega = vee(R0 G^T - G R0^T) +
 * t0 x c (G its rotation block); Adam (beta1, beta2, eps, bias-corrected) with step
 * lr_rot on omega and lr_trans on v gives xi, and E <- exp(xi) E (rotation by Rodrigues'
 * formula, translation v). Evaluated in FP64 by one thread. */
#define SGAD_POSE_STATE_FLOATS 64
sgad_status sgad_pose_adam_step(const float *d_pose, const float *view_pose, float *state,
                                float lr_rot, float lr_trans, float beta1, float beta2, float eps,
                                void *stream);

/* Forward splatting that allocates nothing, for callers that cannot allocate device
 * memory (code running in a host callback or a real-time loop where cudaMalloc would
 * stall the device, or an application whose memory manager owns every allocation and
 * hands this library only its input and output buffers). The paper has no counterpart:
 * this is an interface convenience around sgad_forward().
 *
 * Same arguments and results as sgad_forward(), without the workspace: the scratch is a
 * static device array of SGAD_NOALLOC_SCRATCH_BYTES inside the library, which every GPU
 * that loads the library holds until the process exits. Problems whose workspace does
 * not fit (the workspace of sgad_workspace_size: 64 B per Gaussian, 8 B per Gaussian
 * and view, 8 B per view pixel, 49 B per key and ~1.1 KB per tile) are rejected with
 * SGAD_ERR_WORKSPACE_TOO_SMALL before anything is launched; a forward whose keys exceed
 * the room left returns SGAD_ERR_KEY_OVERFLOW. The call synchronises `stream` to report
 * that status. Every call looks up the array's device address in the current device's
 * context (cudaGetSymbolAddress, a host-side lookup); the first call on a device also
 * loads the library's device code there and should come before any stream capture on
 * that device. All calls share the one array and it keeps the last call's contents:
 * calls that may run concurrently on the GPU (different streams or threads) race and
 * must be serialised by the caller. No backward pass is offered this way (its state
 * would live in the shared array). */
#define SGAD_NOALLOC_SCRATCH_BYTES (64u << 20)
sgad_status sgad_forward_noalloc(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                                 const sgad_camera *views, int32_t n_views, sgad_images *out,
                                 void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SGAD_H */
