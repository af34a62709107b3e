/*
 * FP64 CPU oracle for the splatting of pixel-aligned Gaussians at adjusted depth.
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously-correct definition the
 * CUDA library is checked against. Only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark may load it; the product path never does. It shares no
 * code, header, table or helper with the CUDA library.
 *
 * What it computes (paper: "SGAD-SLAM", Sec. 3.1 simplified Gaussians, Sec. 3.2 mapping,
 * Eq. 1, and the implementation details of the supplementary Sec. A):
 *   - Gaussian j of keyframe i sits on the ray of pixel j at the adjusted depth
 *     |D_i(j) + delta_i(j)| (Sec. 3.2, "Pixel-Aligned Gaussians at Adjusted Depth");
 *   - each Gaussian has colour (3), one isotropic scale, an opacity and the offset
 *     (Sec. 3.1);
 *   - (V'_k, D'_k) = splat(G_i, p_k) is 3DGS-style tile splatting (Sec. 3.2, "Rendering
 *     RGB and Depth by Splatting"); the paper gives no formulas, so the 3DGS conventions
 *     are taken (EWA projection with a 0.3 px dilation, 3-sigma square bounds, 16x16
 *     tiles, alpha capped at 0.99, alpha < 1/255 skipped, stop before T drops below
 *     1e-4, sigmoid opacity, black background, depth composited without normalisation);
 *   - the adjoint of all of the above into delta, colour, opacity logit and scale.
 *
 * Inputs are FP64 arrays; the tests pass exact upcasts of the float32 arrays the CUDA
 * library receives (and perturb them in FP64 for finite differences).
 *
 * Values (positions, conics, alphas, transmittance, images, gradients) are computed in
 * FP64. Every discrete decision (near-plane cull, the integer radius, the tile bounds,
 * power > 0, the alpha floor and cap, the transmittance stop) is an integer decided by
 * floating point, and is taken in the precision the kernel uses, FP32, evaluating the
 * same formulas in the same order with IEEE single-precision operations (fmaf where the
 * kernel fuses). Binning therefore matches the kernel bit for bit. The alpha decisions
 * involve exp, whose single-precision implementations differ in the last bits, so they
 * are reported "near" when within opts.margin (4e-6) relative of their threshold (the
 * transmittance stop, which accumulates those differences, within opts.t_margin, 2e-4).
 * The depth key is t_z
 * evaluated in FP64 and rounded once to f32; it is near when within 1e-12 relative of an
 * f32 rounding midpoint.
 */
#ifndef SGAD_ORACLE_H
#define SGAD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;
    double pose[12];            /* row-major 3x4; keyframes: cam->world, views: world->cam */
} orc_cam;

typedef struct {
    orc_cam cam;
    const double *depth;        /* [H][W] z-depth D */
    const double *offset;       /* [H][W] delta */
    const double *rgb;          /* [3][H][W] */
    const double *logit;        /* [H][W] opacity logit */
    const double *scale;        /* [H][W] isotropic std-dev s (metres) */
    int32_t learnable;          /* 0: fixed neighbour, its gradients are not produced */
} orc_kf;

typedef struct {
    int32_t tile_w, tile_h;
    double bg[3];               /* background colour */
    double margin;              /* relative margin of the alpha floor/cap decisions (4e-6) */
    double t_margin;            /* relative margin of the transmittance stop (2e-4) */
} orc_opts;

/* The f32 rounding of the depth key lies within 1e-12 of a rounding midpoint (the key
 * bits may differ; the order does not, short of an exact depth tie). */
#define ORC_NEAR_Z 64

/* Projection of one Gaussian into one view. The FP32 fields are the decision values
 * (the kernel's arithmetic); the others are FP64 values. */
typedef struct {
    int32_t visible;            /* passed the near plane (FP32 t_z > 0.2) */
    int32_t tx0, tx1, ty0, ty1; /* inclusive tile rectangle; empty when tx0 > tx1 */
    int32_t ntiles;
    int32_t near;               /* ORC_NEAR_Z or 0 */
    int32_t pad_;
    double mu[3];               /* world-space centre */
    double t[3];                /* view-space centre */
    double p[2];                /* pixel-space mean */
    double cov[3];              /* 2D covariance (xx, xy, yy) */
    double conic[3];            /* its inverse (a, b, c) */
    double o;                   /* sigmoid(logit) */
    double rho;                 /* integer pixel radius (FP32 decision) */
    double zf;                  /* t_z rounded once to f32 */
    double s;                   /* scale */
    double color[3];
    float pf[2];                /* FP32 pixel-space mean */
    float conicf[3];            /* FP32 conic */
    float of;                   /* FP32 opacity */
} orc_proj;

/* Per view, per pixel forward outputs. */
typedef struct {
    double *rgb;                /* [3][H][W] */
    double *depth;              /* [H][W] */
    double *alpha;              /* [H][W] */
    double *t_final;            /* [H][W] */
    int32_t *n_contrib;         /* [H][W] 1 + list position of the last contributor, 0 if none */
    uint8_t *near;              /* [H][W] 1 if a decision on this pixel's walk is near */
} orc_image;

/* Gradients of one keyframe (learnable ones only). */
typedef struct {
    double *d_offset;           /* [H][W] */
    double *d_rgb;              /* [3][H][W] */
    double *d_logit;            /* [H][W] */
    double *d_scale;            /* [H][W] */
} orc_kf_grads;

/* Image-space gradient of the loss for one view. */
typedef struct {
    const double *d_rgb;        /* [3][H][W] */
    const double *d_depth;      /* [H][W] */
    const double *d_alpha;      /* [H][W] */
} orc_image_grads;

int64_t orc_num_gaussians(const orc_kf *kfs, int32_t n_kf);
int32_t orc_num_tiles(const orc_cam *views, int32_t n_views, const orc_opts *opt);

/* Project every Gaussian (global index order: keyframe-major, then pixel row-major)
 * into one view. */
int32_t orc_project(const orc_kf *kfs, int32_t n_kf, const orc_cam *view, const orc_opts *opt,
                    orc_proj *out);

/* Brute-force key list: for every view, every tile and every Gaussian, a key
 * (global tile << 32 | f32 bits of z) when the Gaussian's tile rectangle contains the
 * tile; sorted by (key, Gaussian index). Pass keys == NULL to get the count only.
 * near_out[i] = 1 when entry i belongs to a (view, Gaussian) with a near decision. */
int64_t orc_keys(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                 const orc_opts *opt, uint64_t *keys, uint32_t *vals, uint8_t *near_out);

/* Forward render of every view. */
int32_t orc_render(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                   const orc_opts *opt, orc_image *out);

/* Forward render of selected pixels (view index, x, y); outputs are per pixel
 * (rgb interleaved [n][3]). */
int32_t orc_render_pixels(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                          const orc_opts *opt, int64_t n_px, const int32_t *px_view,
                          const int32_t *px_x, const int32_t *px_y, double *rgb, double *depth,
                          double *alpha, double *t_final, int32_t *n_contrib, uint8_t *near);

/* Adjoint: gradients of L = sum_views <grad_in, (rgb, depth, alpha)> with respect to the
 * offset, colour, opacity logit and scale of every learnable keyframe. Overwrites the
 * gradient arrays of learnable keyframes; fixed keyframes are not touched.
 * near_gauss (optional, one byte per Gaussian, global index) is set to 1 for every
 * Gaussian whose alpha passes (or nearly passes) the floor at a pixel with a near
 * decision: its gradient includes a term FP32 may legitimately drop or add.
 * abs_out (optional, [n_gaussians][6] in the order d_offset, d_r, d_g, d_b, d_logit,
 * d_scale) receives, per Gaussian, the sum over views and pixels of the absolute value
 * of each pixel's contribution: the scale against which the rounding error of a sum
 * with cancellation is measured. */
int32_t orc_backward(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                     const orc_opts *opt, const orc_image_grads *grad_in, orc_kf_grads *grads,
                     uint8_t *near_gauss, double *abs_out);

/* Adjoint into the view poses: d_pose[k][12] = d loss / d W_k for the row-major 3x4
 * world->cam matrix W_k = [R_k | t_k] of view k. Through t = R_k mu + t_k only (the 2D
 * covariance s^2 J J^T + 0.3 I does not involve R_k for an isotropic Gaussian):
 * d L / d R_k[a][b] = sum_g d L / d t_g[a] mu_g[b], d L / d t_k[a] = sum_g d L / d t_g[a].
 * abs_pose (optional, [n_views][12]): the sum over pixels and Gaussians of the magnitude
 * of each pixel's contribution (the scale of the sum's rounding error). This is the
 * gradient the rendering-based camera initialisation of tracking (Sec. 3.3,
 * "Initialization": minimise the rendering error of the new frame against the previous
 * frame's Gaussians) descends. */
int32_t orc_backward_pose(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                          const orc_opts *opt, const orc_image_grads *grad_in, double *d_pose,
                          double *abs_pose);

/* Adjoint restricted to a list of Gaussians (global indices): out[n][6] =
 * (d_offset, d_r, d_g, d_b, d_logit, d_scale). Only the tiles these Gaussians touch are
 * walked, so it runs on full-size scenes. near_sel (optional, n bytes) and abs_sel
 * (optional, [n][6]) as near_gauss and abs_out above for the selected Gaussians. */
int32_t orc_backward_gaussians(const orc_kf *kfs, int32_t n_kf, const orc_cam *views,
                               int32_t n_views, const orc_opts *opt,
                               const orc_image_grads *grad_in, int64_t n_sel,
                               const int64_t *sel, double *out, uint8_t *near_sel, double *abs_sel);

/* Fingerprint of every discrete decision of a forward pass (binning and, per pixel, the
 * accepted entries and the stopping point). Two parameter sets with equal fingerprints
 * take the same branches. */
uint64_t orc_decision_hash(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                           const orc_opts *opt);

/* L1 mapping loss of Eq. 1 without the SSIM term, per view:
 *   rgb_w * mean_{px,ch} |V - V'| + depth_w * mean_{px: D > 0} |D - D'|
 * summed over views. Writes d loss / d (V', D') (sign(0) = 0) and returns the loss. */
double orc_l1_loss(int32_t n_views, const orc_cam *views, const double *const *rgb,
                   const double *const *depth, const double *const *target_rgb,
                   const double *const *target_depth, double rgb_w, double depth_w,
                   double *const *d_rgb, double *const *d_depth);

/* One Adam step (PyTorch convention, bias-corrected) on n parameters, in FP64. With
 * log_param != 0 the array holds s = exp(p): the step is taken on p = log s with
 * gradient s * grad, and exp(p) is written back. */
void orc_adam(int64_t n, double *param, const double *grad, double *m, double *v, double lr,
              double beta1, double beta2, double eps, int32_t step, int32_t log_param);

#ifdef __cplusplus
}
#endif
#endif
