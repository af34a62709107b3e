/*
 * sgad_gicp.h - C ABI of the geometric tracking of SGAD-SLAM (Sec. 3.3 "Matching a Frame
 * to a Scene" and "Generalized ICP for Matching", Eq. 2; the scale normalisation of the
 * ablation study; the downsampling ratio R and neighbour count K_c of Supp. A).
 *
 * A depth map D_i becomes a set T_i of geometry Gaussians: the pixels (u, v) with u and v
 * multiples of R and depth > 0, in raster order, back-projected to
 * p = d ((u - cx) / fx, (v - cy) / fy, 1); each with the covariance of its K_c nearest
 * selected points (itself included, FP32 squared distances ((dx dx + dy dy) + dz dz),
 * ties by index, all of them when fewer; (1 / K) sum (p - m)(p - m)^T over the K used),
 * decomposed into scales and rotation
 * (eigen-decomposition of the symmetric matrix, the SVD the paper cites), the scales
 * normalised (s / max s, each floored at sqrt(eps)) and the covariance rebuilt from them;
 * the normal is the axis of the smallest scale. A global set T holds the scene's
 * geometry Gaussians in the world frame. GICP estimates the frame's cam->world pose:
 * every iteration matches each source Gaussian, moved into the world by the current pose
 * (x = R a + t in FP32, each coordinate ((r0 a0 + r1 a1) + r2 a2) + t), to the map
 * Gaussian with the smallest point-to-surface distance |n_b . (mu_b - x)| among its
 * k_match nearest map Gaussians within r_max (ties by squared distance, then index), and
 * takes one Gauss-Newton step on Eq. 2, read with the inverse of GICP:
 *   sum e^T (C_b + R C_a R^T)^-1 e,  e = mu_b - (R a + t),
 * on a left perturbation (Jacobian [[x]_x, -I], covariance term fixed within the step),
 * update R <- Exp(omega) R, t <- Exp(omega) t + v, until |xi| < tol or max_iters. The
 * map then takes the source Gaussians with no map Gaussian within d_overlap (in source
 * order), rotated into the world.
 *
 * Conventions: as in sgad.h. Every array is a caller-owned DEVICE buffer; the caller
 * passes one workspace sized by sgad_gicp_workspace_size(). Poses are row-major 3x4
 * cam->world. Calls are asynchronous on `stream` except sgad_gicp_result (synchronous).
 * Bad host arguments return SGAD_ERR_INVALID_ARG and launch nothing; capacity overflow
 * and degenerate systems found on the device are recorded in the workspace and reported
 * by sgad_gicp_result.
 */
#ifndef SGAD_GICP_H
#define SGAD_GICP_H

#include "sgad.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t stride;       /* R >= 1 (Supp. A: 10 for Replica-like, 5 for TUM-like frames) */
    int32_t k_cov;        /* K_c in [3, 32] (Supp. A: 10, 15 or 23) */
    int32_t k_match;      /* correspondence candidates in [1, 8] */
    int32_t max_iters;    /* GICP iterations in [1, 100] */
    float r_max;          /* correspondence radius in metres (> 0) */
    float d_overlap;      /* map update: overlap distance in metres (>= 0) */
    float tol;            /* stop when |xi| < tol (>= 0) */
    float eps;            /* floor of the normalised variances, in (0, 1] */
    int32_t src_capacity; /* largest source set the workspace serves, in [1, 2^24] */
    int32_t map_capacity; /* largest map the workspace serves, in [1, 2^24] */
} sgad_gicp_params;

/* A set of geometry Gaussians (caller-owned device arrays, `capacity` records each). */
typedef struct {
    float *pos;           /* [capacity][4]: x, y, z, 0 (16-byte aligned) */
    float *cov;           /* [capacity][8]: xx, xy, xz, yy, yz, zz, 0, 0 (normalised; 16-byte aligned) */
    float *normal;        /* [capacity][4]: unit normal, 0 */
    int32_t *count;       /* one device int32: records held (written by the producers) */
    int32_t capacity;
} sgad_gaussian_set;

typedef struct {
    int32_t iterations;   /* GICP iterations taken by the last sgad_gicp_track */
    int32_t converged;    /* 1 if |xi| < tol ended it */
    int32_t n_matches;    /* correspondences of the last iteration */
    int32_t status;       /* bit 0: a set overflowed its capacity (cleared by
                             sgad_gicp_frame, set by it or by sgad_gicp_insert);
                             bit 1: fewer than 6 correspondences or a singular system
                             ended the last sgad_gicp_track */
    double cost;          /* Eq. 2 at the start of the last iteration */
    double step;          /* |xi| of the last iteration */
} sgad_gicp_stats;

/* R 10, K_c 10, k_match 5, 30 iterations, r_max 0.1 m, d_overlap 0.02 m, tol 1e-6,
 * eps 1e-3, capacities 2^16 (source) and 2^20 (map). */
sgad_status sgad_gicp_default_params(sgad_gicp_params *out);

/* Workspace bytes for these parameters (state, the map's and the source's hash grids,
 * per-block partial sums, scratch). Every call computes the workspace's layout from the
 * parameters it is given, so all calls on one workspace take the same capacities; a set
 * passed to a call may be smaller than its capacity in the parameters. */
sgad_status sgad_gicp_workspace_size(const sgad_gicp_params *p, size_t *bytes);

/* T_i of a depth map (device [H][W] FP32, z-depth, 0 = invalid) in the camera frame into
 * `out` (its count is written). pix_out (device int32 [capacity], may be NULL) receives
 * each Gaussian's pixel index v * W + u; knn_out (device int32 [capacity][k_cov], may be
 * NULL) each Gaussian's K_c neighbours, nearest first. Selected pixels beyond
 * out->capacity are dropped and flagged. cam->pose is not used. */
sgad_status sgad_gicp_frame(const sgad_gicp_params *p, const sgad_camera *cam, const float *depth,
                            const sgad_gaussian_set *out, int32_t *pix_out, int32_t *knn_out, void *workspace,
                            size_t ws_bytes, void *stream);

/* The map's spatial hash grid (cells of max(r_max, d_overlap) / 3; searches visit rings
 * of cells until their result is proven). Required after the caller changes the map;
 * sgad_gicp_insert rebuilds it itself. */
sgad_status sgad_gicp_index(const sgad_gicp_params *p, const sgad_gaussian_set *map, void *workspace,
                            size_t ws_bytes, void *stream);

/* Correspondence of every source Gaussian at the host pose (cam->world, row-major 3x4):
 * idx_out (device int32 [src capacity]) = map index or -1. */
sgad_status sgad_gicp_correspond(const sgad_gicp_params *p, const sgad_gaussian_set *src,
                                 const sgad_gaussian_set *map, const float pose[12], int32_t *idx_out,
                                 void *workspace, size_t ws_bytes, void *stream);

/* The Gauss-Newton system of Eq. 2 at the host pose, summed in FP64 over the per-block
 * FP32 partial sums: system_out (device double [29]) = H's upper triangle row by row
 * (21), g = sum J^T M e (6), the cost (1), the number of correspondences (1). */
sgad_status sgad_gicp_linearize(const sgad_gicp_params *p, const sgad_gaussian_set *src,
                                const sgad_gaussian_set *map, const float pose[12], double *system_out,
                                void *workspace, size_t ws_bytes, void *stream);

/* Sets the workspace's pose (cam->world, FP64 host array) without tracking. */
sgad_status sgad_gicp_set_pose(const double pose[12], void *workspace, size_t ws_bytes, void *stream);

/* GICP of the source set against the map (whose index must be current) from the host
 * initial pose, or from the workspace's pose (sgad_gicp_set_pose, or the last estimate)
 * when pose0 is NULL, so that a frame's calls can be captured once in a CUDA graph and
 * replayed with a new starting pose; the estimate stays in the workspace (read by
 * sgad_gicp_result, used by sgad_gicp_insert). 1 + max_iters kernel launches (the last block of each iteration
 * solves and updates the pose); iterations after convergence exit
 * at once. Capturable in a CUDA graph. */
sgad_status sgad_gicp_track(const sgad_gicp_params *p, const sgad_gaussian_set *src,
                            const sgad_gaussian_set *map, const double pose0[12], void *workspace,
                            size_t ws_bytes, void *stream);

/* Adds the source Gaussians that no map Gaussian overlaps, moved by the workspace's pose,
 * to the map (count updated; records beyond map->capacity dropped and flagged), then
 * rebuilds the index. */
sgad_status sgad_gicp_insert(const sgad_gicp_params *p, const sgad_gaussian_set *src,
                             const sgad_gaussian_set *map, void *workspace, size_t ws_bytes, void *stream);

/* Synchronises `stream` and reads the workspace's pose (FP64, may be NULL) and stats
 * (may be NULL). */
sgad_status sgad_gicp_result(void *workspace, size_t ws_bytes, double pose[12], sgad_gicp_stats *stats,
                             void *stream);

#ifdef __cplusplus
}
#endif

#endif
