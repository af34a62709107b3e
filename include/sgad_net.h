/*
 * sgad_net.h - C ABI of the learned proposal net (GB300, sm_103a tensor cores).
 *
 * The paper initialises each new keyframe's Gaussians with a zero depth offset and
 * learns the offsets and opacities during mapping (Sec. 3.2, Supp. A). This small
 * convolutional net has no counterpart in the paper: it is the workload's learned part,
 * predicting a keyframe's initial offsets and opacity logits from its RGB-D, trained on
 * the offsets and logits the plain mapping converges to; the zero initialisation stays
 * the fallback.
 *
 * Architecture: four 3x3 convolutions with zero padding of one pixel,
 * 4 -> 32 -> 32 -> 32 -> 2 channels, ReLU after the first three:
 *   y_l[p, o] = b_l[o] + sum_{ky, kx} sum_i W_l[3 ky + kx][i][o] x_l[p + (ky - 1, kx - 1), i].
 * Input per pixel: R, G, B (observed colour in [0, 1]) and D (observed depth, metres).
 * Output per pixel: delta = 0.01 y[0] metres and the opacity logit y[1].
 *
 * Precision: inputs, weights and activations are stored as bfloat16 (round to nearest
 * even), products are accumulated in FP32 on the tensor cores (tcgen05.mma, operands in
 * shared memory, accumulators in tensor memory); the output and all parameter gradients
 * are FP32.
 *
 * Parameters are FP32 master copies owned by the caller, in a padded layout: layer l
 * (0..3) has weights w[l] = [9][cin_p][cout_p] (tap 3 ky + kx, then input channel, then
 * output channel) and biases b[l] = [cout_p], with cin_p = 16, 32, 32, 32 and
 * cout_p = 32, 32, 32, 16 (sgad_net_layer_shape). Padded entries must be zero; their
 * gradients are zero, so an optimiser keeps them zero.
 *
 * All image tensors are device FP32, frames contiguous: rgb [N][3][H][W], depth, delta,
 * logit and targets [N][H][W]. Calls are asynchronous on `stream` and allocate nothing;
 * the caller provides one workspace (sgad_net_workspace_size) that holds the packed
 * input, the activations and gradients between layers and the bf16 weight copies.
 * Device-side failures (a bounded wait on the tensor cores that gave up) are recorded in
 * the workspace and reported by sgad_net_check(). Errors as in sgad.h.
 */
#ifndef SGAD_NET_H
#define SGAD_NET_H

#include "sgad.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SGAD_NET_LAYERS 4

typedef struct {
    float *w[SGAD_NET_LAYERS];
    float *b[SGAD_NET_LAYERS];
} sgad_net_params;

typedef struct {
    float *dw[SGAD_NET_LAYERS];
    float *db[SGAD_NET_LAYERS];
} sgad_net_grads;

/* Real and padded channel counts of layer 0..3. Host only. */
sgad_status sgad_net_layer_shape(int32_t layer, int32_t *cin, int32_t *cout, int32_t *cin_padded,
                                 int32_t *cout_padded);

/* Workspace bytes for a batch of n_frames frames of height x width. Host only. */
sgad_status sgad_net_workspace_size(int32_t n_frames, int32_t height, int32_t width, size_t *bytes);

/* Forward pass: packs (rgb, depth) to bf16, converts the weights to their bf16 operand
 * layouts, and runs the four convolutions. delta and logit (either may be NULL) receive
 * the outputs; the activations stay in the workspace for sgad_net_loss_grad() and
 * sgad_net_backward(). The workspace's status word must start at zero (zero its first
 * 256 bytes once after allocating it). */
sgad_status sgad_net_forward(const sgad_net_params *params, int32_t n_frames, int32_t height,
                             int32_t width, const float *rgb, const float *depth, float *delta,
                             float *logit, void *workspace, size_t ws_bytes, void *stream);

/* Training loss of the last forward on this workspace against the targets (delta in
 * metres, opacity logit): mean over pixels of (y0 - delta_t / 0.01)^2 +
 * logit_weight (y1 - logit_t)^2, added to *loss_accum (device float; may be NULL), and
 * its gradient with respect to the outputs, kept in the workspace. */
sgad_status sgad_net_loss_grad(int32_t n_frames, int32_t height, int32_t width,
                               const float *target_delta, const float *target_logit,
                               float logit_weight, float *loss_accum, void *workspace,
                               size_t ws_bytes, void *stream);

/* Adjoint of the network for the output gradient left by sgad_net_loss_grad(): input
 * gradients of layers 3, 2, 1 through the ReLUs and the weight and bias gradients of all
 * four layers, written (not accumulated) into grads (padded layout as the parameters). */
sgad_status sgad_net_backward(const sgad_net_params *params, sgad_net_grads *grads, int32_t n_frames,
                              int32_t height, int32_t width, void *workspace, size_t ws_bytes,
                              void *stream);

/* Synchronise `stream` and return the workspace's device status (SGAD_OK, or
 * SGAD_ERR_TIMEOUT if a tensor-core wait gave up), clearing it. */
sgad_status sgad_net_check(void *workspace, size_t ws_bytes, void *stream);

/* Device pointers into the workspace, for inspection and tests: x[0] the packed input
 * (bf16, 16 channels), x[1..3] the post-ReLU activations (bf16, 32 channels), y4 the raw
 * outputs (float pairs per pixel), dy4 the output gradient (bf16, 16 channels, two used)
 * and dpre[0..2] the gradients of the pre-activations of layers 0..2 (bf16, 32
 * channels). The bf16 tensors are chunk-planar: channel c of pixel (frame f, row y,
 * column x) of a tensor with C channels is element c % 8 of the 16-byte unit
 * ((f H + y) C/8 + c / 8) W + x. */
typedef struct {
    const void *x[4];
    const float *y4;
    const void *dy4;
    const void *dpre[3];
} sgad_net_buffers;

sgad_status sgad_net_buffers_view(int32_t n_frames, int32_t height, int32_t width, void *workspace,
                                  size_t ws_bytes, sgad_net_buffers *out);

#ifdef __cplusplus
}
#endif
#endif /* SGAD_NET_H */
