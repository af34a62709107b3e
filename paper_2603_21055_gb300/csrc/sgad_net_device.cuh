// Launch parameters of the proposal-net kernels (k_net.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sgad {
namespace net {

constexpr int kModeRelu = 0;   // out = bf16(relu(acc + bias))
constexpr int kModeMask = 1;   // out = bf16(acc * [mask > 0])  (input gradient through a ReLU)
constexpr int kModeOut = 2;    // y = acc + bias -> y4 (f32 pairs), delta = 0.01 y0, logit = y1

struct ConvArgs {
    const uint4 *in;     // chunk-planar bf16, CI channels
    const uint4 *wB;     // [9][CI / 8][CO] 16-byte units
    const float *bias;   // [CO] (forward modes)
    uint4 *out;          // chunk-planar bf16, CO channels (relu / mask modes)
    const uint4 *mask;   // chunk-planar bf16, CO channels (mask mode)
    float2 *y4;          // [N H W] (out mode)
    float *delta;        // [N H W] metres (out mode; may be null)
    float *logit;        // [N H W] (out mode; may be null)
    int N, H, W;
    uint32_t *status;    // device status word (0 = ok)
};

struct WgradArgs {
    const uint4 *x;      // chunk-planar bf16, CI channels (layer input)
    const uint4 *dy;     // chunk-planar bf16, CO channels (gradient of the pre-activation output)
    float *dw;           // [9][CI][CO] f32, accumulated into
    float *db;           // [CO] f32, accumulated into
    int N, H, W;
    uint32_t *status;
};

template <int CI, int CO, int MODE>
cudaError_t launch_conv(const ConvArgs &a, cudaStream_t st);
template <int CI, int CO>
cudaError_t launch_wgrad(const WgradArgs &a, cudaStream_t st);
cudaError_t launch_pack_input(const float *rgb, const float *depth, uint4 *x0, int n, int h, int w, cudaStream_t st);
cudaError_t launch_prep_weights(const float *w, uint4 *fwd, uint4 *bwd, int ci_p, int co_p, cudaStream_t st);
cudaError_t launch_loss(const float2 *y4, const float *td, const float *tl, float lw, uint4 *dy4, float *loss,
                        size_t total, int w, cudaStream_t st);

}  // namespace net
}  // namespace sgad
