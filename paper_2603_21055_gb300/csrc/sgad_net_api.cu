// C ABI of the proposal net (include/sgad_net.h): argument checks, the workspace layout
// and the launch sequence. No device memory is allocated here.
#include <cstdio>
#include <cstring>

#include "sgad_net.h"
#include "sgad_net_device.cuh"

namespace sgad {
sgad_status report_error(sgad_status code, const char *msg);
}

using namespace sgad;
using namespace sgad::net;

namespace {

constexpr int kCin[4] = {4, 32, 32, 32}, kCout[4] = {32, 32, 32, 2};
constexpr int kCinP[4] = {16, 32, 32, 32}, kCoutP[4] = {32, 32, 32, 16};

sgad_status err(sgad_status code, const char *msg) { return report_error(code, msg); }

sgad_status cuda_err(cudaError_t e, const char *what)
{
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return report_error(SGAD_ERR_CUDA, buf);
}

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct NetLayout {
    size_t x[4], y4, dy4, d[3], wf[4], wb[4], total;
};

NetLayout layout(size_t px)
{
    NetLayout L;
    size_t o = 256;   // status block
    L.x[0] = o; o = a256(o + px * 32);
    for (int l = 1; l < 4; ++l) { L.x[l] = o; o = a256(o + px * 64); }
    L.y4 = o; o = a256(o + px * 8);
    L.dy4 = o; o = a256(o + px * 32);
    for (int l = 0; l < 3; ++l) { L.d[l] = o; o = a256(o + px * 64); }
    for (int l = 0; l < 4; ++l) { L.wf[l] = o; o = a256(o + (size_t)9 * kCinP[l] * kCoutP[l] * 2); }
    for (int l = 0; l < 4; ++l) { L.wb[l] = o; o = a256(o + (size_t)9 * kCinP[l] * kCoutP[l] * 2); }
    L.total = o;
    return L;
}

struct Ws {
    NetLayout L;
    char *base = nullptr;
    uint32_t *status() const { return reinterpret_cast<uint32_t *>(base); }
    uint4 *at(size_t off) const { return reinterpret_cast<uint4 *>(base + off); }
};

sgad_status get_ws(int32_t n, int32_t h, int32_t w, void *workspace, size_t ws_bytes, Ws &ws)
{
    if (n < 1 || h < 1 || w < 1 || h > 16384 || w > 16384 || (long long)n * h * w > (1ll << 31))
        return err(SGAD_ERR_INVALID_ARG, "sgad_net: bad frame count or size");
    ws.L = layout((size_t)n * h * w);
    if (!workspace) return err(SGAD_ERR_INVALID_ARG, "sgad_net: workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return err(SGAD_ERR_INVALID_ARG, "sgad_net: workspace must be 256-byte aligned");
    if (ws_bytes < ws.L.total) return err(SGAD_ERR_WORKSPACE_TOO_SMALL, "sgad_net: workspace too small");
    ws.base = static_cast<char *>(workspace);
    return SGAD_OK;
}

sgad_status check_params(const sgad_net_params *p)
{
    if (!p) return err(SGAD_ERR_INVALID_ARG, "sgad_net: params is NULL");
    for (int l = 0; l < 4; ++l)
        if (!p->w[l] || !p->b[l]) return err(SGAD_ERR_INVALID_ARG, "sgad_net: a parameter pointer is NULL");
    return SGAD_OK;
}

sgad_status launched(cudaError_t e, const char *what) { return e == cudaSuccess ? SGAD_OK : cuda_err(e, what); }

}  // namespace

extern "C" {

sgad_status sgad_net_layer_shape(int32_t layer, int32_t *cin, int32_t *cout, int32_t *cin_padded,
                                 int32_t *cout_padded)
{
    if (layer < 0 || layer >= 4) return err(SGAD_ERR_INVALID_ARG, "sgad_net_layer_shape: layer must be 0..3");
    if (cin) *cin = kCin[layer];
    if (cout) *cout = kCout[layer];
    if (cin_padded) *cin_padded = kCinP[layer];
    if (cout_padded) *cout_padded = kCoutP[layer];
    return SGAD_OK;
}

sgad_status sgad_net_workspace_size(int32_t n_frames, int32_t height, int32_t width, size_t *bytes)
{
    if (!bytes) return err(SGAD_ERR_INVALID_ARG, "sgad_net_workspace_size: bytes is NULL");
    if (n_frames < 1 || height < 1 || width < 1 || height > 16384 || width > 16384 ||
        (long long)n_frames * height * width > (1ll << 31))
        return err(SGAD_ERR_INVALID_ARG, "sgad_net: bad frame count or size");
    *bytes = layout((size_t)n_frames * height * width).total;
    return SGAD_OK;
}

sgad_status sgad_net_forward(const sgad_net_params *params, int32_t n_frames, int32_t height, int32_t width,
                             const float *rgb, const float *depth, float *delta, float *logit, void *workspace,
                             size_t ws_bytes, void *stream)
{
    Ws ws;
    sgad_status s = check_params(params);
    if (!s) s = get_ws(n_frames, height, width, workspace, ws_bytes, ws);
    if (s) return s;
    if (!rgb || !depth) return err(SGAD_ERR_INVALID_ARG, "sgad_net_forward: rgb / depth is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const NetLayout &L = ws.L;
    s = launched(launch_pack_input(rgb, depth, ws.at(L.x[0]), n_frames, height, width, st), "pack input");
    for (int l = 0; l < 4 && !s; ++l)
        s = launched(launch_prep_weights(params->w[l], ws.at(L.wf[l]), l > 0 ? ws.at(L.wb[l]) : nullptr, kCinP[l],
                                         kCoutP[l], st),
                     "weight conversion");
    if (s) return s;
    ConvArgs a = {};
    a.N = n_frames;
    a.H = height;
    a.W = width;
    a.status = ws.status();
    for (int l = 0; l < 4 && !s; ++l) {
        a.in = ws.at(L.x[l]);
        a.wB = ws.at(L.wf[l]);
        a.bias = params->b[l];
        cudaError_t e;
        if (l == 0) {
            a.out = ws.at(L.x[1]);
            e = launch_conv<16, 32, kModeRelu>(a, st);
        } else if (l < 3) {
            a.out = ws.at(L.x[l + 1]);
            e = launch_conv<32, 32, kModeRelu>(a, st);
        } else {
            a.out = nullptr;
            a.y4 = reinterpret_cast<float2 *>(ws.base + L.y4);
            a.delta = delta;
            a.logit = logit;
            e = launch_conv<32, 16, kModeOut>(a, st);
        }
        s = launched(e, "conv forward");
    }
    return s;
}

sgad_status sgad_net_loss_grad(int32_t n_frames, int32_t height, int32_t width, const float *target_delta,
                               const float *target_logit, float logit_weight, float *loss_accum, void *workspace,
                               size_t ws_bytes, void *stream)
{
    Ws ws;
    sgad_status s = get_ws(n_frames, height, width, workspace, ws_bytes, ws);
    if (s) return s;
    if (!target_delta || !target_logit) return err(SGAD_ERR_INVALID_ARG, "sgad_net_loss_grad: a target is NULL");
    return launched(launch_loss(reinterpret_cast<const float2 *>(ws.base + ws.L.y4), target_delta, target_logit,
                                logit_weight, ws.at(ws.L.dy4), loss_accum, (size_t)n_frames * height * width, width,
                                static_cast<cudaStream_t>(stream)),
                    "net loss");
}

sgad_status sgad_net_backward(const sgad_net_params *params, sgad_net_grads *grads, int32_t n_frames, int32_t height,
                              int32_t width, void *workspace, size_t ws_bytes, void *stream)
{
    Ws ws;
    sgad_status s = check_params(params);
    if (!s) s = get_ws(n_frames, height, width, workspace, ws_bytes, ws);
    if (s) return s;
    if (!grads) return err(SGAD_ERR_INVALID_ARG, "sgad_net_backward: grads is NULL");
    for (int l = 0; l < 4; ++l)
        if (!grads->dw[l] || !grads->db[l]) return err(SGAD_ERR_INVALID_ARG, "sgad_net_backward: a gradient is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const NetLayout &L = ws.L;
    for (int l = 0; l < 4; ++l) {
        cudaError_t e = cudaMemsetAsync(grads->dw[l], 0, (size_t)9 * kCinP[l] * kCoutP[l] * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(grads->db[l], 0, (size_t)kCoutP[l] * 4, st);
        if (e != cudaSuccess) return cuda_err(e, "cudaMemsetAsync");
    }
    // layer l's output gradient (pre-activation): dy4 for l = 3, d[l] below
    ConvArgs a = {};
    a.N = n_frames;
    a.H = height;
    a.W = width;
    a.status = ws.status();
    WgradArgs g = {};
    g.N = n_frames;
    g.H = height;
    g.W = width;
    g.status = ws.status();
    for (int l = 3; l >= 0 && !s; --l) {
        const uint4 *dout = l == 3 ? ws.at(L.dy4) : ws.at(L.d[l]);
        if (l > 0) {     // input gradient of layer l = output gradient of layer l - 1, through its ReLU
            a.in = dout;
            a.wB = ws.at(L.wb[l]);
            a.out = ws.at(L.d[l - 1]);
            a.mask = ws.at(L.x[l]);
            s = launched(l == 3 ? launch_conv<16, 32, kModeMask>(a, st) : launch_conv<32, 32, kModeMask>(a, st),
                         "conv input gradient");
            if (s) break;
        }
        g.x = ws.at(L.x[l]);
        g.dy = dout;
        g.dw = grads->dw[l];
        g.db = grads->db[l];
        cudaError_t e;
        if (l == 0)
            e = launch_wgrad<16, 32>(g, st);
        else if (l < 3)
            e = launch_wgrad<32, 32>(g, st);
        else
            e = launch_wgrad<32, 16>(g, st);
        s = launched(e, "conv weight gradient");
    }
    return s;
}

sgad_status sgad_net_check(void *workspace, size_t ws_bytes, void *stream)
{
    if (!workspace || ws_bytes < 256) return err(SGAD_ERR_INVALID_ARG, "sgad_net_check: bad workspace");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, workspace, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && v) e = cudaMemsetAsync(workspace, 0, 4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(e, "sgad_net_check");
    if (v) return err(SGAD_ERR_TIMEOUT, "sgad_net: a tensor-core wait gave up");
    return SGAD_OK;
}

sgad_status sgad_net_buffers_view(int32_t n_frames, int32_t height, int32_t width, void *workspace, size_t ws_bytes,
                                  sgad_net_buffers *out)
{
    Ws ws;
    sgad_status s = get_ws(n_frames, height, width, workspace, ws_bytes, ws);
    if (s) return s;
    if (!out) return err(SGAD_ERR_INVALID_ARG, "sgad_net_buffers_view: out is NULL");
    for (int l = 0; l < 4; ++l) out->x[l] = ws.base + ws.L.x[l];
    out->y4 = reinterpret_cast<const float *>(ws.base + ws.L.y4);
    out->dy4 = ws.base + ws.L.dy4;
    for (int l = 0; l < 3; ++l) out->dpre[l] = ws.base + ws.L.d[l];
    return SGAD_OK;
}

}  // extern "C"
