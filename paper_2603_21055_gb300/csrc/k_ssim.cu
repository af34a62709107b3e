// SSIM term of the mapping loss (Eq. 1, tau L_S) and its gradient, all views of a batch in
// one launch per pass.
//
// L_S = 1 - mean over pixels and colour channels of SSIM(V', V), with an 11 x 11 Gaussian
// window (standard deviation 1.5, weights normalised), zero padding, C1 = 0.01^2 and
// C2 = 0.03^2. With the blurred moments m1 = G * x, m2 = G * x^2, m12 = G * (x y) of the
// rendering x and my = G * y, myy = G * y^2 of the observation y:
//   A1 = 2 m1 my + C1, A2 = 2 (m12 - m1 my) + C2, B1 = m1^2 + my^2 + C1,
//   B2 = (m2 - m1^2) + (myy - my^2) + C2, S = A1 A2 / (B1 B2),
//   d S / d m1 = S (2 my / A1 - 2 my / A2 - 2 m1 / B1 + 2 m1 / B2),
//   d S / d m2 = -S / B2, d S / d m12 = 2 S / A2,
//   d L_S / d x = -(G * dS/dm1 + 2 x (G * dS/dm2) + y (G * dS/dm12)) / N.
//
// Pass 1 (k_ssim_maps): one block per 32 x 32 tile of one channel of one view stages the
// 42 x 42 neighbourhood of x and y in shared memory, blurs the five products separably
// (horizontal then vertical, 11 taps each), and writes the three d S / d m maps; the block
// adds tau sum(1 - S) / N to the loss. Pass 2 (k_ssim_grad) blurs the three maps the same
// way (zero outside the image) and adds tau d L_S / d x to the colour gradient.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "sgad_device.cuh"

namespace sgad {
sgad_status report_error(sgad_status code, const char *msg);

namespace {

constexpr int kWin = 11, kRad = 5, kTile = 32, kExt = kTile + 2 * kRad;    // 42
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// The normalised window weights, computed by the block itself.
__device__ __forceinline__ void window_weights(float *g)
{
    if (threadIdx.x < kWin) {
        const float d = (float)((int)threadIdx.x - kRad);
        g[threadIdx.x] = expf(-d * d / (2.0f * 1.5f * 1.5f));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float sum = 0.f;
        for (int i = 0; i < kWin; ++i) sum += g[i];
        for (int i = 0; i < kWin; ++i) g[i] /= sum;
    }
    // the caller's next barrier publishes the normalised weights
}

struct SsimView {
    const float *x;        // rendered colour [3][H][W]
    const float *y;        // observed colour [3][H][W]
    float *dx;             // colour gradient [3][H][W] (added to)
    float *maps;           // d S / d (m1, m2, m12): [3 maps][3 channels][H][W]
    int32_t W, H, tiles_x, block_base;
};

struct SsimBatch {
    SsimView v[SGAD_MAX_VIEWS];
    int32_t n_views;
    float weight;
    float *loss;
};

__device__ __forceinline__ int view_of_block(const SsimBatch &b, int blk)
{
    int k = 0;
#pragma unroll 1
    for (int i = 1; i < b.n_views; ++i)
        if (blk >= b.v[i].block_base) k = i;
    return k;
}

// Block -> (view, channel, tile origin).
struct TileAt {
    int view, ch, x0, y0;
};

__device__ __forceinline__ TileAt tile_at(const SsimBatch &b)
{
    TileAt t;
    t.view = view_of_block(b, blockIdx.x);
    const SsimView &v = b.v[t.view];
    const int local = blockIdx.x - v.block_base;
    const int tiles = v.tiles_x * ((v.H + kTile - 1) / kTile);
    t.ch = local / tiles;
    const int tl = local - t.ch * tiles;
    t.x0 = (tl % v.tiles_x) * kTile;
    t.y0 = (tl / v.tiles_x) * kTile;
    return t;
}

__global__ void __launch_bounds__(256) k_ssim_maps(const __grid_constant__ SsimBatch b)
{
    __shared__ float sx[kExt][kExt + 1], sy[kExt][kExt + 1];
    __shared__ float h[5][kExt][kTile + 1];
    __shared__ float red[8];
    __shared__ float c_gauss[kWin];
    window_weights(c_gauss);
    const TileAt t = tile_at(b);
    const SsimView &v = b.v[t.view];
    const size_t hw = (size_t)v.W * v.H;
    const float *X = v.x + t.ch * hw, *Y = v.y + t.ch * hw;
    for (int i = threadIdx.x; i < kExt * kExt; i += blockDim.x) {
        const int r = i / kExt, c = i % kExt;
        const int gy = t.y0 + r - kRad, gx = t.x0 + c - kRad;
        const bool in = gx >= 0 && gx < v.W && gy >= 0 && gy < v.H;
        sx[r][c] = in ? X[(size_t)gy * v.W + gx] : 0.f;
        sy[r][c] = in ? Y[(size_t)gy * v.W + gx] : 0.f;
    }
    __syncthreads();
    // horizontal pass: all 42 rows, the 32 output columns
    for (int i = threadIdx.x; i < kExt * kTile; i += blockDim.x) {
        const int r = i / kTile, c = i % kTile;
        float a = 0.f, bb = 0.f, aa = 0.f, bb2 = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; ++k) {
            const float g = c_gauss[k], xv = sx[r][c + k], yv = sy[r][c + k];
            a = fmaf(g, xv, a);
            bb = fmaf(g, yv, bb);
            aa = fmaf(g, xv * xv, aa);
            bb2 = fmaf(g, yv * yv, bb2);
            ab = fmaf(g, xv * yv, ab);
        }
        h[0][r][c] = a;
        h[1][r][c] = bb;
        h[2][r][c] = aa;
        h[3][r][c] = bb2;
        h[4][r][c] = ab;
    }
    __syncthreads();
    const float inv_n = 1.0f / (3.0f * (float)hw);
    float part = 0.f;
    for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) {
        const int r = i / kTile, c = i % kTile;
        const int gy = t.y0 + r, gx = t.x0 + c;
        if (gx >= v.W || gy >= v.H) continue;
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kWin; ++k) {
            const float g = c_gauss[k];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = fmaf(g, h[q][r + k][c], m[q]);
        }
        const float m1 = m[0], my = m[1], m2 = m[2], myy = m[3], m12 = m[4];
        const float A1 = 2.f * m1 * my + kC1, A2 = 2.f * (m12 - m1 * my) + kC2;
        const float B1 = m1 * m1 + my * my + kC1, B2 = (m2 - m1 * m1) + (myy - my * my) + kC2;
        // S / A1 and S / A2 written as A2 P and A1 P (P = 1 / (B1 B2)): no division by
        // A1 or A2, which may vanish; B1 >= C1 and B2 >= C2 up to rounding.
        const float P = 1.f / (B1 * B2);
        const float S = A1 * A2 * P;
        part += 1.f - S;
        const size_t p = (size_t)gy * v.W + gx;
        v.maps[t.ch * hw + p] = 2.f * my * (A2 - A1) * P + 2.f * m1 * S * (1.f / B2 - 1.f / B1);
        v.maps[(3 + t.ch) * hw + p] = -S / B2;
        v.maps[(6 + t.ch) * hw + p] = 2.f * A1 * P;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0 && b.loss) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(b.loss, b.weight * s * inv_n);
    }
}

__global__ void __launch_bounds__(256) k_ssim_grad(const __grid_constant__ SsimBatch b)
{
    __shared__ float sd[3][kExt][kExt + 1];
    __shared__ float h[3][kExt][kTile + 1];
    __shared__ float c_gauss[kWin];
    window_weights(c_gauss);
    const TileAt t = tile_at(b);
    const SsimView &v = b.v[t.view];
    const size_t hw = (size_t)v.W * v.H;
    for (int i = threadIdx.x; i < kExt * kExt; i += blockDim.x) {
        const int r = i / kExt, c = i % kExt;
        const int gy = t.y0 + r - kRad, gx = t.x0 + c - kRad;
        const bool in = gx >= 0 && gx < v.W && gy >= 0 && gy < v.H;
        const size_t p = (size_t)gy * v.W + gx;
#pragma unroll
        for (int q = 0; q < 3; ++q) sd[q][r][c] = in ? v.maps[(3 * q + t.ch) * hw + p] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kExt * kTile; i += blockDim.x) {
        const int r = i / kTile, c = i % kTile;
        float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kWin; ++k) {
            const float g = c_gauss[k];
#pragma unroll
            for (int q = 0; q < 3; ++q) s[q] = fmaf(g, sd[q][r][c + k], s[q]);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) h[q][r][c] = s[q];
    }
    __syncthreads();
    const float scale = -b.weight / (3.0f * (float)hw);
    for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) {
        const int r = i / kTile, c = i % kTile;
        const int gy = t.y0 + r, gx = t.x0 + c;
        if (gx >= v.W || gy >= v.H) continue;
        float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kWin; ++k) {
            const float g = c_gauss[k];
#pragma unroll
            for (int q = 0; q < 3; ++q) s[q] = fmaf(g, h[q][r + k][c], s[q]);
        }
        const size_t p = t.ch * hw + (size_t)gy * v.W + gx;
        v.dx[p] += scale * (s[0] + 2.f * v.x[p] * s[1] + v.y[p] * s[2]);
    }
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

sgad_status fail(sgad_status code, const char *msg) { return report_error(code, msg); }

}  // namespace
}  // namespace sgad

using namespace sgad;

extern "C" sgad_status sgad_ssim_workspace_size(int32_t n_views, const sgad_camera *views, size_t *bytes)
{
    if (!views || !bytes || n_views < 1 || n_views > SGAD_MAX_VIEWS)
        return fail(SGAD_ERR_INVALID_ARG, "sgad_ssim_workspace_size: bad arguments");
    size_t o = 0;
    for (int i = 0; i < n_views; ++i) {
        if (views[i].width <= 0 || views[i].height <= 0 || views[i].width > 16384 || views[i].height > 16384)
            return fail(SGAD_ERR_INVALID_ARG, "sgad_ssim_workspace_size: bad view size");
        o = round256(o + (size_t)9 * views[i].width * views[i].height * sizeof(float));
    }
    *bytes = o;
    return SGAD_OK;
}

extern "C" sgad_status sgad_ssim_loss_grad(int32_t n_views, const sgad_camera *views, const sgad_images *rendered,
                                           const float *const *target_rgb, float weight, float *const *d_rgb,
                                           float *loss_accum, void *workspace, size_t ws_bytes, void *stream)
{
    size_t need = 0;
    sgad_status s = sgad_ssim_workspace_size(n_views, views, &need);
    if (s) return s;
    if (!rendered || !target_rgb || !d_rgb) return fail(SGAD_ERR_INVALID_ARG, "sgad_ssim_loss_grad: NULL argument");
    for (int i = 0; i < n_views; ++i)
        if (!rendered[i].rgb || !target_rgb[i] || !d_rgb[i])
            return fail(SGAD_ERR_INVALID_ARG, "sgad_ssim_loss_grad: a view's image is NULL");
    if (!workspace || ws_bytes < need) return fail(SGAD_ERR_WORKSPACE_TOO_SMALL, "sgad_ssim_loss_grad: workspace too small");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(SGAD_ERR_INVALID_ARG, "sgad_ssim_loss_grad: workspace must be 256-byte aligned");
    if (!std::isfinite(weight)) return fail(SGAD_ERR_INVALID_ARG, "sgad_ssim_loss_grad: weight must be finite");
    SsimBatch b;
    std::memset(&b, 0, sizeof(b));
    b.n_views = n_views;
    b.weight = weight;
    b.loss = loss_accum;
    size_t o = 0;
    int blocks = 0;
    for (int i = 0; i < n_views; ++i) {
        SsimView &v = b.v[i];
        v.x = rendered[i].rgb;
        v.y = target_rgb[i];
        v.dx = d_rgb[i];
        v.maps = reinterpret_cast<float *>(static_cast<char *>(workspace) + o);
        v.W = views[i].width;
        v.H = views[i].height;
        v.tiles_x = (v.W + kTile - 1) / kTile;
        v.block_base = blocks;
        blocks += 3 * v.tiles_x * ((v.H + kTile - 1) / kTile);
        o = round256(o + (size_t)9 * v.W * v.H * sizeof(float));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_ssim_maps<<<blocks, 256, 0, st>>>(b);
    k_ssim_grad<<<blocks, 256, 0, st>>>(b);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SGAD_OK : fail(SGAD_ERR_CUDA, "sgad_ssim_loss_grad: launch failed");
}
