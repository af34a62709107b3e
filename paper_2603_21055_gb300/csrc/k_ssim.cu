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
//
// Staging is asynchronous (cp.async, zero-filled outside the image; 16-byte copies when
// the rows are 16-byte aligned, else 4-byte ones). Both blurs are register-blocked: a
// lane of the horizontal pass reads the 14 neighbours of 4 consecutive outputs of a row
// with five aligned float4 loads, a lane of the vertical pass streams 14 values of a
// column into 4 outputs, so each shared-memory value read feeds several outputs (11 taps
// per output would otherwise mean 11 loads per output and per product).
#include <cmath>
#include <cstdio>
#include <cstring>

#include "sgad_device.cuh"

namespace sgad {
sgad_status report_error(sgad_status code, const char *msg);

namespace {

constexpr int kWin = 11, kRad = 5, kTile = 32, kExt = kTile + 2 * kRad;    // 42
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct SsimView {
    const float *x;        // rendered colour [3][H][W]
    const float *y;        // observed colour [3][H][W]
    float *dx;             // colour gradient [3][H][W] (added to)
    float *maps;           // d S / d (m1, m2, m12): [3 maps][3 channels][H][W]
    int32_t W, H, tiles_x, block_base;
    int32_t vec;           // rows and planes 16-byte aligned: stage with 16-byte copies
};

struct SsimBatch {
    SsimView v[SGAD_MAX_VIEWS];
    int32_t n_views;
    float weight;
    float *loss;
    float gauss[kWin];     // normalised window weights
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

// Staged neighbourhood: rows y0 - 5 .. y0 + 36 and the 48 columns x0 - 8 .. x0 + 39, so
// that every 4-column chunk starts on a multiple of 4 in image coordinates (x0 is a
// multiple of 32): with W a multiple of 4 a chunk is wholly inside or wholly outside the
// image and is one 16-byte copy. Output column c reads frame columns c + 3 .. c + 13.
constexpr int kPitch = 48, kLead = 8 - kRad;                   // frame column of image x0 - 5
// Horizontal pass: a lane computes kRh = 4 consecutive outputs of one row from five
// aligned float4 loads (20 frame columns, of which 14 are used).
constexpr int kRh = 4, kStripsH = kTile / kRh;                 // 8 strips per row
// Vertical pass: a lane computes kRv = 4 consecutive outputs of one column from 14 inputs
// (32 columns x 8 strips = one item per lane of a 256-thread block).
constexpr int kRv = 4;
constexpr int kThreads = 256;
static_assert(kTile * (kTile / kRv) == kThreads, "one vertical item per lane");

// Asynchronous copies global -> shared; src_bytes = 0 writes zeros (the padding).
__device__ __forceinline__ void cp_async4(float *dst, const float *src, uint32_t src_bytes)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async16(float *dst, const float *src, uint32_t src_bytes)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Stage the frame of NP planes (zero outside the image) into s[NP][42][48].
template <int NP>
__device__ __forceinline__ void stage(float (*s)[kExt][kPitch], const float *const (&plane)[NP], int W, int H,
                                      int x0, int y0, bool vec)
{
    const int gx0 = x0 - 8, gy0 = y0 - kRad;
    if (vec) {
        constexpr int kChunks = kPitch / 4;
        for (int i = threadIdx.x; i < kExt * kChunks; i += kThreads) {
            const int r = i / kChunks, k = i - r * kChunks;
            const int gy = gy0 + r, gx = gx0 + 4 * k;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            const int off = in ? gy * W + gx : 0;
#pragma unroll
            for (int q = 0; q < NP; ++q) cp_async16(&s[q][r][4 * k], plane[q] + off, in ? 16u : 0u);
        }
    } else {
        for (int i = threadIdx.x; i < kExt * kPitch; i += kThreads) {
            const int r = i / kPitch, c = i - r * kPitch;
            const int gy = gy0 + r, gx = gx0 + c;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            const int off = in ? gy * W + gx : 0;
#pragma unroll
            for (int q = 0; q < NP; ++q) cp_async4(&s[q][r][c], plane[q] + off, in ? 4u : 0u);
        }
    }
    cp_async_wait_all();
}

__device__ __forceinline__ void load_weights(const SsimBatch &b, float (&g)[kWin])
{
#pragma unroll
    for (int k = 0; k < kWin; ++k) g[k] = b.gauss[k];
}

// The 14 inputs of a horizontal strip at output column c0 (a multiple of 4): five aligned
// float4 loads of frame columns c0 .. c0 + 19, inputs at c0 + 3 .. c0 + 16.
__device__ __forceinline__ void load_strip(const float *row, int c0, float (&v)[kRh + kWin - 1])
{
    float t[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const float4 f = *reinterpret_cast<const float4 *>(row + c0 + 4 * q);
        t[4 * q] = f.x;
        t[4 * q + 1] = f.y;
        t[4 * q + 2] = f.z;
        t[4 * q + 3] = f.w;
    }
#pragma unroll
    for (int m = 0; m < kRh + kWin - 1; ++m) v[m] = t[m + kLead];
}

__global__ void __launch_bounds__(kThreads, 4) k_ssim_maps(const __grid_constant__ SsimBatch b)
{
    __shared__ __align__(16) float sxy[2][kExt][kPitch];       // x, y
    __shared__ __align__(16) float h[5][kExt][kTile];          // m1, my, m2, myy, m12 (horizontal)
    __shared__ float red[kThreads / 32];
    const TileAt t = tile_at(b);
    const SsimView &v = b.v[t.view];
    const size_t hw = (size_t)v.W * v.H;
    const float *const planes[2] = {v.x + t.ch * hw, v.y + t.ch * hw};
    stage<2>(sxy, planes, v.W, v.H, t.x0, t.y0, v.vec != 0);
    float g[kWin];
    load_weights(b, g);
    __syncthreads();
    // horizontal pass: 42 rows x 8 strips of 4 outputs
    for (int i = threadIdx.x; i < kExt * kStripsH; i += kThreads) {
        const int r = i / kStripsH, c0 = (i % kStripsH) * kRh;
        float xv[kRh + kWin - 1], yv[kRh + kWin - 1];
        load_strip(&sxy[0][r][0], c0, xv);
        load_strip(&sxy[1][r][0], c0, yv);
        float acc[5][kRh];
#pragma unroll
        for (int j = 0; j < kRh; ++j)
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[q][j] = 0.f;
#pragma unroll
        for (int m = 0; m < kRh + kWin - 1; ++m) {
            const float a = xv[m], bb = yv[m], aa = a * a, b2 = bb * bb, ab = a * bb;
#pragma unroll
            for (int j = 0; j < kRh; ++j) {
                const int k = m - j;
                if (k >= 0 && k < kWin) {
                    acc[0][j] = fmaf(g[k], a, acc[0][j]);
                    acc[1][j] = fmaf(g[k], bb, acc[1][j]);
                    acc[2][j] = fmaf(g[k], aa, acc[2][j]);
                    acc[3][j] = fmaf(g[k], b2, acc[3][j]);
                    acc[4][j] = fmaf(g[k], ab, acc[4][j]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 5; ++q)
            *reinterpret_cast<float4 *>(&h[q][r][c0]) = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
    }
    __syncthreads();
    // vertical pass: 32 columns x 8 strips of 4 outputs, one per lane
    const int c = threadIdx.x % kTile, r0 = (threadIdx.x / kTile) * kRv;
    float m[5][kRv];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
#pragma unroll
        for (int j = 0; j < kRv; ++j) m[q][j] = 0.f;
#pragma unroll
        for (int s = 0; s < kRv + kWin - 1; ++s) {
            const float val = h[q][r0 + s][c];
#pragma unroll
            for (int j = 0; j < kRv; ++j) {
                const int k = s - j;
                if (k >= 0 && k < kWin) m[q][j] = fmaf(g[k], val, m[q][j]);
            }
        }
    }
    float part = 0.f;
    const int gx = t.x0 + c;
    if (gx < v.W) {
        float *M1 = v.maps + t.ch * hw, *M2 = v.maps + (3 + t.ch) * hw, *M12 = v.maps + (6 + t.ch) * hw;
#pragma unroll
        for (int j = 0; j < kRv; ++j) {
            const int gy = t.y0 + r0 + j;
            if (gy >= v.H) break;
            const float m1 = m[0][j], my = m[1][j], m2 = m[2][j], myy = m[3][j], m12 = m[4][j];
            const float A1 = 2.f * m1 * my + kC1, A2 = 2.f * (m12 - m1 * my) + kC2;
            const float B1 = m1 * m1 + my * my + kC1, B2 = (m2 - m1 * m1) + (myy - my * my) + kC2;
            // S / A1 and S / A2 written as A2 P and A1 P (P = 1 / (B1 B2)): no division by
            // A1 or A2, which may vanish; B1 >= C1 and B2 >= C2 up to rounding, so the
            // fast reciprocals (2 ulp) see normal operands.
            const float rB1 = __fdividef(1.f, B1), rB2 = __fdividef(1.f, B2);
            const float P = rB1 * rB2;
            const float S = A1 * A2 * P;
            part += 1.f - S;
            const int p = gy * v.W + gx;
            M1[p] = 2.f * my * (A2 - A1) * P + 2.f * m1 * S * (rB2 - rB1);
            M2[p] = -S * rB2;
            M12[p] = 2.f * A1 * P;
        }
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0 && b.loss) {
        const float inv_n = 1.0f / (3.0f * (float)hw);
        float s = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        atomicAdd(b.loss, b.weight * s * inv_n);
    }
}

__global__ void __launch_bounds__(kThreads, 4) k_ssim_grad(const __grid_constant__ SsimBatch b)
{
    __shared__ __align__(16) float sd[3][kExt][kPitch];
    __shared__ __align__(16) float h[3][kExt][kTile];
    const TileAt t = tile_at(b);
    const SsimView &v = b.v[t.view];
    const size_t hw = (size_t)v.W * v.H;
    const float *const planes[3] = {v.maps + t.ch * hw, v.maps + (3 + t.ch) * hw, v.maps + (6 + t.ch) * hw};
    stage<3>(sd, planes, v.W, v.H, t.x0, t.y0, v.vec != 0);
    // this lane's outputs: x, y and the gradient so far, loaded while the blurs run
    const int c = threadIdx.x % kTile, r0 = (threadIdx.x / kTile) * kRv;
    const int gx = t.x0 + c;
    const float *X = v.x + t.ch * hw, *Y = v.y + t.ch * hw;
    float *D = v.dx + t.ch * hw;
    float xo[kRv], yo[kRv], dO[kRv];
#pragma unroll
    for (int j = 0; j < kRv; ++j) {
        const int gy = t.y0 + r0 + j;
        const bool in = gx < v.W && gy < v.H;
        const int p = in ? gy * v.W + gx : 0;
        xo[j] = in ? __ldg(X + p) : 0.f;
        yo[j] = in ? __ldg(Y + p) : 0.f;
        dO[j] = in ? D[p] : 0.f;
    }
    float g[kWin];
    load_weights(b, g);
    __syncthreads();
    for (int i = threadIdx.x; i < kExt * kStripsH; i += kThreads) {
        const int r = i / kStripsH, c0 = (i % kStripsH) * kRh;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float dv[kRh + kWin - 1];
            load_strip(&sd[q][r][0], c0, dv);
            float acc[kRh] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int m = 0; m < kRh + kWin - 1; ++m)
#pragma unroll
                for (int j = 0; j < kRh; ++j) {
                    const int k = m - j;
                    if (k >= 0 && k < kWin) acc[j] = fmaf(g[k], dv[m], acc[j]);
                }
            *reinterpret_cast<float4 *>(&h[q][r][c0]) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        }
    }
    __syncthreads();
    float s[3][kRv];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int j = 0; j < kRv; ++j) s[q][j] = 0.f;
#pragma unroll
        for (int m = 0; m < kRv + kWin - 1; ++m) {
            const float val = h[q][r0 + m][c];
#pragma unroll
            for (int j = 0; j < kRv; ++j) {
                const int k = m - j;
                if (k >= 0 && k < kWin) s[q][j] = fmaf(g[k], val, s[q][j]);
            }
        }
    }
    if (gx >= v.W) return;
    const float scale = -b.weight / (3.0f * (float)hw);
#pragma unroll
    for (int j = 0; j < kRv; ++j) {
        const int gy = t.y0 + r0 + j;
        if (gy >= v.H) break;
        D[gy * v.W + gx] = dO[j] + scale * (s[0][j] + 2.f * xo[j] * s[1][j] + yo[j] * s[2][j]);
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
    {
        double w[kWin], sum = 0.0;
        for (int k = 0; k < kWin; ++k) {
            const double d = k - kRad;
            w[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
            sum += w[k];
        }
        for (int k = 0; k < kWin; ++k) b.gauss[k] = (float)(w[k] / sum);
    }
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
        const auto a16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
        v.vec = (v.W % 4 == 0) && a16(v.x) && a16(v.y) && a16(v.maps);
        v.block_base = blocks;
        blocks += 3 * v.tiles_x * ((v.H + kTile - 1) / kTile);
        o = round256(o + (size_t)9 * v.W * v.H * sizeof(float));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the whole unified L1 as shared memory (4 blocks per SM); a preference only, set
    // once per device (outside any stream capture, which replays launches only)
    static int configured[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(SGAD_ERR_CUDA, "sgad_ssim_loss_grad: no device");
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        if (cudaFuncSetAttribute(k_ssim_maps, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess ||
            cudaFuncSetAttribute(k_ssim_grad, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
            return fail(SGAD_ERR_CUDA, "sgad_ssim_loss_grad: cannot set the shared-memory carveout");
        if (dev >= 0 && dev < 64) configured[dev] = 1;
    }
    k_ssim_maps<<<blocks, kThreads, 0, st>>>(b);
    k_ssim_grad<<<blocks, kThreads, 0, st>>>(b);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SGAD_OK : fail(SGAD_ERR_CUDA, "sgad_ssim_loss_grad: launch failed");
}
