// Per-Gaussian and per-pixel elementwise kernels:
//   k_finalize   : last link of the adjoint (a10): d mu -> d delta through
//                  mu = R_i |D + delta| r + t_i, d opacity -> d logit, written into the
//                  caller's gradient planes of learnable keyframes.
//   k_l1_grad    : L1 terms of Eq. 1 and their image gradients (a8).
//   k_adam       : bias-corrected Adam step (a11).
#include "sgad_device.cuh"

namespace sgad {

__global__ void __launch_bounds__(256) k_finalize(const __grid_constant__ Scene sc, const World *__restrict__ world,
                                                  const float4 *__restrict__ gacc)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= sc.n_gauss) return;
    const KfDev &k = sc.kf[find_kf(sc, g)];
    if (!k.learnable) return;
    const uint32_t j = g - k.gbase;
    const size_t hw = (size_t)k.W * k.H;
    const float4 a = gacc[2 * (size_t)g], b = gacc[2 * (size_t)g + 1];
    const float u = (float)(j % (uint32_t)k.W), v = (float)(j / (uint32_t)k.W);
    const float rx = (u - k.cx) / k.fx, ry = (v - k.cy) / k.fy;
    // d mu / d |D + delta| = R_i r
    const float dir_x = k.R[0] * rx + k.R[1] * ry + k.R[2];
    const float dir_y = k.R[3] * rx + k.R[4] * ry + k.R[5];
    const float dir_z = k.R[6] * rx + k.R[7] * ry + k.R[8];
    const float sum = k.depth[j] + k.offset[j];
    const float sgn = sum > 0.0f ? 1.0f : (sum < 0.0f ? -1.0f : 0.0f);
    const float o = world[g].w1.x;
    k.d_offset[j] = sc.freeze_offset ? 0.0f : sgn * (dir_x * a.x + dir_y * a.y + dir_z * a.z);
    k.d_scale[j] = a.w;
    k.d_logit[j] = b.x * o * (1.0f - o);
    k.d_rgb[j] = b.y;
    k.d_rgb[hw + j] = b.z;
    k.d_rgb[2 * hw + j] = b.w;
}

void launch_finalize(const Scene &sc, const World *world, const float4 *gacc, cudaStream_t st)
{
    const unsigned blocks = (sc.n_gauss + 255) / 256;
    if (blocks) k_finalize<<<blocks, 256, 0, st>>>(sc, world, gacc);
}

__device__ __forceinline__ float sgnf(float x) { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); }

__device__ __forceinline__ float block_sum(float x, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

__global__ void k_count_valid(const float *__restrict__ td, size_t hw, uint32_t *count)
{
    __shared__ float red[32];
    float c = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < hw; i += (size_t)gridDim.x * blockDim.x)
        c += td[i] > 0.0f ? 1.0f : 0.0f;
    const float t = block_sum(c, red);
    if (threadIdx.x == 0 && t > 0.f) atomicAdd(count, (uint32_t)t);
}

__global__ void k_l1_grad(const float *__restrict__ rgb, const float *__restrict__ depth,
                          const float *__restrict__ trgb, const float *__restrict__ tdep, size_t hw, float wrgb,
                          float wdep, const uint32_t *__restrict__ nvalid, float *__restrict__ d_rgb,
                          float *__restrict__ d_depth, float *loss)
{
    __shared__ float red[32];
    const float inv_rgb = wrgb / (3.0f * (float)hw);
    const uint32_t nv = nvalid ? *nvalid : 0u;
    const float inv_dep = nv > 0 ? wdep / (float)nv : 0.0f;
    float l = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < hw; i += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = rgb[c * hw + i] - trgb[c * hw + i];
            l += fabsf(d) * inv_rgb;
            d_rgb[c * hw + i] = sgnf(d) * inv_rgb;
        }
        if (d_depth) {
            float gd = 0.f;
            if (tdep && tdep[i] > 0.0f && inv_dep > 0.0f) {
                const float d = depth[i] - tdep[i];
                l += fabsf(d) * inv_dep;
                gd = sgnf(d) * inv_dep;
            }
            d_depth[i] = gd;
        }
    }
    if (loss) {
        const float t = block_sum(l, red);
        if (threadIdx.x == 0) atomicAdd(loss, t);
    }
}

void launch_l1(const float *rgb, const float *depth, const float *trgb, const float *tdep, size_t hw, float wrgb,
               float wdep, uint32_t *nvalid, float *d_rgb, float *d_depth, float *loss, cudaStream_t st)
{
    const int threads = 256;
    int blocks = (int)((hw + threads - 1) / threads);
    if (blocks > 4 * 152) blocks = 4 * 152;
    if (blocks < 1) blocks = 1;
    const bool use_depth = tdep && d_depth && wdep != 0.0f;
    if (use_depth) k_count_valid<<<blocks, threads, 0, st>>>(tdep, hw, nvalid);
    k_l1_grad<<<blocks, threads, 0, st>>>(rgb, depth, trgb, use_depth ? tdep : nullptr, hw, wrgb, wdep,
                                          use_depth ? nvalid : nullptr, d_rgb, d_depth, loss);
}

__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

void launch_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t st)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks > 0) k_adam<<<(unsigned)blocks, 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
}

}  // namespace sgad
