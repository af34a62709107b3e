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
    // the opacity as the projection computed it (same expression: bit-identical), from the
    // 4-byte logit instead of the 32-byte world record
    const float o = 1.0f / (1.0f + expf(-k.logit[j]));
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

// All views of one loss call; every view owns a contiguous range of CTAs.
constexpr int kLossChunk = 4096;    // pixels per CTA

struct LossView {
    const float *rgb, *depth, *alpha, *trgb, *tdep;   // alpha: null unless masking
    float *drgb, *ddep;
    uint32_t *nvalid;
    uint32_t hw;
    uint32_t block0;
    int32_t vec;                    // hw % 4 == 0 and every plane 16-byte aligned
};

struct LossBatch {
    int32_t n;
    float wrgb, wdep, min_alpha;
    LossView v[SGAD_MAX_VIEWS];
};

__device__ __forceinline__ int loss_view(const LossBatch &B)
{
    int k = 0;
    for (int i = 1; i < B.n; ++i)
        if (B.v[i].block0 <= blockIdx.x) k = i;
    return k;
}

__global__ void __launch_bounds__(256) k_count_valid(const __grid_constant__ LossBatch B)
{
    __shared__ float red[32];
    const LossView &v = B.v[loss_view(B)];
    const size_t base = (size_t)(blockIdx.x - v.block0) * kLossChunk;
    const size_t end = base + kLossChunk < v.hw ? base + kLossChunk : v.hw;
    float c = 0.f;
    for (size_t i = base + threadIdx.x; i < end; i += blockDim.x) c += v.tdep[i] > 0.0f ? 1.0f : 0.0f;
    const float t = block_sum(c, red);
    if (threadIdx.x == 0 && t > 0.f) atomicAdd(v.nvalid, (uint32_t)t);
}

__global__ void __launch_bounds__(256) k_l1_grad(const __grid_constant__ LossBatch B, float *loss)
{
    __shared__ float red[32];
    const LossView &v = B.v[loss_view(B)];
    const size_t hw = v.hw;
    const size_t base = (size_t)(blockIdx.x - v.block0) * kLossChunk;
    const size_t end = base + kLossChunk < hw ? base + kLossChunk : hw;
    const float inv_rgb = B.wrgb / (3.0f * (float)hw);
    const uint32_t nv = v.nvalid ? *v.nvalid : 0u;
    const float inv_dep = nv > 0 ? B.wdep / (float)nv : 0.0f;
    float l = 0.f;
    if (v.vec) {                     // four pixels per thread and access
        for (size_t i = base + 4 * threadIdx.x; i < end; i += 4 * blockDim.x) {
            const float4 al = v.alpha ? *reinterpret_cast<const float4 *>(v.alpha + i) : make_float4(1.f, 1.f, 1.f, 1.f);
            const bool keep[4] = {!v.alpha || al.x > B.min_alpha, !v.alpha || al.y > B.min_alpha,
                                  !v.alpha || al.z > B.min_alpha, !v.alpha || al.w > B.min_alpha};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 r = *reinterpret_cast<const float4 *>(v.rgb + c * hw + i);
                const float4 t = *reinterpret_cast<const float4 *>(v.trgb + c * hw + i);
                const float d[4] = {r.x - t.x, r.y - t.y, r.z - t.z, r.w - t.w};
                float gq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (keep[q]) l += fabsf(d[q]) * inv_rgb;
                    gq[q] = keep[q] ? sgnf(d[q]) * inv_rgb : 0.0f;
                }
                *reinterpret_cast<float4 *>(v.drgb + c * hw + i) = make_float4(gq[0], gq[1], gq[2], gq[3]);
            }
            if (v.ddep) {
                float gd[4] = {0.f, 0.f, 0.f, 0.f};
                if (v.tdep && inv_dep > 0.0f) {
                    const float4 dp = *reinterpret_cast<const float4 *>(v.depth + i);
                    const float4 td = *reinterpret_cast<const float4 *>(v.tdep + i);
                    const float dv[4] = {dp.x, dp.y, dp.z, dp.w}, tv[4] = {td.x, td.y, td.z, td.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (keep[q] && tv[q] > 0.0f) {
                            const float d = dv[q] - tv[q];
                            l += fabsf(d) * inv_dep;
                            gd[q] = sgnf(d) * inv_dep;
                        }
                }
                *reinterpret_cast<float4 *>(v.ddep + i) = make_float4(gd[0], gd[1], gd[2], gd[3]);
            }
        }
    } else {
        for (size_t i = base + threadIdx.x; i < end; i += blockDim.x) {
            const bool keep = !v.alpha || v.alpha[i] > B.min_alpha;     // silhouette mask
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float d = v.rgb[c * hw + i] - v.trgb[c * hw + i];
                if (keep) l += fabsf(d) * inv_rgb;
                v.drgb[c * hw + i] = keep ? sgnf(d) * inv_rgb : 0.0f;
            }
            if (v.ddep) {
                float gd = 0.f;
                if (keep && v.tdep && v.tdep[i] > 0.0f && inv_dep > 0.0f) {
                    const float d = v.depth[i] - v.tdep[i];
                    l += fabsf(d) * inv_dep;
                    gd = sgnf(d) * inv_dep;
                }
                v.ddep[i] = gd;
            }
        }
    }
    if (loss) {
        const float t = block_sum(l, red);
        if (threadIdx.x == 0) atomicAdd(loss, t);
    }
}

// views: per view (rgb, depth, target rgb, target depth or NULL, d_rgb, d_depth or NULL,
// valid counter or NULL, pixel count).
void launch_l1_batch(int n, const float *const *rgb, const float *const *depth, const float *const *alpha,
                     const float *const *trgb, const float *const *tdep, float *const *drgb, float *const *ddep,
                     uint32_t *nvalid, const uint32_t *hw, float wrgb, float wdep, float min_alpha, float *loss,
                     cudaStream_t st)
{
    LossBatch B;
    B.n = n;
    B.wrgb = wrgb;
    B.wdep = wdep;
    B.min_alpha = min_alpha;
    uint32_t blocks = 0;
    const bool use_depth = wdep != 0.0f && tdep && ddep && nvalid;
    for (int i = 0; i < n; ++i) {
        LossView &v = B.v[i];
        v.rgb = rgb[i];
        v.depth = depth ? depth[i] : nullptr;
        v.alpha = alpha ? alpha[i] : nullptr;
        v.trgb = trgb[i];
        v.tdep = use_depth ? tdep[i] : nullptr;
        v.drgb = drgb[i];
        v.ddep = ddep ? ddep[i] : nullptr;
        v.nvalid = use_depth ? nvalid + i : nullptr;
        v.hw = hw[i];
        uintptr_t al = reinterpret_cast<uintptr_t>(v.rgb) | reinterpret_cast<uintptr_t>(v.trgb) |
                       reinterpret_cast<uintptr_t>(v.drgb) | reinterpret_cast<uintptr_t>(v.alpha) |
                       reinterpret_cast<uintptr_t>(v.ddep);
        if (v.tdep) al |= reinterpret_cast<uintptr_t>(v.depth) | reinterpret_cast<uintptr_t>(v.tdep);
        v.vec = (hw[i] % 4 == 0 && (al & 15u) == 0) ? 1 : 0;
        v.block0 = blocks;
        blocks += (hw[i] + kLossChunk - 1) / kLossChunk;
    }
    if (use_depth) k_count_valid<<<blocks, 256, 0, st>>>(B);
    k_l1_grad<<<blocks, 256, 0, st>>>(B, loss);
}

template <bool kLog>
__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float pi = p[i];
        const float gi = kLog ? g[i] * pi : g[i];     // d/d(log s) = s d/ds
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float step = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = kLog ? expf(logf(pi) - step) : pi - step;
    }
}

// ---------------------------------------------------------- multi-tensor Adam

constexpr int kAdamChunk = 4096;    // elements per CTA

struct AdamDesc {
    float *p;
    const float *g;
    float *m, *v;
    int64_t n;
    float lr;
    int32_t mode;
    int32_t vec;                    // n % 4 == 0 and all four arrays 16-byte aligned
    int64_t block0;                 // first CTA of this tensor
};

struct AdamBatch {
    int32_t n;
    float b1, b2, eps;
    AdamDesc t[SGAD_ADAM_MAX_TENSORS];
};

// One Adam update of element (p, g, m, v) with the bias corrections' reciprocals.
__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, float b1, float b2, float eps, float lr,
                                         float ic1, float ic2, bool log_mode)
{
    const float gi = log_mode ? g * p : g;
    m = b1 * m + (1.0f - b1) * gi;
    v = b2 * v + (1.0f - b2) * gi * gi;
    const float stp = lr * (m * ic1) / (sqrtf(v * ic2) + eps);
    p = log_mode ? p * expf(-stp) : p - stp;
}

__global__ void __launch_bounds__(256) k_adam_multi(const __grid_constant__ AdamBatch B, const int32_t *step)
{
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {                 // last tensor whose first CTA <= blockIdx.x
        const int mid = (lo + hi + 1) >> 1;
        if (B.t[mid].block0 <= (int64_t)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const AdamDesc &d = B.t[lo];
    const float s = (float)(*step + 1);
    const float ic1 = 1.0f / (1.0f - powf(B.b1, s)), ic2 = 1.0f / (1.0f - powf(B.b2, s));
    const bool log_mode = d.mode == SGAD_ADAM_LOG;
    const int64_t base = ((int64_t)blockIdx.x - d.block0) * kAdamChunk;
    const int64_t end = base + kAdamChunk < d.n ? base + kAdamChunk : d.n;
    if (d.vec) {                      // four elements per thread and access
        for (int64_t i = base + 4 * (int64_t)threadIdx.x; i < end; i += 4 * (int64_t)blockDim.x) {
            float4 p = *reinterpret_cast<const float4 *>(d.p + i);
            const float4 g = *reinterpret_cast<const float4 *>(d.g + i);
            float4 m = *reinterpret_cast<const float4 *>(d.m + i);
            float4 v = *reinterpret_cast<const float4 *>(d.v + i);
            adam_one(p.x, g.x, m.x, v.x, B.b1, B.b2, B.eps, d.lr, ic1, ic2, log_mode);
            adam_one(p.y, g.y, m.y, v.y, B.b1, B.b2, B.eps, d.lr, ic1, ic2, log_mode);
            adam_one(p.z, g.z, m.z, v.z, B.b1, B.b2, B.eps, d.lr, ic1, ic2, log_mode);
            adam_one(p.w, g.w, m.w, v.w, B.b1, B.b2, B.eps, d.lr, ic1, ic2, log_mode);
            *reinterpret_cast<float4 *>(d.m + i) = m;
            *reinterpret_cast<float4 *>(d.v + i) = v;
            *reinterpret_cast<float4 *>(d.p + i) = p;
        }
        return;
    }
    for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x) {
        float p = d.p[i], m = d.m[i], v = d.v[i];
        adam_one(p, d.g[i], m, v, B.b1, B.b2, B.eps, d.lr, ic1, ic2, log_mode);
        d.m[i] = m;
        d.v[i] = v;
        d.p[i] = p;
    }
}

__global__ void k_increment(int32_t *c) { *c += 1; }

cudaError_t launch_adam_multi(int n_t, const sgad_adam_tensor *t, float b1, float b2, float eps, int32_t *step,
                              cudaStream_t st)
{
    AdamBatch B;
    B.n = n_t;
    B.b1 = b1;
    B.b2 = b2;
    B.eps = eps;
    int64_t blocks = 0;
    for (int i = 0; i < n_t; ++i) {
        AdamDesc &d = B.t[i];
        d.p = t[i].param;
        d.g = t[i].grad;
        d.m = t[i].m;
        d.v = t[i].v;
        d.n = t[i].n;
        d.lr = t[i].lr;
        d.mode = t[i].mode;
        const uintptr_t al = reinterpret_cast<uintptr_t>(d.p) | reinterpret_cast<uintptr_t>(d.g) |
                             reinterpret_cast<uintptr_t>(d.m) | reinterpret_cast<uintptr_t>(d.v);
        d.vec = (d.n % 4 == 0 && (al & 15u) == 0) ? 1 : 0;
        d.block0 = blocks;
        blocks += (t[i].n + kAdamChunk - 1) / kAdamChunk;
    }
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    if (blocks > 0) k_adam_multi<<<(unsigned)blocks, 256, 0, st>>>(B, step);
    k_increment<<<1, 1, 0, st>>>(step);
    return cudaGetLastError();
}

void launch_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                 float c1, float c2, bool log_mode, cudaStream_t st)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks <= 0) return;
    if (log_mode)
        k_adam<true><<<(unsigned)blocks, 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
    else
        k_adam<false><<<(unsigned)blocks, 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
}

// ------------------------------------------------- rendering-based camera initialisation
//
// State layout (device floats): E [0, 12), M = W0^-1 E W0 [12, 24), Adam m [24, 30) and
// v [30, 36), step count [36], current pose E W0 [37, 49). 3x4 row-major [R | t].
struct PoseArgs {
    double W0[12];
    double lr[6];
    double b1, b2, eps;
};

__device__ void mat34_mul(const double *A, const double *B, double *C)     // C = A B (as 4x4)
{
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c) {
            double s = c == 3 ? A[4 * r + 3] : 0.0;
            for (int k = 0; k < 3; ++k) s += A[4 * r + k] * B[4 * k + c];
            C[4 * r + c] = s;
        }
    }
}

__global__ void k_pose_adam_step(const float *__restrict__ d_pose, float *__restrict__ st, const PoseArgs a)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double *W = a.W0;
    double G[9], c[3];
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) G[3 * r + k] = d_pose[4 * r + k];
        c[r] = d_pose[4 * r + 3];
    }
    // M = R0 G^T; d/d omega = vee(M - M^T) + t0 x c; d/d v = c
    double Mx[9];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int q = 0; q < 3; ++q) s += W[4 * r + q] * G[3 * k + q];
            Mx[3 * r + k] = s;
        }
    const double t0[3] = {W[3], W[7], W[11]};
    double g[6];
    g[0] = Mx[5] - Mx[7] + (t0[1] * c[2] - t0[2] * c[1]);
    g[1] = Mx[6] - Mx[2] + (t0[2] * c[0] - t0[0] * c[2]);
    g[2] = Mx[1] - Mx[3] + (t0[0] * c[1] - t0[1] * c[0]);
    g[3] = c[0];
    g[4] = c[1];
    g[5] = c[2];
    const double n = (double)st[36] + 1.0;
    st[36] = (float)n;
    double xi[6];
    for (int i = 0; i < 6; ++i) {
        const double m = a.b1 * (double)st[24 + i] + (1.0 - a.b1) * g[i];
        const double v = a.b2 * (double)st[30 + i] + (1.0 - a.b2) * g[i] * g[i];
        st[24 + i] = (float)m;
        st[30 + i] = (float)v;
        const double mh = m / (1.0 - pow(a.b1, n)), vh = v / (1.0 - pow(a.b2, n));
        xi[i] = -a.lr[i] * mh / (sqrt(vh) + a.eps);
    }
    // exp(xi) = [Rodrigues(omega) | v]
    const double th = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    const double K[9] = {0.0, -xi[2], xi[1], xi[2], 0.0, -xi[0], -xi[1], xi[0], 0.0};
    double K2[9];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int q = 0; q < 3; ++q) s += K[3 * r + q] * K[3 * q + k];
            K2[3 * r + k] = s;
        }
    const double sa = th < 1e-12 ? 1.0 : sin(th) / th;
    const double sb = th < 1e-12 ? 0.0 : (1.0 - cos(th)) / (th * th);
    double X[12];
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) X[4 * r + k] = (r == k ? 1.0 : 0.0) + sa * K[3 * r + k] + sb * K2[3 * r + k];
        X[4 * r + 3] = xi[3 + r];
    }
    double E[12], En[12];
    for (int i = 0; i < 12; ++i) E[i] = st[i];
    mat34_mul(X, E, En);
    // M = W0^-1 E W0 with W0^-1 = [R0^T | -R0^T t0]; pose = E W0
    double Wi[12], EW[12], Mn[12];
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) Wi[4 * r + k] = W[4 * k + r];
        Wi[4 * r + 3] = -(W[r] * t0[0] + W[4 + r] * t0[1] + W[8 + r] * t0[2]);
    }
    mat34_mul(En, W, EW);
    mat34_mul(Wi, EW, Mn);
    for (int i = 0; i < 12; ++i) {
        st[i] = (float)En[i];
        st[12 + i] = (float)Mn[i];
        st[37 + i] = (float)EW[i];
    }
}

cudaError_t launch_pose_adam_step(const float *d_pose, const float *W0, float *state, float lr_rot, float lr_trans,
                                  float b1, float b2, float eps, cudaStream_t st)
{
    PoseArgs a;
    for (int i = 0; i < 12; ++i) a.W0[i] = W0[i];
    for (int i = 0; i < 3; ++i) {
        a.lr[i] = lr_rot;
        a.lr[3 + i] = lr_trans;
    }
    a.b1 = b1;
    a.b2 = b2;
    a.eps = eps;
    k_pose_adam_step<<<1, 32, 0, st>>>(d_pose, state, a);
    return cudaGetLastError();
}

}  // namespace sgad
