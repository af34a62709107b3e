// Front-to-back compositing (forward step a7) and its reverse-order adjoint (a9, with
// the per-Gaussian chain rule of a10 down to the world centre, scale, opacity and
// colour).
//
// One CTA of 256 threads per tile, one pixel per thread; each warp owns an 8x4 block of
// pixels. The tile's sorted list is consumed in batches of 256 entries: each thread
// stages one entry (gathering the Gaussian's 32-byte world record and projecting it into
// the view) into shared memory, then every warp tests 32 staged Gaussians at a time
// against its pixel block (one lane per Gaussian, a ballot) and walks only the ones
// whose alpha >= 1/255 box reaches it. A warp stops when all its pixels are done; the
// CTA stops when all warps are.
//
// The backward pass walks the same lists from the tile's largest contributor count down
// to 0. Each pixel starts from its saved final transmittance and recovers the
// transmittance in front of entry i by division, T_i = T_{i+1} / (1 - alpha_i), which is
// stable because alpha <= 0.99. Per (pixel, entry) it forms the gradient of the colour,
// depth and alpha terms, reduces ten moments over the warp with a reduce-scatter,
// accumulates them per staged Gaussian in shared memory, and at the end of the batch the
// staging thread turns them into d mu, d s, d opacity, d colour and adds them to the
// per-Gaussian accumulator with two 16-byte vector atomics.
//
// Defaults (measured on the 8 x 640x480 room): forward one pixel per thread, 512 entries
// per barrier, 6 resident blocks; backward two pixels per thread (k_composite_bwd2, 128
// threads, 8 resident blocks). The other layouts stay selectable at build time.
#include "sgad_device.cuh"

namespace sgad {

constexpr int kBlock = 256;
constexpr unsigned kFull = 0xffffffffu;
// Entries staged per block-wide barrier in the forward pass (a multiple of kBlock), and
// the resident-block target of the backward pass (bounds its registers).
#ifndef SGAD_FWD_BATCH
#define SGAD_FWD_BATCH 512
#endif
#ifndef SGAD_FWD_MINBLOCKS
#define SGAD_FWD_MINBLOCKS 6
#endif
#ifndef SGAD_BWD_MINBLOCKS
#define SGAD_BWD_MINBLOCKS 5
#endif
constexpr int kFwdBatch = SGAD_FWD_BATCH;
static_assert(kFwdBatch % kBlock == 0 && kFwdBatch * 48 <= 48 * 1024, "forward batch");

struct PixelMap {
    int x, y;
    bool inside;
    WarpRect wr;
};

template <int TW, int TH>
__device__ __forceinline__ PixelMap map_pixel(const ViewDev &v, int local_tile)
{
    static_assert(TW * TH == kBlock, "tile must hold 256 pixels");
    const int tx = local_tile % v.tiles_x, ty = local_tile / v.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wx = warp % (TW / 8), wy = warp / (TW / 8);
    PixelMap m;
    const int bx = tx * TW + wx * 8, by = ty * TH + wy * 4;
    m.x = bx + (lane & 7);
    m.y = by + (lane >> 3);
    m.inside = m.x < v.W && m.y < v.H;
    m.wr = {(float)bx, (float)by, (float)(bx + 7), (float)(by + 3)};
    return m;
}

template <int TW, int TH>
__global__ void __launch_bounds__(kBlock, SGAD_FWD_MINBLOCKS) k_composite_fwd(const __grid_constant__ Scene sc,
                                                          const World *__restrict__ world,
                                                          const uint32_t *__restrict__ off,
                                                          const uint64_t *__restrict__ entries,
                                                          float *__restrict__ pix_t, uint32_t *__restrict__ pix_n,
                                                          WsHeader *hdr)
{
    __shared__ Staged sm[kFwdBatch];
    if (hdr->overflow) return;
    uint32_t n_pairs = 0, n_evals = 0;
    const int tile = blockIdx.x;
    const ViewDev &v = sc.view[find_view_of_tile(sc, tile)];
    const PixelMap pm = map_pixel<TW, TH>(v, tile - v.tile_base);
    const float qx = (float)pm.x, qy = (float)pm.y;
    const int lane = threadIdx.x & 31;

    float T = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f, aa = 0.f;
    int last = -1;
    bool done = !pm.inside;
    bool warp_done = __all_sync(kFull, done);
    const uint32_t s = off[tile], e = off[tile + 1];
    for (uint32_t b0 = s; b0 < e; b0 += kFwdBatch) {
        if (__syncthreads_and(done)) break;
#pragma unroll
        for (int r = 0; r < kFwdBatch / kBlock; ++r) {
            const uint32_t i = b0 + r * kBlock + threadIdx.x;
            if (i < e) {
                const uint64_t ent = entries[i];
                Staged st;
                if ((uint32_t)ent < sc.n_gauss) {
                    const World w = world[(uint32_t)ent];
                    stage(project(w.w0, v), w.w1, __uint_as_float((uint32_t)(ent >> 32)), st);
                } else {
                    st.a = make_float4(0.f, 0.f, -1.f, -1.f);     // never reaches a pixel
                }
                sm[r * kBlock + threadIdx.x] = st;
            }
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)kFwdBatch, e - b0);
        if (warp_done) continue;
        for (int c0 = 0; c0 < nb; c0 += 32) {
            const int j = c0 + lane;
            const uint32_t hits = __ballot_sync(kFull, j < nb && overlaps(sm[j], pm.wr));
            uint32_t mask = hits;
            while (mask) {
                const int jj = c0 + __ffs(mask) - 1;
                mask &= mask - 1;
                if (done) continue;
                const Staged st = sm[jj];
                float dx, dy, ep, alpha;
                ++n_evals;
                if (!gauss_alpha(st, qx, qy, dx, dy, ep, alpha)) continue;
                const float test = __fmul_rn(T, __fsub_rn(1.0f, alpha));
                if (test < kTStop) {
                    done = true;
                    continue;
                }
                ++n_pairs;
                const float w = __fmul_rn(alpha, T);
                cr = __fmaf_rn(w, st.c.x, cr);
                cg = __fmaf_rn(w, st.c.y, cg);
                cb = __fmaf_rn(w, st.c.z, cb);
                dd = __fmaf_rn(w, st.c.w, dd);
                aa = __fadd_rn(aa, w);
                T = test;
                last = (int)(b0 + jj - s);
            }
            if (__all_sync(kFull, done)) {
                warp_done = true;
                break;
            }
        }
    }
    if (pm.inside) {
        const size_t hw = (size_t)v.W * v.H, p = (size_t)pm.y * v.W + pm.x;
        v.rgb[p] = cr + T * sc.bg[0];
        v.rgb[hw + p] = cg + T * sc.bg[1];
        v.rgb[2 * hw + p] = cb + T * sc.bg[2];
        v.depth[p] = dd;
        v.alpha[p] = aa;
        pix_t[v.pix_base + p] = T;
        pix_n[v.pix_base + p] = (uint32_t)(last + 1);
    }
    const uint32_t wp = __reduce_add_sync(kFull, n_pairs), we = __reduce_add_sync(kFull, n_evals);
    if (lane == 0 && we) {
        atomicAdd(&hdr->n_pairs, (unsigned long long)wp);
        atomicAdd(&hdr->n_evals, (unsigned long long)we);
    }
}

// ------------------------------------------- forward, two pixels per thread variant
//
// 128 threads per tile, each warp an 8x8 pixel block, each lane the pixels (x, y) and
// (x, y + 4): fewer warps wait at each block barrier and the staged Gaussian read from
// shared memory serves two pixels.
constexpr int kBlock2 = 128;
#ifndef SGAD_FWD_PPT
#define SGAD_FWD_PPT 1
#endif
#ifndef SGAD_FWD2_MINBLOCKS
#define SGAD_FWD2_MINBLOCKS 1
#endif

struct PixelMap2 {
    int x, y[2];
    bool inside[2];
    WarpRect wr;
};

template <int TW, int TH>
__device__ __forceinline__ PixelMap2 map_pixel2(const ViewDev &v, int local_tile)
{
    static_assert(TW * TH == 2 * kBlock2, "tile must hold 256 pixels");
    const int tx = local_tile % v.tiles_x, ty = local_tile / v.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wx = warp % (TW / 8), wy = warp / (TW / 8);
    PixelMap2 m;
    const int bx = tx * TW + wx * 8, by = ty * TH + wy * 8;
    m.x = bx + (lane & 7);
    m.y[0] = by + (lane >> 3);
    m.y[1] = m.y[0] + 4;
    m.inside[0] = m.x < v.W && m.y[0] < v.H;
    m.inside[1] = m.x < v.W && m.y[1] < v.H;
    m.wr = {(float)bx, (float)by, (float)(bx + 7), (float)(by + 7)};
    return m;
}

template <int TW, int TH>
__global__ void __launch_bounds__(kBlock2, SGAD_FWD2_MINBLOCKS) k_composite_fwd2(const __grid_constant__ Scene sc,
                                                                                const World *__restrict__ world,
                                                                                const uint32_t *__restrict__ off,
                                                                                const uint64_t *__restrict__ entries,
                                                                                float *__restrict__ pix_t,
                                                                                uint32_t *__restrict__ pix_n,
                                                                                WsHeader *hdr)
{
    __shared__ Staged sm[kFwdBatch];
    if (hdr->overflow) return;
    uint32_t n_pairs = 0, n_evals = 0;
    const int tile = blockIdx.x;
    const ViewDev &v = sc.view[find_view_of_tile(sc, tile)];
    const PixelMap2 pm = map_pixel2<TW, TH>(v, tile - v.tile_base);
    const float qx = (float)pm.x;
    const float qy[2] = {(float)pm.y[0], (float)pm.y[1]};
    const int lane = threadIdx.x & 31;

    float T[2] = {1.0f, 1.0f}, cr[2] = {0.f, 0.f}, cg[2] = {0.f, 0.f}, cb[2] = {0.f, 0.f};
    float dd[2] = {0.f, 0.f}, aa[2] = {0.f, 0.f};
    int last[2] = {-1, -1};
    bool done[2] = {!pm.inside[0], !pm.inside[1]};
    bool warp_done = __all_sync(kFull, done[0] && done[1]);
    const uint32_t s = off[tile], e = off[tile + 1];
    for (uint32_t b0 = s; b0 < e; b0 += kFwdBatch) {
        if (__syncthreads_and(done[0] && done[1])) break;
#pragma unroll
        for (int r = 0; r < kFwdBatch / kBlock2; ++r) {
            const uint32_t i = b0 + r * kBlock2 + threadIdx.x;
            if (i < e) {
                const uint64_t ent = entries[i];
                Staged st;
                if ((uint32_t)ent < sc.n_gauss) {
                    const World w = world[(uint32_t)ent];
                    stage(project(w.w0, v), w.w1, __uint_as_float((uint32_t)(ent >> 32)), st);
                } else {
                    st.a = make_float4(0.f, 0.f, -1.f, -1.f);     // never reaches a pixel
                }
                sm[r * kBlock2 + threadIdx.x] = st;
            }
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)kFwdBatch, e - b0);
        if (warp_done) continue;
        for (int c0 = 0; c0 < nb; c0 += 32) {
            const int j = c0 + lane;
            const uint32_t hits = __ballot_sync(kFull, j < nb && overlaps(sm[j], pm.wr));
            uint32_t mask = hits;
            while (mask) {
                const int jj = c0 + __ffs(mask) - 1;
                mask &= mask - 1;
                if (done[0] && done[1]) continue;
                const Staged st = sm[jj];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    if (done[p]) continue;
                    float dx, dy, ep, alpha;
                    ++n_evals;
                    if (!gauss_alpha(st, qx, qy[p], dx, dy, ep, alpha)) continue;
                    const float test = __fmul_rn(T[p], __fsub_rn(1.0f, alpha));
                    if (test < kTStop) {
                        done[p] = true;
                        continue;
                    }
                    ++n_pairs;
                    const float w = __fmul_rn(alpha, T[p]);
                    cr[p] = __fmaf_rn(w, st.c.x, cr[p]);
                    cg[p] = __fmaf_rn(w, st.c.y, cg[p]);
                    cb[p] = __fmaf_rn(w, st.c.z, cb[p]);
                    dd[p] = __fmaf_rn(w, st.c.w, dd[p]);
                    aa[p] = __fadd_rn(aa[p], w);
                    T[p] = test;
                    last[p] = (int)(b0 + jj - s);
                }
            }
            if (__all_sync(kFull, done[0] && done[1])) {
                warp_done = true;
                break;
            }
        }
    }
    const size_t hw = (size_t)v.W * v.H;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        if (!pm.inside[p]) continue;
        const size_t q = (size_t)pm.y[p] * v.W + pm.x;
        v.rgb[q] = cr[p] + T[p] * sc.bg[0];
        v.rgb[hw + q] = cg[p] + T[p] * sc.bg[1];
        v.rgb[2 * hw + q] = cb[p] + T[p] * sc.bg[2];
        v.depth[q] = dd[p];
        v.alpha[q] = aa[p];
        pix_t[v.pix_base + q] = T[p];
        pix_n[v.pix_base + q] = (uint32_t)(last[p] + 1);
    }
    const uint32_t wp = __reduce_add_sync(kFull, n_pairs), we = __reduce_add_sync(kFull, n_evals);
    if (lane == 0 && we) {
        atomicAdd(&hdr->n_pairs, (unsigned long long)wp);
        atomicAdd(&hdr->n_evals, (unsigned long long)we);
    }
}

// Reduce-scatter of 16 per-lane values over the warp in 16 shuffles (instead of 80 for
// 16 butterfly all-reductions): at each level a lane sends the half of its slots its
// partner keeps and adds the partner's copy of the half it keeps. Afterwards every lane
// returns the warp total of slot (lane >> 1).
__device__ __forceinline__ float warp_reduce_scatter16(float (&v)[16], int lane)
{
#pragma unroll
    for (int lvl = 0; lvl < 4; ++lvl) {
        const int half = 8 >> lvl, mask = 16 >> lvl;
        const bool upper = (lane & mask) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, mask);
        }
    }
    return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

template <int TW, int TH>
__global__ void __launch_bounds__(kBlock, SGAD_BWD_MINBLOCKS) k_composite_bwd(const __grid_constant__ Scene sc,
                                                          const World *__restrict__ world,
                                                          const uint32_t *__restrict__ off,
                                                          const uint64_t *__restrict__ entries,
                                                          const float *__restrict__ pix_t,
                                                          const uint32_t *__restrict__ pix_n,
                                                          float4 *__restrict__ gacc, const WsHeader *hdr)
{
    __shared__ Staged sm[kBlock];
    __shared__ float acc[kBlock][11];
    __shared__ int s_nmax;
    if (hdr->overflow) return;
    const int tile = blockIdx.x;
    const ViewDev &v = sc.view[find_view_of_tile(sc, tile)];
    const PixelMap pm = map_pixel<TW, TH>(v, tile - v.tile_base);
    const float qx = (float)pm.x, qy = (float)pm.y;
    const int lane = threadIdx.x & 31;
    const uint32_t s = off[tile];
    const int len = (int)(off[tile + 1] - s);

    float Tf = 1.0f, gr = 0.f, gg = 0.f, gb = 0.f, gD = 0.f, gA = 0.f;
    int nc = 0;
    if (pm.inside) {
        const size_t hw = (size_t)v.W * v.H, p = (size_t)pm.y * v.W + pm.x;
        Tf = pix_t[v.pix_base + p];
        nc = min((int)pix_n[v.pix_base + p], len);
        if (v.g_rgb) {
            gr = v.g_rgb[p];
            gg = v.g_rgb[hw + p];
            gb = v.g_rgb[2 * hw + p];
        }
        if (v.g_depth) gD = v.g_depth[p];
        if (v.g_alpha) gA = v.g_alpha[p];
    }
    const int warp_nc = __reduce_max_sync(kFull, (unsigned)nc);
    if (threadIdx.x == 0) s_nmax = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&s_nmax, warp_nc);
    __syncthreads();
    const int nmax = s_nmax;
    const float bgdot = sc.bg[0] * gr + sc.bg[1] * gg + sc.bg[2] * gb;

    float T = Tf, SCr = 0.f, SCg = 0.f, SCb = 0.f, SD = 0.f, SA = 0.f;
    for (int b1 = nmax; b1 > 0; b1 -= kBlock) {
        const int b0 = b1 > kBlock ? b1 - kBlock : 0;
        const int nb = b1 - b0;
        __syncthreads();
        // stage, keeping this thread's Gaussian in registers for the chain rule
        uint32_t g = 0;
        Proj pr = {};
        float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0;
        bool staged = false;
        if ((int)threadIdx.x < nb) {
            const uint64_t ent = entries[s + b0 + threadIdx.x];
            g = (uint32_t)ent;
            Staged st;
            if (g < sc.n_gauss) {
                const World w = world[g];
                w0 = w.w0;
                w1 = w.w1;
                pr = project(w0, v);
                stage(pr, w1, __uint_as_float((uint32_t)(ent >> 32)), st);
                staged = true;
            } else {
                st.a = make_float4(0.f, 0.f, -1.f, -1.f);     // never reaches a pixel
            }
            sm[threadIdx.x] = st;
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[threadIdx.x][q] = 0.f;
        __syncthreads();
        if (b0 < warp_nc) {
            for (int c0 = ((nb - 1) >> 5) << 5; c0 >= 0; c0 -= 32) {
                const int j = c0 + lane;
                const uint32_t hits = __ballot_sync(kFull, j < nb && b0 + j < warp_nc && overlaps(sm[j], pm.wr));
                uint32_t mask = hits;
                while (mask) {
                    const int bit = 31 - __clz(mask);
                    mask &= ~(1u << bit);
                    const int jj = c0 + bit;
                    float val[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) val[q] = 0.f;
                    bool contrib = false;
                    if (b0 + jj < nc) {
                        const Staged st = sm[jj];
                        float dx, dy, ep, alpha;
                        if (gauss_alpha(st, qx, qy, dx, dy, ep, alpha)) {
                            contrib = true;
                            const float om = __fsub_rn(1.0f, alpha);
                            const float rom = __fdividef(1.0f, om);     // om >= 0.01: fast reciprocal
                            const float Ti = T * rom;
                            const float w = alpha * Ti;
                            val[0] = w * gr;
                            val[1] = w * gg;
                            val[2] = w * gb;
                            val[3] = w * gD;
                            const float dal = Ti * ((st.c.x - SCr) * gr + (st.c.y - SCg) * gg + (st.c.z - SCb) * gb +
                                                    (st.c.w - SD) * gD + (1.0f - SA) * gA) -
                                              (Tf * rom) * bgdot;
                            SCr = alpha * st.c.x + om * SCr;
                            SCg = alpha * st.c.y + om * SCg;
                            SCb = alpha * st.c.z + om * SCb;
                            SD = alpha * st.c.w + om * SD;
                            SA = alpha + om * SA;
                            if (!(st.b.w * ep > kAlphaCap)) {
                                const float G = dal * alpha;
                                val[4] = G;
                                val[5] = G * dx;
                                val[6] = G * dy;
                                val[7] = G * dx * dx;
                                val[8] = G * dx * dy;
                                val[9] = G * dy * dy;
                            }
                            T = Ti;
                        }
                    }
                    if (__any_sync(kFull, contrib)) {
                        const float total = warp_reduce_scatter16(val, lane);
                        const int slot = lane >> 1;
                        if ((lane & 1) == 0 && slot < 10) atomicAdd(&acc[jj][slot], total);
                    }
                }
            }
        }
        __syncthreads();
        if (staged) {
            const float *A = acc[threadIdx.x];
            bool any = false;
#pragma unroll
            for (int q = 0; q < 10; ++q) any |= A[q] != 0.f;
            if (any) {
                const Staged &st = sm[threadIdx.x];
                const float ca = st.b.x, cbb = st.b.y, cc = st.b.z, o = st.b.w;
                const float G = A[4], Gx = A[5], Gy = A[6], Gxx = A[7], Gxy = A[8], Gyy = A[9];
                const float d_o = G / o;
                const float da = -0.5f * Gxx, db = -Gxy, dc = -0.5f * Gyy;
                const float dpx = -(ca * Gx + cbb * Gy), dpy = -(cbb * Gx + cc * Gy);
                // conic (a, b, c) = (w, -y, x) / det of Sigma_2D = [[x, y], [y, w]]
                const float x = pr.cxx, y = pr.cxy, wv = pr.cyy;
                const float det = x * wv - y * y, id2 = 1.0f / (det * det);
                const float gx = (-wv * wv * da + y * wv * db - y * y * dc) * id2;
                const float gy = (2.0f * y * wv * da - (det + 2.0f * y * y) * db + 2.0f * x * y * dc) * id2;
                const float gw = (-y * y * da + y * x * db - x * x * dc) * id2;
                // Sigma_2D = s^2 J J^T + 0.3 I
                const float tz = pr.tz, iz = 1.0f / tz, iz2 = iz * iz;
                const float j00 = v.fx * iz, j02 = -v.fx * pr.tx * iz2;
                const float j11 = v.fy * iz, j12 = -v.fy * pr.ty * iz2;
                const float sc_ = w0.w, s2 = sc_ * sc_;
                const float ds = 2.0f * sc_ * ((j00 * j00 + j02 * j02) * gx + j02 * j12 * gy + (j11 * j11 + j12 * j12) * gw);
                const float gj00 = 2.0f * s2 * j00 * gx;
                const float gj02 = s2 * (2.0f * j02 * gx + j12 * gy);
                const float gj11 = 2.0f * s2 * j11 * gw;
                const float gj12 = s2 * (j02 * gy + 2.0f * j12 * gw);
                // p = (fx tx/tz + cx, fy ty/tz + cy); composited depth z = tz
                const float gtx = gj02 * (-v.fx * iz2) + dpx * v.fx * iz;
                const float gty = gj12 * (-v.fy * iz2) + dpy * v.fy * iz;
                const float gtz = gj00 * (-v.fx * iz2) + gj02 * (2.0f * v.fx * pr.tx * iz2 * iz) +
                                  gj11 * (-v.fy * iz2) + gj12 * (2.0f * v.fy * pr.ty * iz2 * iz) +
                                  dpx * (-v.fx * pr.tx * iz2) + dpy * (-v.fy * pr.ty * iz2) + A[3];
                // t = R mu + t_k  ->  d mu = R^T d t
                const float4 ga = make_float4(v.R[0] * gtx + v.R[3] * gty + v.R[6] * gtz,
                                              v.R[1] * gtx + v.R[4] * gty + v.R[7] * gtz,
                                              v.R[2] * gtx + v.R[5] * gty + v.R[8] * gtz, ds);
                const float4 gb4 = make_float4(d_o, A[0], A[1], A[2]);
                atomicAdd(&gacc[2 * (size_t)g], ga);
                atomicAdd(&gacc[2 * (size_t)g + 1], gb4);
            }
        }
    }
}

// ------------------------------------------- backward, two pixels per thread variant
//
// Same walk as k_composite_bwd with 128 threads per tile, each lane owning the pixels
// (x, y) and (x, y + 4) of its warp's 8x8 block: the per-pair moments of both pixels are
// summed in registers before the warp reduction, so each reduce-scatter covers 64 pixels.
#ifndef SGAD_BWD_PPT
#define SGAD_BWD_PPT 2
#endif
#ifndef SGAD_BWD2_MINBLOCKS
#define SGAD_BWD2_MINBLOCKS 8
#endif
constexpr int kBwdBatch2 = 256;

// Chain rule of one staged Gaussian from its ten accumulated pair moments (colour (3),
// depth, G, G dx, G dy, G dx^2, G dx dy, G dy^2 with G = dL/dpower) down to d mu, d s,
// d opacity and d colour, added to its accumulator.
__device__ __forceinline__ void chain_and_accumulate(const float *A, const Staged &st, const Proj &pr, float s_,
                                                     const ViewDev &v, float4 *gacc, uint32_t g)
{
    const float ca = st.b.x, cbb = st.b.y, cc = st.b.z, o = st.b.w;
    const float G = A[4], Gx = A[5], Gy = A[6], Gxx = A[7], Gxy = A[8], Gyy = A[9];
    const float d_o = G / o;
    const float da = -0.5f * Gxx, db = -Gxy, dc = -0.5f * Gyy;
    const float dpx = -(ca * Gx + cbb * Gy), dpy = -(cbb * Gx + cc * Gy);
    // conic (a, b, c) = (w, -y, x) / det of Sigma_2D = [[x, y], [y, w]]
    const float x = pr.cxx, y = pr.cxy, wv = pr.cyy;
    const float det = x * wv - y * y, id2 = 1.0f / (det * det);
    const float gx = (-wv * wv * da + y * wv * db - y * y * dc) * id2;
    const float gy = (2.0f * y * wv * da - (det + 2.0f * y * y) * db + 2.0f * x * y * dc) * id2;
    const float gw = (-y * y * da + y * x * db - x * x * dc) * id2;
    // Sigma_2D = s^2 J J^T + 0.3 I
    const float tz = pr.tz, iz = 1.0f / tz, iz2 = iz * iz;
    const float j00 = v.fx * iz, j02 = -v.fx * pr.tx * iz2;
    const float j11 = v.fy * iz, j12 = -v.fy * pr.ty * iz2;
    const float s2 = s_ * s_;
    const float ds = 2.0f * s_ * ((j00 * j00 + j02 * j02) * gx + j02 * j12 * gy + (j11 * j11 + j12 * j12) * gw);
    const float gj00 = 2.0f * s2 * j00 * gx;
    const float gj02 = s2 * (2.0f * j02 * gx + j12 * gy);
    const float gj11 = 2.0f * s2 * j11 * gw;
    const float gj12 = s2 * (j02 * gy + 2.0f * j12 * gw);
    // p = (fx tx/tz + cx, fy ty/tz + cy); composited depth z = tz
    const float gtx = gj02 * (-v.fx * iz2) + dpx * v.fx * iz;
    const float gty = gj12 * (-v.fy * iz2) + dpy * v.fy * iz;
    const float gtz = gj00 * (-v.fx * iz2) + gj02 * (2.0f * v.fx * pr.tx * iz2 * iz) + gj11 * (-v.fy * iz2) +
                      gj12 * (2.0f * v.fy * pr.ty * iz2 * iz) + dpx * (-v.fx * pr.tx * iz2) +
                      dpy * (-v.fy * pr.ty * iz2) + A[3];
    // t = R mu + t_k  ->  d mu = R^T d t
    const float4 ga = make_float4(v.R[0] * gtx + v.R[3] * gty + v.R[6] * gtz, v.R[1] * gtx + v.R[4] * gty + v.R[7] * gtz,
                                  v.R[2] * gtx + v.R[5] * gty + v.R[8] * gtz, ds);
    atomicAdd(&gacc[2 * (size_t)g], ga);
    atomicAdd(&gacc[2 * (size_t)g + 1], make_float4(d_o, A[0], A[1], A[2]));
}

template <int TW, int TH>
__global__ void __launch_bounds__(kBlock2, SGAD_BWD2_MINBLOCKS) k_composite_bwd2(const __grid_constant__ Scene sc,
                                                                                const World *__restrict__ world,
                                                                                const uint32_t *__restrict__ off,
                                                                                const uint64_t *__restrict__ entries,
                                                                                const float *__restrict__ pix_t,
                                                                                const uint32_t *__restrict__ pix_n,
                                                                                float4 *__restrict__ gacc,
                                                                                const WsHeader *hdr)
{
    __shared__ Staged sm[kBwdBatch2];
    __shared__ uint32_t sg[kBwdBatch2];
    __shared__ float acc[kBwdBatch2][11];
    __shared__ int s_nmax;
    if (hdr->overflow) return;
    const int tile = blockIdx.x;
    const ViewDev &v = sc.view[find_view_of_tile(sc, tile)];
    const PixelMap2 pm = map_pixel2<TW, TH>(v, tile - v.tile_base);
    const float qx = (float)pm.x;
    const float qy[2] = {(float)pm.y[0], (float)pm.y[1]};
    const int lane = threadIdx.x & 31;
    const uint32_t s = off[tile];
    const int len = (int)(off[tile + 1] - s);
    const size_t hw = (size_t)v.W * v.H;

    float Tf[2], gr[2], gg[2], gb[2], gD[2], gA[2], T[2], SCr[2], SCg[2], SCb[2], SD[2], SA[2];
    int nc[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        Tf[p] = 1.0f;
        gr[p] = gg[p] = gb[p] = gD[p] = gA[p] = 0.f;
        nc[p] = 0;
        if (pm.inside[p]) {
            const size_t q = (size_t)pm.y[p] * v.W + pm.x;
            Tf[p] = pix_t[v.pix_base + q];
            nc[p] = min((int)pix_n[v.pix_base + q], len);
            if (v.g_rgb) {
                gr[p] = v.g_rgb[q];
                gg[p] = v.g_rgb[hw + q];
                gb[p] = v.g_rgb[2 * hw + q];
            }
            if (v.g_depth) gD[p] = v.g_depth[q];
            if (v.g_alpha) gA[p] = v.g_alpha[q];
        }
        T[p] = Tf[p];
        SCr[p] = SCg[p] = SCb[p] = SD[p] = SA[p] = 0.f;
    }
    const int warp_nc = __reduce_max_sync(kFull, (unsigned)max(nc[0], nc[1]));
    if (threadIdx.x == 0) s_nmax = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&s_nmax, warp_nc);
    __syncthreads();
    const int nmax = s_nmax;
    float bgdot[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) bgdot[p] = sc.bg[0] * gr[p] + sc.bg[1] * gg[p] + sc.bg[2] * gb[p];

    for (int b1 = nmax; b1 > 0; b1 -= kBwdBatch2) {
        const int b0 = b1 > kBwdBatch2 ? b1 - kBwdBatch2 : 0;
        const int nb = b1 - b0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kBwdBatch2 / kBlock2; ++r) {
            const int k = r * kBlock2 + threadIdx.x;
            if (k < nb) {
                const uint64_t ent = entries[s + b0 + k];
                const uint32_t g = (uint32_t)ent;
                Staged st;
                if (g < sc.n_gauss) {
                    const World w = world[g];
                    stage(project(w.w0, v), w.w1, __uint_as_float((uint32_t)(ent >> 32)), st);
                } else {
                    st.a = make_float4(0.f, 0.f, -1.f, -1.f);     // never reaches a pixel
                }
                sm[k] = st;
                sg[k] = g;
            }
#pragma unroll
            for (int q = 0; q < 10; ++q) acc[k][q] = 0.f;
        }
        __syncthreads();
        if (b0 < warp_nc) {
            for (int c0 = ((nb - 1) >> 5) << 5; c0 >= 0; c0 -= 32) {
                const int j = c0 + lane;
                const uint32_t hits = __ballot_sync(kFull, j < nb && b0 + j < warp_nc && overlaps(sm[j], pm.wr));
                uint32_t mask = hits;
                while (mask) {
                    const int bit = 31 - __clz(mask);
                    mask &= ~(1u << bit);
                    const int jj = c0 + bit;
                    float val[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) val[q] = 0.f;
                    bool contrib = false;
                    const Staged st = sm[jj];
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        if (b0 + jj >= nc[p]) continue;
                        float dx, dy, ep, alpha;
                        if (!gauss_alpha(st, qx, qy[p], dx, dy, ep, alpha)) continue;
                        contrib = true;
                        const float om = __fsub_rn(1.0f, alpha);
                        const float rom = __fdividef(1.0f, om);     // om >= 0.01: fast reciprocal
                        const float Ti = T[p] * rom;
                        const float w = alpha * Ti;
                        val[0] += w * gr[p];
                        val[1] += w * gg[p];
                        val[2] += w * gb[p];
                        val[3] += w * gD[p];
                        const float dal = Ti * ((st.c.x - SCr[p]) * gr[p] + (st.c.y - SCg[p]) * gg[p] +
                                                (st.c.z - SCb[p]) * gb[p] + (st.c.w - SD[p]) * gD[p] +
                                                (1.0f - SA[p]) * gA[p]) -
                                          (Tf[p] * rom) * bgdot[p];
                        SCr[p] = alpha * st.c.x + om * SCr[p];
                        SCg[p] = alpha * st.c.y + om * SCg[p];
                        SCb[p] = alpha * st.c.z + om * SCb[p];
                        SD[p] = alpha * st.c.w + om * SD[p];
                        SA[p] = alpha + om * SA[p];
                        if (!(st.b.w * ep > kAlphaCap)) {
                            const float G = dal * alpha;
                            val[4] += G;
                            val[5] += G * dx;
                            val[6] += G * dy;
                            val[7] += G * dx * dx;
                            val[8] += G * dx * dy;
                            val[9] += G * dy * dy;
                        }
                        T[p] = Ti;
                    }
                    if (__any_sync(kFull, contrib)) {
                        const float total = warp_reduce_scatter16(val, lane);
                        const int slot = lane >> 1;
                        if ((lane & 1) == 0 && slot < 10) atomicAdd(&acc[jj][slot], total);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kBwdBatch2 / kBlock2; ++r) {
            const int k = r * kBlock2 + threadIdx.x;
            if (k >= nb || sg[k] >= sc.n_gauss) continue;
            const float *A = acc[k];
            bool any = false;
#pragma unroll
            for (int q = 0; q < 10; ++q) any |= A[q] != 0.f;
            if (!any) continue;
            const float4 w0 = world[sg[k]].w0;
            chain_and_accumulate(A, sm[k], project(w0, v), w0.w, v, gacc, sg[k]);
        }
    }
}

template <int TW, int TH>
static void launch_pair(bool fwd, const Scene &sc, const World *world, const uint32_t *off, const uint64_t *entries,
                        float *pix_t, uint32_t *pix_n, float4 *gacc, WsHeader *hdr, cudaStream_t st)
{
    if (sc.n_tiles <= 0) return;
    if (fwd && SGAD_FWD_PPT == 2)
        k_composite_fwd2<TW, TH><<<sc.n_tiles, kBlock2, 0, st>>>(sc, world, off, entries, pix_t, pix_n, hdr);
    else if (fwd)
        k_composite_fwd<TW, TH><<<sc.n_tiles, kBlock, 0, st>>>(sc, world, off, entries, pix_t, pix_n, hdr);
    else if (SGAD_BWD_PPT == 2)
        k_composite_bwd2<TW, TH><<<sc.n_tiles, kBlock2, 0, st>>>(sc, world, off, entries, pix_t, pix_n, gacc, hdr);
    else
        k_composite_bwd<TW, TH><<<sc.n_tiles, kBlock, 0, st>>>(sc, world, off, entries, pix_t, pix_n, gacc, hdr);
}

void launch_composite(bool fwd, const Scene &sc, const World *world, const uint32_t *off, const uint64_t *entries,
                      float *pix_t, uint32_t *pix_n, float4 *gacc, WsHeader *hdr, cudaStream_t st)
{
    if (sc.tile_w == 16)
        launch_pair<16, 16>(fwd, sc, world, off, entries, pix_t, pix_n, gacc, hdr, st);
    else if (sc.tile_w == 8)
        launch_pair<8, 32>(fwd, sc, world, off, entries, pix_t, pix_n, gacc, hdr, st);
    else
        launch_pair<32, 8>(fwd, sc, world, off, entries, pix_t, pix_n, gacc, hdr, st);
}

}  // namespace sgad
