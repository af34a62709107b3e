// Device-side definitions shared by the splatting kernels (sm_103a).
//
// Every floating-point step that decides something discrete (culling, the integer
// radius, tile bounds, the alpha floor and cap, the transmittance stop) is written with
// explicit round-to-nearest intrinsics, so each kernel that evaluates it (binning
// count, key emission, forward and backward compositing) executes the same arithmetic
// and reaches the same decision bit for bit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sgad.h"

namespace sgad {

constexpr float kNearPlane = 0.2f;        // cull at view depth <= 0.2 m
constexpr float kDilation = 0.3f;         // px^2 added to the 2D covariance diagonal
constexpr float kAlphaCap = 0.99f;
constexpr float kAlphaFloor = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;
// Below this exponent alpha = o e^power < e^power < (1/255) e^-0.0012 for any opacity
// o <= 1, so the entry is skipped whatever the rounding of exp: ln(1/255) = -5.54126.
constexpr float kPowerSkip = -5.5425f;
constexpr uint32_t kInvalidTile = 0xffffffffu;

// ------------------------------------------------------------ launch parameters

struct KfDev {
    const float *depth, *offset, *rgb, *logit, *scale;
    const float *xform;          // optional world transform of the centres (device 3x4), or null
    float *d_offset, *d_rgb, *d_logit, *d_scale;
    float fx, fy, cx, cy;
    float R[9], t[3];            // cam -> world
    int32_t W, H;
    uint32_t gbase;              // global index of this keyframe's first Gaussian
    int32_t learnable;
};

struct ViewDev {
    float *rgb, *depth, *alpha;
    const float *g_rgb, *g_depth, *g_alpha;
    float *d_pose;               // [12] d loss / d (world -> cam 3x4), or null
    float fx, fy, cx, cy;
    float R[9], t[3];            // world -> cam
    int32_t W, H;
    int32_t tiles_x, tiles_y;
    int32_t tile_base;           // global index of this view's first tile
    uint32_t pix_base;           // offset of this view's pixels in the per-pixel state
};

// Whole problem, passed by value to every kernel (fits the 32 KB parameter space).
struct Scene {
    int32_t n_kf, n_views;
    uint32_t n_gauss;
    int32_t n_tiles;
    int32_t tile_w, tile_h, tw_log2, th_log2;
    float bg[3];
    int32_t freeze_offset;
    KfDev kf[SGAD_MAX_KEYFRAMES];
    ViewDev view[SGAD_MAX_VIEWS];
};

// Device-side status block at the start of the workspace. The first 128 bytes describe
// the last forward and are cleared by every forward; the last 128 bytes accumulate
// failures until sgad_check() reads and clears them.
struct WsHeader {
    uint32_t n_keys;             // keys emitted by the last forward
    uint32_t needed;             // keys the last forward needed
    int32_t err;                 // first SGAD_ERR_* of the last forward, 0 if none
    uint32_t overflow;           // 1 if the last forward's keys did not fit
    uint32_t emit_overrun;       // binning count and emission disagreed (must stay 0)
    uint32_t queue_fwd;          // persistent forward compositing: next tile-order position
    unsigned long long n_pairs;  // (pixel, entry) pairs composited by the last forward
    unsigned long long n_evals;  // (pixel, entry) pairs whose alpha the last forward evaluated
    uint32_t queue_bwd;          // persistent backward compositing: next tile-order position
    uint32_t n_sort_exact;       // tiles the bucket sort handed to the exact radix sort
    uint32_t pad1[20];
    int32_t sticky_err;          // first error since the last sgad_check()
    uint32_t sticky_needed;      // largest key count needed since the last sgad_check()
    uint32_t sticky_overrun;
    uint32_t pad2[29];
};
static_assert(sizeof(WsHeader) == 256, "header is one 256-byte block");
constexpr size_t kHeaderPerCall = 128;   // bytes cleared by every forward

// Per-Gaussian record computed once per forward (view independent):
//   w0 = (mu_x, mu_y, mu_z, s), w1 = (opacity, r, g, b)
struct __align__(16) World {
    float4 w0, w1;
};

__device__ __forceinline__ int find_kf(const Scene &sc, uint32_t g)
{
    int k = 0;
#pragma unroll 1
    for (int i = 1; i < sc.n_kf; ++i)
        if (g >= sc.kf[i].gbase) k = i;
    return k;
}

__device__ __forceinline__ int find_view_of_tile(const Scene &sc, int tile)
{
    int k = 0;
#pragma unroll 1
    for (int i = 1; i < sc.n_views; ++i)
        if (tile >= sc.view[i].tile_base) k = i;
    return k;
}

__device__ __forceinline__ void record_error(WsHeader *h, int code)
{
    atomicCAS(reinterpret_cast<int *>(&h->err), 0, code);
    atomicCAS(reinterpret_cast<int *>(&h->sticky_err), 0, code);
}

// ------------------------------------------------------- FP32 projection (EWA)

// View-space centre, pixel mean and 2D covariance of an isotropic Gaussian of std-dev s
// at world position mu: t = R mu + t_k, p = (fx tx/tz + cx, fy ty/tz + cy),
// J = d p / d t, Sigma_2D = s^2 J J^T + 0.3 I.
struct Proj {
    float tx, ty, tz;
    float px, py;
    float cxx, cxy, cyy;         // Sigma_2D
};

__device__ __forceinline__ Proj project(const float4 w0, const ViewDev &v)
{
    Proj p;
    p.tx = __fmaf_rn(v.R[0], w0.x, __fmaf_rn(v.R[1], w0.y, __fmaf_rn(v.R[2], w0.z, v.t[0])));
    p.ty = __fmaf_rn(v.R[3], w0.x, __fmaf_rn(v.R[4], w0.y, __fmaf_rn(v.R[5], w0.z, v.t[1])));
    p.tz = __fmaf_rn(v.R[6], w0.x, __fmaf_rn(v.R[7], w0.y, __fmaf_rn(v.R[8], w0.z, v.t[2])));
    const float iz = __fdiv_rn(1.0f, p.tz);
    const float ux = __fmul_rn(p.tx, iz), uy = __fmul_rn(p.ty, iz);
    p.px = __fmaf_rn(v.fx, ux, v.cx);
    p.py = __fmaf_rn(v.fy, uy, v.cy);
    const float j00 = __fmul_rn(v.fx, iz), j02 = -__fmul_rn(j00, ux);
    const float j11 = __fmul_rn(v.fy, iz), j12 = -__fmul_rn(j11, uy);
    const float s2 = __fmul_rn(w0.w, w0.w);
    p.cxx = __fmaf_rn(s2, __fmaf_rn(j00, j00, __fmul_rn(j02, j02)), kDilation);
    p.cxy = __fmul_rn(s2, __fmul_rn(j02, j12));
    p.cyy = __fmaf_rn(s2, __fmaf_rn(j11, j11, __fmul_rn(j12, j12)), kDilation);
    return p;
}

// Square bound ceil(3 sqrt(lambda_max)) and the inclusive tile rectangle of the pixel
// box [floor(p - rho), floor(p + rho)] clipped to the image. Returns the tile count
// (0 when culled by the near plane, degenerate, or off the image).
struct Rect {
    int tx0, ty0, nx, ny;
};

__device__ __forceinline__ int bin_rect(const Proj &p, const ViewDev &v, int tw_log2, int th_log2,
                                        Rect &r)
{
    r.tx0 = r.ty0 = r.nx = r.ny = 0;
    if (!(p.tz > kNearPlane)) return 0;
    const float det = __fsub_rn(__fmul_rn(p.cxx, p.cyy), __fmul_rn(p.cxy, p.cxy));
    if (!(det > 0.0f)) return 0;
    const float mid = __fmul_rn(0.5f, __fadd_rn(p.cxx, p.cyy));
    const float disc = fmaxf(0.1f, __fsub_rn(__fmul_rn(mid, mid), det));
    const float lam = __fadd_rn(mid, __fsqrt_rn(disc));
    const float rho = ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam)));
    const float x0 = floorf(__fsub_rn(p.px, rho)), x1 = floorf(__fadd_rn(p.px, rho));
    const float y0 = floorf(__fsub_rn(p.py, rho)), y1 = floorf(__fadd_rn(p.py, rho));
    if (x1 < 0.0f || y1 < 0.0f || x0 > (float)(v.W - 1) || y0 > (float)(v.H - 1)) return 0;
    const int ix0 = x0 < 0.0f ? 0 : (int)x0;
    const int iy0 = y0 < 0.0f ? 0 : (int)y0;
    const int ix1 = x1 > (float)(v.W - 1) ? v.W - 1 : (int)x1;
    const int iy1 = y1 > (float)(v.H - 1) ? v.H - 1 : (int)y1;
    r.tx0 = ix0 >> tw_log2;
    r.ty0 = iy0 >> th_log2;
    r.nx = (ix1 >> tw_log2) - r.tx0 + 1;
    r.ny = (iy1 >> th_log2) - r.ty0 + 1;
    return r.nx * r.ny;
}

// Tile rectangle of a (Gaussian, view) pair as the binning count leaves it for the key
// emission: (tx0 | ty0 << 16, nx | ny << 16); nx = ny = 0 when it lists no tile.
__device__ __forceinline__ uint2 pack_rect(const Rect &r, int n)
{
    return n > 0 ? make_uint2((uint32_t)r.tx0 | ((uint32_t)r.ty0 << 16), (uint32_t)r.nx | ((uint32_t)r.ny << 16))
                 : make_uint2(0u, 0u);
}

__device__ __forceinline__ int unpack_rect(const uint2 q, Rect &r)
{
    r.tx0 = (int)(q.x & 0xffffu);
    r.ty0 = (int)(q.x >> 16);
    r.nx = (int)(q.y & 0xffffu);
    r.ny = (int)(q.y >> 16);
    return r.nx * r.ny;
}

// ------------------------------------------- double-float (Dekker/Knuth) arithmetic
//
// Used only for the view depth that goes into the sort key, so the key equals the
// exactly-rounded f32 of the depth an FP64 evaluation gives (error ~1e-13 relative,
// far below the f32 spacing). A value is the unevaluated sum hi + lo, |lo| <= ulp(hi)/2.
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b)
{
    dfloat s = df_two_sum(a.hi, b.hi);
    const dfloat t = df_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ dfloat df_mul_f(dfloat a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ dfloat df_div_f(dfloat a, float b)
{
    const float q1 = __fdiv_rn(a.hi, b);
    // remainder a - q1 b, exact product via FMA
    const float p = __fmul_rn(q1, b);
    const float pe = __fmaf_rn(q1, b, -p);
    dfloat r = df_two_sum(a.hi, -p);
    r.lo = __fsub_rn(__fadd_rn(r.lo, a.lo), pe);
    const float q2 = __fdiv_rn(__fadd_rn(r.hi, r.lo), b);
    return df_fast_two_sum(q1, q2);
}

// World position of keyframe pixel (u, v) at depth |D + delta|, in double-float.
struct dvec3 {
    dfloat x, y, z;
};

__device__ __forceinline__ dvec3 df_world_point(const KfDev &k, int u, int v, float D, float delta)
{
    dfloat d = df_two_sum(D, delta);
    if (d.hi < 0.0f || (d.hi == 0.0f && d.lo < 0.0f)) { d.hi = -d.hi; d.lo = -d.lo; }
    const dfloat rx = df_div_f(df_two_sum((float)u, -k.cx), k.fx);
    const dfloat ry = df_div_f(df_two_sum((float)v, -k.cy), k.fy);
    const dfloat px = df_mul(d, rx), py = df_mul(d, ry);     // pz = d
    dvec3 m;
    m.x = df_add(df_add(df_add(df_mul_f(px, k.R[0]), df_mul_f(py, k.R[1])), df_mul_f(d, k.R[2])), {k.t[0], 0.0f});
    m.y = df_add(df_add(df_add(df_mul_f(px, k.R[3]), df_mul_f(py, k.R[4])), df_mul_f(d, k.R[5])), {k.t[1], 0.0f});
    m.z = df_add(df_add(df_add(df_mul_f(px, k.R[6]), df_mul_f(py, k.R[7])), df_mul_f(d, k.R[8])), {k.t[2], 0.0f});
    return m;
}

// mu <- R mu + t with the keyframe's device transform (3x4 row-major), in double-float.
__device__ __forceinline__ dvec3 df_transform(const dvec3 &m, const float *X)
{
    dvec3 r;
    r.x = df_add(df_add(df_add(df_mul_f(m.x, X[0]), df_mul_f(m.y, X[1])), df_mul_f(m.z, X[2])), {X[3], 0.0f});
    r.y = df_add(df_add(df_add(df_mul_f(m.x, X[4]), df_mul_f(m.y, X[5])), df_mul_f(m.z, X[6])), {X[7], 0.0f});
    r.z = df_add(df_add(df_add(df_mul_f(m.x, X[8]), df_mul_f(m.y, X[9])), df_mul_f(m.z, X[10])), {X[11], 0.0f});
    return r;
}

__device__ __forceinline__ float df_view_depth(const dvec3 &m, const ViewDev &v)
{
    const dfloat z = df_add(df_add(df_add(df_mul_f(m.x, v.R[6]), df_mul_f(m.y, v.R[7])), df_mul_f(m.z, v.R[8])),
                            {v.t[2], 0.0f});
    return __fadd_rn(z.hi, z.lo);
}

// ------------------------------------------------------------------ compositing

// A Gaussian as staged in shared memory for one view (16-byte aligned pieces):
//   a = (px, py, hx, hy)  mean and half extents of the box outside which alpha < 1/255
//   b = (conic_a, conic_b, conic_c, opacity)
//   c = (r, g, b, z)
struct Staged {
    float4 a, b, c;
};

// Conic, opacity and culling box of a projected Gaussian. hx < 0 marks a Gaussian that
// cannot reach alpha >= 1/255 anywhere (opacity below the floor).
__device__ __forceinline__ void stage(const Proj &p, const float4 w1, float z, Staged &s)
{
    const float det = __fsub_rn(__fmul_rn(p.cxx, p.cyy), __fmul_rn(p.cxy, p.cxy));
    const float id = __fdiv_rn(1.0f, det);
    const float o = w1.x;
    s.b = make_float4(__fmul_rn(p.cyy, id), -__fmul_rn(p.cxy, id), __fmul_rn(p.cxx, id), o);
    s.c = make_float4(w1.y, w1.z, w1.w, z);
    // alpha >= 1/255 needs d^T Sigma^-1 d <= 2 ln(255 o); its bounding box has half
    // extents sqrt(2 ln(255 o) Sigma_ii). The box only prunes evaluations (the alpha test
    // decides), so it may be larger than needed but never smaller: the fast logarithm is
    // raised by 2e-6, above its documented error for arguments up to 255 (2^-21.41
    // absolute on [0.5, 2], 3 ulp of a result below 5.6 elsewhere), and the fast square
    // roots (x rsqrt(x), a few ulp) sit inside the 0.01-pixel pad that also covers the
    // FP32 rounding of the conic.
    const float l = __logf(255.0f * o) + 2e-6f;
    if (!(l > 0.0f)) {
        s.a = make_float4(p.px, p.py, -1.0f, -1.0f);
    } else {
        const float e = 2.0f * l * 1.0001f;
        const float ex = e * p.cxx, ey = e * p.cyy;     // > 0: cxx, cyy >= the dilation
        s.a = make_float4(p.px, p.py, ex * rsqrtf(ex) + 0.01f, ey * rsqrtf(ey) + 0.01f);
    }
}

// Exponent and alpha of a staged Gaussian at pixel (qx, qy), same arithmetic in the
// forward and backward passes. Returns false when the entry is skipped (power > 0 or
// alpha < 1/255).
__device__ __forceinline__ bool gauss_alpha(const Staged &s, float qx, float qy, float &dx, float &dy,
                                            float &ep, float &alpha)
{
    dx = __fsub_rn(s.a.x, qx);
    dy = __fsub_rn(s.a.y, qy);
    const float quad = __fmaf_rn(s.b.x, __fmul_rn(dx, dx), __fmul_rn(s.b.z, __fmul_rn(dy, dy)));
    const float power = __fsub_rn(__fmul_rn(-0.5f, quad), __fmul_rn(s.b.y, __fmul_rn(dx, dy)));
    // the range test and the floor combined without an early return (the exponential is
    // taken either way; the decisions are those of the two tests in turn)
    const bool in_range = !(power > 0.0f) && !(power < kPowerSkip);
    ep = __expf(power);
    const float raw = __fmul_rn(s.b.w, ep);
    alpha = fminf(kAlphaCap, raw);
    return in_range && alpha >= kAlphaFloor;
}

// Workspace layout (byte offsets, 256-aligned sections). Shared by the host API and the
// kernels' launch code.
struct Layout {
    size_t header, world, gacc, rects, tile_off, tile_cnt, tile_order, sort_list, pix_t, pix_n, keys, keys_alt, contrib,
        wmask, total;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline Layout make_layout(uint64_t n_gauss, uint64_t n_views, uint64_t n_tiles, uint64_t n_pix, uint64_t key_cap)
{
    Layout L;
    size_t o = 0;
    L.header = o; o = align256(o + sizeof(WsHeader));
    L.world = o; o = align256(o + n_gauss * sizeof(World));
    L.gacc = o; o = align256(o + n_gauss * 32);
    L.rects = o; o = align256(o + n_gauss * n_views * 8);
    L.tile_off = o; o = align256(o + (n_tiles + 1) * 4);
    L.tile_cnt = o; o = align256(o + (n_tiles + 1) * 4);
    L.tile_order = o; o = align256(o + n_tiles * 4);
    L.sort_list = o; o = align256(o + n_tiles * 4);
    L.pix_t = o; o = align256(o + n_pix * 4);
    L.pix_n = o; o = align256(o + n_pix * 4);
    L.keys = o; o = align256(o + key_cap * 8);
    L.keys_alt = o; o = align256(o + key_cap * 8);
    L.contrib = o; o = align256(o + (key_cap * 8 + (n_tiles + 1) * 256) * 4);
    L.wmask = o; o = align256(o + ((key_cap >> 2) + (n_tiles + 1) * 16 + 8) * 4);
    L.total = o;
    return L;
}

}  // namespace sgad
