/*
 * FP64 CPU oracle for the splatting of pixel-aligned Gaussians at adjusted depth.
 *
 * TEST INFRASTRUCTURE ONLY (see sgad_oracle.h): the plain definition that the CUDA
 * library is checked against. Written for clarity, not speed: every step follows the
 * formulas in the order they are stated, in double precision, with no blocking or
 * fusion beyond what the definition itself says.
 *
 * Paper passages followed (SGAD-SLAM):
 *   Sec. 3.1  simplified Gaussian: colour (3), one variance ("radius"), opacity, offset;
 *   Sec. 3.2  Gaussian j of frame i on the ray of pixel j at depth |D_i(j) + delta_i(j)|;
 *             (V'_k, D'_k) = splat(G_i, p_k); Eq. 1 mapping loss (L1 terms);
 *   Supp. A   r = D/F initial radius; learning rates for Adam.
 * The splatting formulas themselves are not printed in the paper; the 3DGS conventions
 * it builds on are used (EWA projection, 0.3 px dilation, 3-sigma square bounds,
 * alpha = min(0.99, o exp(power)), skip alpha < 1/255, stop before T < 1e-4).
 */
#include "sgad_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NEAR_PLANE 0.2          /* cull at t_z <= 0.2 m */
#define DILATION 0.3            /* added to both diagonal entries of the 2D covariance */
#define ALPHA_CAP 0.99
#define ALPHA_FLOOR (1.0 / 255.0)
#define T_STOP 1e-4
#define Z_ROUND_MARGIN 1e-12    /* relative distance of t_z to an f32 rounding midpoint */

/* ------------------------------------------------------------------ small helpers */

int64_t orc_num_gaussians(const orc_kf *kfs, int32_t n_kf)
{
    int64_t n = 0;
    for (int32_t i = 0; i < n_kf; ++i) n += (int64_t)kfs[i].cam.width * kfs[i].cam.height;
    return n;
}

static int32_t tiles_x(const orc_cam *v, const orc_opts *o) { return (v->width + o->tile_w - 1) / o->tile_w; }
static int32_t tiles_y(const orc_cam *v, const orc_opts *o) { return (v->height + o->tile_h - 1) / o->tile_h; }

int32_t orc_num_tiles(const orc_cam *views, int32_t n_views, const orc_opts *opt)
{
    int32_t n = 0;
    for (int32_t k = 0; k < n_views; ++k) n += tiles_x(&views[k], opt) * tiles_y(&views[k], opt);
    return n;
}

static int32_t tile_base(const orc_cam *views, int32_t view, const orc_opts *opt)
{
    return orc_num_tiles(views, view, opt);
}

/* keyframe owning global Gaussian g, and g's pixel index inside it */
static int32_t owner(const orc_kf *kfs, int32_t n_kf, int64_t g, int64_t *local)
{
    for (int32_t i = 0; i < n_kf; ++i) {
        int64_t n = (int64_t)kfs[i].cam.width * kfs[i].cam.height;
        if (g < n) { *local = g; return i; }
        g -= n;
    }
    *local = -1;
    return -1;
}

static double rel_gap(double x, double thr) { return fabs(x - thr) / fabs(thr); }

/* relative distance of z to the nearest midpoint between adjacent f32 values, i.e. how
 * far it is from a change of its f32 rounding */
static double round_gap(double z)
{
    float f = (float)z;
    double up = 0.5 * ((double)f + (double)nextafterf(f, INFINITY));
    double dn = 0.5 * ((double)f + (double)nextafterf(f, -INFINITY));
    return fmin(fabs(z - up), fabs(z - dn)) / fabs(z);
}

/* ------------------------------------------------------------------- projection */

/* Decision values of one (Gaussian, view) pair in single precision, the way the kernel
 * evaluates them: the world centre from the keyframe ray, the view-space centre, the
 * pixel mean, the dilated 2D covariance, the integer radius and tile rectangle, the
 * conic and the opacity. Each line is one IEEE single operation (fmaf where the kernel
 * fuses), so the integers that come out equal the kernel's. */
static void project_f32(const orc_kf *kf, int64_t j, const orc_cam *view, const orc_opts *opt, orc_proj *P)
{
    const orc_cam *c = &kf->cam;
    const int32_t W = c->width;
    float M[12], V[12];
    for (int i = 0; i < 12; ++i) {
        M[i] = (float)c->pose[i];
        V[i] = (float)view->pose[i];
    }
    const float u = (float)(j % W), v = (float)(j / W);
    const float d = fabsf((float)kf->depth[j] + (float)kf->offset[j]);
    const float rx = (u - (float)c->cx) / (float)c->fx;
    const float ry = (v - (float)c->cy) / (float)c->fy;
    const float qx = d * rx, qy = d * ry;
    const float mx = fmaf(M[0], qx, fmaf(M[1], qy, fmaf(M[2], d, M[3])));
    const float my = fmaf(M[4], qx, fmaf(M[5], qy, fmaf(M[6], d, M[7])));
    const float mz = fmaf(M[8], qx, fmaf(M[9], qy, fmaf(M[10], d, M[11])));
    const float s = (float)kf->scale[j];
    P->of = 1.0f / (1.0f + expf(-(float)kf->logit[j]));
    const float tx = fmaf(V[0], mx, fmaf(V[1], my, fmaf(V[2], mz, V[3])));
    const float ty = fmaf(V[4], mx, fmaf(V[5], my, fmaf(V[6], mz, V[7])));
    const float tz = fmaf(V[8], mx, fmaf(V[9], my, fmaf(V[10], mz, V[11])));
    const float fx = (float)view->fx, fy = (float)view->fy;
    const float iz = 1.0f / tz;
    const float ux = tx * iz, uy = ty * iz;
    const float px = fmaf(fx, ux, (float)view->cx), py = fmaf(fy, uy, (float)view->cy);
    const float j00 = fx * iz, j02 = -(j00 * ux);
    const float j11 = fy * iz, j12 = -(j11 * uy);
    const float s2 = s * s;
    const float cxx = fmaf(s2, fmaf(j00, j00, j02 * j02), (float)DILATION);
    const float cxy = s2 * (j02 * j12);
    const float cyy = fmaf(s2, fmaf(j11, j11, j12 * j12), (float)DILATION);
    const float det = cxx * cyy - cxy * cxy;
    P->pf[0] = px;
    P->pf[1] = py;
    P->tx0 = 1; P->tx1 = 0; P->ty0 = 1; P->ty1 = 0;
    P->visible = 0;
    P->ntiles = 0;
    if (!(tz > (float)NEAR_PLANE) || !(det > 0.0f)) return;
    P->visible = 1;
    const float id = 1.0f / det;
    P->conicf[0] = cyy * id;
    P->conicf[1] = -(cxy * id);
    P->conicf[2] = cxx * id;
    const float mid = 0.5f * (cxx + cyy);
    const float disc = fmaxf(0.1f, mid * mid - det);
    const float lam = mid + sqrtf(disc);
    const float rho = ceilf(3.0f * sqrtf(lam));
    P->rho = rho;
    /* pixel rectangle [floor(p - rho), floor(p + rho)] clipped to the image */
    const float x0 = floorf(px - rho), x1 = floorf(px + rho);
    const float y0 = floorf(py - rho), y1 = floorf(py + rho);
    if (x1 < 0.0f || y1 < 0.0f || x0 > (float)(view->width - 1) || y0 > (float)(view->height - 1)) return;
    const int32_t ix0 = x0 < 0.0f ? 0 : (int32_t)x0, iy0 = y0 < 0.0f ? 0 : (int32_t)y0;
    const int32_t ix1 = x1 > (float)(view->width - 1) ? view->width - 1 : (int32_t)x1;
    const int32_t iy1 = y1 > (float)(view->height - 1) ? view->height - 1 : (int32_t)y1;
    P->tx0 = ix0 / opt->tile_w; P->tx1 = ix1 / opt->tile_w;
    P->ty0 = iy0 / opt->tile_h; P->ty1 = iy1 / opt->tile_h;
    P->ntiles = (P->tx1 - P->tx0 + 1) * (P->ty1 - P->ty0 + 1);
}

/* Sec. 3.2: Gaussian at pixel (u, v) of keyframe kf sits at mu = R_i (|D + delta| r) + t_i
 * with r = ((u - cx)/fx, (v - cy)/fy, 1); it is seen by the view at t = R_k mu + t_k.
 * EWA: J = d(pixel)/d(t), Sigma_2D = s^2 J J^T + 0.3 I for the isotropic 3D covariance
 * s^2 I; its inverse is the conic. FP64 values; the decisions come from project_f32. */
static void project_one(const orc_kf *kf, int64_t j, const orc_cam *view, const orc_opts *opt,
                        orc_proj *P)
{
    const orc_cam *c = &kf->cam;
    const int32_t W = c->width;
    const double u = (double)(j % W), v = (double)(j / W);
    const double D = kf->depth[j], delta = kf->offset[j];
    const double dt = fabs(D + delta);
    const double r[3] = {(u - c->cx) / c->fx, (v - c->cy) / c->fy, 1.0};
    const double *M = c->pose, *V = view->pose;
    const int64_t hw = (int64_t)c->width * c->height;

    memset(P, 0, sizeof(*P));
    for (int a = 0; a < 3; ++a)
        P->mu[a] = M[4 * a] * dt * r[0] + M[4 * a + 1] * dt * r[1] + M[4 * a + 2] * dt * r[2] + M[4 * a + 3];
    for (int a = 0; a < 3; ++a)
        P->t[a] = V[4 * a] * P->mu[0] + V[4 * a + 1] * P->mu[1] + V[4 * a + 2] * P->mu[2] + V[4 * a + 3];
    P->o = 1.0 / (1.0 + exp(-kf->logit[j]));
    P->s = kf->scale[j];
    for (int ch = 0; ch < 3; ++ch) P->color[ch] = kf->rgb[ch * hw + j];
    P->zf = (double)(float)P->t[2];
    if (round_gap(P->t[2]) < Z_ROUND_MARGIN) P->near |= ORC_NEAR_Z;

    const double tz = P->t[2];
    if (tz > 0.0) {
        const double fx = view->fx, fy = view->fy;
        P->p[0] = fx * P->t[0] / tz + view->cx;
        P->p[1] = fy * P->t[1] / tz + view->cy;
        const double J00 = fx / tz, J02 = -fx * P->t[0] / (tz * tz);
        const double J11 = fy / tz, J12 = -fy * P->t[1] / (tz * tz);
        const double s2 = P->s * P->s;
        const double x = s2 * (J00 * J00 + J02 * J02) + DILATION;
        const double y = s2 * (J02 * J12);
        const double w = s2 * (J11 * J11 + J12 * J12) + DILATION;
        const double det = x * w - y * y;
        P->cov[0] = x; P->cov[1] = y; P->cov[2] = w;
        if (det > 0.0) {
            P->conic[0] = w / det;
            P->conic[1] = -y / det;
            P->conic[2] = x / det;
        }
    }
    project_f32(kf, j, view, opt, P);
}

int32_t orc_project(const orc_kf *kfs, int32_t n_kf, const orc_cam *view, const orc_opts *opt,
                    orc_proj *out)
{
    int64_t base = 0;
    for (int32_t i = 0; i < n_kf; ++i) {
        const int64_t n = (int64_t)kfs[i].cam.width * kfs[i].cam.height;
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j) project_one(&kfs[i], j, view, opt, &out[base + j]);
        base += n;
    }
    return 0;
}

static int covers(const orc_proj *P, int32_t tx, int32_t ty)
{
    return P->ntiles > 0 && tx >= P->tx0 && tx <= P->tx1 && ty >= P->ty0 && ty <= P->ty1;
}

/* -------------------------------------------------------------- brute-force keys */

typedef struct { uint64_t key; uint32_t val; uint8_t near; } key_entry;

static int cmp_key(const void *a, const void *b)
{
    const key_entry *x = (const key_entry *)a, *y = (const key_entry *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->val != y->val) return x->val < y->val ? -1 : 1;
    return 0;
}

static uint32_t f32_bits(double zf)
{
    float f = (float)zf;
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

int64_t orc_keys(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                 const orc_opts *opt, uint64_t *keys, uint32_t *vals, uint8_t *near_out)
{
    const int64_t nG = orc_num_gaussians(kfs, n_kf);
    orc_proj *proj = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)nG);
    key_entry *list = NULL;
    int64_t n = 0, cap = 0;
    for (int32_t k = 0; k < n_views; ++k) {
        orc_project(kfs, n_kf, &views[k], opt, proj);
        const int32_t tb = tile_base(views, k, opt);
        const int32_t ntx = tiles_x(&views[k], opt), nty = tiles_y(&views[k], opt);
        for (int32_t ty = 0; ty < nty; ++ty)
            for (int32_t tx = 0; tx < ntx; ++tx)
                for (int64_t g = 0; g < nG; ++g) {
                    if (!covers(&proj[g], tx, ty)) continue;
                    if (keys) {
                        if (n == cap) {
                            cap = cap ? 2 * cap : 1024;
                            list = (key_entry *)realloc(list, sizeof(key_entry) * (size_t)cap);
                        }
                        list[n].key = ((uint64_t)(uint32_t)(tb + ty * ntx + tx) << 32) | f32_bits(proj[g].zf);
                        list[n].val = (uint32_t)g;
                        list[n].near = (uint8_t)proj[g].near;
                    }
                    ++n;
                }
    }
    if (keys) {
        qsort(list, (size_t)n, sizeof(key_entry), cmp_key);
        for (int64_t i = 0; i < n; ++i) {
            keys[i] = list[i].key;
            vals[i] = list[i].val;
            if (near_out) near_out[i] = list[i].near;
        }
    }
    free(list);
    free(proj);
    return n;
}

/* ------------------------------------------------------------------- tile lists */

typedef struct { float zf; uint32_t g; } list_entry;

static int cmp_list(const void *a, const void *b)
{
    const list_entry *x = (const list_entry *)a, *y = (const list_entry *)b;
    if (x->zf != y->zf) return x->zf < y->zf ? -1 : 1;
    if (x->g != y->g) return x->g < y->g ? -1 : 1;
    return 0;
}

typedef struct {
    int32_t ntx, nty;
    int64_t *off;       /* [ntiles + 1] */
    list_entry *e;      /* entries of every tile, each tile sorted by (zf, g) */
} tile_lists;

/* Every visible Gaussian is listed in each tile of its rectangle; each list is sorted
 * front to back by (z rounded to f32, Gaussian index). */
static void build_lists(const orc_proj *proj, int64_t nG, const orc_cam *view, const orc_opts *opt,
                        tile_lists *L)
{
    L->ntx = tiles_x(view, opt);
    L->nty = tiles_y(view, opt);
    const int32_t nt = L->ntx * L->nty;
    L->off = (int64_t *)calloc((size_t)nt + 1, sizeof(int64_t));
    for (int64_t g = 0; g < nG; ++g) {
        const orc_proj *P = &proj[g];
        if (P->ntiles <= 0) continue;
        for (int32_t ty = P->ty0; ty <= P->ty1; ++ty)
            for (int32_t tx = P->tx0; tx <= P->tx1; ++tx) L->off[ty * L->ntx + tx + 1]++;
    }
    for (int32_t t = 0; t < nt; ++t) L->off[t + 1] += L->off[t];
    L->e = (list_entry *)malloc(sizeof(list_entry) * (size_t)(L->off[nt] + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nt);
    memcpy(fill, L->off, sizeof(int64_t) * (size_t)nt);
    for (int64_t g = 0; g < nG; ++g) {
        const orc_proj *P = &proj[g];
        if (P->ntiles <= 0) continue;
        for (int32_t ty = P->ty0; ty <= P->ty1; ++ty)
            for (int32_t tx = P->tx0; tx <= P->tx1; ++tx) {
                list_entry *e = &L->e[fill[ty * L->ntx + tx]++];
                e->zf = (float)P->zf;
                e->g = (uint32_t)g;
            }
    }
    free(fill);
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t t = 0; t < nt; ++t)
        qsort(L->e + L->off[t], (size_t)(L->off[t + 1] - L->off[t]), sizeof(list_entry), cmp_list);
}

static void free_lists(tile_lists *L)
{
    free(L->off);
    free(L->e);
}

/* ------------------------------------------------------------- per-pixel walk */

typedef struct {
    int32_t pos;        /* position in the tile list */
    uint32_t g;
    double alpha;       /* after the cap */
    double T;           /* transmittance in front of this Gaussian */
    double ep;          /* exp(power) */
    double dx, dy;      /* p - pixel */
    int32_t capped;     /* alpha was clamped to the cap */
} walk_rec;

typedef struct {
    double rgb[3], depth, alpha, T;
    int32_t n_contrib;
    int32_t near;
    int32_t n_rec;
    int32_t end;        /* list position where the walk ended (the stop entry, or the length) */
    uint64_t hash;
} walk_out;

static uint64_t fnv(uint64_t h, uint64_t x)
{
    for (int i = 0; i < 8; ++i) { h ^= (x >> (8 * i)) & 0xff; h *= 1099511628211ull; }
    return h;
}

/* Front-to-back compositing of one pixel over a depth-sorted list (3DGS convention):
 * power = -(a dx^2 + c dy^2)/2 - b dx dy with d = p - pixel; skip power > 0; alpha =
 * min(0.99, o e^power); skip alpha < 1/255; stop (excluding this entry) once T (1 - alpha)
 * would fall below 1e-4; otherwise add alpha T (colour, depth, 1) and update T. The
 * branches are taken in single precision as the kernel takes them (the transmittance
 * that decides the stop is the single-precision running product); the accumulated values
 * are double precision. */
static void walk_pixel(const orc_proj *proj, const list_entry *list, int64_t n, double qx, double qy,
                       const orc_opts *opt, walk_rec *rec, walk_out *out)
{
    const float floor_f = (float)ALPHA_FLOOR, cap_f = (float)ALPHA_CAP, stop_f = (float)T_STOP;
    float Tf = 1.0f;
    double T = 1.0, C[3] = {0, 0, 0}, Dp = 0.0, A = 0.0;
    int32_t last = -1, near = 0, nrec = 0;
    int64_t i;
    uint64_t h = 1469598103934665603ull;
    for (i = 0; i < n; ++i) {
        const orc_proj *P = &proj[list[i].g];
        /* decision, single precision */
        const float dxf = P->pf[0] - (float)qx, dyf = P->pf[1] - (float)qy;
        const float quad = fmaf(P->conicf[0], dxf * dxf, P->conicf[2] * (dyf * dyf));
        const float power = -0.5f * quad - P->conicf[1] * (dxf * dyf);
        if (power > 0.0f) continue;
        const float rawf = P->of * expf(power);
        if (rel_gap(rawf, cap_f) < opt->margin) near = 1;
        if (rel_gap(rawf, floor_f) < opt->margin) near = 1;
        const float alphaf = fminf(cap_f, rawf);
        if (alphaf < floor_f) continue;
        const float testf = Tf * (1.0f - alphaf);
        if (rel_gap(testf, stop_f) < opt->t_margin) near = 1;
        if (testf < stop_f) { h = fnv(h, (uint64_t)i | (1ull << 63)); break; }
        Tf = testf;
        /* value, double precision */
        const double dx = P->p[0] - qx, dy = P->p[1] - qy;
        const double pw = -0.5 * (P->conic[0] * dx * dx + P->conic[2] * dy * dy) - P->conic[1] * dx * dy;
        const double ep = exp(pw);
        const int capped = rawf > cap_f;
        const double alpha = capped ? ALPHA_CAP : P->o * ep;
        const double w = alpha * T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += w * P->color[ch];
        Dp += w * P->t[2];
        A += w;
        if (rec) {
            walk_rec *r = &rec[nrec];
            r->pos = (int32_t)i; r->g = list[i].g; r->alpha = alpha; r->T = T; r->ep = ep;
            r->dx = dx; r->dy = dy; r->capped = capped;
        }
        ++nrec;
        T *= 1.0 - alpha;
        last = (int32_t)i;
        h = fnv(h, (uint64_t)i);
    }
    for (int ch = 0; ch < 3; ++ch) out->rgb[ch] = C[ch] + T * opt->bg[ch];
    out->depth = Dp;
    out->alpha = A;
    out->T = T;
    out->n_contrib = last + 1;
    out->near = near;
    out->n_rec = nrec;
    out->end = (int32_t)i;
    out->hash = h;
}

int32_t orc_render(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                   const orc_opts *opt, orc_image *out)
{
    const int64_t nG = orc_num_gaussians(kfs, n_kf);
    orc_proj *proj = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)nG);
    for (int32_t k = 0; k < n_views; ++k) {
        const orc_cam *view = &views[k];
        const int32_t W = view->width, H = view->height;
        const int64_t hw = (int64_t)W * H;
        orc_project(kfs, n_kf, view, opt, proj);
        tile_lists L;
        build_lists(proj, nG, view, opt, &L);
        const int32_t nt = L.ntx * L.nty;
#pragma omp parallel for schedule(dynamic, 1)
        for (int32_t t = 0; t < nt; ++t) {
            const int32_t tx = t % L.ntx, ty = t / L.ntx;
            for (int32_t y = ty * opt->tile_h; y < (ty + 1) * opt->tile_h && y < H; ++y)
                for (int32_t x = tx * opt->tile_w; x < (tx + 1) * opt->tile_w && x < W; ++x) {
                    walk_out o;
                    walk_pixel(proj, L.e + L.off[t], L.off[t + 1] - L.off[t], x, y, opt, NULL, &o);
                    const int64_t pix = (int64_t)y * W + x;
                    for (int ch = 0; ch < 3; ++ch) out[k].rgb[ch * hw + pix] = o.rgb[ch];
                    out[k].depth[pix] = o.depth;
                    out[k].alpha[pix] = o.alpha;
                    out[k].t_final[pix] = o.T;
                    out[k].n_contrib[pix] = o.n_contrib;
                    out[k].near[pix] = (uint8_t)o.near;
                }
        }
        free_lists(&L);
    }
    free(proj);
    return 0;
}

int32_t orc_render_pixels(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                          const orc_opts *opt, int64_t n_px, const int32_t *px_view,
                          const int32_t *px_x, const int32_t *px_y, double *rgb, double *depth,
                          double *alpha, double *t_final, int32_t *n_contrib, uint8_t *near)
{
    const int64_t nG = orc_num_gaussians(kfs, n_kf);
    orc_proj *proj = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)nG);
    for (int32_t k = 0; k < n_views; ++k) {
        int any = 0;
        for (int64_t i = 0; i < n_px; ++i) any |= px_view[i] == k;
        if (!any) continue;
        const orc_cam *view = &views[k];
        orc_project(kfs, n_kf, view, opt, proj);
        tile_lists L;
        build_lists(proj, nG, view, opt, &L);
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < n_px; ++i) {
            if (px_view[i] != k) continue;
            const int32_t t = (px_y[i] / opt->tile_h) * L.ntx + px_x[i] / opt->tile_w;
            walk_out o;
            walk_pixel(proj, L.e + L.off[t], L.off[t + 1] - L.off[t], px_x[i], px_y[i], opt, NULL, &o);
            for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = o.rgb[ch];
            depth[i] = o.depth;
            alpha[i] = o.alpha;
            t_final[i] = o.T;
            n_contrib[i] = o.n_contrib;
            near[i] = (uint8_t)o.near;
        }
        free_lists(&L);
    }
    free(proj);
    return 0;
}

/* --------------------------------------------------------------------- adjoint */

/* 2D gradient slots of one (view, Gaussian) pair */
enum { G_PX, G_PY, G_A, G_B, G_C, G_O, G_Z, G_R, G_G, G_BL, G_N };

/* Reverse pass over one pixel's accepted entries (3DGS adjoint, with T taken from the
 * forward walk rather than recomputed). For entry i with S_X the front-to-back
 * composite of what lies behind it:
 *   dL/dalpha_i = T_i [(c_i - S_C).gC + (z_i - S_D) gD + (1 - S_A) gA]
 *                 - T_final / (1 - alpha_i) bg.gC
 *   dL/dc_i = alpha_i T_i gC,   dL/dz_i = alpha_i T_i gD,
 * and through alpha = o e^power (zero when capped) into o, the conic and the mean. */
static void pixel_adjoint(const orc_proj *proj, const walk_rec *rec, int32_t nrec, double T_final,
                          const double gC[3], double gD, double gA, const orc_opts *opt,
                          double (*acc)[G_N])
{
    double SC[3] = {0, 0, 0}, SD = 0.0, SA = 0.0;
    for (int32_t r = nrec - 1; r >= 0; --r) {
        const walk_rec *e = &rec[r];
        const orc_proj *P = &proj[e->g];
        const double a = e->alpha, T = e->T;
        double dal = 0.0;
        for (int ch = 0; ch < 3; ++ch) dal += (P->color[ch] - SC[ch]) * gC[ch];
        dal += (P->t[2] - SD) * gD + (1.0 - SA) * gA;
        dal *= T;
        double bgterm = 0.0;
        for (int ch = 0; ch < 3; ++ch) bgterm += opt->bg[ch] * gC[ch];
        dal -= T_final / (1.0 - a) * bgterm;
        double *g = acc[r];
        g[G_R] += a * T * gC[0];
        g[G_G] += a * T * gC[1];
        g[G_BL] += a * T * gC[2];
        g[G_Z] += a * T * gD;
        if (!e->capped) {
            const double G = dal * a;                 /* dL/dpower */
            g[G_O] += dal * e->ep;
            g[G_A] += -0.5 * G * e->dx * e->dx;
            g[G_B] += -G * e->dx * e->dy;
            g[G_C] += -0.5 * G * e->dy * e->dy;
            g[G_PX] += -G * (P->conic[0] * e->dx + P->conic[1] * e->dy);
            g[G_PY] += -G * (P->conic[1] * e->dx + P->conic[2] * e->dy);
        }
        for (int ch = 0; ch < 3; ++ch) SC[ch] = a * P->color[ch] + (1.0 - a) * SC[ch];
        SD = a * P->t[2] + (1.0 - a) * SD;
        SA = a + (1.0 - a) * SA;
    }
}

/* Chain the 2D gradients of one (view, Gaussian) pair down to the keyframe parameters:
 * conic -> Sigma_2D -> (s, J) -> t (with the mean and the depth) -> mu -> |D + delta|
 * -> delta; o -> logit. out = (d_offset, d_r, d_g, d_b, d_logit, d_scale). */
static void chain_params(const orc_kf *kf, int64_t j, const orc_cam *view, const orc_proj *P,
                         const double g[G_N], double out[6], double gt_out[3])
{
    const double fx = view->fx, fy = view->fy;
    const double tx = P->t[0], ty = P->t[1], tz = P->t[2];
    const double J00 = fx / tz, J02 = -fx * tx / (tz * tz);
    const double J11 = fy / tz, J12 = -fy * ty / (tz * tz);
    const double x = P->cov[0], y = P->cov[1], w = P->cov[2];
    const double det = x * w - y * y, det2 = det * det;
    const double ga = g[G_A], gb = g[G_B], gc = g[G_C];
    /* conic (a, b, c) = (w, -y, x) / det */
    const double gx = ga * (-w * w / det2) + gb * (y * w / det2) + gc * (-y * y / det2);
    const double gy = ga * (2.0 * y * w / det2) + gb * (-(det + 2.0 * y * y) / det2) + gc * (2.0 * x * y / det2);
    const double gw = ga * (-y * y / det2) + gb * (y * x / det2) + gc * (-x * x / det2);
    /* Sigma_2D = s^2 J J^T + 0.3 I */
    const double s = P->s, s2 = s * s;
    const double gs = 2.0 * s * ((J00 * J00 + J02 * J02) * gx + J02 * J12 * gy + (J11 * J11 + J12 * J12) * gw);
    const double gJ00 = 2.0 * s2 * J00 * gx;
    const double gJ02 = s2 * (2.0 * J02 * gx + J12 * gy);
    const double gJ11 = 2.0 * s2 * J11 * gw;
    const double gJ12 = s2 * (J02 * gy + 2.0 * J12 * gw);
    /* p = (fx tx/tz + cx, fy ty/tz + cy), J as above, composited depth z = tz */
    const double gtx = gJ02 * (-fx / (tz * tz)) + g[G_PX] * (fx / tz);
    const double gty = gJ12 * (-fy / (tz * tz)) + g[G_PY] * (fy / tz);
    const double gtz = gJ00 * (-fx / (tz * tz)) + gJ02 * (2.0 * fx * tx / (tz * tz * tz))
                     + gJ11 * (-fy / (tz * tz)) + gJ12 * (2.0 * fy * ty / (tz * tz * tz))
                     + g[G_PX] * (-fx * tx / (tz * tz)) + g[G_PY] * (-fy * ty / (tz * tz)) + g[G_Z];
    if (gt_out) {                 /* d loss / d t, the view-space centre */
        gt_out[0] = gtx;
        gt_out[1] = gty;
        gt_out[2] = gtz;
    }
    /* t = R_k mu + t_k */
    const double *V = view->pose;
    double gmu[3];
    for (int a = 0; a < 3; ++a) gmu[a] = V[a] * gtx + V[4 + a] * gty + V[8 + a] * gtz;
    /* mu = R_i (|D + delta| r) + t_i */
    const orc_cam *c = &kf->cam;
    const double u = (double)(j % c->width), v = (double)(j / c->width);
    const double r[3] = {(u - c->cx) / c->fx, (v - c->cy) / c->fy, 1.0};
    const double *M = c->pose;
    double gdt = 0.0;
    for (int a = 0; a < 3; ++a) gdt += (M[4 * a] * r[0] + M[4 * a + 1] * r[1] + M[4 * a + 2] * r[2]) * gmu[a];
    const double sum = kf->depth[j] + kf->offset[j];
    const double sgn = sum > 0.0 ? 1.0 : (sum < 0.0 ? -1.0 : 0.0);
    out[0] = sgn * gdt;
    out[1] = g[G_R];
    out[2] = g[G_G];
    out[3] = g[G_BL];
    out[4] = g[G_O] * P->o * (1.0 - P->o);
    out[5] = gs;
}

/* Walk the given tiles of one view and accumulate per-entry 2D gradients into g2d
 * (indexed by global Gaussian). Tiles are processed in parallel in chunks; each chunk's
 * per-entry contributions are merged in tile order, so the sum is deterministic. */
static void view_adjoint_tiles(const orc_kf *kfs, int32_t n_kf, const orc_proj *proj, const tile_lists *L,
                               const orc_cam *view, const orc_opts *opt, const orc_image_grads *gi,
                               const int32_t *tiles, int32_t n_tiles, const int64_t *slot, double (*g2d)[G_N],
                               double (*gabs)[6], uint8_t *near_out, double *pose_abs)
{
    const int32_t W = view->width, H = view->height;
    const int64_t hw = (int64_t)W * H;
    const int32_t chunk = 64;
    for (int32_t c0 = 0; c0 < n_tiles; c0 += chunk) {
        const int32_t c1 = c0 + chunk < n_tiles ? c0 + chunk : n_tiles;
        double (**acc)[G_N] = (double (**)[G_N])calloc((size_t)(c1 - c0), sizeof(*acc));
        double (**aacc)[6] = (double (**)[6])calloc((size_t)(c1 - c0), sizeof(*aacc));
        uint8_t **nacc = (uint8_t **)calloc((size_t)(c1 - c0), sizeof(*nacc));
        double (*pacc)[12] = pose_abs ? (double (*)[12])calloc((size_t)(c1 - c0), sizeof(*pacc)) : NULL;
#pragma omp parallel for schedule(dynamic, 1)
        for (int32_t ci = c0; ci < c1; ++ci) {
            const int32_t t = tiles[ci];
            const int64_t n = L->off[t + 1] - L->off[t];
            const list_entry *list = L->e + L->off[t];
            double (*a)[G_N] = (double (*)[G_N])calloc((size_t)(n + 1), sizeof(*a));
            double (*ab)[6] = gabs ? (double (*)[6])calloc((size_t)(n + 1), sizeof(*ab)) : NULL;
            double *pab = pacc ? pacc[ci - c0] : NULL;
            uint8_t *nf = (uint8_t *)calloc((size_t)(n + 1), 1);
            double (*pa)[G_N] = (double (*)[G_N])calloc((size_t)(n + 1), sizeof(*pa));
            walk_rec *rec = (walk_rec *)malloc(sizeof(walk_rec) * (size_t)(n + 1));
            const int32_t tx = t % L->ntx, ty = t / L->ntx;
            for (int32_t y = ty * opt->tile_h; y < (ty + 1) * opt->tile_h && y < H; ++y)
                for (int32_t x = tx * opt->tile_w; x < (tx + 1) * opt->tile_w && x < W; ++x) {
                    const int64_t pix = (int64_t)y * W + x;
                    walk_out o;
                    walk_pixel(proj, list, n, x, y, opt, rec, &o);
                    const double gC[3] = {gi->d_rgb[pix], gi->d_rgb[hw + pix], gi->d_rgb[2 * hw + pix]};
                    memset(pa, 0, sizeof(*pa) * (size_t)(o.n_rec + 1));
                    pixel_adjoint(proj, rec, o.n_rec, o.T, gC, gi->d_depth[pix], gi->d_alpha[pix], opt, pa);
                    for (int32_t r = 0; r < o.n_rec; ++r)
                        for (int q = 0; q < G_N; ++q) a[rec[r].pos][q] += pa[r][q];
                    if (ab || pab) {
                        /* magnitude of this pixel's contribution to each parameter gradient
                         * and to the view pose gradient */
                        for (int32_t r = 0; r < o.n_rec; ++r) {
                            int64_t j;
                            const int32_t ki = owner(kfs, n_kf, rec[r].g, &j);
                            double o6[6];
                            double gt[3];
                            chain_params(&kfs[ki], j, view, &proj[rec[r].g], pa[r], o6, gt);
                            if (ab)
                                for (int q = 0; q < 6; ++q) ab[rec[r].pos][q] += fabs(o6[q]);
                            if (pab) {
                                const double *mu = proj[rec[r].g].mu;
                                for (int c = 0; c < 3; ++c) {
                                    for (int b = 0; b < 3; ++b) pab[4 * c + b] += fabs(gt[c] * mu[b]);
                                    pab[4 * c + 3] += fabs(gt[c]);
                                }
                            }
                        }
                    }
                    if (o.near) {
                        /* entries up to the stop whose alpha is at or near the floor here */
                        const int64_t end = o.end < n ? o.end + 1 : n;
                        for (int64_t i = 0; i < end; ++i) {
                            const orc_proj *P = &proj[list[i].g];
                            const double dx = P->p[0] - x, dy = P->p[1] - y;
                            const double power =
                                -0.5 * (P->conic[0] * dx * dx + P->conic[2] * dy * dy) - P->conic[1] * dx * dy;
                            if (P->o * exp(power) >= ALPHA_FLOOR * (1.0 - opt->margin)) nf[i] = 1;
                        }
                    }
                }
            free(rec);
            free(pa);
            acc[ci - c0] = a;
            aacc[ci - c0] = ab;
            nacc[ci - c0] = nf;
        }
        for (int32_t ci = c0; ci < c1; ++ci) {
            const int32_t t = tiles[ci];
            const int64_t n = L->off[t + 1] - L->off[t];
            const list_entry *list = L->e + L->off[t];
            for (int64_t i = 0; i < n; ++i) {
                const int64_t s = slot ? slot[list[i].g] : (int64_t)list[i].g;
                if (s < 0) continue;
                for (int q = 0; q < G_N; ++q) g2d[s][q] += acc[ci - c0][i][q];
                if (gabs)
                    for (int q = 0; q < 6; ++q) gabs[s][q] += aacc[ci - c0][i][q];
                if (near_out && nacc[ci - c0][i]) near_out[s] = 1;
            }
            free(acc[ci - c0]);
            free(aacc[ci - c0]);
            free(nacc[ci - c0]);
            if (pacc)
                for (int q = 0; q < 12; ++q) pose_abs[q] += pacc[ci - c0][q];
        }
        free(pacc);
        free(acc);
        free(aacc);
        free(nacc);
    }
}

int32_t orc_backward(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                     const orc_opts *opt, const orc_image_grads *grad_in, orc_kf_grads *grads,
                     uint8_t *near_gauss, double *abs_out)
{
    double (*gabs)[6] = (double (*)[6])abs_out;
    if (gabs) memset(gabs, 0, sizeof(*gabs) * (size_t)orc_num_gaussians(kfs, n_kf));
    const int64_t nG = orc_num_gaussians(kfs, n_kf);
    orc_proj *proj = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)nG);
    double (*g2d)[G_N] = (double (*)[G_N])malloc(sizeof(*g2d) * (size_t)nG);
    double (*gp)[6] = (double (*)[6])calloc((size_t)nG, sizeof(*gp));
    if (near_gauss) memset(near_gauss, 0, (size_t)nG);
    for (int32_t k = 0; k < n_views; ++k) {
        orc_project(kfs, n_kf, &views[k], opt, proj);
        tile_lists L;
        build_lists(proj, nG, &views[k], opt, &L);
        const int32_t nt = L.ntx * L.nty;
        int32_t *tiles = (int32_t *)malloc(sizeof(int32_t) * (size_t)nt);
        for (int32_t t = 0; t < nt; ++t) tiles[t] = t;
        memset(g2d, 0, sizeof(*g2d) * (size_t)nG);
        view_adjoint_tiles(kfs, n_kf, proj, &L, &views[k], opt, &grad_in[k], tiles, nt, NULL, g2d, gabs, near_gauss,
                           NULL);
        for (int64_t g = 0; g < nG; ++g) {
            if (!(proj[g].ntiles > 0)) continue;
            int64_t j;
            const int32_t i = owner(kfs, n_kf, g, &j);
            double o6[6];
            chain_params(&kfs[i], j, &views[k], &proj[g], g2d[g], o6, NULL);
            for (int q = 0; q < 6; ++q) gp[g][q] += o6[q];
        }
        free(tiles);
        free_lists(&L);
    }
    int64_t base = 0;
    for (int32_t i = 0; i < n_kf; ++i) {
        const int64_t n = (int64_t)kfs[i].cam.width * kfs[i].cam.height;
        if (kfs[i].learnable) {
            for (int64_t j = 0; j < n; ++j) {
                const double *q = gp[base + j];
                grads[i].d_offset[j] = q[0];
                grads[i].d_rgb[j] = q[1];
                grads[i].d_rgb[n + j] = q[2];
                grads[i].d_rgb[2 * n + j] = q[3];
                grads[i].d_logit[j] = q[4];
                grads[i].d_scale[j] = q[5];
            }
        }
        base += n;
    }
    free(gp);
    free(g2d);
    free(proj);
    return 0;
}

int32_t orc_backward_pose(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                          const orc_opts *opt, const orc_image_grads *grad_in, double *d_pose, double *abs_pose)
{
    const int64_t nG = orc_num_gaussians(kfs, n_kf);
    orc_proj *proj = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)nG);
    double (*g2d)[G_N] = (double (*)[G_N])malloc(sizeof(*g2d) * (size_t)nG);
    for (int32_t k = 0; k < n_views; ++k) {
        double *dp = d_pose + 12 * (size_t)k;
        double *ap = abs_pose ? abs_pose + 12 * (size_t)k : NULL;
        memset(dp, 0, 12 * sizeof(double));
        if (ap) memset(ap, 0, 12 * sizeof(double));
        orc_project(kfs, n_kf, &views[k], opt, proj);
        tile_lists L;
        build_lists(proj, nG, &views[k], opt, &L);
        const int32_t nt = L.ntx * L.nty;
        int32_t *tiles = (int32_t *)malloc(sizeof(int32_t) * (size_t)nt);
        for (int32_t t = 0; t < nt; ++t) tiles[t] = t;
        memset(g2d, 0, sizeof(*g2d) * (size_t)nG);
        view_adjoint_tiles(kfs, n_kf, proj, &L, &views[k], opt, &grad_in[k], tiles, nt, NULL, g2d, NULL, NULL, ap);
        for (int64_t g = 0; g < nG; ++g) {
            if (!(proj[g].ntiles > 0)) continue;
            int64_t j;
            const int32_t i = owner(kfs, n_kf, g, &j);
            double o6[6], gt[3];
            chain_params(&kfs[i], j, &views[k], &proj[g], g2d[g], o6, gt);
            /* t = R mu + t_k: d t_a / d R_ab = mu_b, d t_a / d t_k,a = 1 */
            for (int a = 0; a < 3; ++a) {
                for (int b = 0; b < 3; ++b) dp[4 * a + b] += gt[a] * proj[g].mu[b];
                dp[4 * a + 3] += gt[a];
            }
        }
        free(tiles);
        free_lists(&L);
    }
    free(g2d);
    free(proj);
    return 0;
}

int32_t orc_backward_gaussians(const orc_kf *kfs, int32_t n_kf, const orc_cam *views,
                               int32_t n_views, const orc_opts *opt,
                               const orc_image_grads *grad_in, int64_t n_sel,
                               const int64_t *sel, double *out, uint8_t *near_sel, double *abs_sel)
{
    if (abs_sel) memset(abs_sel, 0, sizeof(double) * 6 * (size_t)n_sel);
    if (near_sel) memset(near_sel, 0, (size_t)n_sel);
    const int64_t nG = orc_num_gaussians(kfs, n_kf);
    orc_proj *proj = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)nG);
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)nG);
    for (int64_t g = 0; g < nG; ++g) slot[g] = -1;
    for (int64_t s = 0; s < n_sel; ++s) slot[sel[s]] = s;
    double (*g2d)[G_N] = (double (*)[G_N])malloc(sizeof(*g2d) * (size_t)(n_sel + 1));
    memset(out, 0, sizeof(double) * 6 * (size_t)n_sel);
    for (int32_t k = 0; k < n_views; ++k) {
        orc_project(kfs, n_kf, &views[k], opt, proj);
        tile_lists L;
        build_lists(proj, nG, &views[k], opt, &L);
        const int32_t nt = L.ntx * L.nty;
        uint8_t *want = (uint8_t *)calloc((size_t)nt, 1);
        for (int64_t s = 0; s < n_sel; ++s) {
            const orc_proj *P = &proj[sel[s]];
            if (P->ntiles <= 0) continue;
            for (int32_t ty = P->ty0; ty <= P->ty1; ++ty)
                for (int32_t tx = P->tx0; tx <= P->tx1; ++tx) want[ty * L.ntx + tx] = 1;
        }
        int32_t *tiles = (int32_t *)malloc(sizeof(int32_t) * (size_t)nt);
        int32_t nw = 0;
        for (int32_t t = 0; t < nt; ++t)
            if (want[t]) tiles[nw++] = t;
        memset(g2d, 0, sizeof(*g2d) * (size_t)(n_sel + 1));
        view_adjoint_tiles(kfs, n_kf, proj, &L, &views[k], opt, &grad_in[k], tiles, nw, slot, g2d,
                           (double (*)[6])abs_sel, near_sel, NULL);
        for (int64_t s = 0; s < n_sel; ++s) {
            const int64_t g = sel[s];
            if (!(proj[g].ntiles > 0)) continue;
            int64_t j;
            const int32_t i = owner(kfs, n_kf, g, &j);
            if (!kfs[i].learnable) continue;
            double o6[6];
            chain_params(&kfs[i], j, &views[k], &proj[g], g2d[s], o6, NULL);
            for (int q = 0; q < 6; ++q) out[6 * s + q] += o6[q];
        }
        free(tiles);
        free(want);
        free_lists(&L);
    }
    free(g2d);
    free(slot);
    free(proj);
    return 0;
}

uint64_t orc_decision_hash(const orc_kf *kfs, int32_t n_kf, const orc_cam *views, int32_t n_views,
                           const orc_opts *opt)
{
    const int64_t nG = orc_num_gaussians(kfs, n_kf);
    orc_proj *proj = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)nG);
    uint64_t h = 1469598103934665603ull;
    for (int32_t k = 0; k < n_views; ++k) {
        const orc_cam *view = &views[k];
        orc_project(kfs, n_kf, view, opt, proj);
        for (int64_t g = 0; g < nG; ++g) {
            const orc_proj *P = &proj[g];
            h = fnv(h, (uint64_t)(uint32_t)P->ntiles);
            h = fnv(h, ((uint64_t)(uint32_t)P->tx0 << 32) | (uint32_t)P->tx1);
            h = fnv(h, ((uint64_t)(uint32_t)P->ty0 << 32) | (uint32_t)P->ty1);
        }
        tile_lists L;
        build_lists(proj, nG, view, opt, &L);
        for (int64_t i = 0; i < L.off[L.ntx * L.nty]; ++i) h = fnv(h, L.e[i].g);
        for (int32_t t = 0; t < L.ntx * L.nty; ++t) {
            const int32_t tx = t % L.ntx, ty = t / L.ntx;
            for (int32_t y = ty * opt->tile_h; y < (ty + 1) * opt->tile_h && y < view->height; ++y)
                for (int32_t x = tx * opt->tile_w; x < (tx + 1) * opt->tile_w && x < view->width; ++x) {
                    walk_out o;
                    walk_pixel(proj, L.e + L.off[t], L.off[t + 1] - L.off[t], x, y, opt, NULL, &o);
                    h = fnv(h, o.hash);
                }
        }
        free_lists(&L);
    }
    free(proj);
    return h;
}

/* ---------------------------------------------------------------- loss and Adam */

/* Eq. 1 without the SSIM term (tau = 0): rho |V - V'|_1 + sigma U |D - D'|_1, with the
 * L1 norms taken as means (over pixels and channels; over valid-depth pixels). */
double orc_l1_loss(int32_t n_views, const orc_cam *views, const double *const *rgb,
                   const double *const *depth, const double *const *target_rgb,
                   const double *const *target_depth, double rgb_w, double depth_w,
                   double *const *d_rgb, double *const *d_depth)
{
    double loss = 0.0;
    for (int32_t k = 0; k < n_views; ++k) {
        const int64_t hw = (int64_t)views[k].width * views[k].height;
        const double nrgb = 3.0 * (double)hw;
        for (int64_t i = 0; i < 3 * hw; ++i) {
            const double d = rgb[k][i] - target_rgb[k][i];
            loss += rgb_w * fabs(d) / nrgb;
            d_rgb[k][i] = rgb_w * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / nrgb;
        }
        int64_t nvalid = 0;
        for (int64_t i = 0; i < hw; ++i) nvalid += target_depth[k][i] > 0.0;
        for (int64_t i = 0; i < hw; ++i) {
            d_depth[k][i] = 0.0;
            if (!(target_depth[k][i] > 0.0) || nvalid == 0 || depth_w == 0.0) continue;
            const double d = depth[k][i] - target_depth[k][i];
            loss += depth_w * fabs(d) / (double)nvalid;
            d_depth[k][i] = depth_w * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)nvalid;
        }
    }
    return loss;
}

/* m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
 * p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) */
void orc_adam(int64_t n, double *param, const double *grad, double *m, double *v, double lr,
              double beta1, double beta2, double eps, int32_t step, int32_t log_param)
{
    const double c1 = 1.0 - pow(beta1, step), c2 = 1.0 - pow(beta2, step);
    for (int64_t i = 0; i < n; ++i) {
        const double g = log_param ? grad[i] * param[i] : grad[i];
        m[i] = beta1 * m[i] + (1.0 - beta1) * g;
        v[i] = beta2 * v[i] + (1.0 - beta2) * g * g;
        const double p = log_param ? log(param[i]) : param[i];
        const double q = p - lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
        param[i] = log_param ? exp(q) : q;
    }
}
