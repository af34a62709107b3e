// C ABI entry points (include/sgad.h): argument checks, the workspace layout, and the
// launch sequence of each call. No device memory is allocated here.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "sgad_device.cuh"

namespace sgad {
void launch_project_count(const Scene &, World *, uint32_t *, uint2 *, cudaStream_t);
void launch_scan_tiles(uint32_t *, uint32_t *, int, uint64_t, WsHeader *, uint32_t *, cudaStream_t);
void launch_emit(const Scene &, const uint2 *, const uint32_t *, uint32_t *, uint64_t *, WsHeader *, cudaStream_t);
cudaError_t launch_sort_tiles(const uint32_t *, uint64_t *, uint64_t *, int, int, WsHeader *, uint32_t *, cudaStream_t);
cudaError_t launch_composite(bool, int, int, int, const Scene &, const World *, const uint32_t *, const uint64_t *,
                             float *, uint32_t *, float4 *, WsHeader *, const uint32_t *, uint32_t *, uint32_t *,
                             cudaStream_t);
bool valid_batch(int, bool);
void launch_finalize(const Scene &, const World *, const float4 *, cudaStream_t);
void launch_l1_batch(int, const float *const *, const float *const *, const float *const *, const float *const *,
                     const float *const *, float *const *, float *const *, uint32_t *, const uint32_t *, float, float,
                     float, float *, cudaStream_t);
cudaError_t launch_pose_adam_step(const float *, const float *, float *, float, float, float, float, float,
                                  cudaStream_t);
void launch_adam(int64_t, float *, const float *, float *, float *, float, float, float, float, float, float, bool,
                 cudaStream_t);
cudaError_t launch_adam_multi(int, const sgad_adam_tensor *, float, float, float, int32_t *, cudaStream_t);
}  // namespace sgad

using namespace sgad;

struct sgad_ctx {
    sgad_options opt;
    int sort_cap;
    // per-stage events: [0..4] forward boundaries, [5..7] backward boundaries
    bool profile = false;
    bool fwd_recorded = false, bwd_recorded = false;
    cudaEvent_t ev[8] = {};
};

namespace {
inline void mark(sgad_ctx *ctx, int i, cudaStream_t st)
{
    if (ctx->profile) cudaEventRecord(ctx->ev[i], st);
}
}  // namespace

namespace {

thread_local char g_err[512] = "";

sgad_status fail(sgad_status code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

sgad_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(SGAD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

namespace sgad {
// Records the message returned by sgad_last_error() for entry points in other files.
sgad_status report_error(sgad_status code, const char *msg)
{
    return fail(code, "%s", msg);
}
}  // namespace sgad

namespace {

int ilog2_exact(int x)
{
    int l = 0;
    while ((1 << l) < x) ++l;
    return (1 << l) == x ? l : -1;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

bool valid_camera(const sgad_camera &c)
{
    if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384) return false;
    if (!finite_pos(c.fx) || !finite_pos(c.fy) || !std::isfinite(c.cx) || !std::isfinite(c.cy)) return false;
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(c.pose[i])) return false;
    return true;
}

void set_cam(const sgad_camera &c, float &fx, float &fy, float &cx, float &cy, float *R, float *t)
{
    fx = c.fx;
    fy = c.fy;
    cx = c.cx;
    cy = c.cy;
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) R[3 * r + q] = c.pose[4 * r + q];
        t[r] = c.pose[4 * r + 3];
    }
}

// Fills the launch parameters; checks shapes. Pointers are checked by the callers
// according to what each call reads and writes.
sgad_status build_scene(const sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf, const sgad_camera *views,
                        int32_t n_views, Scene &sc, uint64_t &n_pix)
{
    if (!ctx) return fail(SGAD_ERR_INVALID_ARG, "ctx is NULL");
    if (!kfs || n_kf < 1 || n_kf > SGAD_MAX_KEYFRAMES)
        return fail(SGAD_ERR_INVALID_ARG, "n_kf must be in [1, %d] with kfs non-NULL", SGAD_MAX_KEYFRAMES);
    if (!views || n_views < 1 || n_views > SGAD_MAX_VIEWS)
        return fail(SGAD_ERR_INVALID_ARG, "n_views must be in [1, %d] with views non-NULL", SGAD_MAX_VIEWS);
    std::memset(&sc, 0, sizeof(sc));
    sc.n_kf = n_kf;
    sc.n_views = n_views;
    sc.tile_w = ctx->opt.tile_w;
    sc.tile_h = ctx->opt.tile_h;
    sc.tw_log2 = ilog2_exact(sc.tile_w);
    sc.th_log2 = ilog2_exact(sc.tile_h);
    for (int c = 0; c < 3; ++c) sc.bg[c] = ctx->opt.bg[c];
    sc.freeze_offset = ctx->opt.freeze_offset;
    uint64_t ng = 0;
    for (int i = 0; i < n_kf; ++i) {
        const sgad_keyframe &k = kfs[i];
        if (!valid_camera(k.cam)) return fail(SGAD_ERR_INVALID_ARG, "keyframe %d: invalid camera", i);
        KfDev &d = sc.kf[i];
        d.depth = k.depth;
        d.offset = k.offset;
        d.rgb = k.rgb;
        d.logit = k.opacity_logit;
        d.scale = k.scale;
        d.xform = k.world_transform;
        if (k.world_transform && k.learnable)
            return fail(SGAD_ERR_INVALID_ARG, "keyframe %d: a world transform is only allowed on a fixed keyframe", i);
        set_cam(k.cam, d.fx, d.fy, d.cx, d.cy, d.R, d.t);
        d.W = k.cam.width;
        d.H = k.cam.height;
        d.gbase = (uint32_t)ng;
        d.learnable = k.learnable ? 1 : 0;
        ng += (uint64_t)k.cam.width * k.cam.height;
        if (ng >= 0xffffffffull) return fail(SGAD_ERR_INVALID_ARG, "more than 2^32 - 1 Gaussians");
    }
    sc.n_gauss = (uint32_t)ng;
    uint64_t nt = 0;
    n_pix = 0;
    for (int i = 0; i < n_views; ++i) {
        if (!valid_camera(views[i])) return fail(SGAD_ERR_INVALID_ARG, "view %d: invalid camera", i);
        ViewDev &v = sc.view[i];
        set_cam(views[i], v.fx, v.fy, v.cx, v.cy, v.R, v.t);
        v.W = views[i].width;
        v.H = views[i].height;
        v.tiles_x = (v.W + sc.tile_w - 1) / sc.tile_w;
        v.tiles_y = (v.H + sc.tile_h - 1) / sc.tile_h;
        v.tile_base = (int32_t)nt;
        v.pix_base = (uint32_t)n_pix;
        nt += (uint64_t)v.tiles_x * v.tiles_y;
        n_pix += (uint64_t)v.W * v.H;
        if (nt >= (1ull << 30) || n_pix >= 0xffffffffull) return fail(SGAD_ERR_INVALID_ARG, "too many pixels");
    }
    sc.n_tiles = (int32_t)nt;
    return SGAD_OK;
}

struct Ws {
    Layout L;
    char *base;
    WsHeader *hdr() const { return reinterpret_cast<WsHeader *>(base + L.header); }
    World *world() const { return reinterpret_cast<World *>(base + L.world); }
    float4 *gacc() const { return reinterpret_cast<float4 *>(base + L.gacc); }
    uint2 *rects() const { return reinterpret_cast<uint2 *>(base + L.rects); }
    uint32_t *tile_off() const { return reinterpret_cast<uint32_t *>(base + L.tile_off); }
    uint32_t *tile_cnt() const { return reinterpret_cast<uint32_t *>(base + L.tile_cnt); }
    uint32_t *tile_order() const { return reinterpret_cast<uint32_t *>(base + L.tile_order); }
    uint32_t *sort_list() const { return reinterpret_cast<uint32_t *>(base + L.sort_list); }
    float *pix_t() const { return reinterpret_cast<float *>(base + L.pix_t); }
    uint32_t *pix_n() const { return reinterpret_cast<uint32_t *>(base + L.pix_n); }
    uint64_t *keys() const { return reinterpret_cast<uint64_t *>(base + L.keys); }
    uint64_t *keys_alt() const { return reinterpret_cast<uint64_t *>(base + L.keys_alt); }
    uint32_t *contrib() const { return reinterpret_cast<uint32_t *>(base + L.contrib); }
    uint32_t *wmask() const { return reinterpret_cast<uint32_t *>(base + L.wmask); }
};

sgad_status get_ws(const Scene &sc, uint64_t n_pix, void *workspace, size_t ws_bytes, int64_t key_cap, Ws &ws)
{
    if (key_cap < 0 || key_cap >= 0xffffffffll) return fail(SGAD_ERR_INVALID_ARG, "key_capacity out of range");
    ws.L = make_layout(sc.n_gauss, (uint64_t)sc.n_views, (uint64_t)sc.n_tiles, n_pix, (uint64_t)key_cap);
    if (!workspace) return fail(SGAD_ERR_INVALID_ARG, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(SGAD_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < ws.L.total)
        return fail(SGAD_ERR_WORKSPACE_TOO_SMALL, "workspace holds %zu bytes, %zu needed", ws_bytes, ws.L.total);
    ws.base = static_cast<char *>(workspace);
    return SGAD_OK;
}

sgad_status check_kf_inputs(const sgad_keyframe *kfs, int n_kf)
{
    for (int i = 0; i < n_kf; ++i)
        if (!kfs[i].depth || !kfs[i].offset || !kfs[i].rgb || !kfs[i].opacity_logit || !kfs[i].scale)
            return fail(SGAD_ERR_INVALID_ARG, "keyframe %d: a parameter plane is NULL", i);
    return SGAD_OK;
}

sgad_status last_launch(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SGAD_OK : cuda_fail(e, what);
}

bool uses_order(const sgad_options &o)
{
    return o.fwd_schedule == SGAD_SCHEDULE_PERSISTENT || o.bwd_schedule == SGAD_SCHEDULE_PERSISTENT;
}

// Projection, binning count and scan: the part shared by sgad_count_keys and sgad_forward.
sgad_status run_binning_count(const sgad_options &o, const Scene &sc, const Ws &ws, int64_t key_cap,
                              bool clear_sticky, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(ws.hdr(), 0, clear_sticky ? sizeof(WsHeader) : kHeaderPerCall, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.tile_cnt(), 0, ((size_t)sc.n_tiles + 1) * 4, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    launch_project_count(sc, ws.world(), ws.tile_cnt(), ws.rects(), st);
    launch_scan_tiles(ws.tile_cnt(), ws.tile_off(), sc.n_tiles, (uint64_t)key_cap, ws.hdr(),
                      uses_order(o) ? ws.tile_order() : nullptr, st);
    return last_launch("binning");
}

// Forward steps before compositing: binning count and scan, key emission, per-tile sort.
sgad_status run_forward_prep(sgad_ctx *ctx, const Scene &sc, const Ws &ws, int64_t key_cap, cudaStream_t st)
{
    mark(ctx, 0, st);
    sgad_status s = run_binning_count(ctx->opt, sc, ws, key_cap, false, st);
    if (s) return s;
    mark(ctx, 1, st);
    launch_emit(sc, ws.rects(), ws.tile_off(), ws.tile_cnt(), ws.keys(), ws.hdr(), st);
    mark(ctx, 2, st);
    cudaError_t e = launch_sort_tiles(ws.tile_off(), ws.keys(), ws.keys_alt(), sc.n_tiles, ctx->sort_cap, ws.hdr(),
                                      ws.sort_list(), st);
    if (e != cudaSuccess) return cuda_fail(e, "sort launch");
    mark(ctx, 3, st);
    return last_launch("binning / emission / sort");
}

// One compositing pass. batch 0 in the backward selects the pair-parallel kernel; the
// forward records contribution words when the context's backward is pair-parallel.
sgad_status run_composite(const sgad_ctx *ctx, bool fwd, int batch, int schedule, const Scene &sc, const Ws &ws,
                          cudaStream_t st)
{
    uint32_t *contrib = (!fwd || ctx->opt.bwd_algorithm == SGAD_BWD_PAIRS) ? ws.contrib() : nullptr;
    const cudaError_t e = launch_composite(fwd, batch, schedule, ctx->opt.max_blocks, sc, ws.world(), ws.tile_off(), ws.keys(), ws.pix_t(),
                                           ws.pix_n(), fwd ? nullptr : ws.gacc(), ws.hdr(), ws.tile_order(), contrib,
                                           ws.wmask(), st);
    return e == cudaSuccess ? SGAD_OK : cuda_fail(e, fwd ? "forward compositing launch" : "backward compositing launch");
}

// The batch argument of the backward launch: 0 selects the pair-parallel kernel, a
// negative value the warp-local one.
int bwd_batch_of(const sgad_options &o)
{
    if (o.bwd_algorithm == SGAD_BWD_PAIRS) return 0;
    if (o.bwd_algorithm == SGAD_BWD_WARP_LOCAL) return -1;
    return o.bwd_batch;
}

// Output images of sgad_forward into the launch parameters.
sgad_status bind_images(Scene &sc, const sgad_images *out, int n_views)
{
    if (!out) return fail(SGAD_ERR_INVALID_ARG, "out is NULL");
    for (int i = 0; i < n_views; ++i) {
        if (!out[i].rgb || !out[i].depth || !out[i].alpha)
            return fail(SGAD_ERR_INVALID_ARG, "view %d: an output image is NULL", i);
        sc.view[i].rgb = out[i].rgb;
        sc.view[i].depth = out[i].depth;
        sc.view[i].alpha = out[i].alpha;
    }
    return SGAD_OK;
}

// Image gradients in and keyframe gradients out of sgad_backward into the launch parameters.
sgad_status bind_grads(Scene &sc, const sgad_image_grads *grad_in, sgad_keyframe_grads *grads_out, int n_kf,
                       int n_views)
{
    if (!grad_in || !grads_out) return fail(SGAD_ERR_INVALID_ARG, "grad_in / grads_out is NULL");
    for (int i = 0; i < n_views; ++i) {
        sc.view[i].g_rgb = grad_in[i].d_rgb;
        sc.view[i].g_depth = grad_in[i].d_depth;
        sc.view[i].g_alpha = grad_in[i].d_alpha;
        sc.view[i].d_pose = grad_in[i].d_pose;
    }
    for (int i = 0; i < n_kf; ++i) {
        KfDev &d = sc.kf[i];
        d.d_offset = grads_out[i].d_offset;
        d.d_rgb = grads_out[i].d_rgb;
        d.d_logit = grads_out[i].d_opacity_logit;
        d.d_scale = grads_out[i].d_scale;
        if (d.learnable && (!d.d_offset || !d.d_rgb || !d.d_logit || !d.d_scale))
            return fail(SGAD_ERR_INVALID_ARG, "keyframe %d is learnable but a gradient plane is NULL", i);
    }
    return SGAD_OK;
}


// Event pair for the autotuner: times `reps` runs of a launch sequence after one warm-up
// and returns the median in milliseconds.
struct TuneTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~TuneTimer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    cudaError_t init()
    {
        cudaError_t e = cudaEventCreate(&a);
        return e == cudaSuccess ? cudaEventCreate(&b) : e;
    }
    template <class F>
    sgad_status median(int reps, cudaStream_t st, F &&run, float *ms)
    {
        float t[101];
        for (int r = 0; r <= reps; ++r) {
            cudaError_t e = cudaEventRecord(a, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
            const sgad_status s = run();
            if (s) return s;
            e = cudaEventRecord(b, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            if (e == cudaSuccess && r > 0) e = cudaEventElapsedTime(&t[r - 1], a, b);
            if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
        }
        for (int i = 1; i < reps; ++i)      // insertion sort of at most 100 values
            for (int j = i; j > 0 && t[j] < t[j - 1]; --j) {
                const float x = t[j];
                t[j] = t[j - 1];
                t[j - 1] = x;
            }
        *ms = t[reps / 2];
        return SGAD_OK;
    }
};

struct TuneLog {
    sgad_tune_entry *rows;
    int max_rows, n = 0;
    void add(int tw, int th, int stage, int batch, int sched, float ms)
    {
        if (rows && n < max_rows) rows[n] = sgad_tune_entry{tw, th, stage, batch, sched, ms};
        if (rows && n < max_rows) ++n;
    }
};

}  // namespace

extern "C" {

sgad_status sgad_default_options(sgad_options *opt)
{
    if (!opt) return fail(SGAD_ERR_INVALID_ARG, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->tile_w = 16;
    opt->tile_h = 16;
    opt->sort_smem_cap = 0;
    opt->freeze_offset = 0;
    opt->fwd_batch = 512;
    opt->bwd_batch = 256;
    opt->fwd_schedule = SGAD_SCHEDULE_TILES;
    opt->bwd_schedule = SGAD_SCHEDULE_TILES;
    opt->bwd_algorithm = SGAD_BWD_WARP_LOCAL;
    return SGAD_OK;
}

sgad_status sgad_get_options(const sgad_ctx *ctx, sgad_options *opt)
{
    if (!ctx || !opt) return fail(SGAD_ERR_INVALID_ARG, "ctx / opt is NULL");
    *opt = ctx->opt;
    return SGAD_OK;
}

sgad_status sgad_create(sgad_ctx **out, const sgad_options *opt)
{
    if (!out) return fail(SGAD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    sgad_options o;
    if (opt)
        o = *opt;
    else
        sgad_default_options(&o);
    const bool shape_ok = (o.tile_w == 16 && o.tile_h == 16) || (o.tile_w == 8 && o.tile_h == 32) ||
                          (o.tile_w == 32 && o.tile_h == 8);
    if (!shape_ok) return fail(SGAD_ERR_UNSUPPORTED, "tile shape %dx%d not supported", o.tile_w, o.tile_h);
    for (int i = 0; i < 2; ++i)
        if (o.reserved[i] != 0) return fail(SGAD_ERR_INVALID_ARG, "reserved options must be zero");
    if (o.max_blocks < 0) return fail(SGAD_ERR_INVALID_ARG, "max_blocks must be >= 0");
    if (o.bwd_algorithm != SGAD_BWD_PAIRS && o.bwd_algorithm != SGAD_BWD_WARP_REDUCE &&
        o.bwd_algorithm != SGAD_BWD_WARP_LOCAL)
        return fail(SGAD_ERR_INVALID_ARG, "unknown backward algorithm %d", o.bwd_algorithm);
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(o.bg[c])) return fail(SGAD_ERR_INVALID_ARG, "background must be finite");
    if (o.fwd_batch == 0) o.fwd_batch = 512;
    if (o.bwd_batch == 0) o.bwd_batch = 256;
    if (!valid_batch(o.fwd_batch, true) || !valid_batch(o.bwd_batch, false))
        return fail(SGAD_ERR_UNSUPPORTED,
                    "batch sizes must be 128, 192, 256, 384 or 512 (forward also 768 or 1024)");
    for (int sch : {o.fwd_schedule, o.bwd_schedule})
        if (sch != SGAD_SCHEDULE_TILES && sch != SGAD_SCHEDULE_PERSISTENT && sch != SGAD_SCHEDULE_PER_VIEW)
            return fail(SGAD_ERR_INVALID_ARG, "unknown schedule %d", sch);
    const int cap = o.sort_smem_cap == 0 ? 6144 : o.sort_smem_cap;
    if (cap < 64 || cap > 12288) return fail(SGAD_ERR_INVALID_ARG, "sort_smem_cap must be in [64, 12288]");
    sgad_ctx *c = new (std::nothrow) sgad_ctx;
    if (!c) return fail(SGAD_ERR_INVALID_ARG, "out of host memory");
    c->opt = o;
    c->sort_cap = cap;
    *out = c;
    return SGAD_OK;
}

void sgad_destroy(sgad_ctx *ctx)
{
    if (!ctx) return;
    for (cudaEvent_t &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
}

sgad_status sgad_profile_enable(sgad_ctx *ctx, int32_t enable)
{
    if (!ctx) return fail(SGAD_ERR_INVALID_ARG, "ctx is NULL");
    if (enable && !ctx->ev[0]) {
        for (cudaEvent_t &e : ctx->ev) {
            const cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(r, "cudaEventCreate");
        }
    }
    ctx->profile = enable != 0;
    ctx->fwd_recorded = ctx->bwd_recorded = false;
    return SGAD_OK;
}

sgad_status sgad_profile_read(sgad_ctx *ctx, float *ms)
{
    if (!ctx || !ms) return fail(SGAD_ERR_INVALID_ARG, "bad arguments to sgad_profile_read");
    for (int i = 0; i < SGAD_NUM_STAGES; ++i) ms[i] = 0.0f;
    if (ctx->fwd_recorded) {
        cudaError_t r = cudaEventSynchronize(ctx->ev[4]);
        for (int i = 0; i < 4 && r == cudaSuccess; ++i) r = cudaEventElapsedTime(&ms[i], ctx->ev[i], ctx->ev[i + 1]);
        if (r != cudaSuccess) return cuda_fail(r, "sgad_profile_read");
    }
    if (ctx->bwd_recorded) {
        cudaError_t r = cudaEventSynchronize(ctx->ev[7]);
        if (r == cudaSuccess) r = cudaEventElapsedTime(&ms[4], ctx->ev[5], ctx->ev[6]);
        if (r == cudaSuccess) r = cudaEventElapsedTime(&ms[5], ctx->ev[6], ctx->ev[7]);
        if (r != cudaSuccess) return cuda_fail(r, "sgad_profile_read");
    }
    return SGAD_OK;
}

sgad_status sgad_read_stats(sgad_ctx *ctx, void *workspace, size_t ws_bytes, sgad_stats *out, void *stream)
{
    if (!ctx || !workspace || !out || ws_bytes < sizeof(WsHeader)) return fail(SGAD_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WsHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "sgad_read_stats");
    out->n_keys = h.n_keys;
    out->keys_needed = h.needed;
    out->n_pairs = (int64_t)h.n_pairs;
    out->n_evals = (int64_t)h.n_evals;
    out->n_sort_exact = h.n_sort_exact;
    return SGAD_OK;
}

const char *sgad_last_error(void) { return g_err; }

sgad_status sgad_workspace_size(const sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                                const sgad_camera *views, int32_t n_views, int64_t key_capacity, size_t *bytes)
{
    if (!bytes) return fail(SGAD_ERR_INVALID_ARG, "bytes is NULL");
    Scene sc;
    uint64_t n_pix;
    sgad_status s = build_scene(ctx, kfs, n_kf, views, n_views, sc, n_pix);
    if (s) return s;
    if (key_capacity < 0 || key_capacity >= 0xffffffffll)
        return fail(SGAD_ERR_INVALID_ARG, "key_capacity out of range");
    *bytes = make_layout(sc.n_gauss, (uint64_t)sc.n_views, (uint64_t)sc.n_tiles, n_pix, (uint64_t)key_capacity).total;
    return SGAD_OK;
}

sgad_status sgad_count_keys(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf, const sgad_camera *views,
                            int32_t n_views, void *workspace, size_t ws_bytes, int64_t *n_keys, void *stream)
{
    if (!n_keys) return fail(SGAD_ERR_INVALID_ARG, "n_keys is NULL");
    Scene sc;
    uint64_t n_pix;
    Ws ws;
    sgad_status s = build_scene(ctx, kfs, n_kf, views, n_views, sc, n_pix);
    if (!s) s = check_kf_inputs(kfs, n_kf);
    if (!s) s = get_ws(sc, n_pix, workspace, ws_bytes, 0, ws);
    if (s) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = run_binning_count(ctx->opt, sc, ws, 0xfffffffell, true, st);
    if (s) return s;
    WsHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, ws.hdr(), sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "sgad_count_keys");
    *n_keys = (int64_t)h.needed;
    return SGAD_OK;
}

sgad_status sgad_forward(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf, const sgad_camera *views,
                         int32_t n_views, sgad_images *out, void *workspace, size_t ws_bytes, int64_t key_capacity,
                         void *stream)
{
    Scene sc;
    uint64_t n_pix;
    Ws ws;
    sgad_status s = build_scene(ctx, kfs, n_kf, views, n_views, sc, n_pix);
    if (!s) s = check_kf_inputs(kfs, n_kf);
    if (!s) s = get_ws(sc, n_pix, workspace, ws_bytes, key_capacity, ws);
    if (!s) s = bind_images(sc, out, n_views);
    if (s) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = run_forward_prep(ctx, sc, ws, key_capacity, st);
    if (!s) s = run_composite(ctx, true, ctx->opt.fwd_batch, ctx->opt.fwd_schedule, sc, ws, st);
    if (s) return s;
    mark(ctx, 4, st);
    ctx->fwd_recorded = ctx->profile;
    return last_launch("sgad_forward");
}

sgad_status sgad_backward(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf, const sgad_camera *views,
                          int32_t n_views, const sgad_image_grads *grad_in, sgad_keyframe_grads *grads_out,
                          void *workspace, size_t ws_bytes, int64_t key_capacity, void *stream)
{
    Scene sc;
    uint64_t n_pix;
    Ws ws;
    sgad_status s = build_scene(ctx, kfs, n_kf, views, n_views, sc, n_pix);
    if (!s) s = check_kf_inputs(kfs, n_kf);
    if (!s) s = get_ws(sc, n_pix, workspace, ws_bytes, key_capacity, ws);
    if (!s) s = bind_grads(sc, grad_in, grads_out, n_kf, n_views);
    if (s) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mark(ctx, 5, st);
    cudaError_t e = cudaMemsetAsync(ws.gacc(), 0, (size_t)sc.n_gauss * 32, st);
    for (int i = 0; i < n_views && e == cudaSuccess; ++i)
        if (sc.view[i].d_pose) e = cudaMemsetAsync(sc.view[i].d_pose, 0, 12 * sizeof(float), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    s = run_composite(ctx, false, bwd_batch_of(ctx->opt), ctx->opt.bwd_schedule, sc, ws, st);
    if (s) return s;
    mark(ctx, 6, st);
    launch_finalize(sc, ws.world(), ws.gacc(), st);
    mark(ctx, 7, st);
    ctx->bwd_recorded = ctx->profile;
    return last_launch("sgad_backward");
}

sgad_status sgad_check(sgad_ctx *ctx, void *workspace, size_t ws_bytes, int64_t *n_keys, int64_t *keys_needed,
                       void *stream)
{
    if (!ctx || !workspace || ws_bytes < sizeof(WsHeader)) return fail(SGAD_ERR_INVALID_ARG, "bad workspace");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WsHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "sgad_check");
    if (n_keys) *n_keys = h.n_keys;
    const uint32_t need = h.sticky_needed > h.needed ? h.sticky_needed : h.needed;
    if (keys_needed) *keys_needed = need;
    if (h.sticky_err != 0 || h.sticky_overrun != 0) {
        e = cudaMemsetAsync(reinterpret_cast<char *>(workspace) + kHeaderPerCall, 0, sizeof(WsHeader) - kHeaderPerCall,
                            st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "sgad_check");
        if (h.sticky_overrun) return fail(SGAD_ERR_CUDA, "internal: binning count and key emission disagree");
        if (h.sticky_err == SGAD_ERR_KEY_OVERFLOW)
            return fail(SGAD_ERR_KEY_OVERFLOW, "a forward needed %u keys, more than the workspace capacity", need);
        return fail(h.sticky_err, "device reported error %d", h.sticky_err);
    }
    return SGAD_OK;
}

sgad_status sgad_state(const sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf, const sgad_camera *views,
                       int32_t n_views, void *workspace, size_t ws_bytes, int64_t key_capacity, sgad_state_view *out)
{
    if (!out) return fail(SGAD_ERR_INVALID_ARG, "out is NULL");
    Scene sc;
    uint64_t n_pix;
    Ws ws;
    sgad_status s = build_scene(ctx, kfs, n_kf, views, n_views, sc, n_pix);
    if (!s) s = get_ws(sc, n_pix, workspace, ws_bytes, key_capacity, ws);
    if (s) return s;
    out->tile_offsets = ws.tile_off();
    out->entries = ws.keys();
    out->t_final = ws.pix_t();
    out->n_contrib = ws.pix_n();
    out->n_tiles = sc.n_tiles;
    out->n_pixels = (int64_t)n_pix;
    return SGAD_OK;
}

sgad_status sgad_l1_loss_grad(int32_t n_views, const sgad_camera *views, const sgad_images *rendered,
                              const float *const *target_rgb, const float *const *target_depth, float rgb_weight,
                              float depth_weight, float min_alpha, float *const *d_rgb, float *const *d_depth,
                              float *loss_accum, uint32_t *valid_count, void *stream)
{
    if (n_views < 1 || !views || !rendered || !target_rgb || !d_rgb)
        return fail(SGAD_ERR_INVALID_ARG, "bad arguments to sgad_l1_loss_grad");
    if (!std::isfinite(rgb_weight) || !std::isfinite(depth_weight))
        return fail(SGAD_ERR_INVALID_ARG, "loss weights must be finite");
    const bool use_depth = depth_weight != 0.0f;
    if (use_depth && (!target_depth || !d_depth || !valid_count))
        return fail(SGAD_ERR_INVALID_ARG, "depth term needs target_depth, d_depth and valid_count");
    if (n_views > SGAD_MAX_VIEWS) return fail(SGAD_ERR_INVALID_ARG, "too many views");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!std::isfinite(min_alpha)) return fail(SGAD_ERR_INVALID_ARG, "min_alpha must be finite");
    const bool mask = min_alpha >= 0.0f;
    const float *rgb[SGAD_MAX_VIEWS], *dep[SGAD_MAX_VIEWS], *alp[SGAD_MAX_VIEWS];
    uint32_t hw[SGAD_MAX_VIEWS];
    for (int i = 0; i < n_views; ++i) {
        if (!valid_camera(views[i])) return fail(SGAD_ERR_INVALID_ARG, "view %d: invalid camera", i);
        if (!rendered[i].rgb || !target_rgb[i] || !d_rgb[i] || (use_depth && (!rendered[i].depth || !target_depth[i])))
            return fail(SGAD_ERR_INVALID_ARG, "view %d: NULL image", i);
        if (mask && !rendered[i].alpha) return fail(SGAD_ERR_INVALID_ARG, "view %d: NULL alpha image", i);
        rgb[i] = rendered[i].rgb;
        dep[i] = rendered[i].depth;
        alp[i] = rendered[i].alpha;
        hw[i] = (uint32_t)views[i].width * (uint32_t)views[i].height;
    }
    if (use_depth) {
        cudaError_t e = cudaMemsetAsync(valid_count, 0, sizeof(uint32_t) * (size_t)n_views, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    launch_l1_batch(n_views, rgb, dep, mask ? alp : nullptr, target_rgb, use_depth ? target_depth : nullptr, d_rgb,
                    d_depth, use_depth ? valid_count : nullptr, hw, rgb_weight, depth_weight, min_alpha, loss_accum,
                    st);
    return last_launch("sgad_l1_loss_grad");
}

sgad_status sgad_pose_adam_step(const float *d_pose, const float *view_pose, float *state, float lr_rot,
                                float lr_trans, float beta1, float beta2, float eps, void *stream)
{
    if (!d_pose || !view_pose || !state) return fail(SGAD_ERR_INVALID_ARG, "NULL argument to sgad_pose_adam_step");
    if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f) ||
        !std::isfinite(lr_rot) || !std::isfinite(lr_trans))
        return fail(SGAD_ERR_INVALID_ARG, "bad hyper-parameters in sgad_pose_adam_step");
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(view_pose[i])) return fail(SGAD_ERR_INVALID_ARG, "view_pose must be finite");
    const cudaError_t e = launch_pose_adam_step(d_pose, view_pose, state, lr_rot, lr_trans, beta1, beta2, eps,
                                                static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SGAD_OK : cuda_fail(e, "sgad_pose_adam_step");
}

sgad_status sgad_adam_step(int64_t n, float *param, const float *grad, float *m, float *v, float lr, float beta1,
                           float beta2, float eps, int32_t step, int32_t mode, void *stream)
{
    if (n < 0 || (n > 0 && (!param || !grad || !m || !v)) || step < 1)
        return fail(SGAD_ERR_INVALID_ARG, "bad arguments to sgad_adam_step");
    if (mode != SGAD_ADAM_PLAIN && mode != SGAD_ADAM_LOG) return fail(SGAD_ERR_INVALID_ARG, "unknown Adam mode");
    if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !std::isfinite(lr) || !(eps >= 0.0f))
        return fail(SGAD_ERR_INVALID_ARG, "bad Adam hyper-parameters");
    const float c1 = (float)(1.0 - std::pow((double)beta1, (double)step));
    const float c2 = (float)(1.0 - std::pow((double)beta2, (double)step));
    launch_adam(n, param, grad, m, v, lr, beta1, beta2, eps, c1, c2, mode == SGAD_ADAM_LOG,
                static_cast<cudaStream_t>(stream));
    return last_launch("sgad_adam_step");
}

sgad_status sgad_adam_step_multi(int32_t n_tensors, const sgad_adam_tensor *tensors, float beta1, float beta2,
                                 float eps, int32_t *step_counter, void *stream)
{
    if (n_tensors < 1 || n_tensors > SGAD_ADAM_MAX_TENSORS || !tensors || !step_counter)
        return fail(SGAD_ERR_INVALID_ARG, "bad arguments to sgad_adam_step_multi");
    if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f))
        return fail(SGAD_ERR_INVALID_ARG, "bad Adam hyper-parameters");
    for (int i = 0; i < n_tensors; ++i) {
        const sgad_adam_tensor &t = tensors[i];
        if (t.n < 0 || (t.n > 0 && (!t.param || !t.grad || !t.m || !t.v)) || !std::isfinite(t.lr) ||
            (t.mode != SGAD_ADAM_PLAIN && t.mode != SGAD_ADAM_LOG))
            return fail(SGAD_ERR_INVALID_ARG, "Adam tensor %d is invalid", i);
    }
    const cudaError_t e = launch_adam_multi(n_tensors, tensors, beta1, beta2, eps, step_counter,
                                            static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SGAD_OK : cuda_fail(e, "sgad_adam_step_multi");
}

sgad_status sgad_autotune(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf, const sgad_camera *views,
                          int32_t n_views, sgad_images *out, const sgad_image_grads *grad_in,
                          sgad_keyframe_grads *grads_out, void *workspace, size_t ws_bytes, int32_t reps,
                          sgad_tune_entry *entries, int32_t max_entries, int32_t *n_entries, void *stream)
{
    if (n_entries) *n_entries = 0;
    if (!ctx) return fail(SGAD_ERR_INVALID_ARG, "ctx is NULL");
    if (reps < 1 || reps > 100) return fail(SGAD_ERR_INVALID_ARG, "reps must be in [1, 100]");
    if (max_entries < 0 || (max_entries > 0 && !entries)) return fail(SGAD_ERR_INVALID_ARG, "bad entries buffer");
    static const int kShapes[3][2] = {{16, 16}, {8, 32}, {32, 8}};
    static const int kBatches[7] = {128, 192, 256, 384, 512, 768, 1024};     // forward
    static const int kScheds[2] = {SGAD_SCHEDULE_TILES, SGAD_SCHEDULE_PERSISTENT};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TuneTimer timer;
    cudaError_t ce = timer.init();
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaEventCreate");
    TuneLog log{entries, max_entries};
    // Candidates run on a copy of the context: persistent order always computed, no
    // profiling events.
    sgad_ctx trial;
    trial.opt = ctx->opt;
    trial.sort_cap = ctx->sort_cap;
    trial.opt.fwd_schedule = SGAD_SCHEDULE_PERSISTENT;
    float best_total = -1.0f;
    sgad_options best = ctx->opt;
    for (const auto &shape : kShapes) {
        trial.opt.tile_w = shape[0];
        trial.opt.tile_h = shape[1];
        Scene sc;
        uint64_t n_pix;
        Ws ws;
        sgad_status s = build_scene(&trial, kfs, n_kf, views, n_views, sc, n_pix);
        if (!s) s = check_kf_inputs(kfs, n_kf);
        if (!s) s = bind_images(sc, out, n_views);
        if (!s) s = bind_grads(sc, grad_in, grads_out, n_kf, n_views);
        if (s) return s;
        // keys of this shape (synchronises)
        if (get_ws(sc, n_pix, workspace, ws_bytes, 0, ws) != SGAD_OK) {
            log.add(shape[0], shape[1], SGAD_TUNE_PREP, 0, 0, -1.0f);
            continue;
        }
        s = run_binning_count(trial.opt, sc, ws, 0xfffffffell, true, st);
        if (s) return s;
        WsHeader h;
        ce = cudaMemcpyAsync(&h, ws.hdr(), sizeof(h), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return cuda_fail(ce, "sgad_autotune");
        const int64_t keys = (int64_t)h.needed;
        if (get_ws(sc, n_pix, workspace, ws_bytes, keys, ws) != SGAD_OK) {
            log.add(shape[0], shape[1], SGAD_TUNE_PREP, 0, 0, -1.0f);
            continue;
        }
        float prep = 0.f;
        s = timer.median(reps, st, [&] { return run_forward_prep(&trial, sc, ws, keys, st); }, &prep);
        if (s) return s;
        log.add(shape[0], shape[1], SGAD_TUNE_PREP, 0, 0, prep);
        float best_f = -1.f, best_b = -1.f;
        int fb = 0, fs = 0, bb = 0, bs = 0;
        trial.opt.bwd_algorithm = SGAD_BWD_WARP_REDUCE;     // forwards without contribution words
        for (int sched : kScheds)
            for (int batch : kBatches) {
                float ms = 0.f;
                s = timer.median(reps, st, [&] { return run_composite(&trial, true, batch, sched, sc, ws, st); }, &ms);
                if (s) return s;
                log.add(shape[0], shape[1], SGAD_TUNE_FWD, batch, sched, ms);
                if (best_f < 0.f || ms < best_f) {
                    best_f = ms;
                    fb = batch;
                    fs = sched;
                }
            }
        // The pair-parallel backward needs the best forward to record contribution words;
        // that extra forward cost is charged to the pair-parallel candidates.
        trial.opt.bwd_algorithm = SGAD_BWD_PAIRS;
        float fwd_words = 0.f;
        s = timer.median(reps, st, [&] { return run_composite(&trial, true, fb, fs, sc, ws, st); }, &fwd_words);
        if (s) return s;
        const float words_cost = fwd_words > best_f ? fwd_words - best_f : 0.f;
        static const int kBwdBatches[7] = {-1, 0, 128, 192, 256, 384, 512};  // -1: warp-local, 0: pair-parallel
        for (int sched : kScheds)
            for (int batch : kBwdBatches) {
                float ms = 0.f;
                auto run = [&] {
                    const cudaError_t e = cudaMemsetAsync(ws.gacc(), 0, (size_t)sc.n_gauss * 32, st);
                    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
                    return run_composite(&trial, false, batch, sched, sc, ws, st);
                };
                s = timer.median(reps, st, run, &ms);
                if (s) return s;
                if (batch == 0) ms += words_cost;
                log.add(shape[0], shape[1], SGAD_TUNE_BWD, batch, sched, ms);
                if (best_b < 0.f || ms < best_b) {
                    best_b = ms;
                    bb = batch;
                    bs = sched;
                }
            }
        const float total = prep + best_f + best_b;
        if (best_total < 0.f || total < best_total) {
            best_total = total;
            best.tile_w = shape[0];
            best.tile_h = shape[1];
            best.fwd_batch = fb;
            best.fwd_schedule = fs;
            best.bwd_algorithm = bb == 0 ? SGAD_BWD_PAIRS : (bb < 0 ? SGAD_BWD_WARP_LOCAL : SGAD_BWD_WARP_REDUCE);
            best.bwd_batch = bb <= 0 ? ctx->opt.bwd_batch : bb;
            best.bwd_schedule = bs;
        }
    }
    if (n_entries) *n_entries = log.n;
    if (best_total < 0.f)
        return fail(SGAD_ERR_WORKSPACE_TOO_SMALL, "sgad_autotune: the workspace holds the keys of no tile shape");
    ctx->opt = best;
    return SGAD_OK;
}

}  // extern "C"
