// Front-to-back compositing (forward step a7) and its reverse-order adjoint (a9, with
// the per-Gaussian chain rule of a10 down to the world centre, scale, opacity and
// colour), templated on the tile shape (TW x TH = 256 pixels) and on the number of list
// entries staged per block-wide barrier (B).
//
// Forward: 256 threads per tile, one pixel per thread; each warp owns an 8x4 block of
// pixels. The tile's sorted list is consumed in batches of B entries: the threads stage
// them (gathering each Gaussian's 32-byte world record and projecting it into the view)
// into shared memory; then every warp takes 32 staged Gaussians at a time: lane j forms
// the mask of the block's pixels inside Gaussian j's alpha >= 1/255 box, a 32 x 32 bit
// transpose gives each lane the Gaussians whose box covers its pixel, and each lane
// walks only those, in order, until its pixel is done. A warp stops when its pixels are
// done, the block when all warps are. For every 32-entry chunk it walked, a warp also
// writes the OR of its lanes' contribution bits: which entries reached a pixel of its
// block.
//
// Backward: 256 threads per tile, each warp an 8x4 pixel block and each lane one pixel
// (two pixels per lane on 8x8 blocks is a build option). The same lists are walked from
// the tile's largest contributor count down to 0, each warp over exactly the entries that
// reached a pixel of its block (the mask of the forward warp with the same block, or of
// the two that cover an 8x8 block, for the chunks in front of their largest contributor
// counts), so no step is spent on an entry that contributes nowhere in the block. (Splitting the warp into groups as in the forward walks fewer entries
// too, but each step then carries more state and a group-wise reduction, and it measured
// slower.) Each pixel starts from its saved final transmittance and recovers the
// transmittance in front of entry i by division, T_i = T_{i+1} / (1 - alpha_i), which
// is stable because alpha <= 0.99. Per (pixel, entry) it forms the gradient of the
// colour, depth and alpha terms; the moments of the lane's pixels are summed in
// registers, reduced over the warp with a reduce-scatter (two entries at a time) and
// accumulated per staged Gaussian in shared memory. At the end of the batch each staging thread turns them into d mu, d s,
// d opacity and d colour and adds them to the per-Gaussian accumulator with two 16-byte
// vector atomics.
//
// A second backward, the pair-parallel variant further below (k_composite_bwdp), walks
// only the pairs the forward marked as contributing and sums them with shared-memory
// atomics; it is selectable (SGAD_BWD_PAIRS) but slower on the room workloads (same-
// Gaussian atomic conflicts between neighbouring pixels), so the warp-reduced one above
// is the default.
//
// A third backward, the warp-local one (k_composite_bwdl, the default), has no block-wide
// barrier at all: every warp takes (tile, 8x4 pixel block) units from a queue and walks
// only the entries its forward mask marks, 32 at a time. Each lane keeps its pixel's
// reverse-walk state; per (entry, contributing pixel) it leaves two numbers in the warp's
// shared memory (dL/dpower and the blend weight), and then one lane per entry sums its
// pixels' moments and applies the chain rule. No (entry, lane) slot of a warp-wide
// reduction is spent on a pixel the entry does not reach.
//
// Work split (CompositeArgs): either one block per tile (blockIdx.x + tile0), or a
// persistent grid of resident blocks that take tiles from an atomic queue in the
// heavy-first order written by the tile scan.
#pragma once

#include "sgad_device.cuh"

namespace sgad {

constexpr int kFwdThreads = 256;
// Backward pixels per lane: 1 (each warp an 8x4 block, 256 threads per tile; the
// default) or 2 (each warp an 8x8 block, 128 threads per tile). One pixel per lane walks
// more (warp, entry) steps with half the arithmetic each and leaves the registers for
// reducing two entries at a time (SGAD_BWD_PAIRED).
#ifndef SGAD_BWD_PX
#define SGAD_BWD_PX 1
#endif
constexpr int kBwdPx = SGAD_BWD_PX;
static_assert(kBwdPx == 1 || kBwdPx == 2, "one or two backward pixels per lane");
constexpr int kBwdThreads = 256 / kBwdPx;
constexpr unsigned kFull = 0xffffffffu;
// Resident-block targets (they bound the registers per thread).
#ifndef SGAD_FWD_MINBLOCKS
#define SGAD_FWD_MINBLOCKS 6
#endif
#ifndef SGAD_BWD_MINBLOCKS
#define SGAD_BWD_MINBLOCKS (kBwdPx == 2 ? 8 : 4)
#endif

// Launch arguments common to both directions.
struct CompositeArgs {
    const World *world;
    const uint32_t *off;          // [n_tiles + 1] list offsets
    const uint64_t *entries;      // sorted (depth bits << 32 | Gaussian) per tile
    float *pix_t;                 // per-pixel final transmittance
    uint32_t *pix_n;              // per-pixel contributor count
    float4 *gacc;                 // per-Gaussian accumulators (backward)
    WsHeader *hdr;
    const uint32_t *order;        // persistent: heavy-first tile order; nullptr: one block per tile
    uint32_t *queue;              // persistent: next position in `order` (starts at 0)
    int32_t tile0;                // one block per tile: tile of block 0
    int32_t n_launch_tiles;       // warp-local backward: tiles this launch covers (from
                                  // tile0, or through `order` when it is set)
    // Contribution words (forward writes, pair-parallel backward reads; may be null):
    // for tile t, list chunk c (entries 32c .. 32c + 31) and forward thread i (its
    // pixel), word contrib[8 off[t] + 256 t + 256 c + i] has bit j set iff entry 32c + j
    // contributed to that pixel. Written for every chunk the pixel's warp walked.
    uint32_t *contrib;
    // Per-warp contribution masks (forward writes, warp-reduced backward reads): for tile
    // t, list chunk c and forward warp w (its 8x4 pixel block), word
    // wmask[(off[t] >> 2) + 16 t + 8 c + w] has bit j set iff entry 32c + j contributed to
    // a pixel of that block. Written for every chunk the warp walked.
    uint32_t *wmask;
    int32_t pose;                 // some view wants its pose gradient (selects the kernel variant)
};

__device__ __forceinline__ size_t wmask_base(int tile, uint32_t s) { return (size_t)(s >> 2) + 16 * (size_t)tile; }

__device__ __forceinline__ size_t contrib_base(const CompositeArgs &a, int tile, uint32_t s)
{
    return 8 * (size_t)s + 256 * (size_t)tile;
}

// Next tile of this block, or -1 when there is none. s_tile is a shared-memory slot.
__device__ __forceinline__ int next_tile(const Scene &sc, const CompositeArgs &a, bool &first, int *s_tile)
{
    if (!a.order) {
        const bool f = first;
        first = false;
        return f ? a.tile0 + (int)blockIdx.x : -1;
    }
    __syncthreads();     // every thread has read the previous slot value
    if (threadIdx.x == 0) {
        const uint32_t q = atomicAdd(a.queue, 1u);
        *s_tile = q < (uint32_t)sc.n_tiles ? (int)a.order[q] : -1;
    }
    __syncthreads();
    return *s_tile;
}

__device__ __forceinline__ void stage_entry(const Scene &sc, const CompositeArgs &a, const ViewDev &v, uint64_t ent,
                                            Staged &st)
{
    const uint32_t g = (uint32_t)ent;
    if (g < sc.n_gauss) {
        const World w = a.world[g];
        stage(project(w.w0, v), w.w1, __uint_as_float((uint32_t)(ent >> 32)), st);
    } else {
        st.a = make_float4(0.f, 0.f, -1.f, -1.f);     // never reaches a pixel
    }
}

__device__ __forceinline__ uint32_t lane_mask_lt(int lane) { return (1u << lane) - 1u; }

// 32 x 32 bit transpose across the warp: lane j holds row j on entry; on return lane i
// holds column i (bit j = bit i of row j). Swaps the off-diagonal blocks of halving size.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000ffffu : (s == 8 ? 0x00ff00ffu : (s == 4 ? 0x0f0f0f0fu :
                           (s == 2 ? 0x33333333u : 0x55555555u)));
        const uint32_t y = __shfl_xor_sync(kFull, x, s);
        x = (lane & s) ? ((x & ~m) | ((y >> s) & m)) : ((x & m) | ((y << s) & ~m));
    }
    return x;
}

// Pixels (bit p: pixel (bx + p % 8, by + p / 8)) of an 8x4 block inside the box
// |px - x| <= hx, |py - y| <= hy of a staged entry; hx < 0 marks an empty box.
__device__ __forceinline__ uint32_t box_block_mask(const float4 a, float bxf, float byf)
{
    if (!(a.z >= 0.0f)) return 0u;
    const float x0 = fmaxf(ceilf(a.x - a.z) - bxf, 0.0f), x1 = fminf(floorf(a.x + a.z) - bxf, 7.0f);
    const float y0 = fmaxf(ceilf(a.y - a.w) - byf, 0.0f), y1 = fminf(floorf(a.y + a.w) - byf, 3.0f);
    if (!(x0 <= x1) || !(y0 <= y1)) return 0u;
    const int xl = (int)x0, xh = (int)x1, yl = (int)y0, yh = (int)y1;
    const uint32_t cols = (0xffu >> (7 - (xh - xl))) << xl;
    const uint32_t rows = (0xffffffffu >> (8 * (3 - (yh - yl)))) << (8 * yl);
    return (cols * 0x01010101u) & rows;
}

// ------------------------------------------------------------------ forward

// Forward shared memory for batch B: the staged entries.
template <int B>
constexpr size_t fwd_smem_bytes()
{
    return (size_t)B * sizeof(Staged);
}

// Resident-block target of the forward kernel for batch B: as many blocks as the shared
// memory lets share an SM (227 KB), at most SGAD_FWD_MINBLOCKS; it bounds the registers.
template <int B>
constexpr int fwd_min_blocks()
{
    const int fit = (int)((227 * 1024) / (fwd_smem_bytes<B>() + 1024));
    return fit < 1 ? 1 : (fit > SGAD_FWD_MINBLOCKS ? SGAD_FWD_MINBLOCKS : fit);
}

// The box of a staged entry as tile-relative masks, in place of its half extents (a.z,
// a.w): bit i of the column mask is set when tile column i (pixel x = ox + i) lies in
// [ceil(x - hx), floor(x + hx)], the row mask likewise; both zero for an empty box. The
// same pixel sets as box_block_mask, computed once per (entry, tile) instead of per warp.
template <int TW, int TH>
__device__ __forceinline__ void box_tile_masks(float4 &a, float oxf, float oyf)
{
    uint32_t cm = 0u, rm = 0u;
    if (a.z >= 0.0f) {
        const float x0 = fmaxf(ceilf(a.x - a.z) - oxf, 0.0f), x1 = fminf(floorf(a.x + a.z) - oxf, (float)(TW - 1));
        const float y0 = fmaxf(ceilf(a.y - a.w) - oyf, 0.0f), y1 = fminf(floorf(a.y + a.w) - oyf, (float)(TH - 1));
        if (x0 <= x1 && y0 <= y1) {
            const int xl = (int)x0, xh = (int)x1, yl = (int)y0, yh = (int)y1;
            cm = (~0u >> (31 - (xh - xl))) << xl;
            rm = (~0u >> (31 - (yh - yl))) << yl;
        }
    }
    a.z = __uint_as_float(cm);
    a.w = __uint_as_float(rm);
}

// The 8x4 block mask (bit p: pixel (p % 8, p / 8) of the block) of an entry staged with
// tile masks, for the block at tile column 8 cb (csh = 8 cb) and tile row 4 rb (rsh = 4 rb).
__device__ __forceinline__ uint32_t block_mask_from_tile(const float2 m, int csh, int rsh)
{
    const uint32_t cols = (__float_as_uint(m.x) >> csh) & 0xffu;
    const uint32_t rows = (__float_as_uint(m.y) >> rsh) & 0xfu;
    // row bit k -> byte k all ones: the four copies of rows at bit offsets 0, 7, 14, 21
    // put bit k at bit 8 k without overlapping
    return (cols * 0x01010101u) & (((rows * 0x00204081u) & 0x01010101u) * 0xffu);
}

// Stage entries [b0, min(b0 + B, e)) of a tile list whose tile origin is (oxf, oyf).
template <int TW, int TH, int B>
__device__ __forceinline__ void stage_batch(const Scene &sc, const CompositeArgs &a, const ViewDev &v, uint32_t b0,
                                            uint32_t e, float oxf, float oyf, Staged *buf)
{
#pragma unroll
    for (int r = 0; r < (B + kFwdThreads - 1) / kFwdThreads; ++r) {
        const int k = r * kFwdThreads + threadIdx.x;
        if (k < B && b0 + k < e) {
            Staged st;
            stage_entry(sc, a, v, a.entries[b0 + k], st);
            box_tile_masks<TW, TH>(st.a, oxf, oyf);
            buf[k] = st;
        }
    }
}

// Per-pixel running state of the forward walk.
struct FwdPixel {
    float T, cr, cg, cb, dd, aa;
    int last;
    bool done;
};

// Forward pixel of thread (warp, lane) in a TW-wide tile at pixel (ox, oy): the warp's
// 8x4 block, row-major (lane % 8, lane / 8).
template <int TW>
__device__ __forceinline__ int2 fwd_pixel(int ox, int oy, int warp, int lane)
{
    return make_int2(ox + (warp % (TW / 8)) * 8 + (lane & 7), oy + (warp / (TW / 8)) * 4 + (lane >> 3));
}

// The warp walks nb staged entries (list positions b0 - s ...) against its pixel block,
// 32 at a time: lane j forms entry j's block mask (the block's pixels inside its alpha >=
// 1/255 box, from the tile masks staged with it), a bit transpose gives every lane the
// entries whose box covers its pixel, and each lane not yet done walks its own entries in
// order. Lanes are busy only with (pixel, entry) pairs inside the entry's box.
template <bool CONTRIB>
__device__ __forceinline__ void walk_batch(const Staged *sm, int nb, uint32_t b0, uint32_t s, int tile,
                                           const CompositeArgs &a, int csh, int rsh, float qx, float qy, int lane,
                                           FwdPixel &px, bool &warp_done, uint32_t &n_pairs, uint32_t &n_evals,
                                           uint32_t *wmw)
{
    for (int c0 = 0; c0 < nb; c0 += 32) {
        const int j = c0 + lane;
        uint32_t mine = warp_transpose32(
            j < nb ? block_mask_from_tile(*reinterpret_cast<const float2 *>(&sm[j].a.z), csh, rsh) : 0u, lane);
        if (px.done) mine = 0u;
        n_evals += __popc(mine);            // less the candidates left when the pixel stops
        const int pos0 = (int)(b0 + c0 - s);
        uint32_t bits = 0;
        while (__any_sync(kFull, mine != 0u)) {
            if (mine) {
                const int jj = __ffs(mine) - 1;
                mine &= mine - 1u;
                const Staged st = sm[c0 + jj];
                float dx, dy, ep, alpha;
                if (gauss_alpha(st, qx, qy, dx, dy, ep, alpha)) {
                    const float test = __fmul_rn(px.T, __fsub_rn(1.0f, alpha));
                    if (test < kTStop) {
                        px.done = true;
                        n_evals -= __popc(mine);
                        mine = 0u;
                    } else {
                        bits |= 1u << jj;
                        const float w = __fmul_rn(alpha, px.T);
                        px.cr = __fmaf_rn(w, st.c.x, px.cr);
                        px.cg = __fmaf_rn(w, st.c.y, px.cg);
                        px.cb = __fmaf_rn(w, st.c.z, px.cb);
                        px.dd = __fmaf_rn(w, st.c.w, px.dd);
                        px.aa = __fadd_rn(px.aa, w);
                        px.T = test;
                        px.last = pos0 + jj;
                    }
                }
            }
        }
        n_pairs += __popc(bits);
        if (CONTRIB) a.contrib[contrib_base(a, tile, s) + (size_t)((b0 - s + c0) >> 5) * 256 + threadIdx.x] = bits;
        if (wmw) {
            const uint32_t wbits = __reduce_or_sync(kFull, bits);
            if (lane == 0) wmw[(b0 - s + c0) >> 2] = wbits;        // chunk (b0 - s + c0) / 32, 8 words each
        }
        if (__all_sync(kFull, px.done)) {
            warp_done = true;
            break;
        }
    }
}

template <int TW, int TH, int B, bool CONTRIB>
__device__ __forceinline__ void fwd_tile(const Scene &sc, const CompositeArgs &a, int tile, Staged *sm,
                                         uint32_t &n_pairs, uint32_t &n_evals)
{
    static_assert(TW * TH == kFwdThreads, "tile must hold 256 pixels");
    const ViewDev &v = sc.view[find_view_of_tile(sc, tile)];
    const int local = tile - v.tile_base;
    const int tx = local % v.tiles_x, ty = local / v.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 pix = fwd_pixel<TW>(tx * TW, ty * TH, warp, lane);
    const int px = pix.x, py = pix.y;
    const bool inside = px < v.W && py < v.H;
    const float qx = (float)px, qy = (float)py;

    FwdPixel st = {1.0f, 0.f, 0.f, 0.f, 0.f, 0.f, -1, !inside};
    bool warp_done = __all_sync(kFull, st.done);
    const uint32_t s = a.off[tile], e = a.off[tile + 1];
    // this warp's contribution-mask word of chunk 0; chunk c's is 8 c words further, i.e.
    // at offset (32 c) / 4
    uint32_t *wmw = a.wmask ? a.wmask + wmask_base(tile, s) + warp : nullptr;
    for (uint32_t b0 = s; b0 < e; b0 += B) {
        if (__syncthreads_and(st.done)) break;
        // tile origin from this thread's pixel (TW, TH are powers of two)
        stage_batch<TW, TH, B>(sc, a, v, b0, e, (float)(px & ~(TW - 1)), (float)(py & ~(TH - 1)), sm);
        __syncthreads();
        const int nb = (int)min((uint32_t)B, e - b0);
        if (!warp_done)
            walk_batch<CONTRIB>(sm, nb, b0, s, tile, a, 8 * (warp % (TW / 8)), 4 * (warp / (TW / 8)), qx, qy, lane, st,
                       warp_done, n_pairs, n_evals, wmw);
    }
    if (inside) {
        const size_t hw = (size_t)v.W * v.H, p = (size_t)py * v.W + px;
        v.rgb[p] = st.cr + st.T * sc.bg[0];
        v.rgb[hw + p] = st.cg + st.T * sc.bg[1];
        v.rgb[2 * hw + p] = st.cb + st.T * sc.bg[2];
        v.depth[p] = st.dd;
        v.alpha[p] = st.aa;
        a.pix_t[v.pix_base + p] = st.T;
        a.pix_n[v.pix_base + p] = (uint32_t)(st.last + 1);
    }
}

template <int TW, int TH, int B, bool CONTRIB>
__global__ void __launch_bounds__(kFwdThreads, fwd_min_blocks<B>())
    k_composite_fwd(const __grid_constant__ Scene sc, const CompositeArgs a)
{
    extern __shared__ float4 fwd_smem[];
    Staged *sm = reinterpret_cast<Staged *>(fwd_smem);     // B staged entries
    __shared__ int s_tile;
    if (a.hdr->overflow) return;
    uint32_t n_pairs = 0, n_evals = 0;
    bool first = true;
    for (;;) {
        const int tile = next_tile(sc, a, first, &s_tile);
        if (tile < 0) break;
        fwd_tile<TW, TH, B, CONTRIB>(sc, a, tile, sm, n_pairs, n_evals);
    }
    const uint32_t wp = __reduce_add_sync(kFull, n_pairs), we = __reduce_add_sync(kFull, n_evals);
    if ((threadIdx.x & 31) == 0 && we) {
        atomicAdd(&a.hdr->n_pairs, (unsigned long long)wp);
        atomicAdd(&a.hdr->n_evals, (unsigned long long)we);
    }
}

// ------------------------------------------------------------------ backward

// Reduce-scatter of ten per-lane values over the warp by recursive halving with padding:
// at lane distance 16, 8, 4 and 2 a lane sends the part of its slots its partner keeps
// (5, 3, 2 and 1 values) and adds the partner's copy of the part it keeps; a last
// exchange at distance 1 sums the pair. 12 shuffles (a 16-slot scatter takes 16, ten
// all-reductions 50). Both lanes of a pair then hold the warp total of the slot
// scatter10_slot(lane) names (-1: padding).
__device__ __forceinline__ float warp_reduce_scatter10(float (&v)[10], int lane)
{
    {
        const bool up = (lane & 16) != 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float send = up ? v[i] : v[i + 5];
            const float keep = up ? v[i + 5] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, 16);
        }
    }
    {
        const bool up = (lane & 8) != 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float hi = i + 3 < 5 ? v[i + 3] : 0.f;
            const float send = up ? v[i] : hi;
            const float keep = up ? hi : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, 8);
        }
    }
    {
        const bool up = (lane & 4) != 0;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float hi = i + 2 < 3 ? v[i + 2] : 0.f;
            const float send = up ? v[i] : hi;
            const float keep = up ? hi : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, 4);
        }
    }
    {
        const bool up = (lane & 2) != 0;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(kFull, send, 2);
    }
    return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

// Slot held by a lane after warp_reduce_scatter10, -1 for padding.
__device__ __forceinline__ int scatter10_slot(int lane)
{
    const int g = lane >> 4, q = (lane >> 3) & 1, r = (lane >> 1) & 3;
    if (q ? r >= 2 : r >= 3) return -1;
    return 5 * g + (q ? 3 + r : r);
}

// Backward entries per reduction: 1, or 2 (the default: two consecutive entries of a
// warp's walk are evaluated, then their moments reduced together, so that the two
// shuffle chains overlap).
#ifndef SGAD_BWD_PAIRED
#define SGAD_BWD_PAIRED 2
#endif

// warp_reduce_scatter10 of two value sets at once (their shuffles interleaved); each lane
// ends with the totals of the same slot of both.
__device__ __forceinline__ void warp_reduce_scatter10x2(float (&v)[10], float (&u)[10], int lane, float &tv,
                                                        float &tu)
{
    {
        const bool up = (lane & 16) != 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float sv = up ? v[i] : v[i + 5], kv = up ? v[i + 5] : v[i];
            const float su = up ? u[i] : u[i + 5], ku = up ? u[i + 5] : u[i];
            v[i] = kv + __shfl_xor_sync(kFull, sv, 16);
            u[i] = ku + __shfl_xor_sync(kFull, su, 16);
        }
    }
    {
        const bool up = (lane & 8) != 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float hv = i + 3 < 5 ? v[i + 3] : 0.f, hu = i + 3 < 5 ? u[i + 3] : 0.f;
            const float sv = up ? v[i] : hv, kv = up ? hv : v[i];
            const float su = up ? u[i] : hu, ku = up ? hu : u[i];
            v[i] = kv + __shfl_xor_sync(kFull, sv, 8);
            u[i] = ku + __shfl_xor_sync(kFull, su, 8);
        }
    }
    {
        const bool up = (lane & 4) != 0;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float hv = i + 2 < 3 ? v[i + 2] : 0.f, hu = i + 2 < 3 ? u[i + 2] : 0.f;
            const float sv = up ? v[i] : hv, kv = up ? hv : v[i];
            const float su = up ? u[i] : hu, ku = up ? hu : u[i];
            v[i] = kv + __shfl_xor_sync(kFull, sv, 4);
            u[i] = ku + __shfl_xor_sync(kFull, su, 4);
        }
    }
    {
        const bool up = (lane & 2) != 0;
        const float sv = up ? v[0] : v[1], kv = up ? v[1] : v[0];
        const float su = up ? u[0] : u[1], ku = up ? u[1] : u[0];
        v[0] = kv + __shfl_xor_sync(kFull, sv, 2);
        u[0] = ku + __shfl_xor_sync(kFull, su, 2);
    }
    tv = v[0] + __shfl_xor_sync(kFull, v[0], 1);
    tu = u[0] + __shfl_xor_sync(kFull, u[0], 1);
}

// Projection of a Gaussian for the chain rule: the same quantities as project() with a
// fast reciprocal of the depth (the gradients are compared with tolerances; the
// decisions of the walk use project()).
__device__ __forceinline__ Proj project_chain(const float4 w0, const ViewDev &v)
{
    Proj p;
    p.tx = fmaf(v.R[0], w0.x, fmaf(v.R[1], w0.y, fmaf(v.R[2], w0.z, v.t[0])));
    p.ty = fmaf(v.R[3], w0.x, fmaf(v.R[4], w0.y, fmaf(v.R[5], w0.z, v.t[1])));
    p.tz = fmaf(v.R[6], w0.x, fmaf(v.R[7], w0.y, fmaf(v.R[8], w0.z, v.t[2])));
    const float iz = __fdividef(1.0f, p.tz);
    const float ux = p.tx * iz, uy = p.ty * iz;
    p.px = fmaf(v.fx, ux, v.cx);
    p.py = fmaf(v.fy, uy, v.cy);
    const float j00 = v.fx * iz, j02 = -j00 * ux;
    const float j11 = v.fy * iz, j12 = -j11 * uy;
    const float s2 = w0.w * w0.w;
    p.cxx = fmaf(s2, fmaf(j00, j00, j02 * j02), kDilation);
    p.cxy = s2 * (j02 * j12);
    p.cyy = fmaf(s2, fmaf(j11, j11, j12 * j12), kDilation);
    return p;
}

// Chain rule of one staged Gaussian from its ten accumulated pair moments (colour (3),
// depth, G, G dx, G dy, G dx^2, G dx dy, G dy^2 with G = dL/dpower) down to d mu, d s,
// d opacity and d colour, added to its accumulator.
__device__ __forceinline__ float3 chain_and_accumulate(const float *A, const Staged &st, const Proj &pr, float s_,
                                                       const ViewDev &v, float4 *gacc, uint32_t g)
{
    const float ca = st.b.x, cbb = st.b.y, cc = st.b.z, o = st.b.w;
    const float G = A[4], Gx = A[5], Gy = A[6], Gxx = A[7], Gxy = A[8], Gyy = A[9];
    const float d_o = __fdividef(G, o);
    const float da = -0.5f * Gxx, db = -Gxy, dc = -0.5f * Gyy;
    const float dpx = -(ca * Gx + cbb * Gy), dpy = -(cbb * Gx + cc * Gy);
    // conic (a, b, c) = (w, -y, x) / det of Sigma_2D = [[x, y], [y, w]]
    const float x = pr.cxx, y = pr.cxy, wv = pr.cyy;
    const float det = x * wv - y * y, id2 = __fdividef(1.0f, det * det);
    const float gx = (-wv * wv * da + y * wv * db - y * y * dc) * id2;
    const float gy = (2.0f * y * wv * da - (det + 2.0f * y * y) * db + 2.0f * x * y * dc) * id2;
    const float gw = (-y * y * da + y * x * db - x * x * dc) * id2;
    // Sigma_2D = s^2 J J^T + 0.3 I
    const float tz = pr.tz, iz = __fdividef(1.0f, tz), iz2 = iz * iz;
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
    return make_float3(gtx, gty, gtz);
}

// View-pose terms of one Gaussian per lane (zero for lanes without one): t = R mu + t_k,
// so d L / d R[a][b] += dL/dt[a] mu[b] and d L / d t_k[a] += dL/dt[a] (row-major 3x4);
// summed over the warp and added to the block's shared accumulator. Whole warp.
__device__ __forceinline__ void pose_reduce(const float3 gt, const float4 mu, float *s_pose)
{
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const float g = (q >> 2) == 0 ? gt.x : ((q >> 2) == 1 ? gt.y : gt.z);
        const int c = q & 3;
        float x = c == 3 ? g : g * (c == 0 ? mu.x : (c == 1 ? mu.y : mu.z));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if ((threadIdx.x & 31) == 0 && x != 0.f) atomicAdd(&s_pose[q], x);
    }
}

// Shared memory of the backward pass for a batch of B entries: the staged records, their
// Gaussian indices and eleven-float moment rows (odd stride: the per-thread row reads of
// the chain phase hit distinct banks).
template <int B>
constexpr size_t bwd_smem_bytes()
{
    return (size_t)B * (sizeof(Staged) + sizeof(uint32_t) + 11 * sizeof(float));
}

template <int TW, int TH, int B, bool POSE>
__device__ __forceinline__ void bwd_tile(const Scene &sc, const CompositeArgs &a, int tile, Staged *sm, uint32_t *sg,
                                         float (*acc)[11], int *s_nmax, float *s_pose)
{
    static_assert(TW * TH == kBwdPx * kBwdThreads, "tile must hold 256 pixels");
    const ViewDev &v = sc.view[find_view_of_tile(sc, tile)];
    const int local = tile - v.tile_base;
    const int tx = local % v.tiles_x, ty = local / v.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = tx * TW + (warp % (TW / 8)) * 8, by = ty * TH + (warp / (TW / 8)) * (4 * kBwdPx);
    const int px = bx + (lane & 7);
    int py[kBwdPx];
    float qy[kBwdPx];
#pragma unroll
    for (int p = 0; p < kBwdPx; ++p) {
        py[p] = by + (lane >> 3) + 4 * p;
        qy[p] = (float)py[p];
    }
    const float qx = (float)px;
    const uint32_t s = a.off[tile];
    const int len = (int)(a.off[tile + 1] - s);
    const size_t hw = (size_t)v.W * v.H;

    float Tf[kBwdPx], gr[kBwdPx], gg[kBwdPx], gb[kBwdPx], gD[kBwdPx], gA[kBwdPx], T[kBwdPx], SCr[kBwdPx],
        SCg[kBwdPx], SCb[kBwdPx], SD[kBwdPx], SA[kBwdPx];
    int nc[kBwdPx];
#pragma unroll
    for (int p = 0; p < kBwdPx; ++p) {
        Tf[p] = 1.0f;
        gr[p] = gg[p] = gb[p] = gD[p] = gA[p] = 0.f;
        nc[p] = 0;
        if (px < v.W && py[p] < v.H) {
            const size_t q = (size_t)py[p] * v.W + px;
            Tf[p] = a.pix_t[v.pix_base + q];
            nc[p] = min((int)a.pix_n[v.pix_base + q], len);
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
    const int warp_nc = __reduce_max_sync(kFull, (unsigned)(kBwdPx == 2 ? max(nc[0], nc[kBwdPx - 1]) : nc[0]));
    // The forward warps (8x4 blocks) whose pixels are this warp's: their contribution
    // masks hold the entries that reach a pixel here, valid for the chunks in front of
    // their largest contributor count (the chunks the forward walked).
    const int fw0 = ((by - ty * TH) >> 2) * (TW / 8) + ((bx - tx * TW) >> 3);
    const int fnc0 = __reduce_max_sync(kFull, (unsigned)nc[0]);
    const int fnc1 = kBwdPx == 2 ? (int)__reduce_max_sync(kFull, (unsigned)nc[kBwdPx - 1]) : 0;
    const uint32_t *wm = a.wmask + wmask_base(tile, s);
    __syncthreads();     // the previous tile's readers of *s_nmax are done
    if (POSE && threadIdx.x < 12) s_pose[threadIdx.x] = 0.f;
    if (threadIdx.x == 0) *s_nmax = 0;
    __syncthreads();
    if (lane == 0) atomicMax(s_nmax, warp_nc);
    __syncthreads();
    const int nmax = *s_nmax;
    float bgdot[kBwdPx];
#pragma unroll
    for (int p = 0; p < kBwdPx; ++p) bgdot[p] = sc.bg[0] * gr[p] + sc.bg[1] * gg[p] + sc.bg[2] * gb[p];

    for (int b1 = nmax; b1 > 0; b1 -= B) {
        const int b0 = b1 > B ? b1 - B : 0;
        const int nb = b1 - b0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < (B + kBwdThreads - 1) / kBwdThreads; ++r) {
            const int k = r * kBwdThreads + threadIdx.x;
            if (k >= B) continue;
            if (k < nb) {
                const uint64_t ent = a.entries[s + b0 + k];
                stage_entry(sc, a, v, ent, sm[k]);
                sg[k] = (uint32_t)ent;
            }
#pragma unroll
            for (int q = 0; q < 10; ++q) acc[k][q] = 0.f;
        }
        __syncthreads();
        if (b0 < warp_nc) {
            // the gradient terms of one entry at the lane's pixels in front of their
            // contributor counts (list position lim), added to val
            auto pair_terms = [&](const Staged &st, int lim, float (&val)[10]) {
#pragma unroll
                for (int p = 0; p < kBwdPx; ++p) {
                    if (lim >= nc[p]) continue;
                    float dx, dy, ep, alpha;
                    if (!gauss_alpha(st, qx, qy[p], dx, dy, ep, alpha)) continue;
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
            };
            // the tile list's chunks (32 entries from the list start) that meet this batch,
            // last first; each walks the entries that reach a pixel of the warp's block
            for (int c = (b1 - 1) >> 5; c >= (b0 >> 5); --c) {
                uint32_t mask = (32 * c < fnc0 ? wm[8 * c + fw0] : 0u) |
                                (kBwdPx == 2 && 32 * c < fnc1 ? wm[8 * c + fw0 + TW / 8] : 0u);
                const int lo = b0 - 32 * c, hi = b1 - 32 * c;             // batch range in the chunk
                if (lo > 0) mask &= ~0u << lo;
                if (hi < 32) mask &= (1u << hi) - 1u;
                // every marked entry reaches a pixel of the block, so every step reduces
                while (mask) {
                    const int bit = 31 - __clz(mask);
                    mask &= ~(1u << bit);
                    const int jj = 32 * c + bit - b0;
                    int jj2 = -1;
                    if (SGAD_BWD_PAIRED == 2 && mask) {
                        const int bit2 = 31 - __clz(mask);
                        mask &= ~(1u << bit2);
                        jj2 = 32 * c + bit2 - b0;
                    }
                    float val[10], val2[10];
#pragma unroll
                    for (int q = 0; q < 10; ++q) val[q] = val2[q] = 0.f;
                    pair_terms(sm[jj], b0 + jj, val);
                    if (jj2 >= 0) {
                        pair_terms(sm[jj2], b0 + jj2, val2);
                        float t1, t2;
                        warp_reduce_scatter10x2(val, val2, lane, t1, t2);
                        const int slot = scatter10_slot(lane);
                        if ((lane & 1) == 0 && slot >= 0) {
                            atomicAdd(&acc[jj][slot], t1);
                            atomicAdd(&acc[jj2][slot], t2);
                        }
                    } else {
                        const float total = warp_reduce_scatter10(val, lane);
                        const int slot = scatter10_slot(lane);
                        if ((lane & 1) == 0 && slot >= 0) atomicAdd(&acc[jj][slot], total);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < (B + kBwdThreads - 1) / kBwdThreads; ++r) {
            const int k = r * kBwdThreads + threadIdx.x;
            float3 gt = make_float3(0.f, 0.f, 0.f);
            float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < nb && sg[k] < sc.n_gauss) {
                const float *A = acc[k];
                bool any = false;
#pragma unroll
                for (int q = 0; q < 10; ++q) any |= A[q] != 0.f;
                if (any) {
                    w0 = a.world[sg[k]].w0;
                    gt = chain_and_accumulate(A, sm[k], project_chain(w0, v), w0.w, v, a.gacc, sg[k]);
                }
            }
            if (POSE && v.d_pose) pose_reduce(gt, w0, s_pose);
        }
    }
    if (POSE && v.d_pose) {
        __syncthreads();
        if (threadIdx.x < 12 && s_pose[threadIdx.x] != 0.f) atomicAdd(&v.d_pose[threadIdx.x], s_pose[threadIdx.x]);
    }
}

template <int TW, int TH, int B, bool POSE>
__global__ void __launch_bounds__(kBwdThreads, SGAD_BWD_MINBLOCKS)
    k_composite_bwd(const __grid_constant__ Scene sc, const CompositeArgs a)
{
    extern __shared__ float4 dyn_smem[];
    Staged *sm = reinterpret_cast<Staged *>(dyn_smem);
    uint32_t *sg = reinterpret_cast<uint32_t *>(sm + B);
    float(*acc)[11] = reinterpret_cast<float(*)[11]>(sg + B);
    __shared__ int s_tile, s_nmax;
    __shared__ float s_pose[12];
    if (a.hdr->overflow) return;
    bool first = true;
    for (;;) {
        const int tile = next_tile(sc, a, first, &s_tile);
        if (tile < 0) break;
        bwd_tile<TW, TH, B, POSE>(sc, a, tile, sm, sg, acc, &s_nmax, s_pose);
    }
}

// ------------------------------------------------------------------ pair-parallel backward
//
// 256 threads per tile with the forward's pixel map (one pixel per thread, fwd_pixel).
// The list is staged in batches of 256 entries (one per thread, batch starts at
// multiples of 256), walked from the tile's largest contributor count down. Each thread
// walks only its own pixel's contributing entries, read from the forward's contribution
// words (bit j of a chunk word), in reverse order: it recovers the transmittance by
// division, keeps the suffix sums, forms the ten pair moments and adds them to the staged
// entry's shared accumulator row with shared-memory atomics. No (pixel, entry) pair that
// did not contribute is evaluated and no warp-wide reduction is needed. The staging
// thread of each entry then applies the chain rule as in the warp-reduced backward.
constexpr int kPairThreads = 256;
constexpr int kPairBatch = 256;

template <int TW, int TH, bool POSE>
__device__ __forceinline__ void bwdp_tile(const Scene &sc, const CompositeArgs &a, int tile, Staged *sm, uint32_t *sg,
                                          float (*acc)[11], int *s_nmax, float *s_pose)
{
    static_assert(TW * TH == kPairThreads, "tile must hold 256 pixels");
    const ViewDev &v = sc.view[find_view_of_tile(sc, tile)];
    const int local = tile - v.tile_base;
    const int tx = local % v.tiles_x, ty = local / v.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 pix = fwd_pixel<TW>(tx * TW, ty * TH, warp, lane);
    const int px = pix.x, py = pix.y;
    const float qx = (float)px, qy = (float)py;
    const uint32_t s = a.off[tile];
    const int len = (int)(a.off[tile + 1] - s);
    const size_t hw = (size_t)v.W * v.H;
    const uint32_t *words = a.contrib + contrib_base(a, tile, s) + threadIdx.x;

    float Tf = 1.0f, gr = 0.f, gg = 0.f, gb = 0.f, gD = 0.f, gA = 0.f;
    int nc = 0;
    if (px < v.W && py < v.H) {
        const size_t q = (size_t)py * v.W + px;
        Tf = a.pix_t[v.pix_base + q];
        nc = min((int)a.pix_n[v.pix_base + q], len);
        if (v.g_rgb) {
            gr = v.g_rgb[q];
            gg = v.g_rgb[hw + q];
            gb = v.g_rgb[2 * hw + q];
        }
        if (v.g_depth) gD = v.g_depth[q];
        if (v.g_alpha) gA = v.g_alpha[q];
    }
    __syncthreads();     // the previous tile's readers of *s_nmax are done
    if (POSE && threadIdx.x < 12) s_pose[threadIdx.x] = 0.f;
    if (threadIdx.x == 0) *s_nmax = 0;
    __syncthreads();
    const int warp_nc = __reduce_max_sync(kFull, (unsigned)nc);
    if (lane == 0) atomicMax(s_nmax, warp_nc);
    __syncthreads();
    const int nmax = *s_nmax;
    const float bgdot = sc.bg[0] * gr + sc.bg[1] * gg + sc.bg[2] * gb;
    float T = Tf, SCr = 0.f, SCg = 0.f, SCb = 0.f, SD = 0.f, SA = 0.f;

    for (int b0 = nmax > 0 ? ((nmax - 1) / kPairBatch) * kPairBatch : -1; b0 >= 0; b0 -= kPairBatch) {
        const int nb = min(kPairBatch, nmax - b0);
        __syncthreads();
        {
            const int k = threadIdx.x;
            if (k < nb) {
                const uint64_t ent = a.entries[s + b0 + k];
                stage_entry(sc, a, v, ent, sm[k]);
                sg[k] = (uint32_t)ent;
            }
#pragma unroll
            for (int q = 0; q < 10; ++q) acc[k][q] = 0.f;
        }
        __syncthreads();
        // this pixel's contributing entries of the batch, last first, one per step of a
        // warp-uniform loop (each lane advances through its own chunk words)
        const int c_hi = min(b0 + nb, nc), c_lo = b0 >> 5;
        bool active = c_hi > b0;
        int c = active ? (c_hi - 1) >> 5 : c_lo;
        uint32_t bits = active ? words[(size_t)c * 256] : 0u;
        while (__any_sync(kFull, active)) {
            int k = -1;
            if (active) {
                while (bits == 0u && c > c_lo) bits = words[(size_t)(--c) * 256];
                if (bits) {
                    const int bit = 31 - __clz(bits);
                    bits &= ~(1u << bit);
                    k = c * 32 + bit - b0;
                } else {
                    active = false;
                }
            }
            if (k >= 0) {
                const Staged st = sm[k];
                float dx, dy, ep, alpha;
                gauss_alpha(st, qx, qy, dx, dy, ep, alpha);     // contributes (forward decision)
                const float om = __fsub_rn(1.0f, alpha);
                const float rom = __fdividef(1.0f, om);          // om >= 0.01: fast reciprocal
                const float Ti = T * rom;
                const float w = alpha * Ti;
                const float dal = Ti * ((st.c.x - SCr) * gr + (st.c.y - SCg) * gg + (st.c.z - SCb) * gb +
                                        (st.c.w - SD) * gD + (1.0f - SA) * gA) -
                                  (Tf * rom) * bgdot;
                SCr = alpha * st.c.x + om * SCr;
                SCg = alpha * st.c.y + om * SCg;
                SCb = alpha * st.c.z + om * SCb;
                SD = alpha * st.c.w + om * SD;
                SA = alpha + om * SA;
                T = Ti;
                float *row = acc[k];
                atomicAdd(row + 0, w * gr);
                atomicAdd(row + 1, w * gg);
                atomicAdd(row + 2, w * gb);
                atomicAdd(row + 3, w * gD);
                if (!(st.b.w * ep > kAlphaCap)) {
                    const float G = dal * alpha;
                    atomicAdd(row + 4, G);
                    atomicAdd(row + 5, G * dx);
                    atomicAdd(row + 6, G * dy);
                    atomicAdd(row + 7, G * dx * dx);
                    atomicAdd(row + 8, G * dx * dy);
                    atomicAdd(row + 9, G * dy * dy);
                }
            }
        }
        __syncthreads();
        {
            const int k = threadIdx.x;
            float3 gt = make_float3(0.f, 0.f, 0.f);
            float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < nb && sg[k] < sc.n_gauss) {
                const float *A = acc[k];
                bool any = false;
#pragma unroll
                for (int q = 0; q < 10; ++q) any |= A[q] != 0.f;
                if (any) {
                    w0 = a.world[sg[k]].w0;
                    gt = chain_and_accumulate(A, sm[k], project_chain(w0, v), w0.w, v, a.gacc, sg[k]);
                }
            }
            if (POSE && v.d_pose) pose_reduce(gt, w0, s_pose);
        }
    }
    if (POSE && v.d_pose) {
        __syncthreads();
        if (threadIdx.x < 12 && s_pose[threadIdx.x] != 0.f) atomicAdd(&v.d_pose[threadIdx.x], s_pose[threadIdx.x]);
    }
}

template <int TW, int TH, bool POSE>
__global__ void __launch_bounds__(kPairThreads, 4) k_composite_bwdp(const __grid_constant__ Scene sc, const CompositeArgs a)
{
    __shared__ Staged sm[kPairBatch];
    __shared__ uint32_t sg[kPairBatch];
    __shared__ float acc[kPairBatch][11];
    __shared__ int s_tile, s_nmax;
    __shared__ float s_pose[12];
    if (a.hdr->overflow) return;
    bool first = true;
    for (;;) {
        const int tile = next_tile(sc, a, first, &s_tile);
        if (tile < 0) break;
        bwdp_tile<TW, TH, POSE>(sc, a, tile, sm, sg, acc, &s_nmax, s_pose);
    }
}

// ------------------------------------------------------------------ warp-local backward
//
// Work unit: one 8x4 pixel block of one tile, lane = pixel (the block of forward warp wb,
// whose contribution masks mark the entries that reached one of these pixels). Units are
// taken from an atomic queue by single warps, heaviest tile first when the tile order is
// given, so warps never wait for one another. A unit walks its marked entries from the
// largest contributor count down in rounds of up to 32:
//   1. gather: the next (lower) marked positions, highest first, one per lane;
//   2. stage: lane j projects entry j into the warp's shared memory and forms its box
//      mask, the pixels of the block inside the entry's alpha >= 1/255 box;
//   3. transpose the 32 x 32 bit matrix of box masks (five xor-shuffle steps), so that
//      each lane holds the entries whose box covers its pixel, and drop those at or past
//      the pixel's contributor count;
//   4. walk: each lane visits only its own entries, in order, recovers the transmittance
//      by division, forms dL/dalpha from its suffix sums and, where the entry contributes,
//      stores (G = alpha dL/dalpha, zero at the alpha cap; w = alpha T) in the entry's
//      slot range of a per-warp pair buffer (a slot per box pixel);
//   5. reduce: the lanes' contribution bits are transposed back, and lane j sums the ten
//      moments of entry j over the pixels it reached (colour and depth: w times the
//      pixel's image gradients; G, G dx, G dy, G dx^2, G dx dy, G dy^2), applies the chain
//      rule and adds the result with two vector atomics.
// Entries whose box slots do not fit the pair buffer together are walked and reduced in
// consecutive sub-ranges. The per-pair arithmetic is the warp-reduced backward's; no
// lane steps through an entry whose box misses its pixel.
constexpr int kLocalThreads = 256;          // 8 independent warps per block
constexpr int kLocalPairCap = 512;          // (G, w) slots per warp
#ifndef SGAD_BWDL_MINBLOCKS
#define SGAD_BWDL_MINBLOCKS 4
#endif

struct LocalWarpSmem {
    float4 sa[32], sb[32], sc[32];  // the round's entries (Staged a, b, c)
    float4 pg[32];                  // image gradients (r, g, b, depth) of the unit's pixels
    float2 pq[32];                  // their coordinates (x, y)
    float2 pairs[kLocalPairCap];    // (G, w) per box pixel of each entry
    uint32_t row[32];               // box mask of entry j over the block's pixels
    int32_t base[32];               // first pair slot of entry j
    int32_t pos[32];                // list position of entry j (descending in j)
};
constexpr size_t kLocalSmemBytes = (kLocalThreads / 32) * sizeof(LocalWarpSmem);

// Moments of the entries [j0, j1) of a round (lane j holds entry j: the pixels it
// contributed to, cm, its Gaussian g and world record w0; its pair slots start at
// base_j - b0), the chain rule, and the pose terms accumulated per lane. When the range
// holds at most 16 entries, the lane 16 away from entry j's lane sums the moments of the
// entry's bottom two pixel rows and hands them over with one shuffle per moment, so no
// lane is idle and each walks at most half of an entry's pixels. Whole warp.
template <bool POSE>
__device__ __forceinline__ void bwdl_reduce(const ViewDev &v, const CompositeArgs &a, const LocalWarpSmem &S, int j0,
                                            int j1, int lane, uint32_t cm, uint32_t g, float4 w0, int b0,
                                            float (&pose)[12])
{
    const bool split = j1 - j0 <= 16;
    const uint32_t cm_x = __shfl_xor_sync(kFull, cm, 16);
    const bool own = lane >= j0 && lane < j1;
    int e = -1;
    uint32_t m = 0u;
    if (own) {
        e = lane;
        m = split ? (cm & 0xffffu) : cm;
    } else if (split && (lane ^ 16) >= j0 && (lane ^ 16) < j1) {
        e = lane ^ 16;
        m = cm_x & 0xffff0000u;
    }
    float A[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) A[q] = 0.f;
    if (m) {
        const float4 sa = S.sa[e];
        const uint32_t row = S.row[e];
        const int base = S.base[e] - b0;
        while (m) {
            const int p = __ffs(m) - 1;
            m &= m - 1u;
            const float2 gw = S.pairs[base + __popc(row & lane_mask_lt(p))];
            const float4 pg = S.pg[p];
            const float2 pq = S.pq[p];
            const float dx = __fsub_rn(sa.x, pq.x);
            const float dy = __fsub_rn(sa.y, pq.y);
            A[0] += gw.y * pg.x;
            A[1] += gw.y * pg.y;
            A[2] += gw.y * pg.z;
            A[3] += gw.y * pg.w;
            const float G = gw.x;
            A[4] += G;
            A[5] += G * dx;
            A[6] += G * dy;
            A[7] += G * dx * dx;
            A[8] += G * dx * dy;
            A[9] += G * dy * dy;
        }
    }
    if (split) {
#pragma unroll
        for (int q = 0; q < 10; ++q) A[q] += __shfl_xor_sync(kFull, A[q], 16);
    }
    if (!own || cm == 0u) return;
    Staged st;
    st.a = S.sa[lane];
    st.b = S.sb[lane];
    st.c = S.sc[lane];
    const float3 gt = chain_and_accumulate(A, st, project_chain(w0, v), w0.w, v, a.gacc, g);
    if (POSE) {
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float gq = (q >> 2) == 0 ? gt.x : ((q >> 2) == 1 ? gt.y : gt.z);
            const int c = q & 3;
            pose[q] += c == 3 ? gq : gq * (c == 0 ? w0.x : (c == 1 ? w0.y : w0.z));
        }
    }
}

template <int TW, int TH, bool POSE, bool PLAIN>
__device__ __forceinline__ void bwdl_unit(const Scene &sc, const CompositeArgs &a, int tile, int wb, LocalWarpSmem &S,
                                          int lane)
{
    const ViewDev &v = sc.view[find_view_of_tile(sc, tile)];
    const int local = tile - v.tile_base;
    const int tx = local % v.tiles_x, ty = local / v.tiles_x;
    const int bx = tx * TW + (wb % (TW / 8)) * 8, by = ty * TH + (wb / (TW / 8)) * 4;
    const float bxf = (float)bx, byf = (float)by;
    const int px = bx + (lane & 7), py = by + (lane >> 3);
    const float qx = (float)px, qy = (float)py;
    const uint32_t s = a.off[tile];
    const int len = (int)(a.off[tile + 1] - s);
    const size_t hw = (size_t)v.W * v.H;

    float Tf = 1.0f, gr = 0.f, gg = 0.f, gb = 0.f, gD = 0.f, gA = 0.f;
    int nc = 0;
    if (px < v.W && py < v.H) {
        const size_t q = (size_t)py * v.W + px;
        Tf = a.pix_t[v.pix_base + q];
        nc = min((int)a.pix_n[v.pix_base + q], len);
        if (v.g_rgb) {
            gr = v.g_rgb[q];
            gg = v.g_rgb[hw + q];
            gb = v.g_rgb[2 * hw + q];
        }
        if (v.g_depth) gD = v.g_depth[q];
        if (v.g_alpha) gA = v.g_alpha[q];
    }
    const int fnc = (int)__reduce_max_sync(kFull, (unsigned)nc);
    if (fnc == 0) return;
    __syncwarp();                       // the previous unit's readers of S are done
    S.pg[lane] = make_float4(gr, gg, gb, gD);
    S.pq[lane] = make_float2(qx, qy);
    const float bgdot = sc.bg[0] * gr + sc.bg[1] * gg + sc.bg[2] * gb;
    // Reverse-walk state: transmittance, and the suffix sums of colour and depth behind
    // the current entry already dotted with this pixel's image gradients (Sg = S_C . g_C
    // + S_D g_D, updated as Sg <- alpha (c . g) + (1 - alpha) Sg) plus the alpha suffix.
    float T = Tf, Sg = 0.f, SA = 0.f;
    float pose[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) pose[q] = 0.f;

    // chunk c of the tile list (entries 32c .. 32c + 31) has this block's mask at wm[8 c];
    // a window of 32 chunks is held one per lane, lane L the chunk cw - L
    const uint32_t *wm = a.wmask + wmask_base(tile, s) + wb;
    int cw = (fnc - 1) >> 5;
    uint32_t wl = cw - lane >= 0 ? wm[8 * (cw - lane)] : 0u;     // bits of chunk cw - lane not yet taken
    for (;;) {
        // 1. gather up to 32 marked positions, highest first, into S.pos: a scan of the
        // lanes' remaining bit counts orders the window's chunks, and each lane writes the
        // highest bits of its chunk that still fit the round
        int n = 0;
        while (n < 32) {
            const int cnt = __popc(wl);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(kFull, incl, 31);
            if (total == 0) {
                cw -= 32;
                if (cw < 0) break;
                wl = cw - lane >= 0 ? wm[8 * (cw - lane)] : 0u;
                continue;
            }
            const int excl = incl - cnt;
            int take = 32 - n - excl;
            take = take < 0 ? 0 : (take > cnt ? cnt : take);
            for (int t = 0; t < take; ++t) {
                const int bit = 31 - __clz(wl);
                wl &= ~(1u << bit);
                S.pos[n + excl + t] = 32 * (cw - lane) + bit;
            }
            n += total < 32 - n ? total : 32 - n;
        }
        if (n == 0) break;
        __syncwarp();
        const int my_pos = lane < n ? S.pos[lane] : 0;
        // 2. stage (lane j: entry j) and the box masks
        uint32_t my_g = 0u, row = 0u;
        float4 my_w0 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < n) {
            const uint64_t ent = a.entries[s + my_pos];
            my_g = (uint32_t)ent;
            const World w = a.world[my_g];
            my_w0 = w.w0;
            Staged st;
            stage(project(w.w0, v), w.w1, __uint_as_float((uint32_t)(ent >> 32)), st);
            S.sa[lane] = st.a;
            S.sb[lane] = st.b;
            S.sc[lane] = st.c;
            row = box_block_mask(st.a, bxf, byf);
        }
        S.pos[lane] = lane < n ? my_pos : -1;
        // 3. the entries whose box covers this pixel, before its contributor count
        uint32_t mine = warp_transpose32(row, lane);
        __syncwarp();
        {
            int lo = 0, hi = n;                 // first j with pos_j < nc (positions descend)
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (S.pos[mid] >= nc) lo = mid + 1; else hi = mid;
            }
            mine &= lo >= 32 ? 0u : (~0u << lo);
        }
        // pair slots: entry j owns one slot per pixel it may reach (inside its box, before
        // the pixel's contributor count), popc(row_j) slots from base_j (exclusive prefix)
        row = warp_transpose32(mine, lane);
        const int cnt = __popc(row);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        S.row[lane] = row;
        S.base[lane] = incl - cnt;
        __syncwarp();
        // 4./5. walk and reduce, in sub-ranges whose box slots fit the pair buffer
        int j0 = 0;
        while (j0 < n) {
            const int b0 = __shfl_sync(kFull, incl - cnt, j0);
            const uint32_t fit = __ballot_sync(kFull, lane >= j0 && lane < n && incl - b0 <= kLocalPairCap);
            const int j1 = fit ? 32 - __clz(fit) : j0 + 1;   // fit is a run of lanes from j0
            const uint32_t range = (j1 >= 32 ? ~0u : ((1u << j1) - 1u)) & (~0u << j0);
            uint32_t todo = mine & range, done = 0u;
            while (__any_sync(kFull, todo != 0u)) {
                if (todo) {
                    const int j = __ffs(todo) - 1;
                    todo &= todo - 1u;
                    Staged st;
                    st.a = S.sa[j];
                    st.b = S.sb[j];
                    st.c = S.sc[j];
                    float dx, dy, ep, alpha;
                    const bool hit = gauss_alpha(st, qx, qy, dx, dy, ep, alpha);
                    // evaluated for every candidate and kept by selects (no branch): a
                    // candidate that misses writes its own pair slot, which the moment
                    // loop never reads (it takes the hits only)
                    {
                        const float om = __fsub_rn(1.0f, alpha);
                        const float rom = __fdividef(1.0f, om);     // om >= 0.01: fast reciprocal
                        const float Ti = T * rom;
                        const float cg = st.c.x * gr + st.c.y * gg + st.c.z * gb + st.c.w * gD;
                        // PLAIN: no alpha gradient and no background (the terms are zero)
                        const float dal = PLAIN ? Ti * (cg - Sg)
                                                : Ti * ((cg - Sg) + (1.0f - SA) * gA) - (Tf * rom) * bgdot;
                        Sg = hit ? alpha * cg + om * Sg : Sg;
                        if (!PLAIN) SA = hit ? alpha + om * SA : SA;
                        const float G = (st.b.w * ep > kAlphaCap) ? 0.f : dal * alpha;
                        S.pairs[S.base[j] - b0 + __popc(S.row[j] & lane_mask_lt(lane))] = make_float2(G, alpha * Ti);
                        T = hit ? Ti : T;
                        done |= (hit ? 1u : 0u) << j;
                    }
                }
            }
            const uint32_t cm = warp_transpose32(done, lane);
            __syncwarp();
            bwdl_reduce<POSE>(v, a, S, j0, j1, lane, cm, my_g, my_w0, b0, pose);
            __syncwarp();               // the next sub-range overwrites the pair slots
            j0 = j1;
        }
        if (n < 32) break;
    }
    if (POSE && v.d_pose) {
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            float x = pose[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
            if (lane == 0 && x != 0.f) atomicAdd(&v.d_pose[q], x);
        }
    }
}

template <int TW, int TH, bool POSE, bool PLAIN>
__global__ void __launch_bounds__(kLocalThreads, SGAD_BWDL_MINBLOCKS)
    k_composite_bwdl(const __grid_constant__ Scene sc, const CompositeArgs a)
{
    static_assert(TW * TH == 256 && TW % 8 == 0 && TH % 4 == 0, "tile must hold eight 8x4 blocks");
    extern __shared__ float4 bwdl_smem[];
    LocalWarpSmem &S = reinterpret_cast<LocalWarpSmem *>(bwdl_smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    if (a.hdr->overflow) return;
    const uint32_t n_units = (uint32_t)a.n_launch_tiles * 8u;
    for (;;) {
        uint32_t u = 0u;
        if (lane == 0) u = atomicAdd(a.queue, 1u);
        u = __shfl_sync(kFull, u, 0);
        if (u >= n_units) break;
        const int tile = a.order ? (int)a.order[u >> 3] : a.tile0 + (int)(u >> 3);
        bwdl_unit<TW, TH, POSE, PLAIN>(sc, a, tile, (int)(u & 7u), S, lane);
    }
}

// ------------------------------------------------------------------ launch

// Batch sizes the kernels are built for (entries staged per block-wide barrier).
constexpr int kBatchSizes[] = {128, 192, 256, 384, 512};          // both passes
constexpr int kFwdOnlyBatchSizes[] = {768, 1024};                 // forward only

// Launches one direction for tile shape TW x TH with batch B. grid_blocks > 0: that many
// blocks (one per tile from tile0, or the persistent grid); returns the launch error.
template <int TW, int TH, int B>
cudaError_t launch_composite_tb(bool fwd, const Scene &sc, const CompositeArgs &a, int grid_blocks, cudaStream_t st)
{
    if (grid_blocks <= 0) return cudaSuccess;
    if (fwd) {
        // the dynamic staging buffers plus the kernel's static slot may pass the 48 KB
        // default: raise the limit (once per device)
        constexpr size_t smem = fwd_smem_bytes<B>();
        static int configured[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64 || !configured[dev]) {
            e = cudaFuncSetAttribute(k_composite_fwd<TW, TH, B, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_composite_fwd<TW, TH, B, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) configured[dev] = 1;
        }
        if (a.contrib)   // the pair-parallel backward's per-pixel contribution words
            k_composite_fwd<TW, TH, B, true><<<grid_blocks, kFwdThreads, smem, st>>>(sc, a);
        else
            k_composite_fwd<TW, TH, B, false><<<grid_blocks, kFwdThreads, smem, st>>>(sc, a);
    } else if constexpr (B <= 512) {
        constexpr size_t smem = bwd_smem_bytes<B>();
        static int configured[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64 || !configured[dev]) {
            e = cudaFuncSetAttribute(k_composite_bwd<TW, TH, B, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_composite_bwd<TW, TH, B, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) configured[dev] = 1;
        }
        if (a.pose)
            k_composite_bwd<TW, TH, B, true><<<grid_blocks, kBwdThreads, smem, st>>>(sc, a);
        else
            k_composite_bwd<TW, TH, B, false><<<grid_blocks, kBwdThreads, smem, st>>>(sc, a);
    } else {
        return cudaErrorInvalidValue;     // the backward is built for batches up to 512
    }
    return cudaGetLastError();
}

// Resident blocks per SM of one direction for tile shape TW x TH with batch B.
template <int TW, int TH, int B>
cudaError_t occupancy_tb(bool fwd, int *blocks_per_sm)
{
    if (fwd) {
        constexpr size_t smem = fwd_smem_bytes<B>();
        const cudaError_t e = cudaFuncSetAttribute(k_composite_fwd<TW, TH, B, false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_composite_fwd<TW, TH, B, false>, kFwdThreads,
                                                             smem);
    }
    if constexpr (B <= 512)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_composite_bwd<TW, TH, B, false>,
                                                             kBwdThreads, bwd_smem_bytes<B>());
    return cudaErrorInvalidValue;
}

template <int TW, int TH>
cudaError_t launch_bwdp(const Scene &sc, const CompositeArgs &a, int grid_blocks, int *occupancy, cudaStream_t st)
{
    if (occupancy)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, k_composite_bwdp<TW, TH, false>, kPairThreads, 0);
    if (grid_blocks <= 0) return cudaSuccess;
    if (a.pose)
        k_composite_bwdp<TW, TH, true><<<grid_blocks, kPairThreads, 0, st>>>(sc, a);
    else
        k_composite_bwdp<TW, TH, false><<<grid_blocks, kPairThreads, 0, st>>>(sc, a);
    return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t launch_bwdl(const Scene &sc, const CompositeArgs &a, int grid_blocks, int *occupancy, cudaStream_t st)
{
    static int configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(k_composite_bwdl<TW, TH, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kLocalSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_composite_bwdl<TW, TH, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kLocalSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_composite_bwdl<TW, TH, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kLocalSmemBytes);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = 1;
    }
    if (occupancy)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, k_composite_bwdl<TW, TH, false, false>,
                                                             kLocalThreads, kLocalSmemBytes);
    if (grid_blocks <= 0) return cudaSuccess;
    // without an alpha gradient and with a black background the walk drops those terms
    bool plain = sc.bg[0] == 0.0f && sc.bg[1] == 0.0f && sc.bg[2] == 0.0f;
    for (int i = 0; i < sc.n_views && plain; ++i) plain = sc.view[i].g_alpha == nullptr;
    if (a.pose)
        k_composite_bwdl<TW, TH, true, false><<<grid_blocks, kLocalThreads, kLocalSmemBytes, st>>>(sc, a);
    else if (plain)
        k_composite_bwdl<TW, TH, false, true><<<grid_blocks, kLocalThreads, kLocalSmemBytes, st>>>(sc, a);
    else
        k_composite_bwdl<TW, TH, false, false><<<grid_blocks, kLocalThreads, kLocalSmemBytes, st>>>(sc, a);
    return cudaGetLastError();
}

// Dispatch on the batch size for one tile shape (instantiated in one translation unit per
// shape); in the backward, batch 0 selects the pair-parallel kernel and a negative batch
// the warp-local one. occupancy != nullptr: only report the resident blocks per SM.
template <int TW, int TH>
cudaError_t launch_composite_shape(bool fwd, int batch, const Scene &sc, const CompositeArgs &a, int grid_blocks,
                                   int *occupancy, cudaStream_t st)
{
    if (!fwd && batch == 0) return launch_bwdp<TW, TH>(sc, a, grid_blocks, occupancy, st);
    if (!fwd && batch < 0) return launch_bwdl<TW, TH>(sc, a, grid_blocks, occupancy, st);
#define SGAD_BATCH_CASE(Bv)                                                                     \
    case Bv:                                                                                    \
        return occupancy ? occupancy_tb<TW, TH, Bv>(fwd, occupancy)                            \
                         : launch_composite_tb<TW, TH, Bv>(fwd, sc, a, grid_blocks, st);
    switch (batch) {
        SGAD_BATCH_CASE(128)
        SGAD_BATCH_CASE(192)
        SGAD_BATCH_CASE(256)
        SGAD_BATCH_CASE(384)
        SGAD_BATCH_CASE(512)
    case 768:
        if (!fwd) return cudaErrorInvalidValue;
        return occupancy ? occupancy_tb<TW, TH, 768>(true, occupancy)
                         : launch_composite_tb<TW, TH, 768>(true, sc, a, grid_blocks, st);
    case 1024:
        if (!fwd) return cudaErrorInvalidValue;
        return occupancy ? occupancy_tb<TW, TH, 1024>(true, occupancy)
                         : launch_composite_tb<TW, TH, 1024>(true, sc, a, grid_blocks, st);
    default:
        return cudaErrorInvalidValue;
    }
#undef SGAD_BATCH_CASE
}

}  // namespace sgad
