// Projection and tile binning (forward steps a1-a4).
//
//   k_project_count : per Gaussian, the world centre mu = R_i (|D + delta| r) + t_i
//                     (Sec. 3.2), opacity sigmoid(logit), the view-independent record,
//                     and for every view the tile rectangle of its 3-sigma square;
//                     per-tile counts with warp-aggregated atomics.
//   k_scan_tiles    : exclusive scan of the per-tile counts -> list offsets; flags a
//                     key overflow.
//   k_emit          : per Gaussian and view, one 8-byte entry (f32 depth bits << 32 |
//                     Gaussian index) per tile of the rectangle the count kernel left in
//                     the workspace (8 bytes per Gaussian and view), written into the
//                     tile's bucket. The depth is evaluated in double-float so the key is
//                     the exactly-rounded f32 of the view depth.
#include "sgad_device.cuh"

namespace sgad {

constexpr int kOrderClasses = 128;

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(256) k_project_count(const __grid_constant__ Scene sc, World *__restrict__ world,
                                                       uint32_t *__restrict__ tile_cnt, uint2 *__restrict__ rects)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = g < sc.n_gauss;
    float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        const KfDev &k = sc.kf[find_kf(sc, g)];
        const uint32_t j = g - k.gbase;
        const int u = (int)(j % (uint32_t)k.W), v = (int)(j / (uint32_t)k.W);
        const size_t hw = (size_t)k.W * k.H;
        const float D = k.depth[j], delta = k.offset[j];
        const float d = fabsf(__fadd_rn(D, delta));
        const float rx = __fdiv_rn(__fsub_rn((float)u, k.cx), k.fx);
        const float ry = __fdiv_rn(__fsub_rn((float)v, k.cy), k.fy);
        const float qx = __fmul_rn(d, rx), qy = __fmul_rn(d, ry);
        w0.x = __fmaf_rn(k.R[0], qx, __fmaf_rn(k.R[1], qy, __fmaf_rn(k.R[2], d, k.t[0])));
        w0.y = __fmaf_rn(k.R[3], qx, __fmaf_rn(k.R[4], qy, __fmaf_rn(k.R[5], d, k.t[1])));
        w0.z = __fmaf_rn(k.R[6], qx, __fmaf_rn(k.R[7], qy, __fmaf_rn(k.R[8], d, k.t[2])));
        if (k.xform) {          // device transform of the centres: mu <- R mu + t
            const float *X = k.xform;
            const float mx = w0.x, my = w0.y, mz = w0.z;
            w0.x = __fmaf_rn(X[0], mx, __fmaf_rn(X[1], my, __fmaf_rn(X[2], mz, X[3])));
            w0.y = __fmaf_rn(X[4], mx, __fmaf_rn(X[5], my, __fmaf_rn(X[6], mz, X[7])));
            w0.z = __fmaf_rn(X[8], mx, __fmaf_rn(X[9], my, __fmaf_rn(X[10], mz, X[11])));
        }
        w0.w = k.scale[j];
        const float o = 1.0f / (1.0f + expf(-k.logit[j]));
        World w;
        w.w0 = w0;
        w.w1 = make_float4(o, k.rgb[j], k.rgb[hw + j], k.rgb[2 * hw + j]);
        world[g] = w;
    }
    const unsigned full = 0xffffffffu;
    for (int vi = 0; vi < sc.n_views; ++vi) {
        const ViewDev &v = sc.view[vi];
        Rect r;
        int n = 0;
        if (valid) {
            n = bin_rect(project(w0, v), v, sc.tw_log2, sc.th_log2, r);
            if (rects) rects[(size_t)vi * sc.n_gauss + g] = pack_rect(r, n);
        }
        const int maxn = __reduce_max_sync(full, n);
        uint32_t row = (uint32_t)(v.tile_base + r.ty0 * v.tiles_x + r.tx0);   // first tile of the current rectangle row
        int col = 0;
        for (int i = 0; i < maxn; ++i) {
            uint32_t tile = kInvalidTile;
            if (i < n) {
                tile = row + (uint32_t)col;
                if (++col == r.nx) {
                    col = 0;
                    row += (uint32_t)v.tiles_x;
                }
            }
            const uint32_t peers = __match_any_sync(full, tile);
            if (tile != kInvalidTile && (threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAdd(&tile_cnt[tile], (uint32_t)__popc(peers));
        }
    }
}

// Position of a tile with `len` list entries in the heavy-first order: 128 classes, four
// per power of two of the length, longest first (lengths 0 and 1 share the last class).
__device__ __forceinline__ int order_class(uint32_t len)
{
    if (len <= 1) return kOrderClasses - 1;
    const int e = 31 - __clz(len);
    const int sub = e >= 2 ? (int)((len >> (e - 2)) & 3u) : (int)((len << (2 - e)) & 3u);
    return kOrderClasses - 1 - (4 * e + sub);
}

// Single-CTA exclusive scan of the per-tile counts (1024 threads, 4 tiles per thread per
// round). Also resets the counts to serve as emission cursors and, when `order` is
// given, writes the tiles in heavy-first order (by list-length class; the order within a
// class is unspecified) for the persistent compositing schedule.
__global__ void __launch_bounds__(1024) k_scan_tiles(uint32_t *__restrict__ cnt, uint32_t *__restrict__ off, int n_tiles,
                                                     uint64_t key_cap, WsHeader *hdr, uint32_t *__restrict__ order)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint64_t carry_s;
    __shared__ uint32_t cls_cnt[kOrderClasses];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < n_tiles; base += 4096) {
        uint32_t c[4];
        uint32_t sum = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = base + threadIdx.x * 4 + q;
            c[q] = i < n_tiles ? cnt[i] : 0u;
            sum += c[q];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            uint32_t ws = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += y;
            }
            warp_sums[lane] = ws;       // inclusive over warps
        }
        __syncthreads();
        const uint64_t carry = carry_s;
        uint64_t run = carry + (wid > 0 ? warp_sums[wid - 1] : 0u) + (incl - sum);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = base + threadIdx.x * 4 + q;
            if (i < n_tiles) {
                off[i] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
                cnt[i] = 0u;
            }
            run += c[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + warp_sums[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint64_t total = carry_s;
        off[n_tiles] = (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull);
        hdr->n_keys = (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull);
        hdr->needed = (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull);
        hdr->overflow = total > key_cap ? 1u : 0u;
        if (total > key_cap) {
            record_error(hdr, SGAD_ERR_KEY_OVERFLOW);
            atomicMax(&hdr->sticky_needed, (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull));
        }
    }
    if (!order) return;
    // heavy-first order: class histogram, exclusive scan of the classes, scatter
    for (int i = threadIdx.x; i < kOrderClasses; i += blockDim.x) cls_cnt[i] = 0u;
    __syncthreads();     // also makes this block's writes of off[] visible to all its threads
    for (int i = threadIdx.x; i < n_tiles; i += blockDim.x) atomicAdd(&cls_cnt[order_class(off[i + 1] - off[i])], 1u);
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr int kPer = kOrderClasses / 32;
        uint32_t c[kPer], sum = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            c[q] = cls_cnt[threadIdx.x * kPer + q];
            sum += c[q];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            cls_cnt[threadIdx.x * kPer + q] = run;
            run += c[q];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_tiles; i += blockDim.x)
        order[atomicAdd(&cls_cnt[order_class(off[i + 1] - off[i])], 1u)] = (uint32_t)i;
}

__global__ void __launch_bounds__(256) k_emit(const __grid_constant__ Scene sc, const uint2 *__restrict__ rects,
                                              const uint32_t *__restrict__ off, uint32_t *__restrict__ cursor,
                                              uint64_t *__restrict__ entries, WsHeader *hdr)
{
    if (hdr->overflow) return;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = g < sc.n_gauss;
    dvec3 m = {};
    if (valid) {
        const KfDev &k = sc.kf[find_kf(sc, g)];
        const uint32_t j = g - k.gbase;
        m = df_world_point(k, (int)(j % (uint32_t)k.W), (int)(j / (uint32_t)k.W), k.depth[j], k.offset[j]);
        if (k.xform) m = df_transform(m, k.xform);
    }
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int vi = 0; vi < sc.n_views; ++vi) {
        const ViewDev &v = sc.view[vi];
        Rect r;
        int n = 0;
        if (valid) n = unpack_rect(rects[(size_t)vi * sc.n_gauss + g], r);     // the count kernel's rectangle
        const int maxn = __reduce_max_sync(full, n);
        if (maxn == 0) continue;
        uint64_t key = 0;
        if (n > 0) key = ((uint64_t)__float_as_uint(df_view_depth(m, v)) << 32) | g;
        uint32_t row = (uint32_t)(v.tile_base + r.ty0 * v.tiles_x + r.tx0);
        int col = 0;
        for (int i = 0; i < maxn; ++i) {
            uint32_t tile = kInvalidTile;
            if (i < n) {
                tile = row + (uint32_t)col;
                if (++col == r.nx) {
                    col = 0;
                    row += (uint32_t)v.tiles_x;
                }
            }
            const uint32_t peers = __match_any_sync(full, tile);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (tile != kInvalidTile && lane == leader) base = atomicAdd(&cursor[tile], (uint32_t)__popc(peers));
            base = __shfl_sync(full, base, leader);
            if (tile != kInvalidTile) {
                const uint32_t slot = off[tile] + base + __popc(peers & lanemask_lt());
                if (slot < off[tile + 1]) {
                    entries[slot] = key;
                } else {
                    atomicExch(&hdr->emit_overrun, 1u);
                    atomicExch(&hdr->sticky_overrun, 1u);
                }
            }
        }
    }
}

void launch_project_count(const Scene &sc, World *world, uint32_t *tile_cnt, uint2 *rects, cudaStream_t st)
{
    const unsigned blocks = (sc.n_gauss + 255) / 256;
    if (blocks) k_project_count<<<blocks, 256, 0, st>>>(sc, world, tile_cnt, rects);
}

void launch_scan_tiles(uint32_t *cnt, uint32_t *off, int n_tiles, uint64_t key_cap, WsHeader *hdr, uint32_t *order,
                       cudaStream_t st)
{
    k_scan_tiles<<<1, 1024, 0, st>>>(cnt, off, n_tiles, key_cap, hdr, order);
}

void launch_emit(const Scene &sc, const uint2 *rects, const uint32_t *off, uint32_t *cursor, uint64_t *entries,
                 WsHeader *hdr, cudaStream_t st)
{
    const unsigned blocks = (sc.n_gauss + 255) / 256;
    if (blocks) k_emit<<<blocks, 256, 0, st>>>(sc, rects, off, cursor, entries, hdr);
}

}  // namespace sgad
