// Work split of the compositing passes: dispatch on tile shape and batch size, and the
// three schedules of include/sgad.h (one block per tile over all views in one launch; a
// persistent resident grid taking tiles heaviest-first from a queue; one launch per
// view). The kernels themselves are in k_composite.cuh, built once per tile shape.
#include "k_composite.cuh"

namespace sgad {

extern template cudaError_t launch_composite_shape<16, 16>(bool, int, const Scene &, const CompositeArgs &, int, int *,
                                                          cudaStream_t);
extern template cudaError_t launch_composite_shape<8, 32>(bool, int, const Scene &, const CompositeArgs &, int, int *,
                                                         cudaStream_t);
extern template cudaError_t launch_composite_shape<32, 8>(bool, int, const Scene &, const CompositeArgs &, int, int *,
                                                         cudaStream_t);

namespace {

cudaError_t dispatch(bool fwd, int batch, const Scene &sc, const CompositeArgs &a, int grid, int *occ, cudaStream_t st)
{
    if (sc.tile_w == 16) return launch_composite_shape<16, 16>(fwd, batch, sc, a, grid, occ, st);
    if (sc.tile_w == 8) return launch_composite_shape<8, 32>(fwd, batch, sc, a, grid, occ, st);
    return launch_composite_shape<32, 8>(fwd, batch, sc, a, grid, occ, st);
}

}  // namespace

bool valid_batch(int batch, bool fwd)
{
    for (int b : kBatchSizes)
        if (b == batch) return true;
    if (fwd)
        for (int b : kFwdOnlyBatchSizes)
            if (b == batch) return true;
    return false;
}

// Blocks of the persistent grid: resident blocks per SM times SMs, at most one per tile
// and at most max_blocks when that is positive.
cudaError_t persistent_blocks(bool fwd, int batch, const Scene &sc, int max_blocks, int *blocks)
{
    int occ = 0, dev = 0, sms = 0;
    cudaError_t e = dispatch(fwd, batch, sc, CompositeArgs{}, 0, &occ, nullptr);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    long long n = (long long)(occ > 0 ? occ : 1) * sms;
    if (n > sc.n_tiles) n = sc.n_tiles;
    if (max_blocks > 0 && n > max_blocks) n = max_blocks;
    *blocks = (int)n;
    return cudaSuccess;
}

cudaError_t launch_composite(bool fwd, int batch, int schedule, int max_blocks, const Scene &sc, const World *world,
                             const uint32_t *off, const uint64_t *entries, float *pix_t, uint32_t *pix_n, float4 *gacc,
                             WsHeader *hdr, const uint32_t *order, uint32_t *contrib, uint32_t *wmask,
                             cudaStream_t st)
{
    if (sc.n_tiles <= 0) return cudaSuccess;
    CompositeArgs a = {};
    a.contrib = contrib;
    a.wmask = wmask;
    for (int i = 0; i < sc.n_views && !fwd; ++i)
        if (sc.view[i].d_pose) a.pose = 1;
    a.world = world;
    a.off = off;
    a.entries = entries;
    a.pix_t = pix_t;
    a.pix_n = pix_n;
    a.gacc = gacc;
    a.hdr = hdr;
    if (!fwd && batch < 0) {
        // warp-local backward: resident warps take (tile, block) units from a queue, in
        // the heavy-first tile order (persistent), in tile order, or view by view
        int blocks = 0;
        cudaError_t e = persistent_blocks(false, batch, sc, max_blocks, &blocks);
        if (e != cudaSuccess) return e;
        a.queue = &hdr->queue_bwd;
        auto run = [&](int tile0, int n_tiles, const uint32_t *ord) {
            a.tile0 = tile0;
            a.n_launch_tiles = n_tiles;
            a.order = ord;
            cudaError_t r = cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), st);
            if (r != cudaSuccess) return r;
            return dispatch(false, batch, sc, a, blocks < n_tiles ? blocks : n_tiles, nullptr, st);
        };
        if (schedule == SGAD_SCHEDULE_PER_VIEW) {
            for (int i = 0; i < sc.n_views; ++i) {
                const ViewDev &v = sc.view[i];
                e = run(v.tile_base, v.tiles_x * v.tiles_y, nullptr);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
        return run(0, sc.n_tiles, schedule == SGAD_SCHEDULE_PERSISTENT ? order : nullptr);
    }
    if (schedule == SGAD_SCHEDULE_PERSISTENT) {
        int blocks = 0;
        cudaError_t e = persistent_blocks(fwd, batch, sc, max_blocks, &blocks);
        if (e != cudaSuccess) return e;
        a.order = order;
        a.queue = fwd ? &hdr->queue_fwd : &hdr->queue_bwd;
        e = cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), st);
        if (e != cudaSuccess) return e;
        return dispatch(fwd, batch, sc, a, blocks, nullptr, st);
    }
    if (schedule == SGAD_SCHEDULE_PER_VIEW) {
        for (int i = 0; i < sc.n_views; ++i) {
            const ViewDev &v = sc.view[i];
            a.tile0 = v.tile_base;
            const cudaError_t e = dispatch(fwd, batch, sc, a, v.tiles_x * v.tiles_y, nullptr, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    a.tile0 = 0;
    return dispatch(fwd, batch, sc, a, sc.n_tiles, nullptr, st);
}

}  // namespace sgad
