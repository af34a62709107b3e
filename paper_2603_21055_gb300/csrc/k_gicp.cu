// Geometric tracking (Sec. 3.3, Eq. 2): geometry Gaussians of a depth map, a spatial hash
// grid of the global set, point-to-surface correspondences, the GICP Gauss-Newton system
// and its solve, and the map update. The operations, readings and layouts are stated in
// include/sgad_gicp.h.
//
// Where floating point decides an integer (neighbour ranks, correspondences, overlaps)
// the kernels use explicitly rounded FP32 operations (__fmul_rn, __fadd_rn, ...) in a
// fixed order, so the decision does not depend on the compiler's contraction choices.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>

#include <cuda_runtime.h>

#include "sgad_gicp.h"

namespace sgad {
sgad_status report_error(sgad_status code, const char *msg);
}

namespace {

using sgad::report_error;

constexpr int kSys = 29;                 // H upper triangle (21), g (6), cost, count
constexpr int kSelBlock = 1024;          // cells per selection block (4 per thread)
constexpr int kMaxSelBlocks = 16384;     // selection grids of up to 16.7 M cells
constexpr int kStepThreads = 128;        // correspondence step: 16 teams of 8 lanes per block
constexpr int kInsThreads = 256;         // map-update kernels
constexpr int kKMatchMax = 8;

struct GicpState {
    double pose[12];
    float posef[12];
    double cost, step;
    int32_t iters, done, converged, n, status, max_iters;
    float tol;
    int32_t map_old, ins_total;
    int32_t blocks_done;     // step blocks finished in the current iteration
};

struct GLayout {
    size_t state, sel_counts, tile_sums, hash_cnt, hash_off, hash_pts, knn_cnt, knn_off, knn_pts, partial, ins_flags,
        ins_counts, total;
    int32_t table, knn_table, max_blocks, step_blocks;
};

constexpr int kScanTile = 4096;          // buckets per tile of the parallel scan
constexpr int kMaxTiles = 4096;          // tables of up to 2^24 buckets

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int32_t table_for(int32_t cap)
{
    int32_t t = 1024;
    while (t < 2 * cap && t < (1 << 24)) t <<= 1;
    return t;
}

// Every call computes the same layout from the parameters (capacities included).
GLayout glayout(const sgad_gicp_params &p)
{
    GLayout L;
    L.table = table_for(p.map_capacity);
    L.knn_table = table_for(p.src_capacity);
    L.max_blocks = (p.src_capacity + kInsThreads - 1) / kInsThreads;
    // the correspondence step: one team of 8 lanes per source point, 16 per block (blocks
    // small enough to spread a few thousand points evenly over the SMs), grid-stride over
    // at most 4 blocks per SM of a 152-SM part (the solve sums one partial row per block)
    L.step_blocks = std::min((p.src_capacity + 15) / 16, 4 * 152);
    size_t o = 0;
    const auto take = [&o](size_t bytes) {
        const size_t at = o;
        o = a256(o + bytes);
        return at;
    };
    L.state = take(sizeof(GicpState));
    L.sel_counts = take((size_t)kMaxSelBlocks * sizeof(int32_t));
    L.tile_sums = take((size_t)kMaxTiles * sizeof(int32_t));
    L.hash_cnt = take((size_t)L.table * sizeof(int32_t));
    L.hash_off = take((size_t)(L.table + 1) * sizeof(int32_t));
    L.hash_pts = take((size_t)p.map_capacity * sizeof(float4));
    L.knn_cnt = take((size_t)L.knn_table * sizeof(int32_t));
    L.knn_off = take((size_t)(L.knn_table + 1) * sizeof(int32_t));
    L.knn_pts = take((size_t)p.src_capacity * sizeof(float4));
    L.partial = take((size_t)std::max(L.max_blocks, L.step_blocks) * 32 * sizeof(float));
    L.ins_flags = take((size_t)p.src_capacity * sizeof(int32_t));
    L.ins_counts = take((size_t)(L.max_blocks + 1) * sizeof(int32_t));
    L.total = o;
    return L;
}

// ------------------------------------------------------------------ device helpers
struct Pose12 {
    float p[12];
};
struct PoseD {
    double p[12];
};

__device__ __forceinline__ float3 transform(const float *P, float4 a)
{
    float3 x;
    x.x = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P[0], a.x), __fmul_rn(P[1], a.y)), __fmul_rn(P[2], a.z)), P[3]);
    x.y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P[4], a.x), __fmul_rn(P[5], a.y)), __fmul_rn(P[6], a.z)), P[7]);
    x.z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(P[8], a.x), __fmul_rn(P[9], a.y)), __fmul_rn(P[10], a.z)), P[11]);
    return x;
}

// ((dx dx + dy dy) + dz dz), d = b - a, explicitly rounded
__device__ __forceinline__ float sqdist(float bx, float by, float bz, float ax, float ay, float az)
{
    const float dx = __fsub_rn(bx, ax), dy = __fsub_rn(by, ay), dz = __fsub_rn(bz, az);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ int cell_of(float x, float inv_cell) { return (int)floorf(__fmul_rn(x, inv_cell)); }

// Spatial hash of a cell (Teschner et al. 2003: XOR of the coordinates times three
// large primes), masked to the power-of-two table.
__device__ __forceinline__ uint32_t cell_hash(int ix, int iy, int iz, uint32_t mask)
{
    return (((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u)) & mask;
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (the symmetric Schur
// method, Golub & Van Loan Sec. 8.5): A (row-major, symmetric) -> eigenvalues w
// ascending, eigenvectors as the columns of V.
__device__ __forceinline__ void eig3(float A[3][3], float w[3], float V[3][3])
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) V[r][c] = r == c ? 1.f : 0.f;
#pragma unroll 1
    for (int sweep = 0; sweep < 8; ++sweep) {
        const float off = fabsf(A[0][1]) + fabsf(A[0][2]) + fabsf(A[1][2]);
        const float scale = fabsf(A[0][0]) + fabsf(A[1][1]) + fabsf(A[2][2]);
        if (off <= 1e-9f * scale || off == 0.f) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            const float apq = A[p][q];
            if (apq == 0.f) continue;
            const float theta = (A[q][q] - A[p][p]) / (2.f * apq);
            const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float c = rsqrtf(t * t + 1.f), s = t * c;
            // A <- J^T A J with J the rotation in the (p, q) plane
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float akp = A[k][p], akq = A[k][q];
                A[k][p] = c * akp - s * akq;
                A[k][q] = s * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float apk = A[p][k], aqk = A[q][k];
                A[p][k] = c * apk - s * aqk;
                A[q][k] = s * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - s * vkq;
                V[k][q] = s * vkp + c * vkq;
            }
        }
    }
    w[0] = A[0][0];
    w[1] = A[1][1];
    w[2] = A[2][2];
    // sort ascending with the vectors
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2 - a; ++b)
            if (w[b] > w[b + 1]) {
                const float tw = w[b];
                w[b] = w[b + 1];
                w[b + 1] = tw;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float tv = V[k][b];
                    V[k][b] = V[k][b + 1];
                    V[k][b + 1] = tv;
                }
            }
}

// Inverse of a symmetric 3x3 (xx, xy, xz, yy, yz, zz) by its adjugate.
__device__ __forceinline__ void inv_sym3(const float S[6], float M[6])
{
    const float a = S[0], b = S[1], c = S[2], d = S[3], e = S[4], f = S[5];
    const float A = d * f - e * e, B = c * e - b * f, C = b * e - c * d;
    const float det = a * A + b * B + c * C;
    const float r = 1.f / det;
    M[0] = A * r;
    M[1] = B * r;
    M[2] = C * r;
    M[3] = (a * f - c * c) * r;
    M[4] = (b * c - a * e) * r;
    M[5] = (a * d - b * b) * r;
}

// Exclusive prefix of per-block counts [0, upto) summed by the whole block.
__device__ int block_prefix(const int32_t *counts, int upto, int *red)
{
    int s = 0;
    for (int k = threadIdx.x; k < upto; k += blockDim.x) s += counts[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    __syncthreads();
    return tot;
}

// Exclusive scan of one int per thread across the block; returns the block total in *total.
__device__ int block_exclusive_scan(int v, int *red, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) red[warp] = x;
    __syncthreads();
    int base = 0, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if (w < warp) base += red[w];
        tot += red[w];
    }
    __syncthreads();
    *total = tot;
    return base + x - v;
}

}  // namespace

namespace {

// ------------------------------------------------------------------ selection
struct SelArgs {
    const float *depth;
    int32_t W, H, R, ncx, ncells;
    float fx, fy, cx, cy;
    float4 *pos;
    int32_t *pix;
    int32_t *count;
    int32_t capacity;
    int32_t *blk;
    GicpState *state;
};

__device__ __forceinline__ bool cell_valid(const SelArgs &a, int c, int *u, int *v, float *d)
{
    if (c >= a.ncells) return false;
    const int cy = c / a.ncx, cx = c - cy * a.ncx;
    *u = cx * a.R;
    *v = cy * a.R;
    *d = a.depth[(size_t)(*v) * a.W + *u];
    return *d > 0.f;
}

__global__ void __launch_bounds__(256) k_select_count(const __grid_constant__ SelArgs a)
{
    __shared__ int red[8];
    if (blockIdx.x == 0 && threadIdx.x == 0) a.state->status = 0;   // a new frame: fresh flags
    int n = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int u, v;
        float d;
        n += cell_valid(a, blockIdx.x * kSelBlock + threadIdx.x * 4 + k, &u, &v, &d) ? 1 : 0;
    }
    int total;
    block_exclusive_scan(n, red, &total);
    if (threadIdx.x == 0) a.blk[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) k_select_write(const __grid_constant__ SelArgs a)
{
    __shared__ int red[8];
    const int prefix = block_prefix(a.blk, blockIdx.x, red);
    int u[4], v[4];
    float d[4];
    bool ok[4];
    int n = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ok[k] = cell_valid(a, blockIdx.x * kSelBlock + threadIdx.x * 4 + k, &u[k], &v[k], &d[k]);
        n += ok[k] ? 1 : 0;
    }
    int total;
    int o = prefix + block_exclusive_scan(n, red, &total);
    bool over = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!ok[k]) continue;
        if (o < a.capacity) {
            // p = d ((u - cx) / fx, (v - cy) / fy, 1), each step rounded as written
            const float x = __fmul_rn(d[k], __fdiv_rn(__fsub_rn((float)u[k], a.cx), a.fx));
            const float y = __fmul_rn(d[k], __fdiv_rn(__fsub_rn((float)v[k], a.cy), a.fy));
            a.pos[o] = make_float4(x, y, d[k], 0.f);
            if (a.pix) a.pix[o] = v[k] * a.W + u[k];
        } else {
            over = true;
        }
        ++o;
    }
    if (over) atomicOr(&a.state->status, 1);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *a.count = min(prefix + total, a.capacity);
}

// ------------------------------------------------------------------ team search
// Neighbour searches run one query per team of kTeam lanes of a warp: the lanes share the
// cells of each ring, keep their own sorted candidate lists, and rank their candidates
// among the team's through shared memory, which gives the exact team-wide k-th candidate
// after every ring (for the stopping proof) and the final sorted list.
constexpr int kTeam = 8;
constexpr int kRings = 6;                // rings searched before the exhaustive fallback

struct Grid {
    const int32_t *off;       // [table + 1] bucket offsets
    const float4 *pts;        // [indexed count] points sorted by bucket: x, y, z, index bits
    float inv_cell, cell;
    uint32_t mask;
};

__device__ __forceinline__ bool lex_less(float d1, int j1, float d2, int j2)
{
    return d1 < d2 || (d1 == d2 && j1 < j2);
}

__device__ __forceinline__ unsigned team_mask() { return 0xFFu << (threadIdx.x & 24); }

// Sorted insert into a lane's list (entries are unique: every point is seen once);
// (wd, wj) tracks the list's K-th entry for the early rejection.
template <int KMAX>
__device__ __forceinline__ void lane_insert(float d, int j, int K, float (&bd)[KMAX], int (&bj)[KMAX], float &wd,
                                            int &wj)
{
    if (!lex_less(d, j, wd, wj)) return;
    float cd = d;
    int cj = j;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < K && lex_less(cd, cj, bd[k], bj[k])) {
            const float td = bd[k];
            const int tj = bj[k];
            bd[k] = cd;
            bj[k] = cj;
            cd = td;
            cj = tj;
        }
        if (k == K - 1) {
            wd = bd[k];
            wj = bj[k];
        }
    }
}

// Calls f(q) for every point of the cells of ring r around (ix, iy, iz) that this lane
// owns (cube cells c = tl, tl + kTeam, ... with Chebyshev distance r). Points stored in
// a visited bucket but belonging to another cell (hash collisions) are skipped, so each
// point is seen once, in its own cell.
template <typename F>
__device__ __forceinline__ void team_ring(const Grid &g, int ix, int iy, int iz, int r, int tl, F &&f)
{
    const int side = 2 * r + 1, ncube = side * side * side;
#pragma unroll 1
    for (int c = tl; c < ncube; c += kTeam) {
        const int dx = c % side - r, dy = (c / side) % side - r, dz = c / (side * side) - r;
        if (max(abs(dx), max(abs(dy), abs(dz))) != r) continue;
        const int cx = ix + dx, cy = iy + dy, cz = iz + dz;
        const uint32_t h = cell_hash(cx, cy, cz, g.mask);
        const int e1 = g.off[h + 1];
#pragma unroll 1
        for (int e = g.off[h]; e < e1; ++e) {
            const float4 q = g.pts[e];
            if (cell_of(q.x, g.inv_cell) == cx && cell_of(q.y, g.inv_cell) == cy && cell_of(q.z, g.inv_cell) == cz)
                f(q);
        }
    }
}

// The team's K smallest (d, j) entries in order, merged from the lanes' sorted lists
// (copied to the team's shared-memory slots sd/sj [kTeam][KMAX]): K rounds of a team
// argmin over the lanes' heads. Writes out/outd [0, found) and returns found.
template <int KMAX>
__device__ __forceinline__ int team_select(const float (&bd)[KMAX], const int (&bj)[KMAX], int K, float *sd, int *sj,
                                           int tl, int *out, float *outd)
{
    const unsigned m = team_mask();
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
        if (k < K) {
            sd[tl * KMAX + k] = bd[k];
            sj[tl * KMAX + k] = bj[k];
        }
    __syncwarp(m);
    int head = 0;
    float hd = sd[tl * KMAX];
    int hj = sj[tl * KMAX];
    int found = 0;
#pragma unroll 1
    for (; found < K; ++found) {
        float md = hd;
        int mj = hj, ml = tl;
#pragma unroll
        for (int o = kTeam / 2; o > 0; o >>= 1) {
            const float od = __shfl_xor_sync(m, md, o, kTeam);
            const int oj = __shfl_xor_sync(m, mj, o, kTeam), ol = __shfl_xor_sync(m, ml, o, kTeam);
            if (lex_less(od, oj, md, mj) || (od == md && oj == mj && ol < ml)) {
                md = od;
                mj = oj;
                ml = ol;
            }
        }
        if (mj == INT_MAX) break;                             // the lanes hold no more entries
        if (tl == 0) {
            out[found] = mj;
            outd[found] = md;
        }
        if (tl == ml) {
            ++head;
            hd = head < K ? sd[tl * KMAX + head] : FLT_MAX;
            hj = head < K ? sj[tl * KMAX + head] : INT_MAX;
        }
    }
    __syncwarp(m);
    return found;
}

// K nearest points of `me` among the indexed ones (optionally within r_max): on return
// out[0 .. K) (team shared memory) holds their indices nearest first, -1 past the last
// found; returns the number found. `pos`/`n` serve the exhaustive fallback.
template <int KMAX>
__device__ int team_nearest(const Grid &g, float3 me, int K, float r_max, int max_rings, const float4 *pos, int n,
                            float *sd, int *sj, int *out, float *outd)
{
    const int tl = threadIdx.x & (kTeam - 1);
    float bd[KMAX];
    int bj[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        bd[k] = FLT_MAX;
        bj[k] = INT_MAX;
    }
    float wd = FLT_MAX;
    int wj = INT_MAX;
    const float r2 = r_max * r_max;
    const int ix = cell_of(me.x, g.inv_cell), iy = cell_of(me.y, g.inv_cell), iz = cell_of(me.z, g.inv_cell);
    int found = 0;
    bool proven = false;
#pragma unroll 1
    for (int r = 0; r <= max_rings && !proven; ++r) {
        team_ring(g, ix, iy, iz, r, tl, [&](float4 q) {
            const float d = sqdist(q.x, q.y, q.z, me.x, me.y, me.z);
            if (d <= r2) lane_insert<KMAX>(d, __float_as_int(q.w), K, bd, bj, wd, wj);
        });
        if (r == 0) continue;                               // nothing is proven at radius 0
        found = team_select<KMAX>(bd, bj, K, sd, sj, tl, out, outd);
        const float reach = (float)r * g.cell * (1.f - 1e-4f);
        // every point outside the searched rings lies at least `reach` away
        proven = reach >= r_max || (found == K && outd[K - 1] < reach * reach);
    }
    if (!proven) {                                          // exhaustive over the set, from scratch
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            bd[k] = FLT_MAX;
            bj[k] = INT_MAX;
        }
        wd = FLT_MAX;
        wj = INT_MAX;
#pragma unroll 1
        for (int j = tl; j < n; j += kTeam) {
            const float4 q = pos[j];
            const float d = sqdist(q.x, q.y, q.z, me.x, me.y, me.z);
            if (d <= r2) lane_insert<KMAX>(d, j, K, bd, bj, wd, wj);
        }
        found = team_select<KMAX>(bd, bj, K, sd, sj, tl, out, outd);
    }
    return found;
}

// ------------------------------------------------------------------ shapes
// One team per selected point: its K_c nearest selected points (FP32 squared distance,
// ties by index) from a ring search of the points' own hash grid, then (lane 0) the
// covariance, its eigen-decomposition and the normalised shape.
template <int KMAX>
__global__ void __launch_bounds__(128) k_shape(const float4 *__restrict__ pos, const int32_t *count, int K, float eps,
                                               Grid g, float4 *cov, float4 *normal, int32_t *knn_out)
{
    __shared__ float s_d[128 / kTeam][kTeam * KMAX];
    __shared__ int s_j[128 / kTeam][kTeam * KMAX];
    __shared__ int s_out[128 / kTeam][KMAX];
    __shared__ float s_outd[128 / kTeam][KMAX];
    const int kcov = K;
    const int n = *count;
    const int team = threadIdx.x / kTeam, tl = threadIdx.x & (kTeam - 1);
    const int i = blockIdx.x * (128 / kTeam) + team;
    if (i >= n) return;                                       // whole team
    K = min(K, n);                                            // fewer points than K_c: all of them
    const float4 me4 = pos[i];
    const float3 me = make_float3(me4.x, me4.y, me4.z);
    team_nearest<KMAX>(g, me, K, FLT_MAX, kRings, pos, n, s_d[team], s_j[team], s_out[team], s_outd[team]);
    const int *nb = s_out[team];
    if (knn_out)
        for (int k = tl; k < kcov; k += kTeam) knn_out[(size_t)i * kcov + k] = k < K ? nb[k] : -1;
    if (tl != 0) return;
    // covariance of the K neighbours (FP32): mean, then centred second moments
    float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        const float4 q = pos[nb[k]];
        mx += q.x;
        my += q.y;
        mz += q.z;
    }
    const float invk = 1.f / (float)K;
    mx *= invk;
    my *= invk;
    mz *= invk;
    float A[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        const float4 q = pos[nb[k]];
        const float dx = q.x - mx, dy = q.y - my, dz = q.z - mz;
        A[0][0] += dx * dx;
        A[0][1] += dx * dy;
        A[0][2] += dx * dz;
        A[1][1] += dy * dy;
        A[1][2] += dy * dz;
        A[2][2] += dz * dz;
    }
    A[0][0] *= invk;
    A[0][1] *= invk;
    A[0][2] *= invk;
    A[1][1] *= invk;
    A[1][2] *= invk;
    A[2][2] *= invk;
    A[1][0] = A[0][1];
    A[2][0] = A[0][2];
    A[2][1] = A[1][2];
    float w[3], V[3][3];
    eig3(A, w, V);
    float sc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sc[k] = sqrtf(fmaxf(w[k], 0.f));
    const float smax = sc[2];
    const float floor_s = sqrtf(eps);
#pragma unroll
    for (int k = 0; k < 3; ++k) sc[k] = fmaxf(smax > 0.f ? sc[k] / smax : 1.f, floor_s);
    float C[6];
    const int rr[6] = {0, 0, 0, 1, 1, 2}, cc[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) acc += V[rr[e]][k] * (sc[k] * sc[k]) * V[cc[e]][k];
        C[e] = acc;
    }
    cov[2 * i] = make_float4(C[0], C[1], C[2], C[3]);
    cov[2 * i + 1] = make_float4(C[4], C[5], 0.f, 0.f);
    normal[i] = make_float4(V[0][0], V[1][0], V[2][0], 0.f);
}

// ------------------------------------------------------------------ hash grid


__global__ void k_hash_count(const float4 *pos, const int32_t *count, float inv_cell, uint32_t mask, int32_t *cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const float4 p = pos[i];
    atomicAdd(&cnt[cell_hash(cell_of(p.x, inv_cell), cell_of(p.y, inv_cell), cell_of(p.z, inv_cell), mask)], 1);
}

// Exclusive offsets of the bucket counts in three parallel passes (tile sums, a scan of
// the tile sums, offsets within each tile); the counts are reset to 0 for use as fill
// cursors.
__global__ void __launch_bounds__(256) k_scan_tiles(const int32_t *cnt, int table, int32_t *tile_sums)
{
    __shared__ int red[8];
    const int b0 = blockIdx.x * kScanTile;
    int s = 0;
    for (int t = threadIdx.x; t < kScanTile; t += 256)
        if (b0 + t < table) s += cnt[b0 + t];
    int total;
    block_exclusive_scan(s, red, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(int32_t *tile_sums, int ntiles)
{
    __shared__ int red[32];
    int v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = threadIdx.x * 4 + k;
        v[k] = i < ntiles ? tile_sums[i] : 0;
        s += v[k];
    }
    int total;
    int o = block_exclusive_scan(s, red, &total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = threadIdx.x * 4 + k;
        if (i < ntiles) tile_sums[i] = o;
        o += v[k];
    }
}

__global__ void __launch_bounds__(256) k_scan_write(int32_t *cnt, int32_t *off, int table, const int32_t *tile_sums)
{
    __shared__ int red[8];
    const int b0 = blockIdx.x * kScanTile + threadIdx.x * 16;
    int v[16], s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[k] = b0 + k < table ? cnt[b0 + k] : 0;
        s += v[k];
    }
    int total;
    int o = tile_sums[blockIdx.x] + block_exclusive_scan(s, red, &total);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (b0 + k < table) {
            off[b0 + k] = o;
            cnt[b0 + k] = 0;
        }
        o += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 255) off[table] = o;
}

__global__ void k_hash_fill(const float4 *pos, const int32_t *count, float inv_cell, uint32_t mask,
                            const int32_t *off, int32_t *cnt, float4 *pts)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const float4 p = pos[i];
    const uint32_t h = cell_hash(cell_of(p.x, inv_cell), cell_of(p.y, inv_cell), cell_of(p.z, inv_cell), mask);
    pts[off[h] + atomicAdd(&cnt[h], 1)] = make_float4(p.x, p.y, p.z, __int_as_float(i));
}

// ------------------------------------------------------------------ Gauss-Newton step
struct StepArgs {
    const float4 *spos, *scov;
    const int32_t *scount;
    const float4 *mpos, *mcov, *mnorm;
    const int32_t *mcount;
    Grid grid;
    float r_max;
    int32_t kmatch;
    int32_t system;          // accumulate the Gauss-Newton system
    int32_t use_state;       // pose from the state (tracking) instead of `pose`
    GicpState *state;
    Pose12 pose;
    int32_t *idx_out;
    float *partial;          // [gridDim.x][32]
};

constexpr int kStepTeams = kStepThreads / kTeam;         // source points per block and round

__device__ void sum_partials(const float *partial, int nblocks, double *sys);
__device__ void solve_state(GicpState *st, const double *sys);

// The contribution of one correspondence to the Gauss-Newton system (H upper triangle,
// g = J^T M e, cost, count) in FP32.
__device__ __forceinline__ void gn_terms(const float *P, float3 x, float4 b, float4 cb0, float4 cb1, float4 ca0,
                                         float4 ca1, float (&acc)[kSys])
{
    const float Ca[3][3] = {{ca0.x, ca0.y, ca0.z}, {ca0.y, ca0.w, ca1.x}, {ca0.z, ca1.x, ca1.y}};
    const float R[3][3] = {{P[0], P[1], P[2]}, {P[4], P[5], P[6]}, {P[8], P[9], P[10]}};
    float RC[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) RC[r][c] = R[r][0] * Ca[0][c] + R[r][1] * Ca[1][c] + R[r][2] * Ca[2][c];
    float S[6];
    const int rr[6] = {0, 0, 0, 1, 1, 2}, cc[6] = {0, 1, 2, 1, 2, 2};
    const float cb[6] = {cb0.x, cb0.y, cb0.z, cb0.w, cb1.x, cb1.y};
#pragma unroll
    for (int e = 0; e < 6; ++e)
        S[e] = cb[e] + RC[rr[e]][0] * R[cc[e]][0] + RC[rr[e]][1] * R[cc[e]][1] + RC[rr[e]][2] * R[cc[e]][2];
    float Mi[6];
    inv_sym3(S, Mi);
    const float M[3][3] = {{Mi[0], Mi[1], Mi[2]}, {Mi[1], Mi[3], Mi[4]}, {Mi[2], Mi[4], Mi[5]}};
    const float e3[3] = {b.x - x.x, b.y - x.y, b.z - x.z};
    // J = [[x]_x, -I]
    const float J[3][6] = {{0.f, -x.z, x.y, -1.f, 0.f, 0.f}, {x.z, 0.f, -x.x, 0.f, -1.f, 0.f},
                           {-x.y, x.x, 0.f, 0.f, 0.f, -1.f}};
    float MJ[3][6];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) MJ[r][c] = M[r][0] * J[0][c] + M[r][1] * J[1][c] + M[r][2] * J[2][c];
    int t = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) acc[t++] += J[0][r] * MJ[0][c] + J[1][r] * MJ[1][c] + J[2][r] * MJ[2][c];
    float Me[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) Me[r] = M[r][0] * e3[0] + M[r][1] * e3[1] + M[r][2] * e3[2];
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[21 + c] += J[0][c] * Me[0] + J[1][c] * Me[1] + J[2][c] * Me[2];
    acc[27] += e3[0] * Me[0] + e3[1] * Me[1] + e3[2] * Me[2];
    acc[28] += 1.f;
}

// One team per source point (grid-stride over the points): the k_match nearest map
// Gaussians within r_max by a ring search of the map's grid (cells of r_max / 3, at most
// 3 rings), the smallest point-to-surface distance among them (ties by squared
// distance, then index), and that correspondence's Gauss-Newton terms, reduced per block.
__global__ void __launch_bounds__(kStepThreads) k_gicp_step(const __grid_constant__ StepArgs a)
{
    __shared__ float red[kStepThreads / 32][kSys + 3];
    __shared__ float s_d[kStepTeams][kTeam * kKMatchMax];
    __shared__ int s_j[kStepTeams][kTeam * kKMatchMax];
    __shared__ int s_out[kStepTeams][kKMatchMax];
    __shared__ float s_outd[kStepTeams][kKMatchMax];
    if (a.use_state && a.state->done) return;                  // uniform across the grid
    float P[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) P[k] = a.use_state ? a.state->posef[k] : a.pose.p[k];
    const int team = threadIdx.x / kTeam, tl = threadIdx.x & (kTeam - 1);
    const int n = *a.scount, nm = *a.mcount;
    const unsigned m = team_mask();
    float acc[kSys];
#pragma unroll
    for (int k = 0; k < kSys; ++k) acc[k] = 0.f;
#pragma unroll 1
    for (int base = blockIdx.x * kStepTeams; base < n; base += gridDim.x * kStepTeams) {
        const int i = base + team;
        if (i >= n) continue;                                  // whole team
        const float3 x = transform(P, a.spos[i]);
        const int found = team_nearest<kKMatchMax>(a.grid, x, a.kmatch, a.r_max, 3, a.mpos, nm, s_d[team], s_j[team],
                                                  s_out[team], s_outd[team]);
        // point-to-surface choice among the found candidates (lane k takes candidate k)
        float bm = FLT_MAX, bd2 = FLT_MAX;
        int bj = INT_MAX;
        if (tl < found) {
            const int j = s_out[team][tl];
            const float4 b = a.mpos[j], nr = a.mnorm[j];
            const float dx = __fsub_rn(b.x, x.x), dy = __fsub_rn(b.y, x.y), dz = __fsub_rn(b.z, x.z);
            bm = fabsf(__fadd_rn(__fadd_rn(__fmul_rn(nr.x, dx), __fmul_rn(nr.y, dy)), __fmul_rn(nr.z, dz)));
            bd2 = s_outd[team][tl];
            bj = j;
        }
#pragma unroll
        for (int o = kTeam / 2; o > 0; o >>= 1) {
            const float om = __shfl_xor_sync(m, bm, o, kTeam), od = __shfl_xor_sync(m, bd2, o, kTeam);
            const int oj = __shfl_xor_sync(m, bj, o, kTeam);
            if (om < bm || (om == bm && (od < bd2 || (od == bd2 && oj < bj)))) {
                bm = om;
                bd2 = od;
                bj = oj;
            }
        }
        const int jbest = found > 0 ? bj : -1;
        if (tl == 0) {
            if (a.idx_out) a.idx_out[i] = jbest;
            if (a.system && jbest >= 0)
                gn_terms(P, x, a.mpos[jbest], a.mcov[2 * jbest], a.mcov[2 * jbest + 1], a.scov[2 * i],
                         a.scov[2 * i + 1], acc);
        }
    }
    if (!a.system) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSys; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSys) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kStepThreads / 32; ++w) s += red[w][threadIdx.x];
        a.partial[blockIdx.x * 32 + threadIdx.x] = s;
    }
    if (!a.use_state) return;
    // tracking: the last block to finish sums the partials and takes the step
    __shared__ int s_last;
    __shared__ double sys[kSys];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&a.state->blocks_done, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    sum_partials(a.partial, gridDim.x, sys);
    if (threadIdx.x == 0) {
        solve_state(a.state, sys);
        a.state->blocks_done = 0;
    }
}

// Sum of the per-block partials in FP64 in a fixed order (warp w takes rows w, w + nw,
// ...; the warps' sums are added in warp order), so the result does not depend on
// scheduling. Partials are read through L2 (written by other blocks of the same grid).
__device__ void sum_partials(const float *partial, int nblocks, double *sys)
{
    __shared__ double part[8][kSys];                    // blocks of up to 256 threads
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, k = threadIdx.x & 31;
    if (k < kSys) {
        // eight independent sums keep eight row loads in flight; added in a fixed order
        double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int b = w;
        for (; b + 7 * nw < nblocks; b += 8 * nw) {
#pragma unroll
            for (int u = 0; u < 8; ++u) s[u] += (double)__ldcg(partial + (b + u * nw) * 32 + k);
        }
        for (int u = 0; b < nblocks; b += nw, ++u) s[u & 7] += (double)__ldcg(partial + b * 32 + k);
        part[w][k] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
    }
    __syncthreads();
    if (threadIdx.x < kSys) {
        double s = 0.0;
        for (int q = 0; q < nw; ++q) s += part[q][threadIdx.x];
        sys[threadIdx.x] = s;
    }
    __syncthreads();
}

__global__ void k_gicp_sum(const float *partial, int nblocks, double *out)
{
    __shared__ double sys[kSys];
    sum_partials(partial, nblocks, sys);
    if (threadIdx.x < kSys) out[threadIdx.x] = sys[threadIdx.x];
}

__device__ void exp_so3(const double w[3], double E[3][3])
{
    const double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    const double K[3][3] = {{0.0, -w[2], w[1]}, {w[2], 0.0, -w[0]}, {-w[1], w[0], 0.0}};
    double a, b;
    if (th < 1e-12) {
        a = 1.0;
        b = 0.5;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / (th * th);
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double kk = 0.0;
            for (int m = 0; m < 3; ++m) kk += K[r][m] * K[m][c];
            E[r][c] = (r == c ? 1.0 : 0.0) + a * K[r][c] + b * kk;
        }
}

// One thread: from the summed system, a Cholesky solve of H xi = -g in FP64 and the
// pose update (R, t) <- (Exp(omega) R, Exp(omega) t + v).
__device__ void solve_state(GicpState *st, const double *sys)
{
    st->n = (int)sys[28];
    st->cost = sys[27];
    if (sys[28] < 6.0) {
        st->status |= 2;
        st->done = 1;
        return;
    }
    double H[6][6], g[6];
    int t = 0;
    for (int r = 0; r < 6; ++r)
        for (int c = r; c < 6; ++c) {
            H[r][c] = sys[t];
            H[c][r] = sys[t];
            ++t;
        }
    for (int c = 0; c < 6; ++c) g[c] = sys[21 + c];
    // Cholesky H = L L^T
    double L[6][6] = {};
    for (int j = 0; j < 6; ++j) {
        double d = H[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0.0)) {
            st->status |= 2;
            st->done = 1;
            return;
        }
        L[j][j] = sqrt(d);
        for (int i = j + 1; i < 6; ++i) {
            double s = H[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            L[i][j] = s / L[j][j];
        }
    }
    double y[6], xi[6];
    for (int i = 0; i < 6; ++i) {
        double s = -g[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[k][i] * xi[k];
        xi[i] = s / L[i][i];
    }
    double E[3][3];
    exp_so3(xi, E);
    double Pn[12];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
            Pn[4 * r + c] = E[r][0] * st->pose[c] + E[r][1] * st->pose[4 + c] + E[r][2] * st->pose[8 + c];
        Pn[4 * r + 3] = E[r][0] * st->pose[3] + E[r][1] * st->pose[7] + E[r][2] * st->pose[11] + xi[3 + r];
    }
    for (int k = 0; k < 12; ++k) {
        st->pose[k] = Pn[k];
        st->posef[k] = (float)Pn[k];
    }
    double nrm = 0.0;
    for (int k = 0; k < 6; ++k) nrm += xi[k] * xi[k];
    st->step = sqrt(nrm);
    st->iters += 1;
    if (st->step < (double)st->tol) {
        st->converged = 1;
        st->done = 1;
    } else if (st->iters >= st->max_iters) {
        st->done = 1;
    }
}

__global__ void k_gicp_init(GicpState *st, PoseD p0, int keep_pose, int max_iters, float tol, int done)
{
    if (!keep_pose)
        for (int k = 0; k < 12; ++k) st->pose[k] = p0.p[k];
    for (int k = 0; k < 12; ++k) st->posef[k] = (float)st->pose[k];
    st->iters = 0;
    st->done = done;
    st->converged = 0;
    st->n = 0;
    st->cost = 0.0;
    st->step = 0.0;
    st->max_iters = max_iters;
    st->tol = tol;
    st->status &= 1;                 // keep the source's overflow flag, clear the rest
    st->blocks_done = 0;
}

// ------------------------------------------------------------------ map update
struct InsArgs {
    const float4 *spos, *scov, *snorm;
    const int32_t *scount;
    float4 *mpos, *mcov, *mnorm;
    int32_t *mcount;
    int32_t mcap;
    Grid grid;
    float d_ov;
    GicpState *state;
    int32_t *flags;
    int32_t *blk;
};

__device__ __forceinline__ bool overlaps(float3 x, const Grid &g, float d_ov)
{
    const float d2ov = d_ov * d_ov;
    const int ix = cell_of(x.x, g.inv_cell), iy = cell_of(x.y, g.inv_cell), iz = cell_of(x.z, g.inv_cell);
    // cells of a third of max(r_max, d_ov) >= d_ov / 3: the three rings reach d_ov
#pragma unroll 1
    for (int r = 0; r <= 3; ++r) {
        const int side = 2 * r + 1, ncube = side * side * side;
#pragma unroll 1
        for (int c = 0; c < ncube; ++c) {
            const int dx = c % side - r, dy = (c / side) % side - r, dz = c / (side * side) - r;
            if (max(abs(dx), max(abs(dy), abs(dz))) != r) continue;
            const uint32_t h = cell_hash(ix + dx, iy + dy, iz + dz, g.mask);
            const int e1 = g.off[h + 1];
#pragma unroll 1
            for (int e = g.off[h]; e < e1; ++e) {
                const float4 b = g.pts[e];
                if (sqdist(b.x, b.y, b.z, x.x, x.y, x.z) <= d2ov) return true;
            }
        }
        if ((float)r * g.cell * (1.f - 1e-4f) >= d_ov) break;
    }
    return false;
}

__global__ void __launch_bounds__(256) k_insert_flag(const __grid_constant__ InsArgs a)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    bool keep = false;
    if (i < *a.scount) {
        const float3 x = transform(a.state->posef, a.spos[i]);
        keep = *a.mcount == 0 || !overlaps(x, a.grid, a.d_ov);
        a.flags[i] = keep ? 1 : 0;
    }
    const int n = __syncthreads_count(keep);
    if (threadIdx.x == 0) a.blk[blockIdx.x] = n;
}

__global__ void __launch_bounds__(256) k_insert_write(const __grid_constant__ InsArgs a)
{
    __shared__ int red[8];
    const int prefix = block_prefix(a.blk, blockIdx.x, red);
    const int i = blockIdx.x * 256 + threadIdx.x;
    const int n = *a.scount;
    const bool keep = i < n && a.flags[i] != 0;
    int total;
    const int local = block_exclusive_scan(keep ? 1 : 0, red, &total);
    const int old = *a.mcount;
    if (keep) {
        const int o = old + prefix + local;
        if (o < a.mcap) {
            const float *P = a.state->posef;
            const float3 x = transform(P, a.spos[i]);
            const float R[3][3] = {{P[0], P[1], P[2]}, {P[4], P[5], P[6]}, {P[8], P[9], P[10]}};
            const float4 c0 = a.scov[2 * i], c1 = a.scov[2 * i + 1], nr = a.snorm[i];
            const float C[3][3] = {{c0.x, c0.y, c0.z}, {c0.y, c0.w, c1.x}, {c0.z, c1.x, c1.y}};
            float RC[3][3], W[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) RC[r][c] = R[r][0] * C[0][c] + R[r][1] * C[1][c] + R[r][2] * C[2][c];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) W[r][c] = RC[r][0] * R[c][0] + RC[r][1] * R[c][1] + RC[r][2] * R[c][2];
            a.mpos[o] = make_float4(x.x, x.y, x.z, 0.f);
            a.mcov[2 * o] = make_float4(W[0][0], W[0][1], W[0][2], W[1][1]);
            a.mcov[2 * o + 1] = make_float4(W[1][2], W[2][2], 0.f, 0.f);
            a.mnorm[o] = make_float4(R[0][0] * nr.x + R[0][1] * nr.y + R[0][2] * nr.z,
                                     R[1][0] * nr.x + R[1][1] * nr.y + R[1][2] * nr.z,
                                     R[2][0] * nr.x + R[2][1] * nr.y + R[2][2] * nr.z, 0.f);
        } else {
            atomicOr(&a.state->status, 1);
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        a.state->map_old = old;
        a.state->ins_total = prefix + total;
    }
}

__global__ void k_insert_commit(GicpState *st, int32_t *mcount, int32_t mcap)
{
    *mcount = min(st->map_old + st->ins_total, mcap);
}

}  // namespace

// ====================================================================== host entry points
namespace {

sgad_status fail(const char *msg) { return report_error(SGAD_ERR_INVALID_ARG, msg); }

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

sgad_status check_params(const sgad_gicp_params *p)
{
    if (!p) return fail("sgad_gicp: NULL params");
    if (p->stride < 1 || p->k_cov < 3 || p->k_cov > 32 || p->k_match < 1 || p->k_match > kKMatchMax ||
        p->max_iters < 1 || p->max_iters > 100 || !(p->r_max > 0.f) || !(p->d_overlap >= 0.f) || !(p->tol >= 0.f) ||
        !(p->eps > 0.f && p->eps <= 1.f) || !std::isfinite(p->r_max) || !std::isfinite(p->d_overlap) ||
        p->src_capacity < 1 || p->map_capacity < 1 || p->src_capacity > (1 << 24) || p->map_capacity > (1 << 24))
        return fail("sgad_gicp: parameter out of range");
    return SGAD_OK;
}

sgad_status check_set(const sgad_gaussian_set *s, int32_t max_capacity, const char *what)
{
    if (!s || !s->pos || !s->cov || !s->normal || !s->count || s->capacity < 1 || s->capacity > max_capacity)
        return fail(what);
    if (!aligned(s->pos, 16) || !aligned(s->cov, 16) || !aligned(s->normal, 16) || !aligned(s->count, 4))
        return fail(what);
    return SGAD_OK;
}

sgad_status check_ws(void *ws, size_t bytes, size_t need)
{
    if (!ws || !aligned(ws, 256)) return fail("sgad_gicp: workspace NULL or not 256-byte aligned");
    if (bytes < need) return report_error(SGAD_ERR_WORKSPACE_TOO_SMALL, "sgad_gicp: workspace too small");
    return SGAD_OK;
}

template <typename T>
T *at(void *ws, size_t off) { return reinterpret_cast<T *>(static_cast<char *>(ws) + off); }

// Map grid cells of a third of the larger search radius: correspondence and overlap
// searches visit rings of cells until their result is proven (at most 3 rings).
float cell_size(const sgad_gicp_params *p) { return fmaxf(p->r_max, p->d_overlap) * (1.001f / 3.f); }

Grid grid_of(const sgad_gicp_params *p, void *ws, const GLayout &L)
{
    Grid g;
    g.off = at<int32_t>(ws, L.hash_off);
    g.pts = at<float4>(ws, L.hash_pts);
    g.cell = cell_size(p);
    g.inv_cell = 1.f / g.cell;
    g.mask = (uint32_t)L.table - 1u;
    return g;
}

sgad_status launched(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SGAD_OK : report_error(SGAD_ERR_CUDA, what);
}

// Counting sort of a set's indices by the hash of their cells: counts, parallel scan,
// fill (entries within a bucket in arbitrary order; queries do not depend on it).
sgad_status hash_build(const float4 *pos, const int32_t *count, int32_t capacity, float inv_cell, int32_t table,
                       int32_t *cnt, int32_t *off, float4 *pts, int32_t *tile_sums, cudaStream_t st)
{
    if (cudaMemsetAsync(cnt, 0, (size_t)table * sizeof(int32_t), st) != cudaSuccess)
        return report_error(SGAD_ERR_CUDA, "sgad_gicp: memset failed");
    const uint32_t mask = (uint32_t)table - 1u;
    const int blocks = (capacity + 255) / 256;
    const int tiles = (table + kScanTile - 1) / kScanTile;
    k_hash_count<<<blocks, 256, 0, st>>>(pos, count, inv_cell, mask, cnt);
    k_scan_tiles<<<tiles, 256, 0, st>>>(cnt, table, tile_sums);
    k_scan_top<<<1, 1024, 0, st>>>(tile_sums, tiles);
    k_scan_write<<<tiles, 256, 0, st>>>(cnt, off, table, tile_sums);
    k_hash_fill<<<blocks, 256, 0, st>>>(pos, count, inv_cell, mask, off, cnt, pts);
    return launched("sgad_gicp: index launch failed");
}

sgad_status build_index(const sgad_gicp_params *p, const sgad_gaussian_set *map, void *ws, const GLayout &L,
                        cudaStream_t st)
{
    return hash_build(reinterpret_cast<const float4 *>(map->pos), map->count, map->capacity, 1.f / cell_size(p),
                      L.table, at<int32_t>(ws, L.hash_cnt), at<int32_t>(ws, L.hash_off), at<float4>(ws, L.hash_pts),
                      at<int32_t>(ws, L.tile_sums), st);
}

StepArgs step_args(const sgad_gicp_params *p, const sgad_gaussian_set *src, const sgad_gaussian_set *map, void *ws,
                   const GLayout &L)
{
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.spos = reinterpret_cast<const float4 *>(src->pos);
    a.scov = reinterpret_cast<const float4 *>(src->cov);
    a.scount = src->count;
    a.mpos = reinterpret_cast<const float4 *>(map->pos);
    a.mcov = reinterpret_cast<const float4 *>(map->cov);
    a.mnorm = reinterpret_cast<const float4 *>(map->normal);
    a.mcount = map->count;
    a.grid = grid_of(p, ws, L);
    a.r_max = p->r_max;
    a.kmatch = p->k_match;
    a.state = at<GicpState>(ws, L.state);
    a.partial = at<float>(ws, L.partial);
    return a;
}

}  // namespace

extern "C" sgad_status sgad_gicp_default_params(sgad_gicp_params *out)
{
    if (!out) return fail("sgad_gicp_default_params: NULL");
    out->stride = 10;
    out->k_cov = 10;
    out->k_match = 5;
    out->max_iters = 30;
    out->r_max = 0.1f;
    out->d_overlap = 0.02f;
    out->tol = 1e-6f;
    out->eps = 1e-3f;
    out->src_capacity = 1 << 16;
    out->map_capacity = 1 << 20;
    return SGAD_OK;
}

extern "C" sgad_status sgad_gicp_workspace_size(const sgad_gicp_params *p, size_t *bytes)
{
    sgad_status s = check_params(p);
    if (s) return s;
    if (!bytes) return fail("sgad_gicp_workspace_size: NULL");
    *bytes = glayout(*p).total;
    return SGAD_OK;
}

extern "C" sgad_status sgad_gicp_frame(const sgad_gicp_params *p, const sgad_camera *cam, const float *depth,
                                       const sgad_gaussian_set *out, int32_t *pix_out, int32_t *knn_out,
                                       void *workspace, size_t ws_bytes, void *stream)
{
    sgad_status s = check_params(p);
    if (s) return s;
    if ((s = check_set(out, p->src_capacity, "sgad_gicp_frame: bad output set"))) return s;
    if (!cam || !depth || cam->width < 1 || cam->height < 1 || !(cam->fx > 0.f) || !(cam->fy > 0.f))
        return fail("sgad_gicp_frame: bad camera or depth");
    const GLayout L = glayout(*p);
    if ((s = check_ws(workspace, ws_bytes, L.total))) return s;
    SelArgs a;
    a.depth = depth;
    a.W = cam->width;
    a.H = cam->height;
    a.R = p->stride;
    a.ncx = (cam->width + p->stride - 1) / p->stride;
    const long long ncells = (long long)a.ncx * ((cam->height + p->stride - 1) / p->stride);
    if (ncells > (long long)kMaxSelBlocks * kSelBlock) return fail("sgad_gicp_frame: too many selection cells");
    a.ncells = (int32_t)ncells;
    a.fx = cam->fx;
    a.fy = cam->fy;
    a.cx = cam->cx;
    a.cy = cam->cy;
    a.pos = reinterpret_cast<float4 *>(out->pos);
    a.pix = pix_out;
    a.count = out->count;
    a.capacity = out->capacity;
    a.blk = at<int32_t>(workspace, L.sel_counts);
    a.state = at<GicpState>(workspace, L.state);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = (int)((ncells + kSelBlock - 1) / kSelBlock);
    k_select_count<<<nb, 256, 0, st>>>(a);
    k_select_write<<<nb, 256, 0, st>>>(a);
    const float4 *pos = reinterpret_cast<const float4 *>(out->pos);
    // the points' own hash grid for the neighbour search; its cells are about twice the
    // selection spacing at 2 m (a performance choice only: the search proves its result)
    const float cell = fmaxf(5e-3f, 2.f * (float)p->stride * 2.f / cam->fx);
    Grid g;
    g.off = at<int32_t>(workspace, L.knn_off);
    g.pts = at<float4>(workspace, L.knn_pts);
    g.cell = cell;
    g.inv_cell = 1.f / cell;
    g.mask = (uint32_t)L.knn_table - 1u;
    if ((s = hash_build(pos, out->count, out->capacity, g.inv_cell, L.knn_table, at<int32_t>(workspace, L.knn_cnt),
                        at<int32_t>(workspace, L.knn_off), at<float4>(workspace, L.knn_pts),
                        at<int32_t>(workspace, L.tile_sums), st)))
        return s;
    const int sb = (out->capacity + (128 / kTeam) - 1) / (128 / kTeam);
    float4 *cov = reinterpret_cast<float4 *>(out->cov), *nrm = reinterpret_cast<float4 *>(out->normal);
    if (p->k_cov <= 8)
        k_shape<8><<<sb, 128, 0, st>>>(pos, out->count, p->k_cov, p->eps, g, cov, nrm, knn_out);
    else if (p->k_cov <= 16)
        k_shape<16><<<sb, 128, 0, st>>>(pos, out->count, p->k_cov, p->eps, g, cov, nrm, knn_out);
    else if (p->k_cov <= 24)
        k_shape<24><<<sb, 128, 0, st>>>(pos, out->count, p->k_cov, p->eps, g, cov, nrm, knn_out);
    else
        k_shape<32><<<sb, 128, 0, st>>>(pos, out->count, p->k_cov, p->eps, g, cov, nrm, knn_out);
    return launched("sgad_gicp_frame: launch failed");
}

extern "C" sgad_status sgad_gicp_index(const sgad_gicp_params *p, const sgad_gaussian_set *map, void *workspace,
                                       size_t ws_bytes, void *stream)
{
    sgad_status s = check_params(p);
    if (s) return s;
    if ((s = check_set(map, p->map_capacity, "sgad_gicp_index: bad map set"))) return s;
    const GLayout L = glayout(*p);
    if ((s = check_ws(workspace, ws_bytes, L.total))) return s;
    return build_index(p, map, workspace, L, static_cast<cudaStream_t>(stream));
}

namespace {
sgad_status pair_checks(const sgad_gicp_params *p, const sgad_gaussian_set *src, const sgad_gaussian_set *map,
                        void *ws, size_t bytes, GLayout *L)
{
    sgad_status s = check_params(p);
    if (s) return s;
    if ((s = check_set(src, p->src_capacity, "sgad_gicp: bad source set"))) return s;
    if ((s = check_set(map, p->map_capacity, "sgad_gicp: bad map set"))) return s;
    *L = glayout(*p);
    return check_ws(ws, bytes, L->total);
}

bool finite_pose(const float *P)
{
    for (int k = 0; k < 12; ++k)
        if (!std::isfinite(P[k])) return false;
    return true;
}
}  // namespace

extern "C" sgad_status sgad_gicp_correspond(const sgad_gicp_params *p, const sgad_gaussian_set *src,
                                            const sgad_gaussian_set *map, const float pose[12], int32_t *idx_out,
                                            void *workspace, size_t ws_bytes, void *stream)
{
    GLayout L;
    sgad_status s = pair_checks(p, src, map, workspace, ws_bytes, &L);
    if (s) return s;
    if (!pose || !idx_out || !finite_pose(pose)) return fail("sgad_gicp_correspond: bad pose or output");
    StepArgs a = step_args(p, src, map, workspace, L);
    std::memcpy(a.pose.p, pose, sizeof(a.pose.p));
    a.idx_out = idx_out;
    k_gicp_step<<<L.step_blocks, kStepThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return launched("sgad_gicp_correspond: launch failed");
}

extern "C" sgad_status sgad_gicp_linearize(const sgad_gicp_params *p, const sgad_gaussian_set *src,
                                           const sgad_gaussian_set *map, const float pose[12], double *system_out,
                                           void *workspace, size_t ws_bytes, void *stream)
{
    GLayout L;
    sgad_status s = pair_checks(p, src, map, workspace, ws_bytes, &L);
    if (s) return s;
    if (!pose || !system_out || !finite_pose(pose)) return fail("sgad_gicp_linearize: bad pose or output");
    StepArgs a = step_args(p, src, map, workspace, L);
    std::memcpy(a.pose.p, pose, sizeof(a.pose.p));
    a.system = 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_gicp_step<<<L.step_blocks, kStepThreads, 0, st>>>(a);
    k_gicp_sum<<<1, 32, 0, st>>>(a.partial, L.step_blocks, system_out);
    return launched("sgad_gicp_linearize: launch failed");
}

extern "C" sgad_status sgad_gicp_set_pose(const double pose[12], void *workspace, size_t ws_bytes, void *stream)
{
    if (!pose) return fail("sgad_gicp_set_pose: NULL pose");
    for (int k = 0; k < 12; ++k)
        if (!std::isfinite(pose[k])) return fail("sgad_gicp_set_pose: non-finite pose");
    sgad_status s = check_ws(workspace, ws_bytes, sizeof(GicpState));
    if (s) return s;
    PoseD p0;
    std::memcpy(p0.p, pose, sizeof(p0.p));
    k_gicp_init<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(at<GicpState>(workspace, 0), p0, 0, 0, 0.f, 1);
    return launched("sgad_gicp_set_pose: launch failed");
}

extern "C" sgad_status sgad_gicp_track(const sgad_gicp_params *p, const sgad_gaussian_set *src,
                                       const sgad_gaussian_set *map, const double pose0[12], void *workspace,
                                       size_t ws_bytes, void *stream)
{
    GLayout L;
    sgad_status s = pair_checks(p, src, map, workspace, ws_bytes, &L);
    if (s) return s;
    PoseD p0;
    std::memset(&p0, 0, sizeof(p0));
    if (pose0) {                              // else: start from the workspace's pose
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(pose0[k])) return fail("sgad_gicp_track: non-finite pose");
        std::memcpy(p0.p, pose0, sizeof(p0.p));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    StepArgs a = step_args(p, src, map, workspace, L);
    a.system = 1;
    a.use_state = 1;
    k_gicp_init<<<1, 1, 0, st>>>(a.state, p0, pose0 ? 0 : 1, p->max_iters, p->tol, 0);
    // one launch per iteration: each step's last block solves and updates the pose
    for (int it = 0; it < p->max_iters; ++it) {
        k_gicp_step<<<L.step_blocks, kStepThreads, 0, st>>>(a);
    }
    return launched("sgad_gicp_track: launch failed");
}

extern "C" sgad_status sgad_gicp_insert(const sgad_gicp_params *p, const sgad_gaussian_set *src,
                                        const sgad_gaussian_set *map, void *workspace, size_t ws_bytes, void *stream)
{
    GLayout L;
    sgad_status s = pair_checks(p, src, map, workspace, ws_bytes, &L);
    if (s) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    InsArgs a;
    a.spos = reinterpret_cast<const float4 *>(src->pos);
    a.scov = reinterpret_cast<const float4 *>(src->cov);
    a.snorm = reinterpret_cast<const float4 *>(src->normal);
    a.scount = src->count;
    a.mpos = reinterpret_cast<float4 *>(map->pos);
    a.mcov = reinterpret_cast<float4 *>(map->cov);
    a.mnorm = reinterpret_cast<float4 *>(map->normal);
    a.mcount = map->count;
    a.mcap = map->capacity;
    a.grid = grid_of(p, workspace, L);
    a.d_ov = p->d_overlap;
    a.state = at<GicpState>(workspace, L.state);
    a.flags = at<int32_t>(workspace, L.ins_flags);
    a.blk = at<int32_t>(workspace, L.ins_counts);
    k_insert_flag<<<L.max_blocks, 256, 0, st>>>(a);
    k_insert_write<<<L.max_blocks, 256, 0, st>>>(a);
    k_insert_commit<<<1, 1, 0, st>>>(a.state, map->count, map->capacity);
    if ((s = launched("sgad_gicp_insert: launch failed"))) return s;
    return build_index(p, map, workspace, L, st);
}

extern "C" sgad_status sgad_gicp_result(void *workspace, size_t ws_bytes, double pose[12], sgad_gicp_stats *stats,
                                        void *stream)
{
    sgad_status s = check_ws(workspace, ws_bytes, sizeof(GicpState));
    if (s) return s;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return report_error(SGAD_ERR_CUDA, "sgad_gicp_result: stream failed");
    GicpState h;
    if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return report_error(SGAD_ERR_CUDA, "sgad_gicp_result: copy failed");
    if (pose) std::memcpy(pose, h.pose, sizeof(h.pose));
    if (stats) {
        stats->iterations = h.iters;
        stats->converged = h.converged;
        stats->n_matches = h.n;
        stats->status = h.status;
        stats->cost = h.cost;
        stats->step = h.step;
    }
    return SGAD_OK;
}
