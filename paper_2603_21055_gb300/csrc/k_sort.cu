// Per-tile depth sort (forward step a5).
//
// After binning every tile owns a contiguous bucket of 8-byte entries
// (f32 depth bits << 32 | global Gaussian index), in arbitrary order. Entries of one tile
// are distinct (a Gaussian is listed at most once per tile), so sorting them as unsigned
// 64-bit integers gives exactly the front-to-back order by (depth, index) with ties
// broken by the lower index; positive floats order like their bit patterns.
//
// Default path (k_sort_tiles_bucket): one CTA per tile of up to 6,144 entries (and at
// most `cap`) sorts it in one pass through shared memory. The depth field minus the
// tile's smallest depth, shifted right so that the tile's range spans as many buckets as
// the power of two at or above its entry count (at most 4,096), picks each entry's
// bucket; a shared-memory atomic per entry gives both the bucket counts and each entry's
// slot in its bucket; after a scan of the counts every entry is written to its bucket,
// and then to its place in the list: the bucket's start plus the number of the bucket's
// entries below it in exact order (depth, then index), one thread per bucketed position.
// Buckets are small because the bucket width follows the tile's own depth range
// (room workload: at most ~20 entries). A tile with a bucket of more than kBucketMax
// entries (many equal or nearly equal depths), or with more entries than the bucket
// path holds, is listed and sorted afterwards by the exact radix sort below.
//
// Exact path (k_sort_tiles over the listed tiles): a bucket of up to `cap` entries is
// sorted in shared memory by a least-significant-digit radix sort on the depth field only: the bits that vary within
// the tile (depth bits minus the tile's smallest, 8 bits per pass, so a tile whose
// depths share their exponent needs three passes) are ranked stably, warp by warp, with
// one match per 32 entries. Equal depths then sit in runs in input order; each run is
// put in index order by one thread. A run longer than kRunMax (a tile of equal depths,
// e.g. a fronto-parallel plane seen from its own camera) sends the tile through the
// exact 64-bit LSD order instead: passes on the index field, then on the depth field.
// Larger buckets are sorted in cap-sized chunks the same way and then merged through
// global memory, ping-ponging with a scratch key array.
#include "sgad_device.cuh"

namespace sgad {

constexpr unsigned kFull32 = 0xffffffffu;
constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadixBins = 256;
constexpr int kCntStride = kSortWarps + 1;          // one padding word per digit row
constexpr int kCntWords = kRadixBins * kCntStride;
constexpr int kRunMax = 32;
static_assert(kRadixBins * kSortWarps == kSortThreads * 8, "the scan gives each thread 8 counters");

// Merged positions [k0, k1) of the sorted runs src[a0 .. a0+la) and src[b0 .. b0+lb),
// written to dst[d0 + k0 .. d0 + k1).
__device__ __forceinline__ void merge_segment(const uint64_t *src, int a0, int la, int b0, int lb, int k0, int k1,
                                              uint64_t *dst, int d0)
{
    int lo = k0 - lb > 0 ? k0 - lb : 0;
    int hi = k0 < la ? k0 : la;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (src[a0 + mid] <= src[b0 + k0 - 1 - mid])
            lo = mid + 1;
        else
            hi = mid;
    }
    int i = lo, j = k0 - lo;
    uint64_t va = i < la ? src[a0 + i] : ~0ull;
    uint64_t vb = j < lb ? src[b0 + j] : ~0ull;
    for (int k = k0; k < k1; ++k) {
        const bool take_a = j >= lb || (i < la && va <= vb);
        if (take_a) {
            dst[d0 + k] = va;
            ++i;
            va = i < la ? src[a0 + i] : ~0ull;
        } else {
            dst[d0 + k] = vb;
            ++j;
            vb = j < lb ? src[b0 + j] : ~0ull;
        }
    }
}

struct SortSmem {
    uint32_t cnt[kCntWords];       // per (digit, warp) counts, then their exclusive offsets
    uint32_t wsum[kSortWarps];
    uint32_t red[2][kSortWarps];   // block min / max scratch
    int flag;
};

__device__ __forceinline__ uint32_t field_of(uint64_t key, int field) { return (uint32_t)(key >> field); }

// Block-wide (min, max) of one 32-bit field over the valid registers; every thread
// returns the same pair. Ends with a barrier after the scratch is read.
template <int kPer>
__device__ __forceinline__ void field_range(const uint64_t (&k)[kPer], int C, int p0, int n, int field, SortSmem &s,
                                            uint32_t &mn, uint32_t &mx)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    mn = 0xffffffffu;
    mx = 0u;
#pragma unroll
    for (int r = 0; r < kPer; ++r)
        if (r < C && p0 + r * 32 < n) {
            const uint32_t f = field_of(k[r], field);
            mn = min(mn, f);
            mx = max(mx, f);
        }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        s.red[0][w] = mn;
        s.red[1][w] = mx;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortWarps; ++i) {
        mn = min(mn, s.red[0][i]);
        mx = max(mx, s.red[1][i]);
    }
    __syncthreads();
}

// One stable pass: entries move to ks in the order of digit ((field - base) >> shift) & 255,
// equal digits keeping the order of positions p = w * 32 C + r * 32 + lane. The caller's
// registers hold the entries at those positions; on return ks holds the pass's output.
template <int kPer>
__device__ __forceinline__ void radix_pass(uint64_t *ks, SortSmem &s, const uint64_t (&k)[kPer], int C, int p0, int n,
                                           int field, uint32_t base, int shift)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kCntWords; i += kSortThreads) s.cnt[i] = 0u;
    __syncthreads();
    // rank within the warp: earlier rounds' count of the digit + earlier lanes of this
    // round; kept with the digit as rank << 8 | digit
    uint32_t rd[kPer];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        if (r >= C) continue;
        const bool valid = p0 + r * 32 < n;
        const uint32_t d = valid ? ((field_of(k[r], field) - base) >> shift) & (kRadixBins - 1) : kRadixBins;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && lane == leader) {
            uint32_t *c = &s.cnt[d * kCntStride + w];
            old = *c;
            *c = old + __popc(peers);
        }
        rd[r] = ((__shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt)) << 8) | (d & (kRadixBins - 1));
    }
    __syncthreads();
    // exclusive scan of the counts in (digit, warp) order: thread t owns digit t / 2,
    // warps (t & 1) * 8 .. + 7
    {
        const int t = threadIdx.x;
        uint32_t *row = &s.cnt[(t >> 1) * kCntStride + (t & 1) * 8];
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            v[j] = row[j];
            sum += v[j];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s.wsum[w] = inc;
        __syncthreads();
        uint32_t run = inc - sum;
        for (int i = 0; i < w; ++i) run += s.wsum[i];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            row[j] = run;
            run += v[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        if (r < C && p0 + r * 32 < n) ks[s.cnt[(rd[r] & (kRadixBins - 1)) * kCntStride + w] + (rd[r] >> 8)] = k[r];
    }
    __syncthreads();
}

template <int kPer>
__device__ __forceinline__ void load_regs(const uint64_t *src, uint64_t (&k)[kPer], int C, int p0, int n)
{
#pragma unroll
    for (int r = 0; r < kPer; ++r)
        if (r < C && p0 + r * 32 < n) k[r] = src[p0 + r * 32];
}

// LSD passes over the bits of (field - min) that vary within the tile. On entry the
// registers hold the entries at positions p; on return ks holds them in the pass order
// (the registers are stale if any pass ran: `in_smem` tells the caller).
template <int kPer>
__device__ __forceinline__ void sort_field(uint64_t *ks, SortSmem &s, uint64_t (&k)[kPer], int C, int p0, int n, int field,
                           bool &in_smem)
{
    uint32_t mn, mx;
    field_range<kPer>(k, C, p0, n, field, s, mn, mx);
    const int bits = mx == mn ? 0 : 32 - __clz(mx - mn);
    for (int shift = 0; shift < bits; shift += 8) {
        if (in_smem) load_regs<kPer>(ks, k, C, p0, n);
        radix_pass<kPer>(ks, s, k, C, p0, n, field, mn, shift);
        in_smem = true;
    }
}

// Sorts the n <= kSortThreads * kPer entries of src into ks (shared memory), exactly by
// their 64-bit value. Phase 0 sorts by depth and orders runs of equal depth by index;
// a run longer than kRunMax sends the tile through phases 1 (index field) and 2 (depth
// field), the exact LSD order. One instance of the pass code serves every phase.
template <int kPer>
__device__ __forceinline__ void block_sort(const uint64_t *src, uint64_t *ks, SortSmem &s, int n)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int C = (n + kSortThreads - 1) / kSortThreads;
    const int p0 = w * 32 * C + lane;
    uint64_t k[kPer];
    load_regs<kPer>(src, k, C, p0, n);
    bool in_smem = false;
    for (int phase = 0;; ++phase) {
        if (phase > 0) load_regs<kPer>(ks, k, C, p0, n);
        sort_field<kPer>(ks, s, k, C, p0, n, phase == 1 ? 0 : 32, in_smem);
        if (phase == 1) continue;
        if (phase == 2) return;
        if (!in_smem) {
#pragma unroll
            for (int r = 0; r < kPer; ++r)
                if (r < C && p0 + r * 32 < n) ks[p0 + r * 32] = k[r];
            in_smem = true;
        }
        if (threadIdx.x == 0) s.flag = 0;
        __syncthreads();
        // runs of equal depth: find them (read only), then order each by index. Position
        // m of this thread (i = thread + m * threads) records (run length - 1) in 5 bits,
        // 0 if no run of 2 .. kRunMax entries starts there.
        constexpr int kCodes = (kPer + 5) / 6;
        uint32_t code[kCodes];
#pragma unroll
        for (int q = 0; q < kCodes; ++q) code[q] = 0u;
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
            const int i = threadIdx.x + m * kSortThreads;
            if (m < C && i + 1 < n) {
                const uint32_t h = field_of(ks[i], 32);
                if ((i == 0 || field_of(ks[i - 1], 32) != h) && field_of(ks[i + 1], 32) == h) {
                    int j = i + 2;
                    while (j < n && j - i <= kRunMax && field_of(ks[j], 32) == h) ++j;
                    if (j - i > kRunMax)
                        s.flag = 1;
                    else
                        code[m / 6] |= (uint32_t)(j - i - 1) << (5 * (m % 6));
                }
            }
        }
        __syncthreads();
        if (s.flag) continue;        // uniform: read after the barrier
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
            const int len = (int)((code[m / 6] >> (5 * (m % 6))) & 31u) + 1;
            if (len < 2) continue;
            uint64_t *a = ks + threadIdx.x + m * kSortThreads;
            for (int i = 1; i < len; ++i) {
                const uint64_t x = a[i];
                int j = i - 1;
                while (j >= 0 && a[j] > x) {
                    a[j + 1] = a[j];
                    --j;
                }
                a[j + 1] = x;
            }
        }
        __syncthreads();
        return;
    }
}

template <int kPer>
__device__ __forceinline__ void sort_tile_exact(const uint32_t *__restrict__ off, uint64_t *__restrict__ entries,
                                                uint64_t *__restrict__ alt, int cap, int t, SortSmem &s,
                                                uint64_t *ks);

// The tiles the bucket sort listed (hdr->n_sort_exact of them in `list`), taken by the
// blocks of a fixed grid in turn.
template <int kPer>
__global__ void __launch_bounds__(kSortThreads, kPer <= 12 ? 2 : 1)
    k_sort_tiles(const uint32_t *__restrict__ off, uint64_t *__restrict__ entries, uint64_t *__restrict__ alt, int cap,
                 const WsHeader *hdr, const uint32_t *__restrict__ list)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &s = *reinterpret_cast<SortSmem *>(smem_raw);
    uint64_t *ks = reinterpret_cast<uint64_t *>(smem_raw + ((sizeof(SortSmem) + 15) & ~size_t(15)));
    if (hdr->overflow) return;
    const uint32_t n_list = hdr->n_sort_exact;
    for (uint32_t k = blockIdx.x; k < n_list; k += gridDim.x) {
        sort_tile_exact<kPer>(off, entries, alt, cap, (int)list[k], s, ks);
        __syncthreads();
    }
}

template <int kPer>
__device__ __forceinline__ void sort_tile_exact(const uint32_t *__restrict__ off, uint64_t *__restrict__ entries,
                                                uint64_t *__restrict__ alt, int cap, int t, SortSmem &s,
                                                uint64_t *ks)
{
    const uint32_t s0 = off[t];
    const int n = (int)(off[t + 1] - s0);
    if (n <= 1) return;
    uint64_t *gk = entries + s0;
    // sort cap-sized chunks in shared memory ...
    for (int c0 = 0; c0 < n; c0 += cap) {
        const int m = n - c0 < cap ? n - c0 : cap;
        block_sort<kPer>(gk + c0, ks, s, m);
        for (int i = threadIdx.x; i < m; i += kSortThreads) gk[c0 + i] = ks[i];
        __syncthreads();
    }
    if (n <= cap) return;
    // ... then merge the sorted chunks through global memory
    uint64_t *src = gk, *dst = alt + s0;
    const int per = (n + kSortThreads - 1) / kSortThreads;
    for (int w = cap; w < n; w <<= 1) {
        const int k0 = threadIdx.x * per;
        const int kend = k0 + per < n ? k0 + per : n;
        for (int k = k0; k < kend;) {
            const int base = (k / (2 * w)) * (2 * w);
            const int la = n - base < w ? n - base : w;
            const int rest = n - base - la;
            const int lb = rest < w ? rest : w;
            const int seg_end = kend < base + la + lb ? kend : base + la + lb;
            merge_segment(src, base, la, base + la, lb, k - base, seg_end - base, dst, base);
            k = seg_end;
        }
        __syncthreads();
        uint64_t *tmp = src;
        src = dst;
        dst = tmp;
    }
    if (src != gk)
        for (int i = threadIdx.x; i < n; i += kSortThreads) gk[i] = src[i];
}

// ------------------------------------------------------------------ bucket sort
constexpr int kBucketThreads = 512;
constexpr int kBucketPer = 12;                          // entries per thread
constexpr int kBucketEntries = kBucketThreads * kBucketPer;
constexpr int kBucketBinsLog2 = 12;                     // at most 4,096 buckets
constexpr int kBucketMax = 64;                          // larger buckets: exact path

__global__ void __launch_bounds__(kBucketThreads, 3)
    k_sort_tiles_bucket(const uint32_t *__restrict__ off, uint64_t *__restrict__ entries, int cap, WsHeader *hdr,
                        uint32_t *__restrict__ list)
{
    __shared__ __align__(16) uint32_t start[1 << kBucketBinsLog2];    // bucket counts, then bucket starts
    __shared__ uint32_t red[2][kBucketThreads / 32];
    __shared__ int heavy;
    extern __shared__ uint64_t ks[];                     // the tile's entries, bucket by bucket
    if (hdr->overflow) return;
    const int t = blockIdx.x;
    const uint32_t s0 = off[t];
    const int n = (int)(off[t + 1] - s0);
    if (n <= 1) return;
    if (n > cap || n > kBucketEntries) {
        if (threadIdx.x == 0) list[atomicAdd(&hdr->n_sort_exact, 1u)] = (uint32_t)t;
        return;
    }
    const uint64_t *gk = entries + s0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // depth range of the tile
    uint32_t mn = 0xffffffffu, mx = 0u;
#pragma unroll
    for (int r = 0; r < kBucketPer; ++r) {
        const int i = threadIdx.x + r * kBucketThreads;
        if (i < n) {
            const uint32_t z = (uint32_t)(gk[i] >> 32);
            mn = min(mn, z);
            mx = max(mx, z);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(kFull32, mn, o));
        mx = max(mx, __shfl_xor_sync(kFull32, mx, o));
    }
    if (lane == 0) {
        red[0][w] = mn;
        red[1][w] = mx;
    }
    const int bins_log2 = min(kBucketBinsLog2, 32 - __clz(n - 1));     // 2^bins_log2 >= n
    const int nbins = 1 << bins_log2;
    for (int i = threadIdx.x; i < nbins; i += kBucketThreads) start[i] = 0u;
    if (threadIdx.x == 0) heavy = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kBucketThreads / 32; ++i) {
        mn = min(mn, red[0][i]);
        mx = max(mx, red[1][i]);
    }
    const int range_bits = mx == mn ? 0 : 32 - __clz(mx - mn);
    const int shift = range_bits > bins_log2 ? range_bits - bins_log2 : 0;
    // counts, and each entry's slot in its bucket
    uint32_t slot[kBucketPer];
#pragma unroll
    for (int r = 0; r < kBucketPer; ++r) {
        const int i = threadIdx.x + r * kBucketThreads;
        slot[r] = i < n ? atomicAdd(&start[((uint32_t)(gk[i] >> 32) - mn) >> shift], 1u) : 0u;
    }
    __syncthreads();
    // exclusive scan of the counts (each thread nbins / 512 or one consecutive bins, read
    // and written as 16-byte vectors when there are four or eight: conflict-free)
    {
        const int per = nbins > kBucketThreads ? nbins / kBucketThreads : 1;
        const int b0 = threadIdx.x * per;
        uint32_t v[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u}, sum = 0u;
        bool big = false;
        if (per >= 4) {
            const uint4 lo = reinterpret_cast<const uint4 *>(start + b0)[0];
            v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
            if (per == 8) {
                const uint4 hi = reinterpret_cast<const uint4 *>(start + b0)[1];
                v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < per && b0 + j < nbins) v[j] = start[b0 + j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            sum += v[j];
            big |= v[j] > (uint32_t)kBucketMax;
        }
        if (big) heavy = 1;
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull32, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) red[0][w] = inc;
        __syncthreads();
        uint32_t run = inc - sum;
        for (int i = 0; i < w; ++i) run += red[0][i];
        uint32_t o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            o[j] = run;
            run += v[j];
        }
        if (per >= 4) {
            reinterpret_cast<uint4 *>(start + b0)[0] = make_uint4(o[0], o[1], o[2], o[3]);
            if (per == 8) reinterpret_cast<uint4 *>(start + b0)[1] = make_uint4(o[4], o[5], o[6], o[7]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < per && b0 + j < nbins) start[b0 + j] = o[j];
        }
    }
    __syncthreads();
    if (heavy) {                                         // uniform: read after the barrier
        if (threadIdx.x == 0) list[atomicAdd(&hdr->n_sort_exact, 1u)] = (uint32_t)t;
        return;
    }
#pragma unroll
    for (int r = 0; r < kBucketPer; ++r) {
        const int i = threadIdx.x + r * kBucketThreads;
        if (i < n) {
            const uint64_t key = gk[i];
            ks[start[((uint32_t)(key >> 32) - mn) >> shift] + slot[r]] = key;
        }
    }
    __syncthreads();
    // exact 64-bit order (depth, then index) inside each bucket: an entry's place is its
    // bucket's start plus the number of the bucket's entries below it (the entries of a
    // tile are distinct, so the places are too), written straight to the list. Threads
    // take consecutive bucketed positions, so the lanes of one bucket read the same words.
    uint64_t *out = entries + s0;
    for (int i = threadIdx.x; i < n; i += kBucketThreads) {
        const uint64_t key = ks[i];
        const uint32_t b = ((uint32_t)(key >> 32) - mn) >> shift;
        const int lo = (int)start[b], hi = b + 1 < (uint32_t)nbins ? (int)start[b + 1] : n;
        int r = lo;
#pragma unroll 4
        for (int j = lo; j < hi; ++j) r += ks[j] < key ? 1 : 0;
        out[r] = key;
    }
}

template <int kPer>
static cudaError_t launch_sort(const uint32_t *off, uint64_t *entries, uint64_t *alt, int n_tiles, int cap,
                               WsHeader *hdr, uint32_t *list, cudaStream_t st)
{
    // Raise the kernel's dynamic shared-memory limit once per device and size (outside
    // any stream capture, which only replays launches).
    static int configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t smem = ((sizeof(SortSmem) + 15) & ~size_t(15)) + (size_t)cap * sizeof(uint64_t);
    if (dev < 0 || dev >= 64 || configured[dev] < (int)smem) {
        e = cudaFuncSetAttribute(k_sort_tiles<kPer>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = (int)smem;
    }
    static int bucket_configured[64] = {};
    constexpr int bucket_smem = kBucketEntries * (int)sizeof(uint64_t);
    if (dev < 0 || dev >= 64 || !bucket_configured[dev]) {
        e = cudaFuncSetAttribute(k_sort_tiles_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, bucket_smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) bucket_configured[dev] = 1;
    }
    if (n_tiles <= 0) return cudaSuccess;
    k_sort_tiles_bucket<<<n_tiles, kBucketThreads, bucket_smem, st>>>(off, entries, cap, hdr, list);
    // the listed tiles: a fixed grid (two blocks per SM) so the launch can be captured
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = n_tiles < 2 * sms ? n_tiles : 2 * sms;
    k_sort_tiles<kPer><<<grid, kSortThreads, smem, st>>>(off, entries, alt, cap, hdr, list);
    return cudaSuccess;
}

// cap in [64, 12288] (checked by the caller). list: n_tiles words of workspace for the
// tiles the bucket sort hands to the exact radix sort (counted in hdr->n_sort_exact,
// which the forward clears).
cudaError_t launch_sort_tiles(const uint32_t *off, uint64_t *entries, uint64_t *alt, int n_tiles, int cap,
                              WsHeader *hdr, uint32_t *list, cudaStream_t st)
{
    if (cap <= kSortThreads * 12) return launch_sort<12>(off, entries, alt, n_tiles, cap, hdr, list, st);
    return launch_sort<24>(off, entries, alt, n_tiles, cap, hdr, list, st);
}

}  // namespace sgad
