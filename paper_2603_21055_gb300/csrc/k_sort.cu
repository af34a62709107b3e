// Per-tile depth sort (forward step a5).
//
// After binning every tile owns a contiguous bucket of 8-byte entries
// (f32 depth bits << 32 | global Gaussian index), in arbitrary order. Entries of one tile
// are distinct (a Gaussian is listed at most once per tile), so sorting them as unsigned
// 64-bit integers gives exactly the front-to-back order by (depth, index) with ties
// broken by the lower index; positive floats order like their bit patterns.
//
// One CTA per tile. Buckets up to `cap` entries are sorted in shared memory by a
// merge sort (per-thread insertion sort of a short run, then log2(threads) rounds of
// merge-path merging); larger buckets are sorted in cap-sized chunks the same way and
// then merged through global memory, ping-ponging with a scratch key array.
#include "sgad_device.cuh"

namespace sgad {

#ifndef SGAD_SORT_THREADS
#define SGAD_SORT_THREADS 512
#endif
constexpr int kSortThreads = SGAD_SORT_THREADS;

// Shared-memory index with one padding slot per 16 entries: each thread works on its own
// run of consecutive entries, and without padding the 64-bit accesses of lanes whose runs
// start 128 bytes apart would all hit the same two banks.
template <bool kPad>
__device__ __forceinline__ int pidx(int i)
{
    return kPad ? i + (i >> 4) : i;
}

template <bool kPad>
__device__ __forceinline__ void insertion_sort(uint64_t *a, int lo, int n)
{
    for (int i = 1; i < n; ++i) {
        const uint64_t x = a[pidx<kPad>(lo + i)];
        int j = i - 1;
        while (j >= 0 && a[pidx<kPad>(lo + j)] > x) {
            a[pidx<kPad>(lo + j + 1)] = a[pidx<kPad>(lo + j)];
            --j;
        }
        a[pidx<kPad>(lo + j + 1)] = x;
    }
}

// Merged positions [k0, k1) of the sorted runs src[a0 .. a0+la) and src[b0 .. b0+lb),
// written to dst[d0 + k0 .. d0 + k1) (indices before padding).
template <bool kPad>
__device__ __forceinline__ void merge_segment(const uint64_t *src, int a0, int la, int b0, int lb, int k0, int k1,
                                              uint64_t *dst, int d0)
{
    int lo = k0 - lb > 0 ? k0 - lb : 0;
    int hi = k0 < la ? k0 : la;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (src[pidx<kPad>(a0 + mid)] <= src[pidx<kPad>(b0 + k0 - 1 - mid)])
            lo = mid + 1;
        else
            hi = mid;
    }
    int i = lo, j = k0 - lo;
    uint64_t va = i < la ? src[pidx<kPad>(a0 + i)] : ~0ull;
    uint64_t vb = j < lb ? src[pidx<kPad>(b0 + j)] : ~0ull;
    for (int k = k0; k < k1; ++k) {
        const bool take_a = j >= lb || (i < la && va <= vb);
        if (take_a) {
            dst[pidx<kPad>(d0 + k)] = va;
            ++i;
            va = i < la ? src[pidx<kPad>(a0 + i)] : ~0ull;
        } else {
            dst[pidx<kPad>(d0 + k)] = vb;
            ++j;
            vb = j < lb ? src[pidx<kPad>(b0 + j)] : ~0ull;
        }
    }
}

// Sorts a[0..n) using b as scratch (both padded shared-memory buffers when kPad); returns
// the buffer holding the result.
template <bool kPad>
__device__ uint64_t *block_merge_sort(uint64_t *a, uint64_t *b, int n)
{
    const int T = blockDim.x;
    const int C = n > T ? (n + T - 1) / T : 1;
    const int lo = threadIdx.x * C;
    if (lo < n) insertion_sort<kPad>(a, lo, n - lo < C ? n - lo : C);
    __syncthreads();
    for (int w = C; w < n; w <<= 1) {
        const int k0 = threadIdx.x * C;
        if (k0 < n) {
            const int base = (k0 / (2 * w)) * (2 * w);
            const int la = n - base < w ? n - base : w;
            const int rest = n - base - la;
            const int lb = rest < w ? rest : w;
            int k1 = k0 + C;
            if (k1 > base + la + lb) k1 = base + la + lb;
            merge_segment<kPad>(a, base, la, base + la, lb, k0 - base, k1 - base, b, base);
        }
        __syncthreads();
        uint64_t *t = a;
        a = b;
        b = t;
    }
    return a;
}

__host__ __device__ constexpr int padded(int n) { return n + (n >> 4) + 16; }

__global__ void __launch_bounds__(kSortThreads) k_sort_tiles(const uint32_t *__restrict__ off,
                                                             uint64_t *__restrict__ entries,
                                                             uint64_t *__restrict__ alt, int cap,
                                                             const WsHeader *hdr)
{
    extern __shared__ uint64_t smem[];
    if (hdr->overflow) return;
    const int t = blockIdx.x;
    const uint32_t s = off[t];
    const int n = (int)(off[t + 1] - s);
    if (n <= 1) return;
    uint64_t *a = smem, *b = smem + padded(cap);
    uint64_t *gk = entries + s;
    if (n <= cap) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) a[pidx<true>(i)] = gk[i];
        __syncthreads();
        const uint64_t *r = block_merge_sort<true>(a, b, n);
        for (int i = threadIdx.x; i < n; i += blockDim.x) gk[i] = r[pidx<true>(i)];
        return;
    }
    // large bucket: sort cap-sized chunks in shared memory ...
    for (int c0 = 0; c0 < n; c0 += cap) {
        const int m = n - c0 < cap ? n - c0 : cap;
        for (int i = threadIdx.x; i < m; i += blockDim.x) a[pidx<true>(i)] = gk[c0 + i];
        __syncthreads();
        const uint64_t *r = block_merge_sort<true>(a, b, m);
        for (int i = threadIdx.x; i < m; i += blockDim.x) gk[c0 + i] = r[pidx<true>(i)];
        __syncthreads();
    }
    // ... then merge the sorted chunks through global memory
    uint64_t *src = gk, *dst = alt + s;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    for (int w = cap; w < n; w <<= 1) {
        const int k0 = threadIdx.x * per;
        const int kend = k0 + per < n ? k0 + per : n;
        for (int k = k0; k < kend;) {
            const int base = (k / (2 * w)) * (2 * w);
            const int la = n - base < w ? n - base : w;
            const int rest = n - base - la;
            const int lb = rest < w ? rest : w;
            const int seg_end = kend < base + la + lb ? kend : base + la + lb;
            merge_segment<false>(src, base, la, base + la, lb, k - base, seg_end - base, dst, base);
            k = seg_end;
        }
        __syncthreads();
        uint64_t *tmp = src;
        src = dst;
        dst = tmp;
    }
    if (src != gk)
        for (int i = threadIdx.x; i < n; i += blockDim.x) gk[i] = src[i];
}

cudaError_t launch_sort_tiles(const uint32_t *off, uint64_t *entries, uint64_t *alt, int n_tiles, int cap,
                              const WsHeader *hdr, cudaStream_t st)
{
    // Raise the kernel's dynamic shared-memory limit once per device and size (outside
    // any stream capture, which only replays launches).
    static int configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)padded(cap) * 2 * sizeof(uint64_t);
    if (dev < 0 || dev >= 64 || configured[dev] < (int)smem) {
        e = cudaFuncSetAttribute(k_sort_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = (int)smem;
    }
    if (n_tiles > 0) k_sort_tiles<<<n_tiles, kSortThreads, smem, st>>>(off, entries, alt, cap, hdr);
    return cudaSuccess;
}

}  // namespace sgad
