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

constexpr int kSortThreads = 512;

__device__ __forceinline__ void insertion_sort(uint64_t *a, int n)
{
    for (int i = 1; i < n; ++i) {
        const uint64_t x = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > x) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = x;
    }
}

// Merged positions [k0, k1) of sorted runs A[0..la) and B[0..lb), written to out[k0..k1).
__device__ __forceinline__ void merge_segment(const uint64_t *A, int la, const uint64_t *B, int lb, int k0, int k1,
                                              uint64_t *out)
{
    int lo = k0 - lb > 0 ? k0 - lb : 0;
    int hi = k0 < la ? k0 : la;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid] <= B[k0 - 1 - mid])
            lo = mid + 1;
        else
            hi = mid;
    }
    int i = lo, j = k0 - lo;
    for (int k = k0; k < k1; ++k) {
        const bool take_a = j >= lb || (i < la && A[i] <= B[j]);
        out[k] = take_a ? A[i++] : B[j++];
    }
}

// Sorts a[0..n) (n <= blockDim * C for the C computed here) using b as scratch; returns
// the buffer holding the result. Works on shared or global pointers.
__device__ uint64_t *block_merge_sort(uint64_t *a, uint64_t *b, int n)
{
    const int T = blockDim.x;
    const int C = n > T ? (n + T - 1) / T : 1;
    const int lo = threadIdx.x * C;
    if (lo < n) insertion_sort(a + lo, n - lo < C ? n - lo : C);
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
            merge_segment(a + base, la, a + base + la, lb, k0 - base, k1 - base, b + base);
        }
        __syncthreads();
        uint64_t *t = a;
        a = b;
        b = t;
    }
    return a;
}

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
    uint64_t *a = smem, *b = smem + cap;
    uint64_t *gk = entries + s;
    if (n <= cap) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = gk[i];
        __syncthreads();
        const uint64_t *r = block_merge_sort(a, b, n);
        for (int i = threadIdx.x; i < n; i += blockDim.x) gk[i] = r[i];
        return;
    }
    // large bucket: sort cap-sized chunks in shared memory ...
    for (int c0 = 0; c0 < n; c0 += cap) {
        const int m = n - c0 < cap ? n - c0 : cap;
        for (int i = threadIdx.x; i < m; i += blockDim.x) a[i] = gk[c0 + i];
        __syncthreads();
        const uint64_t *r = block_merge_sort(a, b, m);
        for (int i = threadIdx.x; i < m; i += blockDim.x) gk[c0 + i] = r[i];
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
            merge_segment(src + base, la, src + base + la, lb, k - base, seg_end - base, dst + base);
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
    const size_t smem = (size_t)cap * 2 * sizeof(uint64_t);
    if (dev < 0 || dev >= 64 || configured[dev] < (int)smem) {
        e = cudaFuncSetAttribute(k_sort_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = (int)smem;
    }
    if (n_tiles > 0) k_sort_tiles<<<n_tiles, kSortThreads, smem, st>>>(off, entries, alt, cap, hdr);
    return cudaSuccess;
}

}  // namespace sgad
