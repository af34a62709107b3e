// Forward splatting without any allocation, for callers that cannot allocate device
// memory: for example code running inside a host callback or a real-time loop where
// cudaMalloc would block the device, an embedding application whose memory manager
// owns every device allocation, or a plug-in that is handed its input and output buffers
// and nothing else. The paper has no counterpart; this is an interface convenience.
//
// The scratch that sgad_forward() normally takes from the caller's workspace lives here
// in one file-scope device array. Every GPU that loads this library holds the array
// (SGAD_NOALLOC_SCRATCH_BYTES) until the process exits.
#include <mutex>

#include "sgad_device.cuh"

// The array itself. In host code this name is only a stand-in for the symbol: its
// device address must be obtained with cudaGetSymbolAddress() on the device in use.
static __device__ __align__(256) unsigned char g_sgad_noalloc_scratch[SGAD_NOALLOC_SCRATCH_BYTES];

namespace sgad {
sgad_status report_error(sgad_status code, const char *msg);
}

namespace {

// Device address of the array in the current device's context. Looked up on every call
// (a host-side lookup, no device work): a pointer cached across calls could outlive the
// context it came from (after cudaDeviceReset the module is loaded again, possibly at
// another address).
cudaError_t scratch_address(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sgad_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

// Bytes of workspace each key adds (make_layout: 8 B in each of the two key arrays, 32 B
// of pair-parallel contribution words and 1 B of per-warp masks), and the most the
// 256-byte alignment of those four sections can add on top.
constexpr size_t kBytesPerKey = 8 + 8 + 32 + 1;
constexpr size_t kKeySectionSlack = 4 * 256;

}  // namespace

extern "C" sgad_status sgad_forward_noalloc(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                                            const sgad_camera *views, int32_t n_views, sgad_images *out,
                                            void *stream)
{
    // Size of the problem with no keys, then the most keys the rest of the array holds,
    // in closed form from the per-key bytes of the layout (checked once, and trimmed by
    // a bounded bisection should the layout ever need more).
    const size_t kScratch = SGAD_NOALLOC_SCRATCH_BYTES;
    size_t base = 0;
    sgad_status s = sgad_workspace_size(ctx, kfs, n_kf, views, n_views, 0, &base);
    if (s) return s;
    const int64_t kMinKeys = 4096;
    if (base + kKeySectionSlack + (size_t)kMinKeys * kBytesPerKey > kScratch)
        return sgad::report_error(SGAD_ERR_WORKSPACE_TOO_SMALL,
                                  "sgad_forward_noalloc: problem too large for the static scratch "
                                  "(SGAD_NOALLOC_SCRATCH_BYTES); use sgad_forward with a workspace");
    int64_t cap = (int64_t)((kScratch - base - kKeySectionSlack) / kBytesPerKey);
    size_t need = 0;
    s = sgad_workspace_size(ctx, kfs, n_kf, views, n_views, cap, &need);
    if (s) return s;
    if (need > kScratch) {     // [lo fits, hi does not]
        int64_t lo = kMinKeys, hi = cap;
        for (int it = 0; it < 40 && hi - lo > 1; ++it) {
            const int64_t mid = lo + (hi - lo) / 2;
            s = sgad_workspace_size(ctx, kfs, n_kf, views, n_views, mid, &need);
            if (s) return s;
            (need <= kScratch ? lo : hi) = mid;
        }
        cap = lo;
    }
    void *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return sgad::report_error(SGAD_ERR_CUDA, "sgad_forward_noalloc: cudaGetSymbolAddress failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: clear the status block (the rest is
    // overwritten or cleared by the forward pass itself).
    e = cudaMemsetAsync(scratch, 0, sizeof(sgad::WsHeader), st);
    if (e != cudaSuccess) return sgad::report_error(SGAD_ERR_CUDA, "sgad_forward_noalloc: cudaMemsetAsync failed");
    s = sgad_forward(ctx, kfs, n_kf, views, n_views, out, scratch, SGAD_NOALLOC_SCRATCH_BYTES, cap, stream);
    if (s) return s;
    // Report a key overflow now: the caller has no workspace to ask later.
    return sgad_check(ctx, scratch, SGAD_NOALLOC_SCRATCH_BYTES, nullptr, nullptr, stream);
}
