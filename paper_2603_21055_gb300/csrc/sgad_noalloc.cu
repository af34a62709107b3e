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

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
cudaError_t scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sgad_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sgad_status sgad_forward_noalloc(sgad_ctx *ctx, const sgad_keyframe *kfs, int32_t n_kf,
                                            const sgad_camera *views, int32_t n_views, sgad_images *out,
                                            void *stream)
{
    // Size of the problem with no keys, then the most keys the rest of the array holds
    // (each key takes 8 bytes in each of the two key arrays).
    size_t base = 0;
    sgad_status s = sgad_workspace_size(ctx, kfs, n_kf, views, n_views, 0, &base);
    if (s) return s;
    if (base + 4096 * 16 > (size_t)SGAD_NOALLOC_SCRATCH_BYTES)
        return sgad::report_error(SGAD_ERR_WORKSPACE_TOO_SMALL,
                                  "sgad_forward_noalloc: problem too large for the static scratch "
                                  "(SGAD_NOALLOC_SCRATCH_BYTES); use sgad_forward with a workspace");
    int64_t cap = (int64_t)(((size_t)SGAD_NOALLOC_SCRATCH_BYTES - base) / 16);
    size_t need = 0;
    while (cap > 0) {          // the per-section 256-byte rounding can cost a few keys
        s = sgad_workspace_size(ctx, kfs, n_kf, views, n_views, cap, &need);
        if (s) return s;
        if (need <= (size_t)SGAD_NOALLOC_SCRATCH_BYTES) break;
        cap -= 64;
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
