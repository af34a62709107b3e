// Compositing kernels for 32x8-pixel tiles, every batch size.
#include "k_composite.cuh"

namespace sgad {
template cudaError_t launch_composite_shape<32, 8>(bool, int, const Scene &, const CompositeArgs &, int, int *,
                                                   cudaStream_t);
template cudaError_t launch_bwdp<32, 8>(const Scene &, const CompositeArgs &, int, int *, cudaStream_t);
template cudaError_t launch_bwdl<32, 8>(const Scene &, const CompositeArgs &, int, int *, cudaStream_t);
}  // namespace sgad
