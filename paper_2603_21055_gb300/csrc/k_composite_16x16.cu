// Compositing kernels for 16x16-pixel tiles, every batch size.
#include "k_composite.cuh"

namespace sgad {
template cudaError_t launch_composite_shape<16, 16>(bool, int, const Scene &, const CompositeArgs &, int, int *,
                                                   cudaStream_t);
template cudaError_t launch_bwdp<16, 16>(const Scene &, const CompositeArgs &, int, int *, cudaStream_t);
template cudaError_t launch_bwdl<16, 16>(const Scene &, const CompositeArgs &, int, int *, cudaStream_t);
}  // namespace sgad
