// Compositing kernels for 8x32-pixel tiles, every batch size.
#include "k_composite.cuh"

namespace sgad {
template cudaError_t launch_composite_shape<8, 32>(bool, int, const Scene &, const CompositeArgs &, int, int *,
                                                   cudaStream_t);
template cudaError_t launch_bwdp<8, 32>(const Scene &, const CompositeArgs &, int, int *, cudaStream_t);
template cudaError_t launch_bwdl<8, 32>(const Scene &, const CompositeArgs &, int, int *, cudaStream_t);
}  // namespace sgad
