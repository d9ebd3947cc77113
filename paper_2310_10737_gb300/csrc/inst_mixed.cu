// inst_mixed.cu -- the mixed form: frames of codes with different n in one launch.
#include "kernels.cuh"

namespace sg {
template cudaError_t launch_product_mixed<uint32_t, 6>(const MixArgs &, int, cudaStream_t);
template cudaError_t launch_product_mixed<uint64_t, 6>(const MixArgs &, int, cudaStream_t);
}  // namespace sg
