// inst_mixed8.cu -- the mixed form compiled for 8 resident blocks per SM (64
// registers a thread), for mixes whose codes all run that schedule.
#include "kernels.cuh"

namespace sg {
template cudaError_t launch_product_mixed<uint32_t, 8>(const MixArgs &, int, cudaStream_t);
}  // namespace sg
