// inst_npl1.cu -- kernels for codes with up to 32 bits (1 bit(s) per lane).
#include "kernels.cuh"

namespace sg {
SG_INSTANTIATE(1, uint32_t)
SG_INSTANTIATE(1, uint64_t)
}  // namespace sg
