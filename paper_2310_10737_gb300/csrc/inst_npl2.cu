// inst_npl2.cu -- kernels for codes with 33..64 bits (2 bit(s) per lane).
#include "kernels.cuh"

namespace sg {
SG_INSTANTIATE(2, uint32_t)
SG_INSTANTIATE(2, uint64_t)
}  // namespace sg
