// inst_npl4.cu -- kernels for codes with 65..128 bits (4 bit(s) per lane).
#include "kernels.cuh"

namespace sg {
SG_INSTANTIATE(4, uint32_t)
SG_INSTANTIATE(4, uint64_t)
}  // namespace sg
