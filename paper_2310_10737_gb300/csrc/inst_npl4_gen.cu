// inst_npl4_gen.cu -- general-geometry product kernels (two codes, or wrapped
// diagonals) for codes with 65..128 bits (4 bit(s) per lane).
#include "kernels.cuh"

namespace sg {
SG_INSTANTIATE_GEN(4, uint32_t)
SG_INSTANTIATE_GEN(4, uint64_t)
}  // namespace sg
