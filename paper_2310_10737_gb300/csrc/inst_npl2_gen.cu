// inst_npl2_gen.cu -- general-geometry product kernels (two codes, or wrapped
// diagonals) for codes with 33..64 bits (2 bit(s) per lane).
#include "kernels.cuh"

namespace sg {
SG_INSTANTIATE_GEN(2, uint32_t)
SG_INSTANTIATE_GEN(2, uint64_t)
}  // namespace sg
