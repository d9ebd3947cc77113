// inst_npl1_gen.cu -- general-geometry product kernels (two codes, or wrapped
// diagonals) for codes with 1..32 bits (1 bit(s) per lane).
#include "kernels.cuh"

namespace sg {
SG_INSTANTIATE_GEN(1, uint32_t)
SG_INSTANTIATE_GEN(1, uint64_t)
}  // namespace sg
