// ms_resident_inst4.cu -- rows 16..18 of the resident engine's variant table
// (single-reduction CG).
#include "ms_resident_kernels.cuh"

namespace ms {
template cudaError_t res_prep<16>(int, size_t, void**, int);
template cudaError_t res_prep<17>(int, size_t, void**, int);
template cudaError_t res_prep<18>(int, size_t, void**, int);
}  // namespace ms
