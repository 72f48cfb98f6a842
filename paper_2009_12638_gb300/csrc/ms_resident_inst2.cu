// ms_resident_inst2.cu -- rows 8..11 of the resident engine's variant table.
#include "ms_resident_kernels.cuh"

namespace ms {
template cudaError_t res_prep<8>(int, size_t, void**, int);
template cudaError_t res_prep<9>(int, size_t, void**, int);
template cudaError_t res_prep<10>(int, size_t, void**, int);
template cudaError_t res_prep<11>(int, size_t, void**, int);
}  // namespace ms
