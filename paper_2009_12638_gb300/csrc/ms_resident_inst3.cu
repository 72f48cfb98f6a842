// ms_resident_inst3.cu -- rows 12..15 of the resident engine's variant table.
#include "ms_resident_kernels.cuh"

namespace ms {
template cudaError_t res_prep<12>(int, size_t, void**, int);
template cudaError_t res_prep<13>(int, size_t, void**, int);
template cudaError_t res_prep<14>(int, size_t, void**, int);
template cudaError_t res_prep<15>(int, size_t, void**, int);
}  // namespace ms
