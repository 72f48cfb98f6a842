// ms_resident_inst0.cu -- rows 0..3 of the resident engine's variant table.
#include "ms_resident_kernels.cuh"

namespace ms {
template cudaError_t res_prep<0>(int, size_t, void**, int);
template cudaError_t res_prep<1>(int, size_t, void**, int);
template cudaError_t res_prep<2>(int, size_t, void**, int);
template cudaError_t res_prep<3>(int, size_t, void**, int);
}  // namespace ms
