// ms_resident_inst1.cu -- rows 4..7 of the resident engine's variant table.
#include "ms_resident_kernels.cuh"

namespace ms {
template cudaError_t res_prep<4>(int, size_t, void**, int);
template cudaError_t res_prep<5>(int, size_t, void**, int);
template cudaError_t res_prep<6>(int, size_t, void**, int);
template cudaError_t res_prep<7>(int, size_t, void**, int);
}  // namespace ms
