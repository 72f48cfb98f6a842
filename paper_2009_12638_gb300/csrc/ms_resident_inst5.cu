// ms_resident_inst5.cu -- rows 19..20 of the resident engine's variant table
// (single-reduction CG).
#include "ms_resident_kernels.cuh"

namespace ms {
template cudaError_t res_prep<19>(int, size_t, void**, int);
template cudaError_t res_prep<20>(int, size_t, void**, int);
}  // namespace ms
