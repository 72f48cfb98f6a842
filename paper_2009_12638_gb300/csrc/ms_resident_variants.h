// ms_resident_variants.h -- the resident engine's table of on-chip layouts
// (see ms_resident.cuh) and the per-row preparation entry res_prep<V>.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace ms {

// ---------------------------------------------------------------- variants
// (NT threads, KC strips per thread, ZS planes per CTA at most, d in shared
// memory, qr: 0 = two stencils per CG iteration, 1 = q = A p kept in
// registers between passes A and B, 2 = the single-reduction CG, which keeps
// p, s = A p and w = A r in registers and needs d in shared memory)
struct ResVariant {
  int nt, kc, zs, ds, qr;
};
constexpr ResVariant kResVariants[] = {
    {512, 2, 4, 0, 0},  {512, 1, 8, 0, 0},  {256, 2, 4, 0, 0},  {256, 1, 8, 0, 0},  {512, 4, 2, 0, 0},
    {1024, 1, 4, 1, 0}, {1024, 2, 2, 1, 0}, {1024, 1, 8, 1, 0}, {512, 2, 4, 1, 0},  {512, 2, 4, 0, 1},
    {512, 1, 8, 0, 1},  {256, 2, 4, 0, 1},  {256, 1, 8, 0, 1},  {512, 2, 4, 1, 1},  {512, 4, 2, 0, 1},
    {1024, 1, 4, 1, 1}, {512, 2, 4, 1, 2},  {256, 1, 8, 1, 2},  {256, 2, 4, 1, 2},  {512, 1, 8, 1, 2},
    {1024, 1, 4, 1, 2}};
constexpr int kNumResVariants = sizeof(kResVariants) / sizeof(kResVariants[0]);


// floats of dynamic shared memory: p (zs + 2 planes), 2 r-halo planes, and
// (d_in_smem) d as zs compact planes of 4*spr*by floats.
__host__ __device__ inline long long res_smem_floats(int bx, int by, int zs, bool d_in_smem) {
  const long long spr = (bx + 3) / 4;
  const long long rp = 4 * spr + 4;
  const long long ps = (by + 2) * rp + 4;  // + the right pad of the last row
  return (zs + 4) * ps + (d_in_smem ? zs * 4 * spr * by : 0);
}

// Sets the kernel attributes of row V for one launch kind (0 sweep, 1 async,
// 2 persistent dataflow) and returns its kernel in *fn.  Defined in
// ms_resident_kernels.cuh, instantiated in the ms_resident_inst*.cu files.
template <int V>
cudaError_t res_prep(int cluster, size_t smem_bytes, void** fn, int kind);

}  // namespace ms
