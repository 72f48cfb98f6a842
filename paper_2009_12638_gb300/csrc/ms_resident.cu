// ms_resident.cu -- host side of the resident engine: variant table
// queries, occupancy and the launchers of its sweep, async and persistent
// dataflow kernels (ms_resident_kernels.cuh; the rows are instantiated in the
// ms_resident_inst*.cu files).
#include <cuda_runtime.h>

#include "ms_internal.h"
#include "ms_resident_variants.h"

namespace ms {

static_assert(kNumResVariants == 21, "one case per variant row");

static cudaError_t res_fn(int variant, int cluster, size_t smem_bytes, void** fn, int am = 0) {
  switch (variant) {
    case 0: return res_prep<0>(cluster, smem_bytes, fn, am);
    case 1: return res_prep<1>(cluster, smem_bytes, fn, am);
    case 2: return res_prep<2>(cluster, smem_bytes, fn, am);
    case 3: return res_prep<3>(cluster, smem_bytes, fn, am);
    case 4: return res_prep<4>(cluster, smem_bytes, fn, am);
    case 5: return res_prep<5>(cluster, smem_bytes, fn, am);
    case 6: return res_prep<6>(cluster, smem_bytes, fn, am);
    case 7: return res_prep<7>(cluster, smem_bytes, fn, am);
    case 8: return res_prep<8>(cluster, smem_bytes, fn, am);
    case 9: return res_prep<9>(cluster, smem_bytes, fn, am);
    case 10: return res_prep<10>(cluster, smem_bytes, fn, am);
    case 11: return res_prep<11>(cluster, smem_bytes, fn, am);
    case 12: return res_prep<12>(cluster, smem_bytes, fn, am);
    case 13: return res_prep<13>(cluster, smem_bytes, fn, am);
    case 14: return res_prep<14>(cluster, smem_bytes, fn, am);
    case 15: return res_prep<15>(cluster, smem_bytes, fn, am);
    case 16: return res_prep<16>(cluster, smem_bytes, fn, am);
    case 17: return res_prep<17>(cluster, smem_bytes, fn, am);
    case 18: return res_prep<18>(cluster, smem_bytes, fn, am);
    case 19: return res_prep<19>(cluster, smem_bytes, fn, am);
    case 20: return res_prep<20>(cluster, smem_bytes, fn, am);
    default: return cudaErrorInvalidValue;
  }
}

int res_variant_count() { return kNumResVariants; }

void res_variant_info(int v, int* nt, int* kc, int* zs, int* ds, int* qr) {
  *nt = kResVariants[v].nt;
  *kc = kResVariants[v].kc;
  *zs = kResVariants[v].zs;
  *ds = kResVariants[v].ds;
  *qr = kResVariants[v].qr;
}

static void res_cfg(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at, int nt, int cluster, int slots, size_t smem,
                    cudaStream_t s) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3((unsigned)(cluster * slots), 1, 1);
  cfg->blockDim = dim3((unsigned)nt, 1, 1);
  cfg->dynamicSmemBytes = smem;
  cfg->stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg->attrs = at;
  cfg->numAttrs = 1;
}

cudaError_t res_max_clusters(int variant, int cluster, size_t smem_bytes, int* out, bool async_mode) {
  void* fn = nullptr;
  cudaError_t e = res_fn(variant, cluster, smem_bytes, &fn, async_mode ? 1 : 0);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  res_cfg(&cfg, at, kResVariants[variant].nt, cluster, 64, smem_bytes, nullptr);
  return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

cudaError_t launch_res_sweep(int variant, int cluster, int slots, size_t smem_bytes, const SweepArgs& a,
                             cudaStream_t s) {
  void* fn = nullptr;
  cudaError_t e = res_fn(variant, cluster, smem_bytes, &fn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  res_cfg(&cfg, at, kResVariants[variant].nt, cluster, slots, smem_bytes, s);
  const int smem_f4 = (int)(smem_bytes / 16);
  void* args[] = {(void*)&a, (void*)&smem_f4};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_res_async(int variant, int cluster, int slots, size_t smem_bytes, const AsyncArgs& a,
                             cudaStream_t s) {
  void* fn = nullptr;
  cudaError_t e = res_fn(variant, cluster, smem_bytes, &fn, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  res_cfg(&cfg, at, kResVariants[variant].nt, cluster, slots, smem_bytes, s);
  const int smem_f4 = (int)(smem_bytes / 16);
  void* args[] = {(void*)&a, (void*)&smem_f4};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_res_flow(int variant, int cluster, int slots, size_t smem_bytes, const FlowArgs& a,
                            cudaStream_t s) {
  void* fn = nullptr;
  cudaError_t e = res_fn(variant, cluster, smem_bytes, &fn, 2);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  res_cfg(&cfg, at, kResVariants[variant].nt, cluster, slots, smem_bytes, s);
  const int smem_f4 = (int)(smem_bytes / 16);
  void* args[] = {(void*)&a, (void*)&smem_f4};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t res_flow_max_clusters(int variant, int cluster, size_t smem_bytes, int* out) {
  void* fn = nullptr;
  cudaError_t e = res_fn(variant, cluster, smem_bytes, &fn, 2);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  res_cfg(&cfg, at, kResVariants[variant].nt, cluster, 64, smem_bytes, nullptr);
  return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

}  // namespace ms
