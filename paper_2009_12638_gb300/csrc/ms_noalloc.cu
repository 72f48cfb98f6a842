// ms_noalloc.cu -- ms_residual_noalloc: the true relative residual of
// ms_residual, computed without allocating any device memory.
//
// Who needs it: callers that cannot call cudaMalloc at this point -- a
// latency-critical loop in which cudaMalloc's implicit device
// synchronisation is not acceptable, or an application whose device memory
// is entirely owned by its own pool allocator and may not be allocated
// behind its back.  ms_residual itself grows a per-handle workspace with
// cudaMalloc on first use; this variant never does.
//
// Its scratch (per-CTA partial sums) is the file-scope device array below,
// of fixed size.  Host code must not hand the symbol itself to a kernel (on
// the host it is only a stand-in, not a device address): the address is
// resolved once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on that device (make that call before any
// stream capture on the device), and cached; after cudaDeviceReset the cached
// address may be stale, so the function must not be used again on that
// device in the same process.  Every call on a device
// shares the one array: calls whose kernels overlap on the GPU (different
// streams, no ordering between them) race on it.  Each call writes every
// partial it later reads, so nothing needs clearing between calls.
#include <cuda_runtime.h>

#include <mutex>

#include "ms.h"
#include "ms_device.cuh"
#include "ms_internal.h"

namespace {

constexpr long long kScratchDoubles = 131072;  // 1 MiB of partial sums per device
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;
constexpr int kMaxBlocksPerRhs = 152 * 8;

static __device__ __align__(256) double g_noalloc_partials[kScratchDoubles];

std::mutex g_mu;
double* g_addr[kMaxDevices];  // device address of g_noalloc_partials, per device

// Resolve the array's device address for the current device (once per device).
cudaError_t partials_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// grid (nblk, nrhs): per-CTA sums of r^2 and bhat^2 into part[(s*nblk + b)*2 + {0,1}]
__global__ void __launch_bounds__(kThreads) noalloc_resid_kernel(const ms::Geo g, const double* __restrict__ f,
                                                                 const double* __restrict__ bnd,
                                                                 const double* __restrict__ x, double* part,
                                                                 int nblk) {
  const int s = blockIdx.y;
  const long long rb = (long long)s * g.npts;
  const double* xs = x + rb;
  const double* fs = f ? f + rb : nullptr;
  const double* bs = bnd ? bnd + (long long)s * g.nbnd : nullptr;
  const long long nxy = (long long)g.nx * g.ny;
  double sr = 0.0, sb = 0.0;
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < g.npts;
       gi += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(gi % g.nx);
    const int gy = (int)((gi / g.nx) % g.ny);
    const int gz = (int)(gi / nxy);
    double si, so;
    ms::nbr_sums(g, xs, bs, gx, gy, gz, gi, si, so);
    const double bh = fs ? fs[gi] + so : so;
    const double r = bh - (6.0 * xs[gi] - si);
    sr += r * r;
    sb += bh * bh;
  }
  __shared__ double w[2][kThreads / 32];
  sr = ms::warp_sum_to_lane0(sr);
  sb = ms::warp_sum_to_lane0(sb);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    w[0][warp] = sr;
    w[1][warp] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) {
      a0 += w[0][i];
      a1 += w[1][i];
    }
    part[((long long)s * nblk + blockIdx.x) * 2 + 0] = a0;
    part[((long long)s * nblk + blockIdx.x) * 2 + 1] = a1;
  }
}

// rel_out[s] = ||bhat - A x|| / ||bhat|| (absolute norm where ||bhat|| = 0)
__global__ void noalloc_finish_kernel(int nrhs, int nblk, const double* part, double* rel_out) {
  for (int s = threadIdx.x; s < nrhs; s += blockDim.x) {
    double r2 = 0.0, b2 = 0.0;
    for (int b = 0; b < nblk; ++b) {
      r2 += part[((long long)s * nblk + b) * 2 + 0];
      b2 += part[((long long)s * nblk + b) * 2 + 1];
    }
    rel_out[s] = b2 > 0.0 ? sqrt(r2) / sqrt(b2) : sqrt(r2);
  }
}

}  // namespace

extern "C" int ms_residual_noalloc(ms_grid* grid, const double* f, const double* bnd, const double* x,
                                   double* rel_out, void* stream) {
  if (!grid) return MS_ERR_ARG;
  if (!x || !rel_out) return ms::grid_fail(grid, MS_ERR_ARG, "ms_residual_noalloc: x and rel_out must be non-NULL");
  const ms::Geo g = ms::grid_geo(grid);
  if (g.nrhs > MS_NOALLOC_MAX_RHS)
    return ms::grid_fail(grid, MS_ERR_ARG,
                         "ms_residual_noalloc: nrhs = %d exceeds the fixed scratch limit MS_NOALLOC_MAX_RHS = %d",
                         g.nrhs, MS_NOALLOC_MAX_RHS);
  double* part = nullptr;
  cudaError_t e = partials_address(&part);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ms::grid_fail(grid, MS_ERR_CUDA, "ms_residual_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  }
  long long nblk = (g.npts + kThreads - 1) / kThreads;
  if (nblk > kMaxBlocksPerRhs) nblk = kMaxBlocksPerRhs;
  const long long fit = kScratchDoubles / (2LL * g.nrhs);  // >= 64 for nrhs <= MS_NOALLOC_MAX_RHS
  if (nblk > fit) nblk = fit;
  if (nblk < 1) nblk = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  noalloc_resid_kernel<<<dim3((unsigned)nblk, (unsigned)g.nrhs), kThreads, 0, s>>>(g, f, bnd, x, part, (int)nblk);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    noalloc_finish_kernel<<<1, 128, 0, s>>>(g.nrhs, (int)nblk, part, rel_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return ms::grid_fail(grid, MS_ERR_CUDA, "ms_residual_noalloc: launch failed: %s", cudaGetErrorString(e));
  return MS_OK;
}
