// ms_gcg.cu -- one global conjugate-gradient solve of A x = bhat on the whole
// grid (no block splitting), FP64: the single-matrix Krylov method the
// two-stage multisplitting is compared against on the same GPU.  CG itself
// is the inner method of sections 2.2 and 3 (here applied to A instead of
// A_ii); the stop rule is the outer one of section 2.1 on the CG recurrence
// residual, ||r_k|| < tol ||bhat||, tested before iteration k (k = 0
// included).
//
// One iteration is three kernels over (row blocks, rhs), replayed from a CUDA
// graph with a conditional WHILE node:
//   gcg_p_kernel     gamma_k = r.r (fixed-order sum of the previous kernel's
//                    per-CTA partials, computed identically by every CTA),
//                    stop decision, beta = gamma_k / gamma_{k-1}, p = r + beta p
//   gcg_q_kernel     q = A p (7-point stencil, zero outside the grid), p.q partials
//   gcg_x_kernel     alpha = gamma_k / p.q, x += alpha p, r -= alpha q, r.r partials
// The r.r partials alternate between two buffers by iteration parity, so
// gamma_{k-1} is still there when beta is formed.  Threads run along x rows
// (coalesced), CTAs stride over the ny*nz rows.  On GB300 this path is FP64
// ALU bound (about 12 FP64 instructions per point and iteration).
#include <cuda_runtime.h>

#include <algorithm>

#include "ms_device.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kGT = 256;  // threads per CTA

// Fixed-order sum of the nb partials at `part` by one warp: lane l adds
// partials l, l + 32, ..., then an xor butterfly; every lane (and every CTA
// that calls it on the same data) gets the same bits.
__device__ __forceinline__ double warp_sum_parts(const double* part, int nb) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int i = lane; i < nb; i += 32) v += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA sum of v into part[blockIdx.x] (thread 0 stores).
__device__ __forceinline__ void cta_partial(double v, double* part) {
  __shared__ double w[kGT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kGT / 32; ++i) t += w[i];
    part[blockIdx.x] = t;
  }
}

// r = bhat - A x0, p = 0, r.r partials into part_rr[parity 0]
__global__ void __launch_bounds__(kGT) gcg_init_kernel(const GcgArgs a) {
  const Geo& g = a.g;
  const int s = blockIdx.y;
  const long long rb = (long long)s * g.npts;
  const double* __restrict__ xs = a.x + rb;
  const double* __restrict__ fs = a.f ? a.f + rb : nullptr;
  const double* __restrict__ bs = a.bnd ? a.bnd + (long long)s * g.nbnd : nullptr;
  double* __restrict__ rs = a.r + rb;
  double* __restrict__ ps = a.p + rb;
  const int rows = g.ny * g.nz;
  double acc = 0.0;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int gy = row % g.ny, gz = row / g.ny;
    const long long base = (long long)row * g.nx;
    for (int gx = threadIdx.x; gx < g.nx; gx += kGT) {
      const long long gi = base + gx;
      double si, so;
      nbr_sums(g, xs, bs, gx, gy, gz, gi, si, so);
      const double bh = fs ? fs[gi] + so : so;
      const double r = bh - (6.0 * xs[gi] - si);
      rs[gi] = r;
      ps[gi] = 0.0;
      acc += r * r;
    }
  }
  cta_partial(acc, a.part_rr + (long long)s * a.nb);
}

// iteration k: stop decision, beta, p = r + beta p
__global__ void __launch_bounds__(kGT) gcg_p_kernel(const GcgArgs a) {
  const Geo& g = a.g;
  const int s = blockIdx.y, k = *a.k_dev;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int s_run;
  __shared__ double s_beta;
  // stop decision of rhs t at iteration k (identical in every CTA: same data, same order)
  auto decide = [&](int t, double* gamma_out) -> int {
    const double gam = warp_sum_parts(a.part_rr + ((long long)(k & 1) * g.nrhs + t) * a.nb, a.nb);
    if (gamma_out) *gamma_out = gam;
    const double b2 = a.norms[2 * t + 1];
    const double thresh = b2 > 0.0 ? a.tol * sqrt(b2) : a.tol;
    if (sqrt(gam) < thresh) return kConverged;
    if (k >= a.maxit || *a.stop_all) return kStopped;
    return kActive;
  };
  if (warp == 0) {
    int run = 0;
    double beta = 0.0;
    if (__shfl_sync(0xffffffffu, a.state[s], 0) == kActive) {
      double gam;
      const int st = decide(s, &gam);
      if (st != kActive) {
        if (blockIdx.x == 0 && lane == 0) {
          a.state[s] = st;
          a.k_final[s] = k;
        }
      } else {
        run = 1;
        if (k > 0) {
          const double gprev = warp_sum_parts(a.part_rr + ((long long)((k + 1) & 1) * g.nrhs + s) * a.nb, a.nb);
          beta = gam / gprev;
        }
      }
    }
    if (lane == 0) {
      s_run = run;
      s_beta = beta;
    }
    if (blockIdx.x == 0 && s == 0) {
      // the graph loop continues while any rhs still iterates
      int any = 0;
      for (int t = 0; t < g.nrhs; ++t)
        if (__shfl_sync(0xffffffffu, a.state[t], 0) == kActive && decide(t, nullptr) == kActive) any = 1;
      if (lane == 0 && a.use_cond) cudaGraphSetConditional(a.cond, any ? 1u : 0u);
    }
  }
  __syncthreads();
  if (!s_run) return;
  const double beta = s_beta;
  const long long rb = (long long)s * g.npts;
  const double* __restrict__ rs = a.r + rb;
  double* __restrict__ ps = a.p + rb;
  const long long n = g.npts;
  for (long long i = (long long)blockIdx.x * kGT + threadIdx.x; i < n; i += (long long)gridDim.x * kGT)
    ps[i] = fma(beta, ps[i], rs[i]);
}

// iteration k: q = A p, p.q partials
__global__ void __launch_bounds__(kGT) gcg_q_kernel(const GcgArgs a) {
  const Geo& g = a.g;
  const int s = blockIdx.y;
  if (blockIdx.x == 0 && s == 0 && threadIdx.x == 0) {
    // no other CTA of this kernel reads k_dev or stop_all; the time budget
    // takes effect at the next iteration's stop decision, identically in every CTA
    *a.k_dev = *a.k_dev + 1;
    if (a.budget_ns > 0) {
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (*a.t_start == 0ull) *a.t_start = now;
      else if ((long long)(now - *a.t_start) > a.budget_ns) *a.stop_all = 1;
    }
  }
  if (a.state[s] != kActive) return;
  const long long rb = (long long)s * g.npts;
  const double* __restrict__ ps = a.p + rb;
  double* __restrict__ qs = a.q + rb;
  const long long nxy = (long long)g.nx * g.ny;
  const int rows = g.ny * g.nz;
  double acc = 0.0;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int gy = row % g.ny, gz = row / g.ny;
    const long long base = (long long)row * g.nx;
    for (int gx = threadIdx.x; gx < g.nx; gx += kGT) {
      const long long gi = base + gx;
      const double c = ps[gi];
      double sn = 0.0;
      if (gx > 0) sn += ps[gi - 1];
      if (gx < g.nx - 1) sn += ps[gi + 1];
      if (gy > 0) sn += ps[gi - g.nx];
      if (gy < g.ny - 1) sn += ps[gi + g.nx];
      if (gz > 0) sn += ps[gi - nxy];
      if (gz < g.nz - 1) sn += ps[gi + nxy];
      const double q = fma(6.0, c, -sn);
      qs[gi] = q;
      acc = fma(c, q, acc);
    }
  }
  cta_partial(acc, a.part_pq + (long long)s * a.nb);
}

// iteration k (k_dev = k + 1 here): alpha, x += alpha p, r -= alpha q, r.r partials
__global__ void __launch_bounds__(kGT) gcg_x_kernel(const GcgArgs a) {
  const Geo& g = a.g;
  const int s = blockIdx.y, k1 = *a.k_dev;
  if (a.state[s] != kActive) return;
  __shared__ double s_alpha;
  if (threadIdx.x < 32) {
    const double gam = warp_sum_parts(a.part_rr + ((long long)((k1 - 1) & 1) * g.nrhs + s) * a.nb, a.nb);
    const double eta = warp_sum_parts(a.part_pq + (long long)s * a.nb, a.nb);
    if (threadIdx.x == 0) s_alpha = eta > 0.0 ? gam / eta : 0.0;  // eta = 0 only for p = 0
  }
  __syncthreads();
  const double alpha = s_alpha;
  const long long rb = (long long)s * g.npts;
  const double* __restrict__ ps = a.p + rb;
  const double* __restrict__ qs = a.q + rb;
  double* __restrict__ xs = a.x + rb;
  double* __restrict__ rs = a.r + rb;
  const long long n = g.npts;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kGT + threadIdx.x; i < n; i += (long long)gridDim.x * kGT) {
    xs[i] = fma(alpha, ps[i], xs[i]);
    const double r = fma(-alpha, qs[i], rs[i]);
    rs[i] = r;
    acc = fma(r, r, acc);
  }
  cta_partial(acc, a.part_rr + ((long long)(k1 & 1) * g.nrhs + s) * a.nb);
}

}  // namespace

int gcg_blocks(const Geo& g) {
  const long long rows = (long long)g.ny * g.nz;
  return (int)std::max(1LL, std::min(rows, 152LL * 4));
}

cudaError_t launch_gcg_init(const GcgArgs& a, cudaStream_t s) {
  gcg_init_kernel<<<dim3((unsigned)a.nb, (unsigned)a.g.nrhs), kGT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gcg_iteration(const GcgArgs& a, cudaStream_t s) {
  const dim3 grid((unsigned)a.nb, (unsigned)a.g.nrhs);
  gcg_p_kernel<<<grid, kGT, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gcg_q_kernel<<<grid, kGT, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gcg_x_kernel<<<grid, kGT, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ms
