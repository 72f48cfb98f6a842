// ms_kernels.cu -- synchronous outer sweep, convergence check, true residual
// and the adjoint face gather.
//
// One synchronous outer sweep k (block Jacobi, section 3 of the paper; the
// loop of Listing 1) is ONE launch of sweep_kernel: a grid of thread-block
// clusters, each cluster a "slot" that pulls (block, rhs) tasks from a
// queue.  For its task a cluster
//   1. forms the block residual r = bhat - A x^k in FP64 from x^k (the halo
//      is read straight from the neighbours' part of x^k: every block reads
//      the same x^k, strict Jacobi) and the block partial ||r_i||^2;
//   2. runs the inner CG on A_ii d = r (ms_cg.cuh) -- or restarted GMRES
//      (ms_gmres.cuh) -- in T = float or double;
//   3. writes x^{k+1}_i = x^k_i + d in FP64 into the other buffer.
// x is double buffered, so the kernel boundary is the only grid-wide
// synchronisation a sweep needs.  A one-CTA check kernel then sums the block
// partials in a fixed order (section 3: the global residual is the square
// root of the sum of the block sums of squares), applies the stop rule of
// section 2.1 per rhs and advances the sweep counter kept in device memory,
// so the same [sweep, check] pair can be replayed from a CUDA graph.
//
// Because the residual of x^k is formed inside sweep k, the stop decision for
// x^k lands after sweep k's inner solves; the solver then returns x^k (still
// in its buffer) and sweep k's update is discarded.
#include <cuda_runtime.h>

#include "ms_cg.cuh"
#include "ms_gmres.cuh"
#include "ms_device.cuh"
#include "ms_internal.h"

namespace ms {

template <typename T, int NT>
__global__ void __launch_bounds__(NT, 1) sweep_kernel(const SweepArgs a) {
  __shared__ RedSmem sm;
  __shared__ GmresSmem gs;
  __shared__ int s_task[2];
  if (*a.all_done) return;
  const unsigned rank = cl_rank(), csize = cl_size(), slot = cl_id();
  const int tid = threadIdx.x;
  const int k = *a.k_dev;
  const double* __restrict__ xin = (k & 1) ? a.xbuf1 : a.xbuf0;
  double* __restrict__ xout = (k & 1) ? a.xbuf0 : a.xbuf1;
  const bool residual_only = (k >= a.outer_maxit);
  const bool gmres = a.inner_method == 1;
  const CgVecs<T> v = slot_vecs<T>(a.scratch, a.vec_stride, slot);
  const GmresVecs<T> gv = gmres_slot_vecs<T>(a.scratch, a.vec_stride, slot, a.gmres_restart);
  T* const rvec = gmres ? gv.r : v.r;  // the slot layout differs between the two inner methods
  T* const dvec = gmres ? gv.d : v.d;
  const Geo g = a.g;
  const long long nxy = (long long)g.nx * g.ny;
  int par = 0;
  for (;;) {
    if (rank == 0 && tid == 0) {
      const int t = (int)atomicAdd(a.counter, 1u);
      for (unsigned j = 0; j < csize; ++j) cl_store(&s_task[par], j, t);
    }
    cl_barrier();
    const int t = s_task[par];
    par ^= 1;
    if (t >= a.ntasks) break;
    const Task tk = a.tasks[t];
    if (a.rhs_state[tk.rhs] != kActive) continue;
    if ((long long)tk.bx * tk.by * tk.bz > a.vec_stride) {  // host guarantees this; never trust it blindly
      if (tid == 0) atomicOr(a.err, kErrGeometry);
      continue;
    }
    const Slab sl = make_slab(tk.bx, tk.by, tk.bz, rank, csize);
    const long long rb = (long long)tk.rhs * g.npts;
    const double* __restrict__ xr = xin + rb;
    const double* __restrict__ fr = a.f ? a.f + rb : nullptr;
    const double* __restrict__ br = a.bnd ? a.bnd + (long long)tk.rhs * g.nbnd : nullptr;
    // ---- 1. block residual in FP64, stored as T (FP32: times a power of two ~ 1/||bhat||, undone in 3.)
    const double scale = inner_scale<T>(a.inv_bnorm[tk.rhs]), unscale = 1.0 / scale;
    double red0[2] = {0.0, 0.0};
    {
      double s_loc = 0.0;
      T g_loc = 0;
      for (int c = tid; c < sl.plane; c += NT) {
        const int gx = tk.ox + c % tk.bx, gy = tk.oy + c / tk.bx;
        for (int z = sl.z0; z < sl.z1; ++z) {
          const int gz = tk.oz + z;
          const long long gi = (long long)gz * nxy + (long long)gy * g.nx + gx;
          double si, so;
          nbr_sums(g, xr, br, gx, gy, gz, gi, si, so);
          const double bh = fr ? fr[gi] + so : so;
          const double rr = bh - (6.0 * xr[gi] - si);
          if (owns(tk, c % tk.bx, c / tk.bx, z)) s_loc += rr * rr;  // the global norm counts owned points
          const T rt = (T)(rr * scale);
          rvec[z * sl.plane + c] = rt;
          g_loc += rt * rt;
        }
      }
      red0[0] = s_loc;
      red0[1] = (double)g_loc;
    }
    cluster_reduce<NT, 2>(red0, sm.slots[0], sm.wsum, rank, csize, [&](double (&t)[2]) {
      sm.tot[0] = t[0];
      sm.tot[1] = t[1];
    });
    red0[0] = sm.tot[0];
    red0[1] = sm.tot[1];
    if (rank == 0 && tid == 0) a.partial[t] = red0[0];
    if (residual_only) continue;
    // ---- 2. inner solve
    const int m = gmres ? block_gmres<T, NT>(gv, a.gmres_restart, sl, red0[1], sweep_inner_rtol(a, tk.rhs),
                                             a.inner_maxit, sm, gs, rank, csize)
                        : block_cg<T, NT>(v, sl, red0[1], sweep_inner_rtol(a, tk.rhs), a.inner_maxit, sm, rank, csize);
    // ---- 3. outer update into the other buffer (owned points only)
    double* __restrict__ xo = xout + rb;
    for (int c = tid; c < sl.plane; c += NT) {
      const int gx = tk.ox + c % tk.bx, gy = tk.oy + c / tk.bx;
      for (int z = sl.z0; z < sl.z1; ++z) {
        if (!owns(tk, c % tk.bx, c / tk.bx, z)) continue;
        const long long gi = (long long)(tk.oz + z) * nxy + (long long)gy * g.nx + gx;
        xo[gi] = (m > 0) ? xr[gi] + (double)dvec[z * sl.plane + c] * unscale : xr[gi];
      }
    }
    if (rank == 0 && tid == 0 && m > 0) {
      atomicAdd(a.inner_count + 2 * tk.rhs, (unsigned long long)m);
      atomicAdd(a.inner_count + 2 * tk.rhs + 1, (unsigned long long)m * (unsigned long long)(sl.plane * tk.bz));
    }
    if (rank == 0 && tid == 0 && a.tr.rec) trace_push(a.tr, *a.k_dev, tk.block, tk.rhs, m, a.partial[t]);
  }
}

// Rung of sweep j under the round schedule of `st` (see AdaptState).
__device__ __forceinline__ int adapt_rung_of(const AdaptState& st, int j) {
  if (j < st.rs || j >= st.rs + 3 * kAdaptWindow) return st.c;
  const int w = (j - st.rs) / kAdaptWindow;
  int r = st.c + (w == 1 ? -1 : (w == 2 ? 1 : 0));
  if (r < 0) r = st.c + kAdaptEdgeProbe;
  else if (r >= kAdaptRungs) r = st.c - kAdaptEdgeProbe;
  return r < 0 ? 0 : (r >= kAdaptRungs ? kAdaptRungs - 1 : r);
}

// Controller step at check k for an rhs that continues: charge sweep k-1 to
// its rung, close the round when its last sweep is charged, and set the
// inner tolerance of sweep k+1.
__device__ void adapt_step(const CheckArgs& a, int s, int k, double rho) {
  AdaptState& st = a.adapt[s];
  const double lr = log(fmax(rho, 1e-300));
  const double cum = (double)a.inner_count[2 * s + 1] + kAdaptSweepCost * a.npts * (double)(k + 1);
  if (k >= 1) {
    const int j = k - 1;
    if (j >= st.rs && j < st.rs + 3 * kAdaptWindow) {
      const int w = (j - st.rs) / kAdaptWindow;
      if ((j - st.rs) % kAdaptWindow >= kAdaptSkip) {
        st.acc_d[w] += st.lr_prev - lr;
        st.acc_w[w] += st.cum_prev - st.cum_prev2;
      }
      if (j == st.rs + 3 * kAdaptWindow - 1) {
        for (int r = 0; r < kAdaptRungs; ++r) {
          st.mem_d[r] *= kAdaptMemory;
          st.mem_w[r] *= kAdaptMemory;
        }
        int rq[3];
        for (int q = 0; q < 3; ++q) {
          rq[q] = adapt_rung_of(st, st.rs + q * kAdaptWindow);
          st.mem_d[rq[q]] += st.acc_d[q];
          st.mem_w[rq[q]] += st.acc_w[q];
        }
        int best = 0;
        double be = -1e300;
        for (int q = 0; q < 3; ++q) {
          const double e = st.mem_w[rq[q]] > 0.0 ? st.mem_d[rq[q]] / st.mem_w[rq[q]] : -1e300;
          if (e > be) {
            be = e;
            best = q;
          }
        }
        for (int q = 0; q < 3; ++q) st.acc_d[q] = st.acc_w[q] = 0.0;
        st.c = rq[best];
        st.rs = k + 1;
      }
    }
  }
  st.cum_prev2 = st.cum_prev;
  st.cum_prev = cum;
  st.lr_prev = lr;
  st.cur = adapt_rung_of(st, k + 1);
  a.inner_rtol_rhs[s] = adapt_rung_rtol(st.cur);
}

// One CTA: per-rhs global norm from the block partials (fixed task order),
// stop rule, bookkeeping for the next sweep (and the inner-tolerance
// controller when enabled).
__global__ void check_kernel(const CheckArgs a) {
  const int k = *a.k_dev;
  __shared__ int timed_out;
  if (threadIdx.x == 0) {
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (*a.t_start == 0ull) *a.t_start = now;
    timed_out = (a.time_budget_ns && now - *a.t_start > a.time_budget_ns) ? 1 : 0;
    if (a.thist && k <= a.outer_maxit) a.thist[k] = (double)(now - *a.t_start) * 1e-6;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int s = warp; s < a.nrhs; s += nwarps) {  // one warp per rhs
    if (a.rhs_state[s] != kActive) continue;
    const double sum = rhs_partial_sum_warp(a.tasks, a.partial, a.ntasks, s);
    if (lane != 0) continue;
    const double rho = sqrt(sum) * a.inv_bnorm[s];
    if (a.hist) a.hist[(long long)s * (a.outer_maxit + 1) + k] = rho;
    if (rho < a.outer_tol) {
      a.rhs_state[s] = kConverged;
      a.k_final[s] = k;
    } else if (k >= a.outer_maxit || timed_out) {
      a.rhs_state[s] = kStopped;
      a.k_final[s] = k;
    } else if (a.adapt) {
      adapt_step(a, s, k, rho);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int done = 1;
    for (int s = 0; s < a.nrhs; ++s)
      if (a.rhs_state[s] == kActive) done = 0;
    if (timed_out) atomicOr(a.err, kErrTimeout);
    *a.all_done = done;
    *a.counter = 0u;
    *a.k_dev = k + 1;
    // the enclosing WHILE node of a whole-solve graph runs another sweep only if work is left
    if (a.use_cond) cudaGraphSetConditional(a.cond, done ? 0u : 1u);
  }
}

// ---------------------------------------------------------------- true residual
// grid (nblk, nrhs): per-CTA sums of r^2 and bhat^2, r = bhat - A x.
__global__ void __launch_bounds__(256) resid_kernel(const ResidArgs a) {
  const Geo g = a.g;
  const int s = blockIdx.y;
  const long long rb = (long long)s * g.npts;
  const double* __restrict__ x = a.x + rb;
  const double* __restrict__ f = a.f ? a.f + rb : nullptr;
  const double* __restrict__ bnd = a.bnd ? a.bnd + (long long)s * g.nbnd : nullptr;
  const long long nxy = (long long)g.nx * g.ny;
  double sr = 0.0, sb = 0.0;
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < g.npts;
       gi += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(gi % g.nx);
    const int gy = (int)((gi / g.nx) % g.ny);
    const int gz = (int)(gi / nxy);
    double si, so;
    nbr_sums(g, x, bnd, gx, gy, gz, gi, si, so);
    const double bh = f ? f[gi] + so : so;
    const double r = bh - (6.0 * x[gi] - si);
    sr += r * r;
    sb += bh * bh;
  }
  __shared__ double w[2][8];
  sr = warp_sum_to_lane0(sr);
  sb = warp_sum_to_lane0(sb);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    w[0][warp] = sr;
    w[1][warp] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a0 += w[0][i];
      a1 += w[1][i];
    }
    a.part[((long long)s * a.nblk + blockIdx.x) * 2 + 0] = a0;
    a.part[((long long)s * a.nblk + blockIdx.x) * 2 + 1] = a1;
  }
}

__global__ void resid_finish_kernel(int nrhs, int nblk, const double* part, double* out, double* inv_bnorm) {
  for (int s = threadIdx.x; s < nrhs; s += blockDim.x) {
    double a0 = 0.0, a1 = 0.0;
    for (int b = 0; b < nblk; ++b) {
      a0 += part[((long long)s * nblk + b) * 2 + 0];
      a1 += part[((long long)s * nblk + b) * 2 + 1];
    }
    out[2 * s + 0] = a0;
    out[2 * s + 1] = a1;
    if (inv_bnorm) inv_bnorm[s] = a1 > 0.0 ? 1.0 / sqrt(a1) : 1.0;
  }
}

// ---------------------------------------------------------------- ||bhat||^2 alone
// grid (nblk, nrhs): per-CTA sums of bhat^2 (bhat = f + lift(bnd)).  Without f
// only the points next to the boundary carry data, so only they are visited:
// the x faces (i = 0, nx-1), then the y faces without the x edges, then the z
// faces without the x and y edges -- every point of that shell once.
__global__ void __launch_bounds__(256) bhat_sq_kernel(const Geo g, const double* f, const double* bnd, double* part,
                                                      int nblk) {
  const int s = blockIdx.y;
  const double* __restrict__ fs = f ? f + (long long)s * g.npts : nullptr;
  const double* __restrict__ bs = bnd ? bnd + (long long)s * g.nbnd : nullptr;
  const long long nxy = (long long)g.nx * g.ny;
  const long long fyz = (long long)g.nz * g.ny, fxz = (long long)g.nz * g.nx;
  // boundary values next to interior point (gx, gy, gz)
  auto lifted = [&](int gx, int gy, int gz) {
    double so = 0.0;
    if (!bs) return so;
    if (gx == 0) so += bs[(long long)gz * g.ny + gy];
    if (gx == g.nx - 1) so += bs[fyz + (long long)gz * g.ny + gy];
    if (gy == 0) so += bs[2 * fyz + (long long)gz * g.nx + gx];
    if (gy == g.ny - 1) so += bs[2 * fyz + fxz + (long long)gz * g.nx + gx];
    if (gz == 0) so += bs[2 * fyz + 2 * fxz + (long long)gy * g.nx + gx];
    if (gz == g.nz - 1) so += bs[2 * fyz + 2 * fxz + nxy + (long long)gy * g.nx + gx];
    return so;
  };
  double sb = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (fs) {
    for (long long gi = t0; gi < g.npts; gi += stride) {
      const int gx = (int)(gi % g.nx), gy = (int)((gi / g.nx) % g.ny), gz = (int)(gi / nxy);
      const double bh = fs[gi] + lifted(gx, gy, gz);
      sb += bh * bh;
    }
  } else if (bs) {
    const int ix = g.nx > 1 ? 2 : 1, iy = g.ny > 1 ? 2 : 1, iz = g.nz > 1 ? 2 : 1;  // x faces present
    const long long ny_in = g.ny > 2 ? g.ny - 2 : 0, nx_in = g.nx > 2 ? g.nx - 2 : 0;
    const long long n_x = (long long)ix * g.ny * g.nz;               // the x faces
    const long long n_y = (long long)iy * nx_in * g.nz;              // y faces, x edges excluded
    const long long n_z = (long long)iz * nx_in * ny_in;             // z faces, x and y edges excluded
    for (long long e = t0; e < n_x + n_y + n_z; e += stride) {
      int gx, gy, gz;
      if (e < n_x) {
        const long long q = e % ((long long)g.ny * g.nz);
        gx = e < (long long)g.ny * g.nz ? 0 : g.nx - 1;
        gy = (int)(q % g.ny);
        gz = (int)(q / g.ny);
      } else if (e < n_x + n_y) {
        const long long p = e - n_x, plane = nx_in * g.nz;
        const long long q = p % plane;
        gy = p < plane ? 0 : g.ny - 1;
        gx = 1 + (int)(q % nx_in);
        gz = (int)(q / nx_in);
      } else {
        const long long p = e - n_x - n_y, plane = nx_in * ny_in;
        const long long q = p % plane;
        gz = p < plane ? 0 : g.nz - 1;
        gx = 1 + (int)(q % nx_in);
        gy = 1 + (int)(q / nx_in);
      }
      const double bh = lifted(gx, gy, gz);
      sb += bh * bh;
    }
  }
  __shared__ double w[8];
  sb = warp_sum_to_lane0(sb);
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = sb;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < 8; ++i) a += w[i];
    part[(long long)s * nblk + blockIdx.x] = a;
  }
}

// out[s] = sum of the per-CTA parts; inv_bnorm[s] = 1/||bhat|| (1 if bhat = 0)
__global__ void bhat_sq_finish_kernel(int nrhs, int nblk, const double* part, double* out, double* inv_bnorm) {
  for (int s = threadIdx.x; s < nrhs; s += blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < nblk; ++b) a += part[(long long)s * nblk + b];
    out[s] = a;
    inv_bnorm[s] = a > 0.0 ? 1.0 / sqrt(a) : 1.0;
  }
}

// out[s] = the sum of the block partials of rhs s (one warp per rhs, the fixed
// order of rhs_partial_sum_warp)
__global__ void task_sums_kernel(const Task* tasks, const double* partial, int ntasks, int nrhs, double* out) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int s = warp; s < nrhs; s += nw) {
    const double v = rhs_partial_sum_warp(tasks, partial, ntasks, s);
    if ((threadIdx.x & 31) == 0) out[s] = v;
  }
}

// ---------------------------------------------------------------- adjoint face gather
__global__ void face_gather_kernel(const Geo g, const double* __restrict__ lam, double* __restrict__ grad) {
  const long long total = g.nbnd * g.nrhs;
  const long long fyz = (long long)g.nz * g.ny, fxz = (long long)g.nz * g.nx, fxy = (long long)g.ny * g.nx;
  const long long nxy = (long long)g.nx * g.ny;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / g.nbnd;
    long long p = e - s * g.nbnd;
    int i, j, k;
    if (p < 2 * fyz) {  // x- / x+ : (k, j)
      const bool hi = p >= fyz;
      const long long q = hi ? p - fyz : p;
      k = (int)(q / g.ny);
      j = (int)(q % g.ny);
      i = hi ? g.nx - 1 : 0;
    } else if ((p -= 2 * fyz) < 2 * fxz) {  // y- / y+ : (k, i)
      const bool hi = p >= fxz;
      const long long q = hi ? p - fxz : p;
      k = (int)(q / g.nx);
      i = (int)(q % g.nx);
      j = hi ? g.ny - 1 : 0;
    } else {  // z- / z+ : (j, i)
      p -= 2 * fxz;
      const bool hi = p >= fxy;
      const long long q = hi ? p - fxy : p;
      j = (int)(q / g.nx);
      i = (int)(q % g.nx);
      k = hi ? g.nz - 1 : 0;
    }
    grad[e] = lam[s * g.npts + (long long)k * nxy + (long long)j * g.nx + i];
  }
}

// ---------------------------------------------------------------- launchers
template <typename T, int NT>
static cudaError_t launch_sweep_t(int cluster, int slots, const SweepArgs& a, cudaStream_t s) {
  auto kern = sweep_kernel<T, NT>;
  if (cluster > 8) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(cluster * slots), 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename T, int NT>
static cudaError_t max_clusters_t(int cluster, int* out) {
  auto kern = sweep_kernel<T, NT>;
  if (cluster > 8) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(cluster * 64), 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(out, kern, &cfg);
}

#define MS_DISPATCH(prec, threads, FN, ...)                                    \
  do {                                                                         \
    if (prec == 1) {                                                           \
      if (threads == 256) return FN<float, 256>(__VA_ARGS__);                  \
      if (threads == 512) return FN<float, 512>(__VA_ARGS__);                  \
      if (threads == 1024) return FN<float, 1024>(__VA_ARGS__);                \
    } else {                                                                   \
      if (threads == 256) return FN<double, 256>(__VA_ARGS__);                 \
      if (threads == 512) return FN<double, 512>(__VA_ARGS__);                 \
      if (threads == 1024) return FN<double, 1024>(__VA_ARGS__);               \
    }                                                                          \
    return cudaErrorInvalidValue;                                              \
  } while (0)

cudaError_t launch_sweep(int prec, int threads, int cluster, int slots, const SweepArgs& a, cudaStream_t s) {
  MS_DISPATCH(prec, threads, launch_sweep_t, cluster, slots, a, s);
}

cudaError_t sweep_max_clusters(int prec, int threads, int cluster, int* out) {
  MS_DISPATCH(prec, threads, max_clusters_t, cluster, out);
}

cudaError_t launch_check(const CheckArgs& a, cudaStream_t s) {
  check_kernel<<<1, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_resid(const ResidArgs& a, double* out, double* inv_bnorm, cudaStream_t s) {
  resid_kernel<<<dim3((unsigned)a.nblk, (unsigned)a.g.nrhs), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  resid_finish_kernel<<<1, 128, 0, s>>>(a.g.nrhs, a.nblk, a.part, out, inv_bnorm);
  return cudaGetLastError();
}

cudaError_t launch_bhat_sq(const Geo& g, const double* f, const double* bnd, double* part, int nblk, double* out,
                           double* inv_bnorm, cudaStream_t s) {
  bhat_sq_kernel<<<dim3((unsigned)nblk, (unsigned)g.nrhs), 256, 0, s>>>(g, f, bnd, part, nblk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bhat_sq_finish_kernel<<<1, 128, 0, s>>>(g.nrhs, nblk, part, out, inv_bnorm);
  return cudaGetLastError();
}

cudaError_t launch_task_sums(const Task* tasks, const double* partial, int ntasks, int nrhs, double* out,
                             cudaStream_t s) {
  task_sums_kernel<<<1, 256, 0, s>>>(tasks, partial, ntasks, nrhs, out);
  return cudaGetLastError();
}

cudaError_t launch_face_gather(const Geo& g, const double* lam, double* grad, cudaStream_t s) {
  const long long total = g.nbnd * g.nrhs;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  face_gather_kernel<<<(unsigned)blocks, 256, 0, s>>>(g, lam, grad);
  return cudaGetLastError();
}

}  // namespace ms
