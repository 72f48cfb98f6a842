// ms_resident_kernels.cuh -- kernels of the resident engine: the synchronous
// outer sweep with the on-chip inner CG (ms_resident.cuh), FP32 inner / FP64
// outer, its asynchronous and persistent-dataflow forms, and res_prep<V>,
// which readies the three kernels of variant table row V.  Included only by
// the ms_resident_inst*.cu files, each of which instantiates a few rows so
// that the rows compile in parallel.
//
// The sweep kernel has the contract of sweep_kernel in ms_kernels.cu (one
// launch per sweep, dynamic task queue, x double buffered, block partials for
// the check kernel), but the CG state of the block being solved never leaves
// the cluster: the residual phase writes r straight into registers, and the
// update reads d from registers (or shared memory).
#pragma once
#include <cuda_runtime.h>

#include "ms_async.cuh"
#include "ms_device.cuh"
#include "ms_internal.h"
#include "ms_resident.cuh"
#include "ms_resident_variants.h"

namespace ms {

// Residual r = bhat - A x^k on this CTA's strips (FP64), multiplied by the
// power-of-two `scale` (~1/||bhat||, exact) and rounded into r4, so that the
// FP32 inner solve sees O(relative residual) values whatever the problem's
// magnitude; the boundary planes of r are pushed to the neighbour CTAs'
// r-halo planes.  s64: FP64 sum of squares of the unscaled r; g32: FP32 sum
// of squares of the scaled, rounded r.
// nb(x, y, z, gi, si, so): neighbour sums of block point (x, y, z) (block
// coordinates, grid index gi) -- straight from x^k (sync) or through the
// halo cache (async).
template <int NT, int KC, int ZS, bool XL2 = false, typename NB>
__device__ __forceinline__ void resident_residual(float4 (&r4)[KC][ZS], const ResGeo& g, const Strips<KC>& s,
                                                  const Task& tk, const Geo& G, const double* xr,
                                                  const double* __restrict__ fr, double scale, float* sp,
                                                  unsigned rank, unsigned csize, double& s64, float& g32, NB&& nb) {
  float* rh_lo = sp + (long long)(ZS + 2) * g.ps;
  float* rh_hi = rh_lo + g.ps;
  const long long nxy = (long long)G.nx * G.ny;
  double sl = 0.0;
  float gl = 0.f;
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int y = s.st[k] >= 0 ? s.st[k] / g.spr : 0;
    const int gx0 = tk.ox + 4 * (s.st[k] >= 0 ? s.st[k] - y * g.spr : 0), gy = tk.oy + y;
#pragma unroll
    for (int z = 0; z < ZS; ++z) {
      float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s.msk[k] && z < g.nzs) {
        const int gz = tk.oz + g.z0 + z;
        float rv[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          rv[l] = 0.f;
          if (s.msk[k] & (1u << l)) {
            const int gx = gx0 + l;
            const long long gi = (long long)gz * nxy + (long long)gy * G.nx + gx;
            double si, so;
            nb(gx - tk.ox, gy - tk.oy, g.z0 + z, gi, si, so);
            const double bh = fr ? fr[gi] + so : so;
            const double rr = bh - (6.0 * ldx<XL2>(xr, gi) - si);
            sl += rr * rr;
            rv[l] = (float)(rr * scale);
          }
        }
        r = make_float4(rv[0], rv[1], rv[2], rv[3]);
        gl += dot4(r, r);
        if (z == 0 && rank > 0) st_cluster_v4(rh_hi + s.off[k], rank - 1, r);
        if (z == g.nzs - 1 && rank + 1 < csize) st_cluster_v4(rh_lo + s.off[k], rank + 1, r);
      }
      r4[k][z] = r;
    }
  }
  s64 = sl;
  g32 = gl;
}

// power of two closest (within a factor 2) to v > 0, 1 otherwise
__device__ __forceinline__ double pow2_near(double v) {
  if (!(v > 0.0) || !isfinite(v)) return 1.0;
  int e;
  frexp(v, &e);
  return ldexp(1.0, e - 1);
}

template <int NT>
__device__ __forceinline__ void zero_smem(float4* p, int n4) {
  for (int i = threadIdx.x; i < n4; i += NT) p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int NT, int KC, int ZS, bool DS, int QR>
__global__ void __launch_bounds__(NT, 1) res_sweep_kernel(const SweepArgs a, int smem_f4) {
  extern __shared__ float4 dyn4[];
  float* sp = reinterpret_cast<float*>(dyn4);
  __shared__ RedSmem red;
  __shared__ ResRed rred;
  __shared__ int s_task[2];
  if (*a.all_done) return;
  res_red_init(rred, a.err, a.sum_polls);
  const unsigned rank = cl_rank(), csize = cl_size();
  const int tid = threadIdx.x;
  const int k = *a.k_dev;
  const double* __restrict__ xin = (k & 1) ? a.xbuf1 : a.xbuf0;
  double* __restrict__ xout = (k & 1) ? a.xbuf0 : a.xbuf1;
  const bool residual_only = (k >= a.outer_maxit);
  const Geo G = a.g;
  const long long nxy = (long long)G.nx * G.ny;
  zero_smem<NT>(dyn4, smem_f4);
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
    // capacity check, identical in every CTA of the cluster
    {
      const int spr = (tk.bx + 3) >> 2;
      const int nzs_max = (tk.bz + (int)csize - 1) / (int)csize;
      if (tk.bz < (int)csize || nzs_max > ZS || spr * tk.by > KC * NT ||
          res_smem_floats(tk.bx, tk.by, ZS, DS) > 4LL * smem_f4) {
        if (tid == 0) atomicOr(a.err, kErrGeometry);
        continue;
      }
    }
    const ResGeo g = make_res_geo(tk.bx, tk.by, tk.bz, rank, csize);
    const Strips<KC> s = make_strips<NT, KC>(g);
    const double scale = pow2_near(a.inv_bnorm[tk.rhs]), unscale = 1.0 / scale;
    const long long rb = (long long)tk.rhs * G.npts;
    const double* __restrict__ xr = xin + rb;
    const double* __restrict__ fr = a.f ? a.f + rb : nullptr;
    const double* __restrict__ br = a.bnd ? a.bnd + (long long)tk.rhs * G.nbnd : nullptr;
    float4 r4[KC][ZS], d4[DS ? 1 : KC][DS ? 1 : ZS];
    double red0[2];
    {
      double s64;
      float g32;
      resident_residual<NT, KC, ZS>(r4, g, s, tk, G, xr, fr, scale, sp, rank, csize, s64, g32,
                                    [&](int bxl, int byl, int bzl, long long gi, double& si, double& so) {
                                      nbr_sums(G, xr, br, tk.ox + bxl, tk.oy + byl, tk.oz + bzl, gi, si, so);
                                    });
      red0[0] = s64;
      red0[1] = (double)g32;
    }
    cluster_reduce<NT, 2>(red0, red.slots[0], red.wsum, rank, csize, [&](double (&t)[2]) {
      red.tot[0] = t[0];
      red.tot[1] = t[1];
    });
    red0[0] = red.tot[0];
    red0[1] = red.tot[1];
    if (rank == 0 && tid == 0) a.partial[t] = red0[0];
    int m = 0;
    if (!residual_only)
      m = resident_cg<NT, KC, ZS, DS, QR>(r4, d4, g, s, sp, (float)red0[1], (float)sweep_inner_rtol(a, tk.rhs),
                                          a.inner_maxit, rred,
                                      rank, csize);
    // every cluster barrier of this task is behind us: with d in registers the
    // smem can be cleared for the next task right away (with d in smem, after the update)
    if (residual_only || !DS) zero_smem<NT>(dyn4, smem_f4);
    if (residual_only) continue;
    double* __restrict__ xo = xout + rb;
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      if (!s.msk[kk]) continue;
      const int y = s.st[kk] / g.spr;
      const long long row = (long long)(tk.oy + y) * G.nx + tk.ox + 4 * (s.st[kk] - y * g.spr);
#pragma unroll
      for (int z = 0; z < ZS; ++z) {
        if (z >= g.nzs) continue;
        const long long gi0 = (long long)(tk.oz + g.z0 + z) * nxy + row;
        float4 d;
        if constexpr (DS) d = *d_slot<NT, KC, ZS, DS>(sp, g, z, s.st[kk]);
        else d = d4[kk][z];
        const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          if (!(s.msk[kk] & (1u << l))) continue;
          xo[gi0 + l] = (m > 0) ? xr[gi0 + l] + (double)dv[l] * unscale : xr[gi0 + l];
        }
      }
    }
    if constexpr (DS) {
      __syncthreads();  // d has been consumed by every thread
      zero_smem<NT>(dyn4, smem_f4);
    }
    if (rank == 0 && tid == 0 && m > 0) {
      atomicAdd(a.inner_count + 2 * tk.rhs, (unsigned long long)m);
      atomicAdd(a.inner_count + 2 * tk.rhs + 1, (unsigned long long)m * (unsigned long long)tk.bx * tk.by * tk.bz);
    }
    if (rank == 0 && tid == 0 && a.tr.rec) trace_push(a.tr, *a.k_dev, tk.block, tk.rhs, m, a.partial[t]);
  }
}

// Asynchronous outer iteration with the on-chip inner CG (protocol in
// ms_async.cuh): halo refresh, residual through the halo cache, resident CG,
// in-place update fused with face publication, stale-estimate monitor.
template <int NT, int KC, int ZS, bool DS, int QR>
__global__ void __launch_bounds__(NT, 1) res_async_kernel(const AsyncArgs a, int smem_f4) {
  extern __shared__ float4 dyn4[];
  float* sp = reinterpret_cast<float*>(dyn4);
  __shared__ RedSmem red;
  __shared__ ResRed rred;
  __shared__ int bc[2][32];
  const unsigned rank = cl_rank(), csize = cl_size(), cid = cl_id(), ncl = cl_count();
  const int tid = threadIdx.x;
  const Geo G = a.g;
  const long long nxy = (long long)G.nx * G.ny;
  __shared__ unsigned snap[12];
  res_red_init(rred, a.err, a.sum_polls);
  AsyncCtl c = async_ctl_init(a, cid, ncl, snap);
  zero_smem<NT>(dyn4, smem_f4);
  for (;; c.par ^= 1) {
    const int t = async_pick(a, c, bc, rank, csize, cid, ncl);
    if (t < 0) break;
    const Task tk = a.tasks[t];
    {
      const int spr = (tk.bx + 3) >> 2;
      const int nzs_max = (tk.bz + (int)csize - 1) / (int)csize;
      if (tk.bz < (int)csize || nzs_max > ZS || spr * tk.by > KC * NT ||
          res_smem_floats(tk.bx, tk.by, ZS, DS) > 4LL * smem_f4 || face_size(0, tk.bx, tk.by, tk.bz) > a.face_stride ||
          face_size(2, tk.bx, tk.by, tk.bz) > a.face_stride || face_size(4, tk.bx, tk.by, tk.bz) > a.face_stride) {
        if (rank == 0 && tid == 0) {
          atomicOr(a.err, kErrGeometry);
          st_rlx_s32(a.stop, 1);
        }
        continue;
      }
    }
    if (a.slow_block == tk.block && a.slow_ns > 0 && rank == 0 && tid == 0)
      __nanosleep((unsigned)min(a.slow_ns, 1000000));
    async_halo_refresh<NT>(a, tk, t, bc, c, rank, csize);
    const int* hcur = bc[c.par] + 20;
    const ResGeo g = make_res_geo(tk.bx, tk.by, tk.bz, rank, csize);
    const Strips<KC> s = make_strips<NT, KC>(g);
    const double scale = pow2_near(a.inv_bnorm[tk.rhs]), unscale = 1.0 / scale;
    const long long rb = (long long)tk.rhs * G.npts;
    double* xr = a.x + rb;
    const double* __restrict__ fr = a.f ? a.f + rb : nullptr;
    const double* __restrict__ br = a.bnd ? a.bnd + (long long)tk.rhs * G.nbnd : nullptr;
    float4 r4[KC][ZS], d4[DS ? 1 : KC][DS ? 1 : ZS];
    double red0[2];
    {
      double s64;
      float g32;
      resident_residual<NT, KC, ZS>(r4, g, s, tk, G, xr, fr, scale, sp, rank, csize, s64, g32,
                                    [&](int bxl, int byl, int bzl, long long gi, double& si, double& so) {
                                      async_nbr_sums(a, tk, t, hcur, xr, br, bxl, byl, bzl, gi, si, so);
                                    });
      red0[0] = s64;
      red0[1] = (double)g32;
    }
    cluster_reduce<NT, 2>(red0, red.slots[0], red.wsum, rank, csize, [&](double (&tt)[2]) {
      red.tot[0] = tt[0];
      red.tot[1] = tt[1];
    });
    if (rank == 0 && tid == 0) st_rlx_f64(a.partial + t, red.tot[0]);
    const int m = resident_cg<NT, KC, ZS, DS, QR>(r4, d4, g, s, sp, (float)red.tot[1], (float)a.inner_rtol,
                                              a.inner_maxit, rred, rank, csize);
    if constexpr (!DS) zero_smem<NT>(dyn4, smem_f4);  // all cluster barriers of the CG are behind us
    async_publish_begin(a, tk, t, bc, c, rank, csize);
    const int* fslot = bc[c.par] + 26;
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      if (!s.msk[kk]) continue;
      const int y = s.st[kk] / g.spr, x0 = 4 * (s.st[kk] - y * g.spr);
      const long long row = (long long)(tk.oy + y) * G.nx + tk.ox + x0;
#pragma unroll
      for (int z = 0; z < ZS; ++z) {
        if (z >= g.nzs) continue;
        const long long gi0 = (long long)(tk.oz + g.z0 + z) * nxy + row;
        float4 d;
        if constexpr (DS) d = *d_slot<NT, KC, ZS, DS>(sp, g, z, s.st[kk]);
        else d = d4[kk][z];
        const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          if (!(s.msk[kk] & (1u << l))) continue;
          const double xn = (m > 0) ? xr[gi0 + l] + (double)dv[l] * unscale : xr[gi0 + l];
          xr[gi0 + l] = xn;
          async_face_store(a, tk, t, fslot, x0 + l, y, g.z0 + z, xn);
        }
      }
    }
    async_publish_end(a, tk, t, fslot, rank, m);
    if constexpr (DS) {
      __syncthreads();
      zero_smem<NT>(dyn4, smem_f4);
    }
    async_monitor(a, rank);
  }
}

// ---------------------------------------------------------------- dataflow sync
__device__ __forceinline__ int ld_acq_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_s32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until *p >= v (warp 0 of rank 0 only).  Returns 1 when the
// flag is reached, -1 when *abort is set meanwhile (another cluster ended the
// launch: leave without an error of our own), 0 when `limit` polls (summed
// over the launch) are spent.  Backs off with __nanosleep.
__device__ __forceinline__ int flow_wait_ge(const int* p, int v, const int* abort, long long& limit) {
  unsigned ns = 32;
  while (ld_acq_s32(p) < v) {
    if (ld_acq_s32(abort)) return -1;
    if (--limit < 0) return 0;
    __nanosleep(ns);
    ns = ns < 1024 ? 2 * ns : 1024;
  }
  return 1;
}

// Stop decision for sweep k (relative kr) -- the one-CTA check kernel's work,
// done by the cluster that counted the last residual of the sweep: per rhs
// the fixed-order sum of the block partials, the stop rule, bookkeeping.
__device__ __forceinline__ void flow_decide(const FlowArgs& fa, int kr) {
  // called by a whole warp (warp 0 of the cluster's rank 0)
  const CheckArgs& c = fa.c;
  const int lane = threadIdx.x & 31;
  const int k = fa.k0 + kr;
  __threadfence();  // acquire side of the other clusters' partial-then-count pattern
  int timed_out = 0;
  if (lane == 0) {
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (*c.t_start == 0ull) *c.t_start = now;
    timed_out = (c.time_budget_ns && now - *c.t_start > c.time_budget_ns) ? 1 : 0;
    if (timed_out) atomicOr(c.err, kErrTimeout);
    if (c.thist && k <= c.outer_maxit) c.thist[k] = (double)(now - *c.t_start) * 1e-6;
  }
  timed_out = __shfl_sync(0xffffffffu, timed_out, 0);
  int done = 1;
  for (int s = 0; s < c.nrhs; ++s) {
    if (c.rhs_state[s] != kActive) continue;
    const double sum = rhs_partial_sum_warp(c.tasks, c.partial, c.ntasks, s);
    const double rho = sqrt(sum) * c.inv_bnorm[s];
    int st = kActive;
    if (rho < c.outer_tol) st = kConverged;
    else if (k >= c.outer_maxit || timed_out) st = kStopped;
    else done = 0;
    __syncwarp();
    if (lane == 0) {
      if (c.hist) c.hist[(long long)s * (c.outer_maxit + 1) + k] = rho;
      if (st != kActive) {
        c.rhs_state[s] = st;
        c.k_final[s] = k;
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    *c.k_dev = k + 1;
    if (done) st_rel_s32(c.all_done, 1);
    __threadfence();
    st_rel_s32(fa.decided_rel, kr);
  }
  __syncwarp();
}

__device__ __forceinline__ int flow_nbr(const FlowArgs& fa, const Task& tk, int f) {
  int bi = tk.block % fa.px, bj = (tk.block / fa.px) % fa.py, bk = tk.block / (fa.px * fa.py);
  switch (f) {
    case 0: bi -= 1; break;
    case 1: bi += 1; break;
    case 2: bj -= 1; break;
    case 3: bj += 1; break;
    case 4: bk -= 1; break;
    default: bk += 1; break;
  }
  if (bi < 0 || bi >= fa.px || bj < 0 || bj >= fa.py || bk < 0 || bk >= fa.pz) return -1;
  return fa.task_of[(long long)tk.rhs * fa.nblocks + bi + fa.px * (bj + fa.py * bk)];
}

template <int NT, int KC, int ZS, bool DS, int QR>
__global__ void __launch_bounds__(NT, 1) res_flow_kernel(const FlowArgs fa, int smem_f4) {
  extern __shared__ float4 dyn4[];
  float* sp = reinterpret_cast<float*>(dyn4);
  __shared__ RedSmem red;
  __shared__ ResRed rred;
  __shared__ int bc[2][4];  // cmd (0 run, 1 skip, 2 leave), relative sweep, task
  // poll budgets of the bounded waits, one per lane of warp 0 of rank 0 (kept in
  // shared memory: no register stays live across the inner CG for them)
  __shared__ long long wait_budget[32];
  const SweepArgs& a = fa.s;
  const unsigned rank = cl_rank(), csize = cl_size();
  const int tid = threadIdx.x;
  const Geo G = a.g;
  const long long nxy = (long long)G.nx * G.ny;
  if (tid < 32) wait_budget[tid] = fa.spin_limit;
  res_red_init(rred, a.err, a.sum_polls);
  zero_smem<NT>(dyn4, smem_f4);
  int par = 0;
  for (;; par ^= 1) {
    if (rank == 0 && tid < 32) {  // warp 0 of rank 0 takes the control decisions
      const int lane = tid;
      int cmd = 0, kr = 0, t = 0;
      if (lane == 0) {
        const unsigned long long j = atomicAdd(fa.ticket, 1ull);
        kr = (int)(j / (unsigned long long)a.ntasks);
        t = (int)(j % (unsigned long long)a.ntasks);
        if (kr > a.outer_maxit - fa.k0 || ld_acq_s32(a.all_done)) {  // past the residual-only sweep
          cmd = 2;
        } else {
          const int w = kr > 0 ? flow_wait_ge(fa.decided_rel, kr - 1, a.all_done, wait_budget[0]) : 1;
          if (w == 0) {
            atomicOr(a.err, kErrTimeout);
            st_rel_s32(const_cast<int*>(a.all_done), 1);
            cmd = 2;
          } else if (w < 0 || ld_acq_s32(a.all_done)) {
            cmd = 2;
          } else if (a.rhs_state[a.tasks[t].rhs] != kActive) {
            cmd = 1;
          }
        }
      }
      cmd = __shfl_sync(0xffffffffu, cmd, 0);
      kr = __shfl_sync(0xffffffffu, kr, 0);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (cmd == 0) {
        // lanes 0..6 wait for the block itself and its six neighbours to finish sweep kr-1
        int w = 1;
        if (lane < 7) {
          const int who = lane == 0 ? t : flow_nbr(fa, a.tasks[t], lane - 1);
          if (who >= 0) w = flow_wait_ge(fa.done_rel + who, kr, a.all_done, wait_budget[lane]);
        }
        if (!__all_sync(0xffffffffu, w > 0)) {
          // a lane that ran out of polls ends the launch with kErrTimeout; a lane
          // that saw another cluster end it leaves quietly
          if (!__all_sync(0xffffffffu, w != 0) && lane == 0) {
            atomicOr(a.err, kErrTimeout);
            st_rel_s32(const_cast<int*>(a.all_done), 1);
          }
          cmd = 2;
        }
      }
      if (lane == 0)
        for (unsigned q = 0; q < csize; ++q) {
          cl_store(&bc[par][0], q, cmd);
          cl_store(&bc[par][1], q, kr);
          cl_store(&bc[par][2], q, t);
        }
    }
    cl_barrier();
    const int cmd = bc[par][0], kr = bc[par][1], t = bc[par][2];
    if (cmd == 2) break;
    if (cmd == 1) {  // rhs already stopped: count the (empty) residual, mark the sweep done
      if (rank == 0 && tid < 32) {
        int last = 0;
        if (tid == 0) {
          __threadfence();
          last = atomicAdd(fa.res_cnt + kr, 1) == a.ntasks - 1;
        }
        if (__shfl_sync(0xffffffffu, last, 0)) flow_decide(fa, kr);
        if (tid == 0) st_rel_s32(fa.done_rel + t, kr + 1);
      }
      continue;
    }
    const int k = fa.k0 + kr;
    if (fa.slow_block == a.tasks[t].block && fa.slow_ns > 0 && rank == 0 && tid == 0)
      __nanosleep((unsigned)min(fa.slow_ns, 1000000));
    // x is written by other clusters during this launch, so it is never read through the
    // non-coherent read-only path (no const __restrict__ on it); ordinary loads see the
    // producers' writes through the acquire chain (done flag ld.acquire.gpu by rank 0 ->
    // cluster barrier with acquire semantics)
    const double* xin = (k & 1) ? a.xbuf1 : a.xbuf0;
    double* xout = (k & 1) ? a.xbuf0 : a.xbuf1;
    const Task tk = a.tasks[t];
    const ResGeo g = make_res_geo(tk.bx, tk.by, tk.bz, rank, csize);
    const Strips<KC> s = make_strips<NT, KC>(g);
    const double scale = pow2_near(a.inv_bnorm[tk.rhs]), unscale = 1.0 / scale;
    const long long rb = (long long)tk.rhs * G.npts;
    const double* xr = xin + rb;
    const double* __restrict__ fr = a.f ? a.f + rb : nullptr;
    const double* __restrict__ br = a.bnd ? a.bnd + (long long)tk.rhs * G.nbnd : nullptr;
    float4 r4[KC][ZS], d4[DS ? 1 : KC][DS ? 1 : ZS];
    double red0[2];
    {
      double s64;
      float g32;
      resident_residual<NT, KC, ZS>(r4, g, s, tk, G, xr, fr, scale, sp, rank, csize, s64, g32,
                                    [&](int bxl, int byl, int bzl, long long gi, double& si, double& so) {
                                      nbr_sums(G, xr, br, tk.ox + bxl, tk.oy + byl, tk.oz + bzl, gi, si, so);
                                    });
      red0[0] = s64;
      red0[1] = (double)g32;
    }
    cluster_reduce<NT, 2>(red0, red.slots[0], red.wsum, rank, csize, [&](double (&tt)[2]) {
      red.tot[0] = tt[0];
      red.tot[1] = tt[1];
    });
    if (rank == 0 && tid < 32) {
      int last = 0;
      if (tid == 0) {
        a.partial[t] = red.tot[0];
        __threadfence();
        last = atomicAdd(fa.res_cnt + kr, 1) == a.ntasks - 1;
      }
      if (__shfl_sync(0xffffffffu, last, 0)) flow_decide(fa, kr);
    }
    if (kr == a.outer_maxit - fa.k0) {  // the residual-only sweep: nothing more to do for it
      zero_smem<NT>(dyn4, smem_f4);
      if (rank == 0 && tid == 0) st_rel_s32(fa.done_rel + t, kr + 1);
      continue;
    }
    const int m = resident_cg<NT, KC, ZS, DS, QR>(r4, d4, g, s, sp, (float)red.tot[1], (float)sweep_inner_rtol(a, tk.rhs),
                                              a.inner_maxit, rred, rank, csize);
    if constexpr (!DS) zero_smem<NT>(dyn4, smem_f4);
    double* xo = xout + rb;
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      if (!s.msk[kk]) continue;
      const int y = s.st[kk] / g.spr;
      const long long row = (long long)(tk.oy + y) * G.nx + tk.ox + 4 * (s.st[kk] - y * g.spr);
#pragma unroll
      for (int z = 0; z < ZS; ++z) {
        if (z >= g.nzs) continue;
        const long long gi0 = (long long)(tk.oz + g.z0 + z) * nxy + row;
        float4 d;
        if constexpr (DS) d = *d_slot<NT, KC, ZS, DS>(sp, g, z, s.st[kk]);
        else d = d4[kk][z];
        const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          if (!(s.msk[kk] & (1u << l))) continue;
          const double xv = xr[gi0 + l];
          xo[gi0 + l] = (m > 0) ? xv + (double)dv[l] * unscale : xv;
        }
      }
    }
    // x^{k+1} of this block is complete in every CTA before the flag says so
    __threadfence();
    cl_barrier();
    if constexpr (DS) zero_smem<NT>(dyn4, smem_f4);
    if (rank == 0 && tid == 0) {
      st_rel_s32(fa.done_rel + t, kr + 1);
      if (m > 0) {
        atomicAdd(a.inner_count + 2 * tk.rhs, (unsigned long long)m);
        atomicAdd(a.inner_count + 2 * tk.rhs + 1, (unsigned long long)m * (unsigned long long)tk.bx * tk.by * tk.bz);
      }
      if (a.tr.rec) trace_push(a.tr, fa.k0 + kr, tk.block, tk.rhs, m, a.partial[t]);
    }
  }
}

template <int NT, int KC, int ZS, bool DS, int QR>
inline cudaError_t prep_res(int cluster, size_t smem_bytes, void** fn, int kind) {
  void (*kern)(const SweepArgs, int) = res_sweep_kernel<NT, KC, ZS, DS, QR>;
  void (*akern)(const AsyncArgs, int) = res_async_kernel<NT, KC, ZS, DS, QR>;
  void (*fkern)(const FlowArgs, int) = res_flow_kernel<NT, KC, ZS, DS, QR>;
  if (kind == 2) {
    cudaError_t e = cudaFuncSetAttribute(fkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    if (cluster > 8) {
      e = cudaFuncSetAttribute(fkern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    *fn = (void*)fkern;
    return cudaSuccess;
  }
  if (kind == 1) {
    cudaError_t e = cudaFuncSetAttribute(akern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    if (cluster > 8) {
      e = cudaFuncSetAttribute(akern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    *fn = (void*)akern;
    return cudaSuccess;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  *fn = (void*)kern;
  return cudaSuccess;
}

template <int V>
cudaError_t res_prep(int cluster, size_t smem_bytes, void** fn, int kind) {
  constexpr ResVariant r = kResVariants[V];
  return prep_res<r.nt, r.kc, r.zs, r.ds != 0, r.qr>(cluster, smem_bytes, fn, kind);
}

}  // namespace ms
