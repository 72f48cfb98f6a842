// ms_async.cu -- asynchronous outer iteration (sections 2.1, 2.3 and 3 of
// the paper): blocks never wait for one another.  One persistent launch; task
// t = (block, rhs) is owned by cluster t % nclusters and visited round-robin.
// A visit is one local outer sweep of that block:
//
//   1. halo refresh: for each neighbouring block, take its most recently
//      published face if a consistent copy can be read (seqlock), else keep
//      the halo already held -- the paper's "latest completed receive,
//      otherwise continue with existing data";
//   2. block residual r = bhat_i - A_ii x_i - sum_j A_ij (halo) in FP64, and
//      its sum of squares published (racy) for the global estimate;
//   3. inner CG on A_ii d = r (ms_cg.cuh);
//   4. x_i += d in place, fused with publishing the six boundary layers into
//      the block's face slots (two slots per face, seqlock counters);
//   5. the stale global estimate sqrt(sum_i ||r_i||^2)/||bhat|| (section 3:
//      an estimate that may be some iterations old) is formed from the
//      published partials; when it is below tol for a rhs its tasks stop.
//
// No wait anywhere depends on another cluster: readers that see a slot being
// rewritten simply keep their old halo.  The host checks the true residual
// after the launch and relaunches (state kept) if the estimate was optimistic.
#include <cuda_runtime.h>

#include "ms_cg.cuh"
#include "ms_device.cuh"
#include "ms_internal.h"

namespace ms {

__device__ __forceinline__ unsigned ld_acq_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_rlx_u32(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_rlx_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rlx_s32(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ double ld_rlx_f64(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rlx_f64(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// face f of a bx*by*bz block: 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+
__device__ __forceinline__ int face_size(int f, int bx, int by, int bz) {
  return f < 2 ? bz * by : (f < 4 ? bz * bx : by * bx);
}

// neighbouring task across face f, or -1 at the domain boundary
__device__ __forceinline__ int nbr_task(const AsyncArgs& a, const Task& tk, int f) {
  const int b = tk.block;
  int bi = b % a.px, bj = (b / a.px) % a.py, bk = b / (a.px * a.py);
  switch (f) {
    case 0: bi -= 1; break;
    case 1: bi += 1; break;
    case 2: bj -= 1; break;
    case 3: bj += 1; break;
    case 4: bk -= 1; break;
    default: bk += 1; break;
  }
  if (bi < 0 || bi >= a.px || bj < 0 || bj >= a.py || bk < 0 || bk >= a.pz) return -1;
  return a.task_of[(long long)tk.rhs * a.nblocks + bi + a.px * (bj + a.py * bk)];
}

// ---------------------------------------------------------------- init
// Publish every block's faces of x^0 into slot 0 and fill every halo slot 0
// with the neighbours' faces; partial sums start at +huge so no rhs can stop
// before all of its blocks have reported once.
__global__ void async_init_kernel(const AsyncArgs a) {
  const long long fs = a.face_stride;
  const long long total = (long long)a.ntasks * 6 * fs;
  const long long nxy = (long long)a.g.nx * a.g.ny;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / (6 * fs));
    const int f = (int)((e / fs) % 6);
    const int idx = (int)(e % fs);
    const Task tk = a.tasks[t];
    if (idx == 0 && f == 0) {
      a.partial[t] = 1.0e300;
      a.sweeps[t] = 0;
    }
    if (idx >= face_size(f, tk.bx, tk.by, tk.bz)) continue;
    // coordinates (in block) of face element idx, and of the point just outside
    int x, y, z;
    if (f < 2) {
      z = idx / tk.by;
      y = idx % tk.by;
      x = f == 0 ? 0 : tk.bx - 1;
    } else if (f < 4) {
      z = idx / tk.bx;
      x = idx % tk.bx;
      y = f == 2 ? 0 : tk.by - 1;
    } else {
      y = idx / tk.bx;
      x = idx % tk.bx;
      z = f == 4 ? 0 : tk.bz - 1;
    }
    const double* xr = a.x + (long long)tk.rhs * a.g.npts;
    const int gx = tk.ox + x, gy = tk.oy + y, gz = tk.oz + z;
    a.faces[(((long long)t * 6 + f) * 2 + 0) * fs + idx] = xr[(long long)gz * nxy + (long long)gy * a.g.nx + gx];
    const int dx = f == 0 ? -1 : (f == 1 ? 1 : 0), dy = f == 2 ? -1 : (f == 3 ? 1 : 0),
              dz = f == 4 ? -1 : (f == 5 ? 1 : 0);
    const int ox = gx + dx, oy = gy + dy, oz = gz + dz;
    double hv = 0.0;
    if (ox >= 0 && ox < a.g.nx && oy >= 0 && oy < a.g.ny && oz >= 0 && oz < a.g.nz)
      hv = xr[(long long)oz * nxy + (long long)oy * a.g.nx + ox];
    a.halo[(((long long)t * 6 + f) * 2 + 0) * fs + idx] = hv;
  }
}

// After an optimistic stop, every block of a re-armed rhs must report a fresh
// partial before the estimate of that rhs can stop the launch again.
__global__ void async_rearm_kernel(const AsyncArgs a) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a.ntasks; t += gridDim.x * blockDim.x)
    if (!a.rhs_stop[a.tasks[t].rhs]) a.partial[t] = 1.0e300;
}

// ---------------------------------------------------------------- persistent kernel
template <typename T, int NT>
__global__ void __launch_bounds__(NT, 1) async_kernel(const AsyncArgs a) {
  __shared__ RedSmem sm;
  __shared__ int bc[2][32];  // rank 0 -> cluster broadcast, double buffered
  const unsigned rank = cl_rank(), csize = cl_size(), cid = cl_id(), ncl = cl_count();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const CgVecs<T> v = slot_vecs<T>(a.scratch, a.vec_stride, cid);
  const Geo g = a.g;
  const long long nxy = (long long)g.nx * g.ny;
  const long long fs = a.face_stride;
  const unsigned long long t_start = globaltimer();
  int par = 0;
  int next = (int)cid;   // rank-0 thread 0 only: round-robin cursor
  unsigned s1v[6], vvv[6];  // rank-0 thread 0 only: seqlock snapshot
  const int owned = (int)cid < a.ntasks ? (a.ntasks - (int)cid + (int)ncl - 1) / (int)ncl : 0;
  const unsigned cl_threads = csize * NT;
  const unsigned cl_tid = rank * NT + tid;

  for (;;) {
    // ---------------- control: pick the next runnable owned task
    if (rank == 0 && tid == 0) {
      int cmd = 0, t = -1;
      if (ld_rlx_s32(a.stop)) {
        cmd = 1;
      } else if (a.time_budget_ns && globaltimer() - t_start > a.time_budget_ns) {
        atomicOr(a.err, kErrTimeout);
        st_rlx_s32(a.stop, 1);
        cmd = 1;
      } else if (a.slice_ns && globaltimer() - t_start > a.slice_ns) {
        cmd = 1;  // end of this launch's time slice: state is kept, the host relaunches
      } else {
        for (int j = 0; j < owned; ++j) {
          const int cand = next;
          next += (int)ncl;
          if (next >= a.ntasks) next = (int)cid;
          if (a.sweeps[cand] < a.outer_maxit && !ld_rlx_s32(a.rhs_stop + a.tasks[cand].rhs)) {
            t = cand;
            break;
          }
        }
        if (t < 0) cmd = 1;
      }
      for (unsigned j = 0; j < csize; ++j) {
        cl_store(&bc[par][0], j, cmd);
        cl_store(&bc[par][1], j, t);
      }
    }
    cl_barrier();
    const int cmd = bc[par][0], t = bc[par][1];
    if (cmd) break;
    const Task tk = a.tasks[t];
    if ((long long)tk.bx * tk.by * tk.bz > a.vec_stride || face_size(0, tk.bx, tk.by, tk.bz) > fs ||
        face_size(2, tk.bx, tk.by, tk.bz) > fs || face_size(4, tk.bx, tk.by, tk.bz) > fs) {
      if (rank == 0 && tid == 0) {
        atomicOr(a.err, kErrGeometry);
        st_rlx_s32(a.stop, 1);
      }
      par ^= 1;
      continue;
    }
    if (a.slow_block == tk.block && a.slow_ns > 0 && rank == 0 && tid == 0)
      __nanosleep((unsigned)min(a.slow_ns, 1000000));

    // ---------------- 1. halo refresh (seqlock read of the neighbours' latest faces)
    if (rank == 0 && tid == 0) {
      for (int f = 0; f < 6; ++f) {
        const int nb = nbr_task(a, tk, f);
        int want = 0, sl = 0;
        const int cur = a.halo_cur[t * 6 + f];
        if (nb >= 0) {
          const unsigned vv = ld_acq_u32(a.face_ver + nb * 6 + (f ^ 1));
          if (vv != a.halo_ver[t * 6 + f]) {
            sl = (int)(vv & 1u);
            const unsigned s1 = ld_acq_u32(a.face_seq + (nb * 6 + (f ^ 1)) * 2 + sl);
            if (!(s1 & 1u)) {
              want = 1;
              s1v[f] = s1;
              vvv[f] = vv;
            }
          }
        }
        for (unsigned j = 0; j < csize; ++j) {
          cl_store(&bc[par][2 + f], j, want ? nb : -1);
          cl_store(&bc[par][8 + f], j, sl);
          cl_store(&bc[par][14 + f], j, cur);
        }
      }
    }
    cl_barrier();
    int hcur[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int nb = bc[par][2 + f];
      hcur[f] = bc[par][14 + f];
      if (nb < 0) continue;
      const int sl = bc[par][8 + f];
      const int nel = face_size(f, tk.bx, tk.by, tk.bz);
      const double* src = a.faces + (((long long)nb * 6 + (f ^ 1)) * 2 + sl) * fs;
      double* dst = a.halo + (((long long)t * 6 + f) * 2 + (hcur[f] ^ 1)) * fs;
      for (unsigned e = cl_tid; e < (unsigned)nel; e += cl_threads) dst[e] = __ldcg(src + e);
    }
    __threadfence();
    cl_barrier();
    if (rank == 0 && tid == 0) {
      for (int f = 0; f < 6; ++f) {
        const int nb = bc[par][2 + f];
        int cur = bc[par][14 + f];
        if (nb >= 0) {
          const unsigned s2 = ld_acq_u32(a.face_seq + (nb * 6 + (f ^ 1)) * 2 + bc[par][8 + f]);
          if (s2 == s1v[f]) {  // consistent copy: switch to it
            cur ^= 1;
            a.halo_cur[t * 6 + f] = cur;
            a.halo_ver[t * 6 + f] = vvv[f];
          }
        }
        for (unsigned j = 0; j < csize; ++j) cl_store(&bc[par][20 + f], j, cur);
      }
    }
    cl_barrier();
    const double* hp[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      hcur[f] = bc[par][20 + f];
      hp[f] = a.halo + (((long long)t * 6 + f) * 2 + hcur[f]) * fs;
    }

    // ---------------- 2. block residual from own x and the halo, FP64
    // (FP32 inner: r times a power of two ~ 1/||bhat||, undone in the update)
    const double scale = inner_scale<T>(a.inv_bnorm[tk.rhs]), unscale = 1.0 / scale;
    const Slab sl = make_slab(tk.bx, tk.by, tk.bz, rank, csize);
    const long long rb = (long long)tk.rhs * g.npts;
    double* xr = a.x + rb;
    const double* __restrict__ fr = a.f ? a.f + rb : nullptr;
    const double* __restrict__ br = a.bnd ? a.bnd + (long long)tk.rhs * g.nbnd : nullptr;
    const long long fyz = (long long)g.nz * g.ny, fxz = (long long)g.nz * g.nx;
    double red0[2] = {0.0, 0.0};
    {
      double s_loc = 0.0;
      T g_loc = 0;
      for (int c = tid; c < sl.plane; c += NT) {
        const int x = c % tk.bx, y = c / tk.bx;
        const int gx = tk.ox + x, gy = tk.oy + y;
        for (int z = sl.z0; z < sl.z1; ++z) {
          const int gz = tk.oz + z;
          const long long gi = (long long)gz * nxy + (long long)gy * g.nx + gx;
          double si = 0.0, so = 0.0;
          // x-
          if (x > 0) si += xr[gi - 1];
          else if (gx > 0) si += hp[0][z * tk.by + y];
          else if (br) so += br[(long long)gz * g.ny + gy];
          // x+
          if (x < tk.bx - 1) si += xr[gi + 1];
          else if (gx < g.nx - 1) si += hp[1][z * tk.by + y];
          else if (br) so += br[fyz + (long long)gz * g.ny + gy];
          // y-
          if (y > 0) si += xr[gi - g.nx];
          else if (gy > 0) si += hp[2][z * tk.bx + x];
          else if (br) so += br[2 * fyz + (long long)gz * g.nx + gx];
          // y+
          if (y < tk.by - 1) si += xr[gi + g.nx];
          else if (gy < g.ny - 1) si += hp[3][z * tk.bx + x];
          else if (br) so += br[2 * fyz + fxz + (long long)gz * g.nx + gx];
          // z-
          if (z > 0) si += xr[gi - nxy];
          else if (gz > 0) si += hp[4][y * tk.bx + x];
          else if (br) so += br[2 * fyz + 2 * fxz + (long long)gy * g.nx + gx];
          // z+
          if (z < tk.bz - 1) si += xr[gi + nxy];
          else if (gz < g.nz - 1) si += hp[5][y * tk.bx + x];
          else if (br) so += br[2 * fyz + 2 * fxz + nxy + (long long)gy * g.nx + gx];
          const double bh = fr ? fr[gi] + so : so;
          const double rr = bh - (6.0 * xr[gi] - si);
          s_loc += rr * rr;
          const T rt = (T)(rr * scale);
          v.r[z * sl.plane + c] = rt;
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
    if (rank == 0 && tid == 0) st_rlx_f64(a.partial + t, red0[0]);

    // ---------------- 3. inner CG
    const int m = block_cg<T, NT>(v, sl, red0[1], a.inner_rtol, a.inner_maxit, sm, rank, csize);

    // ---------------- 4. update in place + publish faces
    if (rank == 0 && tid == 0) {
      for (int f = 0; f < 6; ++f) {
        int slot = -1;
        if (nbr_task(a, tk, f) >= 0) {
          const unsigned vv = a.face_ver[t * 6 + f];
          slot = (int)((vv + 1u) & 1u);
          unsigned* sp = a.face_seq + (t * 6 + f) * 2 + slot;
          st_rlx_u32(sp, *sp + 1u);  // odd: slot being written
        }
        for (unsigned j = 0; j < csize; ++j) cl_store(&bc[par][26 + f], j, slot);
      }
      __threadfence();
    }
    cl_barrier();
    __threadfence();
    int fslot[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) fslot[f] = bc[par][26 + f];
    for (int c = tid; c < sl.plane; c += NT) {
      const int x = c % tk.bx, y = c / tk.bx;
      const int gx = tk.ox + x, gy = tk.oy + y;
      for (int z = sl.z0; z < sl.z1; ++z) {
        const long long gi = (long long)(tk.oz + z) * nxy + (long long)gy * g.nx + gx;
        const double xn = (m > 0) ? xr[gi] + (double)v.d[z * sl.plane + c] * unscale : xr[gi];
        xr[gi] = xn;
        if (x == 0 && fslot[0] >= 0) a.faces[(((long long)t * 6 + 0) * 2 + fslot[0]) * fs + z * tk.by + y] = xn;
        if (x == tk.bx - 1 && fslot[1] >= 0)
          a.faces[(((long long)t * 6 + 1) * 2 + fslot[1]) * fs + z * tk.by + y] = xn;
        if (y == 0 && fslot[2] >= 0) a.faces[(((long long)t * 6 + 2) * 2 + fslot[2]) * fs + z * tk.bx + x] = xn;
        if (y == tk.by - 1 && fslot[3] >= 0)
          a.faces[(((long long)t * 6 + 3) * 2 + fslot[3]) * fs + z * tk.bx + x] = xn;
        if (z == 0 && fslot[4] >= 0) a.faces[(((long long)t * 6 + 4) * 2 + fslot[4]) * fs + y * tk.bx + x] = xn;
        if (z == tk.bz - 1 && fslot[5] >= 0)
          a.faces[(((long long)t * 6 + 5) * 2 + fslot[5]) * fs + y * tk.bx + x] = xn;
      }
    }
    __threadfence();
    cl_barrier();
    if (rank == 0 && tid == 0) {
      for (int f = 0; f < 6; ++f) {
        if (fslot[f] < 0) continue;
        unsigned* sp = a.face_seq + (t * 6 + f) * 2 + fslot[f];
        st_rel_u32(sp, *sp + 1u);  // even: slot complete
        st_rel_u32(a.face_ver + t * 6 + f, a.face_ver[t * 6 + f] + 1u);
      }
      a.sweeps[t] += 1;
      if (m > 0) {
        atomicAdd(a.inner_count + 2 * tk.rhs, (unsigned long long)m);
        atomicAdd(a.inner_count + 2 * tk.rhs + 1, (unsigned long long)m * (unsigned long long)(sl.plane * tk.bz));
      }
    }

    // ---------------- 5. stale global estimate per rhs (warp 0 of rank 0)
    if (rank == 0 && warp == 0) {
      int all = 1;
      for (int r = 0; r < g.nrhs; ++r) {
        if (ld_rlx_s32(a.rhs_stop + r)) continue;
        double s = 0.0;
        for (int b = lane; b < a.nblocks; b += 32) s += ld_rlx_f64(a.partial + a.task_of[(long long)r * a.nblocks + b]);
        s = warp_sum_to_lane0(s);
        s = __shfl_sync(0xffffffffu, s, 0);
        if (sqrt(s) * a.inv_bnorm[r] < a.outer_tol) {
          if (lane == 0) st_rlx_s32(a.rhs_stop + r, 1);
        } else {
          all = 0;
        }
      }
      if (all && lane == 0) st_rlx_s32(a.stop, 1);
    }
    par ^= 1;
  }
}

// ---------------------------------------------------------------- launchers
template <typename T, int NT>
static cudaError_t launch_async_t(int cluster, int slots, const AsyncArgs& a, cudaStream_t s) {
  auto kern = async_kernel<T, NT>;
  if (cluster > 8) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(cluster * slots), 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
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
static cudaError_t async_occ_t(int cluster, int* out) {
  auto kern = async_kernel<T, NT>;
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

#define MS_ADISPATCH(prec, threads, FN, ...)                    \
  do {                                                          \
    if (prec == 1) {                                            \
      if (threads == 256) return FN<float, 256>(__VA_ARGS__);   \
      if (threads == 512) return FN<float, 512>(__VA_ARGS__);   \
      if (threads == 1024) return FN<float, 1024>(__VA_ARGS__); \
    } else {                                                    \
      if (threads == 256) return FN<double, 256>(__VA_ARGS__);  \
      if (threads == 512) return FN<double, 512>(__VA_ARGS__);  \
      if (threads == 1024) return FN<double, 1024>(__VA_ARGS__);\
    }                                                           \
    return cudaErrorInvalidValue;                               \
  } while (0)

cudaError_t launch_async(int prec, int threads, int cluster, int slots, const AsyncArgs& a, cudaStream_t s) {
  MS_ADISPATCH(prec, threads, launch_async_t, cluster, slots, a, s);
}

cudaError_t async_max_clusters(int prec, int threads, int cluster, int* out) {
  MS_ADISPATCH(prec, threads, async_occ_t, cluster, out);
}

cudaError_t launch_async_rearm(const AsyncArgs& a, cudaStream_t s) {
  async_rearm_kernel<<<(a.ntasks + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_async_init(const AsyncArgs& a, cudaStream_t s) {
  const long long total = (long long)a.ntasks * 6 * a.face_stride;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  async_init_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ms
