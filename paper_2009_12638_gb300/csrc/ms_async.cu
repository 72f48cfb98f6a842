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

#include "ms_async.cuh"
#include "ms_cg.cuh"
#include "ms_device.cuh"
#include "ms_internal.h"

namespace ms {

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
  const int tid = threadIdx.x;
  const CgVecs<T> v = slot_vecs<T>(a.scratch, a.vec_stride, cid);
  const Geo g = a.g;
  const long long nxy = (long long)g.nx * g.ny;
  const long long fs = a.face_stride;
  __shared__ unsigned snap[12];
  AsyncCtl c = async_ctl_init(a, cid, ncl, snap);
  for (;; c.par ^= 1) {
    const int t = async_pick(a, c, bc, rank, csize, cid, ncl);
    if (t < 0) break;
    const Task tk = a.tasks[t];
    if ((long long)tk.bx * tk.by * tk.bz > a.vec_stride || face_size(0, tk.bx, tk.by, tk.bz) > fs ||
        face_size(2, tk.bx, tk.by, tk.bz) > fs || face_size(4, tk.bx, tk.by, tk.bz) > fs) {
      if (rank == 0 && tid == 0) {
        atomicOr(a.err, kErrGeometry);
        st_rlx_s32(a.stop, 1);
      }
      continue;
    }
    if (a.slow_block == tk.block && a.slow_ns > 0 && rank == 0 && tid == 0)
      __nanosleep((unsigned)min(a.slow_ns, 1000000));
    // ---------------- 1. halo refresh
    async_halo_refresh<NT>(a, tk, t, bc, c, rank, csize);
    const int* hcur = bc[c.par] + 20;
    // ---------------- 2. block residual from own x and the halo, FP64
    // (FP32 inner: r times a power of two ~ 1/||bhat||, undone in the update)
    const double scale = inner_scale<T>(a.inv_bnorm[tk.rhs]), unscale = 1.0 / scale;
    const Slab sl = make_slab(tk.bx, tk.by, tk.bz, rank, csize);
    const long long rb = (long long)tk.rhs * g.npts;
    double* xr = a.x + rb;
    const double* __restrict__ fr = a.f ? a.f + rb : nullptr;
    const double* __restrict__ br = a.bnd ? a.bnd + (long long)tk.rhs * g.nbnd : nullptr;
    double red0[2] = {0.0, 0.0};
    {
      double s_loc = 0.0;
      T g_loc = 0;
      for (int cc = tid; cc < sl.plane; cc += NT) {
        const int x = cc % tk.bx, y = cc / tk.bx;
        for (int z = sl.z0; z < sl.z1; ++z) {
          const long long gi = (long long)(tk.oz + z) * nxy + (long long)(tk.oy + y) * g.nx + tk.ox + x;
          double si, so;
          async_nbr_sums(a, tk, t, hcur, xr, br, x, y, z, gi, si, so);
          const double bh = fr ? fr[gi] + so : so;
          const double rr = bh - (6.0 * xr[gi] - si);
          s_loc += rr * rr;
          const T rt = (T)(rr * scale);
          v.r[z * sl.plane + cc] = rt;
          g_loc += rt * rt;
        }
      }
      red0[0] = s_loc;
      red0[1] = (double)g_loc;
    }
    cluster_reduce<NT, 2>(red0, sm.slots[0], sm.wsum, rank, csize, [&](double (&tt)[2]) {
      sm.tot[0] = tt[0];
      sm.tot[1] = tt[1];
    });
    if (rank == 0 && tid == 0) st_rlx_f64(a.partial + t, sm.tot[0]);
    // ---------------- 3. inner CG
    const int m = block_cg<T, NT>(v, sl, sm.tot[1], a.inner_rtol, a.inner_maxit, sm, rank, csize);
    // ---------------- 4. update in place + publish faces
    async_publish_begin(a, tk, t, bc, c, rank, csize);
    const int* fslot = bc[c.par] + 26;
    for (int cc = tid; cc < sl.plane; cc += NT) {
      const int x = cc % tk.bx, y = cc / tk.bx;
      for (int z = sl.z0; z < sl.z1; ++z) {
        const long long gi = (long long)(tk.oz + z) * nxy + (long long)(tk.oy + y) * g.nx + tk.ox + x;
        const double xn = (m > 0) ? xr[gi] + (double)v.d[z * sl.plane + cc] * unscale : xr[gi];
        xr[gi] = xn;
        async_face_store(a, tk, t, fslot, x, y, z, xn);
      }
    }
    async_publish_end(a, tk, t, fslot, rank, m);
    // ---------------- 5. stale global estimate
    async_monitor(a, rank);
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
