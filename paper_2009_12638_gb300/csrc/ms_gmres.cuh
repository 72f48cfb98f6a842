// ms_gmres.cuh -- alternative inner stage: restarted GMRES(m) on one block
// system A_ii d = r, run by one thread-block cluster of the (scalar)
// streaming engine.  GMRES is the Krylov method of the paper's own runs
// (PETSc's GMRES, section 3.2); Arnoldi orthogonalises with classical
// Gram-Schmidt (PETSc's default): every projection h_ij of a step comes from
// the same w = A v_j, so one step is two passes over the slab with one
// cluster-wide reduction after each:
//
//   pass 1: w = A_ii v_j, stored as the next basis vector; h_ij = w.v_i, i <= j
//   pass 2: w -= sum_i h_ij v_i; ||w||^2
//
// Projections are reduced kGmresChunk at a time: steps j < kGmresChunk (every
// step when m <= 16) take the single reduction above; a later step re-reads
// the stored w once per further chunk of kGmresChunk basis vectors, so
// registers and shared memory stay bounded up to m = kGmresMaxRestart.
// Basis vectors are stored unnormalised, v_i = sigma_i u_i (sigma_i =
// 1/||w|| of the step that made it), so normalising costs no pass.  Thread 0
// keeps the Hessenberg column, the Givens rotations, the residual estimate
// |g_{j+1}| and the small triangular solve in FP64.  A cycle ends with
// d += sum_i y_i v_i; the next cycle starts from the true residual r - A d.
// Stops when |g_{j+1}| <= inner_rtol ||r|| or after inner_maxit Arnoldi
// steps (the iteration count, one stencil application each).
#pragma once
#include "ms_cg.cuh"
#include "ms_device.cuh"

namespace ms {

constexpr int kGmresMaxRestart = 50;
constexpr int kGmresChunk = 16;  // projections per cluster reduction

template <typename T>
struct GmresVecs {
  T* r;                // block residual on entry (left unchanged)
  T* d;                // correction
  T* u0;               // basis vectors u_0 .. u_m (unnormalised), `stride` apart
  long long stride;
  __device__ __forceinline__ T* u(int i) const { return u0 + (long long)i * stride; }
};

// slot layout: r, d, u_0 .. u_m (m + 3 vectors of vec_stride elements)
template <typename T>
__device__ __forceinline__ GmresVecs<T> gmres_slot_vecs(void* scratch, long long vec_stride, unsigned slot,
                                                        int restart) {
  T* base = reinterpret_cast<T*>(scratch) + (long long)slot * (restart + 3) * vec_stride;
  return GmresVecs<T>{base, base + vec_stride, base + 2 * vec_stride, vec_stride};
}

// Shared state of one cluster's GMRES (thread 0 writes the scalars).
struct GmresSmem {
  double slots[2][kGmresChunk][kMaxCluster];  // consecutive chunk reductions alternate buffers
  double wsum[kGmresChunk][32];
  double H[kGmresMaxRestart + 1][kGmresMaxRestart];  // rotated Hessenberg columns (upper triangle)
  double cs[kGmresMaxRestart], sn[kGmresMaxRestart];
  double g[kGmresMaxRestart + 1];
  double sigma[kGmresMaxRestart + 1];  // v_i = sigma_i u_i
  double coef[kGmresMaxRestart + 1];   // per-pass coefficients on u_i
  double beta0, stop;
  int k, total, done, cycle_end;
};

// 7-point stencil A_ii u at slab point (c, z) of a compact block vector (zero outside the block).
template <typename T>
__device__ __forceinline__ T block_apply(const T* u, const Slab& sl, int c, int z) {
  const int x = c % sl.bx, y = c / sl.bx;
  const int i = z * sl.plane + c;
  T s = 0;
  if (x > 0) s += u[i - 1];
  if (x < sl.bx - 1) s += u[i + 1];
  if (y > 0) s += u[i - sl.bx];
  if (y < sl.by - 1) s += u[i + sl.bx];
  if (z > 0) s += u[i - sl.plane];
  if (z < sl.bz - 1) s += u[i + sl.plane];
  return (T)6 * u[i] - s;
}

// Runs GMRES(restart) from d = 0 on r (gamma0 = r.r already reduced).  Returns
// the number of Arnoldi steps; d holds the correction when it is > 0.
template <typename T, int NT>
__device__ int block_gmres(const GmresVecs<T>& v, int restart, const Slab& sl, double gamma0, double inner_rtol,
                           int inner_maxit, RedSmem& sm, GmresSmem& gs, unsigned rank, unsigned csize) {
  constexpr int C = kGmresChunk;
  const int tid = threadIdx.x;
  if (tid == 0) {
    gs.beta0 = sqrt(gamma0);
    gs.stop = inner_rtol * gs.beta0;
    gs.total = 0;
    gs.done = (!(gamma0 > 0.0) || inner_maxit <= 0) ? 1 : 0;
  }
  __syncthreads();
  if (gs.done) return 0;
  bool first_cycle = true;
  for (;;) {
    // ---- residual of the current iterate into u_0: r (first cycle, d = 0) or r - A d
    {
      T acc = 0;
      T* u0 = v.u(0);
      for (int c = tid; c < sl.plane; c += NT)
        for (int z = sl.z0; z < sl.z1; ++z) {
          const int i = z * sl.plane + c;
          const T w = first_cycle ? v.r[i] : v.r[i] - block_apply(v.d, sl, c, z);
          u0[i] = w;
          acc += w * w;
        }
      const T red[1] = {acc};
      cluster_reduce<NT, 1>(red, sm.slots[2], sm.wsum, rank, csize, [&](double (&t)[1]) {
        const double beta = sqrt(t[0]);
        if (!(beta > gs.stop) || gs.total >= inner_maxit) {
          gs.done = 1;
        } else {
          gs.sigma[0] = 1.0 / beta;
          for (int q = 0; q <= kGmresMaxRestart; ++q) gs.g[q] = 0.0;
          gs.g[0] = beta;
          gs.k = 0;
          gs.cycle_end = 0;
        }
      });
    }
    if (gs.done) break;
    for (int j = 0; j < restart; ++j) {
      const int nch = j / C + 1;  // chunks of projections in this step
      T* un = v.u(j + 1);
      // ---- pass 1: w = A v_j into u_{j+1}; projections on u_0..u_{min(j, C-1)}
      // ---- pass 1b (j >= C): projections of the stored w on the further chunks
      for (int ch = 0; ch < nch; ++ch) {
        const int q0 = ch * C;
        T hp[C];
#pragma unroll
        for (int q = 0; q < C; ++q) hp[q] = 0;
        const T sj = (T)gs.sigma[j];
        const T* uj = v.u(j);
        for (int c = tid; c < sl.plane; c += NT)
          for (int z = sl.z0; z < sl.z1; ++z) {
            const int i = z * sl.plane + c;
            T w;
            if (ch == 0) {
              w = sj * block_apply(uj, sl, c, z);
              un[i] = w;
            } else {
              w = un[i];
            }
#pragma unroll
            for (int q = 0; q < C; ++q)
              if (q0 + q <= j) hp[q] += w * v.u(q0 + q)[i];
          }
        cluster_reduce<NT, C>(hp, gs.slots[ch & 1], gs.wsum, rank, csize, [&](double (&t)[C]) {
          for (int q = 0; q < C && q0 + q <= j; ++q) {
            gs.H[q0 + q][j] = gs.sigma[q0 + q] * t[q];           // h_qj = w . v_q
            gs.coef[q0 + q] = gs.H[q0 + q][j] * gs.sigma[q0 + q];  // on u_q in pass 2
          }
        });
      }
      // ---- pass 2: w -= sum_q h_qj v_q (one pass per chunk), ||w||^2 in the last
      {
        T acc = 0;
        for (int ch = 0; ch < nch; ++ch) {
          const int q0 = ch * C;
          const bool last = ch == nch - 1;
          T cq[C];
#pragma unroll
          for (int q = 0; q < C; ++q) cq[q] = q0 + q <= j ? (T)gs.coef[q0 + q] : (T)0;
          for (int c = tid; c < sl.plane; c += NT)
            for (int z = sl.z0; z < sl.z1; ++z) {
              const int i = z * sl.plane + c;
              T w = un[i];
#pragma unroll
              for (int q = 0; q < C; ++q)
                if (q0 + q <= j) w -= cq[q] * v.u(q0 + q)[i];
              un[i] = w;
              if (last) acc += w * w;
            }
        }
        const T red[1] = {acc};
        cluster_reduce<NT, 1>(red, sm.slots[1], sm.wsum, rank, csize, [&](double (&t)[1]) {
          const double hn = sqrt(t[0]);
          gs.sigma[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
          // earlier rotations on column j, then the one that zeroes h_{j+1,j}
          for (int q = 0; q < j; ++q) {
            const double a = gs.H[q][j], b = gs.H[q + 1][j];
            gs.H[q][j] = gs.cs[q] * a + gs.sn[q] * b;
            gs.H[q + 1][j] = -gs.sn[q] * a + gs.cs[q] * b;
          }
          const double a = gs.H[j][j], b = hn;
          const double rho = sqrt(a * a + b * b);
          gs.cs[j] = rho > 0.0 ? a / rho : 1.0;
          gs.sn[j] = rho > 0.0 ? b / rho : 0.0;
          gs.H[j][j] = rho;
          gs.g[j + 1] = -gs.sn[j] * gs.g[j];
          gs.g[j] = gs.cs[j] * gs.g[j];
          gs.total += 1;
          gs.k = j + 1;
          if (fabs(gs.g[j + 1]) <= gs.stop || gs.total >= inner_maxit || hn == 0.0) gs.cycle_end = 1;
        });
      }
      if (gs.cycle_end) break;
    }
    // ---- y = R^{-1} g, then d (+)= sum_q y_q v_q (one pass per chunk)
    if (tid == 0) {
      const int k = gs.k;
      double y[kGmresMaxRestart];
      for (int q = k - 1; q >= 0; --q) {
        double s = gs.g[q];
        for (int c = q + 1; c < k; ++c) s -= gs.H[q][c] * y[c];
        y[q] = gs.H[q][q] != 0.0 ? s / gs.H[q][q] : 0.0;
      }
      for (int q = 0; q <= kGmresMaxRestart; ++q) gs.coef[q] = q < k ? y[q] * gs.sigma[q] : 0.0;
      // the cycle's last estimate decides whether another cycle runs
      if (fabs(gs.g[k]) <= gs.stop || gs.total >= inner_maxit) gs.done = 1;
    }
    __syncthreads();
    {
      const int k = gs.k;
      const int nch = k > C ? (k + C - 1) / C : 1;
      for (int ch = 0; ch < nch; ++ch) {
        const int q0 = ch * C;
        const bool fresh = first_cycle && ch == 0;
        T cq[C];
#pragma unroll
        for (int q = 0; q < C; ++q) cq[q] = q0 + q < k ? (T)gs.coef[q0 + q] : (T)0;
        for (int c = tid; c < sl.plane; c += NT)
          for (int z = sl.z0; z < sl.z1; ++z) {
            const int i = z * sl.plane + c;
            T acc = 0;
#pragma unroll
            for (int q = 0; q < C; ++q)
              if (q0 + q < k) acc += cq[q] * v.u(q0 + q)[i];
            v.d[i] = fresh ? acc : v.d[i] + acc;
          }
      }
    }
    first_cycle = false;
    if (gs.done) break;
    // the next residual reads d across the slabs of the other CTAs
    cl_barrier();
  }
  return gs.total;
}

}  // namespace ms
