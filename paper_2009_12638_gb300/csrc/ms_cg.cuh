// ms_cg.cuh -- the inner stage: conjugate gradients on one block system
// A_ii d = r (sections 2.2 and 3 of the paper), run by one thread-block
// cluster.  A_ii is the 7-point stencil restricted to the block, zero outside.
//
// Work split: the block (bx*by*bz points, x fastest, compact in a per-cluster
// scratch slot) is cut into z-slabs, one per CTA of the cluster; inside a
// slab a thread owns whole z-columns of the (x, y) plane and marches up z
// keeping the column's neighbours in registers.  Each CG iteration is two
// streaming passes over the slab with one cluster-wide reduction after each:
//
//   pass A: p_new = r + beta p_old at the point and its six neighbours
//           (formed on the fly), q = A_ii p_new, store p_new, eta = p.q
//   pass B: q = A_ii p_new again (recomputed, not stored), d += alpha p_new,
//           r -= alpha q, gamma = r.r
//
// which moves 32 bytes per point per iteration at FP32 (r and p_old read,
// p_new written; p_new read, d and r read and written).  p is double
// buffered so pass A never reads what it writes.
#pragma once
#include "ms_device.cuh"

namespace ms {

template <typename T>
struct CgVecs {
  T* r;
  T* p0;
  T* p1;
  T* d;
};

template <typename T>
__device__ __forceinline__ CgVecs<T> slot_vecs(void* scratch, long long vec_stride, unsigned slot) {
  T* base = reinterpret_cast<T*>(scratch) + (long long)slot * 4 * vec_stride;
  return CgVecs<T>{base, base + vec_stride, base + 2 * vec_stride, base + 3 * vec_stride};
}

struct Slab {
  int bx, by, bz, plane, z0, z1;
};

__device__ __forceinline__ Slab make_slab(int bx, int by, int bz, unsigned rank, unsigned csize) {
  Slab s;
  s.bx = bx;
  s.by = by;
  s.bz = bz;
  s.plane = bx * by;
  s.z0 = (int)(((long long)bz * rank) / csize);
  s.z1 = (int)(((long long)bz * (rank + 1)) / csize);
  return s;
}

// Scale applied to the residual before it is rounded to the inner precision:
// for FP32 a power of two (exact) close to 1/||bhat||, so the inner solve
// works on O(relative residual) numbers whatever the magnitude of the data;
// FP64 needs none.
template <typename T>
__device__ __forceinline__ double inner_scale(double inv_bnorm) {
  if (sizeof(T) == sizeof(double) || !(inv_bnorm > 0.0) || !isfinite(inv_bnorm)) return 1.0;
  int e;
  frexp(inv_bnorm, &e);
  return ldexp(1.0, e - 1);
}

template <typename T>
__device__ __forceinline__ T step_alpha(const RedSmem& sm);
template <>
__device__ __forceinline__ float step_alpha<float>(const RedSmem& sm) { return sm.alpha; }
template <>
__device__ __forceinline__ double step_alpha<double>(const RedSmem& sm) { return sm.alpha_d; }
template <typename T>
__device__ __forceinline__ T step_beta(const RedSmem& sm);
template <>
__device__ __forceinline__ float step_beta<float>(const RedSmem& sm) { return sm.beta; }
template <>
__device__ __forceinline__ double step_beta<double>(const RedSmem& sm) { return sm.beta_d; }

// CG scalar bookkeeping, run by thread 0 only (see cluster_reduce).
__device__ __forceinline__ void cg_begin(RedSmem& sm, double gamma0, double inner_rtol, int inner_maxit) {
  if (threadIdx.x == 0) {
    sm.gamma = gamma0;
    sm.gamma0 = gamma0;
    sm.stop = inner_rtol * sqrt(gamma0);
    sm.m = 0;
    sm.done = (!(gamma0 > 0.0) || inner_maxit <= 0) ? 1 : 0;
    sm.beta = 0.f;
    sm.beta_d = 0.0;
  }
  __syncthreads();
}
// after eta = p.q: curvature breakdown (or NaN) ends the solve, else alpha = gamma / eta
__device__ __forceinline__ void cg_after_eta(RedSmem& sm, double eta) {
  if (!(eta > 0.0)) {
    sm.done = 1;
  } else {
    sm.alpha_d = sm.gamma / eta;
    sm.alpha = (float)sm.alpha_d;
  }
}
// after gamma_new = r.r: count the step, stop test ||r|| <= rtol ||r0||, else beta
__device__ __forceinline__ void cg_after_gamma(RedSmem& sm, double gnew, int inner_maxit) {
  sm.m += 1;
  if (sqrt(gnew) <= sm.stop || sm.m >= inner_maxit) {
    sm.done = 1;
  } else {
    sm.beta_d = gnew / sm.gamma;
    sm.beta = (float)sm.beta_d;
    sm.gamma = gnew;
  }
}

// Runs CG from d = 0 on r (gamma0 = r.r already reduced).  Returns the
// number of iterations m; d holds the correction when m > 0.
template <typename T, int NT>
__device__ int block_cg(const CgVecs<T>& v, const Slab& sl, double gamma0, double inner_rtol, int inner_maxit,
                        RedSmem& sm, unsigned rank, unsigned csize) {
  cg_begin(sm, gamma0, inner_rtol, inner_maxit);
  if (sm.done) return 0;
  const int tid = threadIdx.x;
  const int plane = sl.plane, bx = sl.bx, by = sl.by, bz = sl.bz, z0 = sl.z0, z1 = sl.z1;
  T* po = v.p0;
  T* pn = v.p1;
  T* const rv = v.r;  // written by pass B, read by pass A: plain coherent loads
  bool first = true;
  for (;;) {
    const T bT = step_beta<T>(sm);
    // ---------------- pass A
    T eta_loc = 0;
    for (int c = tid; c < plane; c += NT) {
      const int x = c % bx, y = c / bx;
      const bool xm = x > 0, xp = x < bx - 1, ym = y > 0, yp = y < by - 1;
#define MS_PVAL(idx) (first ? rv[(idx)] : rv[(idx)] + bT * po[(idx)])
      T pzm = (z0 > 0 && z0 < z1) ? MS_PVAL((z0 - 1) * plane + c) : (T)0;
      T pc = (z0 < z1) ? MS_PVAL(z0 * plane + c) : (T)0;
      for (int z = z0; z < z1; ++z) {
        const int i = z * plane + c;
        const T pzp = (z + 1 < bz) ? MS_PVAL(i + plane) : (T)0;
        T s = pzm + pzp;
        if (xm) s += MS_PVAL(i - 1);
        if (xp) s += MS_PVAL(i + 1);
        if (ym) s += MS_PVAL(i - bx);
        if (yp) s += MS_PVAL(i + bx);
        const T q = (T)6 * pc - s;
        pn[i] = pc;
        eta_loc += pc * q;
        pzm = pc;
        pc = pzp;
      }
#undef MS_PVAL
    }
    {
      const T red1[1] = {eta_loc};
      cluster_reduce<NT, 1>(red1, sm.slots[1], sm.wsum, rank, csize,
                            [&](double (&t)[1]) { cg_after_eta(sm, t[0]); });
    }
    if (sm.done) break;
    const T aT = step_alpha<T>(sm);
    // ---------------- pass B
    T g_loc = 0;
    for (int c = tid; c < plane; c += NT) {
      const int x = c % bx, y = c / bx;
      const bool xm = x > 0, xp = x < bx - 1, ym = y > 0, yp = y < by - 1;
      T pzm = (z0 > 0 && z0 < z1) ? pn[(z0 - 1) * plane + c] : (T)0;
      T pc = (z0 < z1) ? pn[z0 * plane + c] : (T)0;
      for (int z = z0; z < z1; ++z) {
        const int i = z * plane + c;
        const T pzp = (z + 1 < bz) ? pn[i + plane] : (T)0;
        T s = pzm + pzp;
        if (xm) s += pn[i - 1];
        if (xp) s += pn[i + 1];
        if (ym) s += pn[i - bx];
        if (yp) s += pn[i + bx];
        const T q = (T)6 * pc - s;
        v.d[i] = first ? aT * pc : v.d[i] + aT * pc;
        const T rn = v.r[i] - aT * q;
        v.r[i] = rn;
        g_loc += rn * rn;
        pzm = pc;
        pc = pzp;
      }
    }
    {
      const T red2[1] = {g_loc};
      cluster_reduce<NT, 1>(red2, sm.slots[2], sm.wsum, rank, csize,
                            [&](double (&t)[1]) { cg_after_gamma(sm, t[0], inner_maxit); });
    }
    if (sm.done) break;
    first = false;
    T* t = po;
    po = pn;
    pn = t;
  }
  return sm.m;
}

}  // namespace ms
