// ms_stream4.cu -- streaming engine, vectorised, FP32 (mixed precision) or
// FP64: the inner CG of one block per thread-block cluster with the CG
// vectors in the cluster's global scratch slot (L2-resident), for blocks too
// large to keep on chip.
//
// Same method and pass structure as block_cg (ms_cg.cuh) -- pass A forms
// p_new = r + beta p_old on the fly at the point and its neighbours, applies
// the stencil and accumulates p.q; pass B recomputes q from p_new and updates
// d, r and r.r -- but every thread owns 4-point x-strips of a pitch-padded
// layout (pitch 4*ceil(bx/4), padding lanes kept at zero), so a point costs a
// quarter of a 128-bit load instead of a scalar load, and the x-neighbours at
// the strip ends come from the adjacent lanes by warp shuffle.  Warps walk the
// strips in lockstep (uniform trip counts) so the shuffles always see 32 lanes.
#include <cuda_runtime.h>

#include "ms_cg.cuh"
#include "ms_device.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

struct StripGeo {
  int bx, by, bz, spr, pitch, plane, nstrips, z0, z1;
  unsigned magic;  // st / spr == __umulhi(st, magic) when magic != 0, else exact division
};

__device__ __forceinline__ StripGeo strip_geo(int bx, int by, int bz, unsigned rank, unsigned csize) {
  StripGeo g;
  g.bx = bx;
  g.by = by;
  g.bz = bz;
  g.spr = (bx + 3) >> 2;
  g.pitch = 4 * g.spr;
  g.plane = by * g.pitch;
  g.nstrips = g.spr * by;
  g.z0 = (int)(((long long)bz * rank) / csize);
  g.z1 = (int)(((long long)bz * (rank + 1)) / csize);
  // ceil(2^32 / spr) divides exactly while st * spr < 2^32 for every strip id
  // st < nstrips; spr = 1 (the multiplier would be 2^32) and larger planes
  // divide directly
  const unsigned long long m = (0x100000000ULL + (unsigned long long)g.spr - 1) / (unsigned long long)g.spr;
  g.magic = (m <= 0xFFFFFFFFULL && (unsigned long long)g.nstrips * (unsigned long long)g.spr < 0x100000000ULL)
                ? (unsigned)m
                : 0u;
  return g;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 msk4(float4 v, unsigned m) {
  return make_float4((m & 1u) ? v.x : 0.f, (m & 2u) ? v.y : 0.f, (m & 4u) ? v.z : 0.f, (m & 8u) ? v.w : 0.f);
}
__device__ __forceinline__ float dot4f(float4 a, float4 b) { return (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w); }

// Per-lane strip position for the current warp step.
struct StripPos {
  bool has;      // the lane holds a strip
  int y, xs;     // row and strip-in-row
  int off;       // offset of the strip in a plane
  unsigned msk;  // lanes with x < bx
  bool lin, rin; // left / right neighbour strip is held by lane-1 / lane+1 (same row)
};

__device__ __forceinline__ StripPos strip_pos(const StripGeo& g, int st, int lane) {
  StripPos s;
  s.has = st < g.nstrips;
  const int stc = s.has ? st : 0;
  s.y = g.magic ? (int)__umulhi((unsigned)stc, g.magic) : stc / g.spr;
  s.xs = stc - s.y * g.spr;
  s.off = s.y * g.pitch + 4 * s.xs;
  const int rem = g.bx - 4 * s.xs;
  s.msk = !s.has ? 0u : (rem >= 4 ? 0xFu : ((1u << rem) - 1u));
  s.lin = lane > 0 && s.xs > 0;
  s.rin = lane < 31 && s.xs + 1 < g.spr;
  return s;
}

// 7-point stencil on a strip: c centre, zm/zp below/above, ym/yp rows (0 when
// outside the block), xl/xr the scalar x-neighbours of the strip ends.
__device__ __forceinline__ float4 stencil_strip(float4 c, float4 zm, float4 zp, float4 ym, float4 yp, float xl,
                                                float xr) {
  float4 q;
  q.x = 6.f * c.x - (((xl + c.y) + (ym.x + yp.x)) + (zm.x + zp.x));
  q.y = 6.f * c.y - (((c.x + c.z) + (ym.y + yp.y)) + (zm.y + zp.y));
  q.z = 6.f * c.z - (((c.y + c.w) + (ym.z + yp.z)) + (zm.z + zp.z));
  q.w = 6.f * c.w - (((c.z + xr) + (ym.w + yp.w)) + (zm.w + zp.w));
  return q;
}

// The FP64 strip: 4 doubles (32 bytes), moved as two 16-byte accesses.
struct __align__(16) dbl4 {
  double x, y, z, w;
};
__device__ __forceinline__ dbl4 ld4(const double* p) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  return dbl4{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st4(double* p, dbl4 v) {
  *reinterpret_cast<double2*>(p) = make_double2(v.x, v.y);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v.z, v.w);
}
__device__ __forceinline__ dbl4 fma4(double a, dbl4 x, dbl4 y) {
  return dbl4{fma(a, x.x, y.x), fma(a, x.y, y.y), fma(a, x.z, y.z), fma(a, x.w, y.w)};
}
__device__ __forceinline__ dbl4 msk4(dbl4 v, unsigned m) {
  return dbl4{(m & 1u) ? v.x : 0.0, (m & 2u) ? v.y : 0.0, (m & 4u) ? v.z : 0.0, (m & 8u) ? v.w : 0.0};
}
__device__ __forceinline__ double dot4f(dbl4 a, dbl4 b) { return (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w); }
__device__ __forceinline__ dbl4 stencil_strip(dbl4 c, dbl4 zm, dbl4 zp, dbl4 ym, dbl4 yp, double xl, double xr) {
  dbl4 q;
  q.x = 6.0 * c.x - (((xl + c.y) + (ym.x + yp.x)) + (zm.x + zp.x));
  q.y = 6.0 * c.y - (((c.x + c.z) + (ym.y + yp.y)) + (zm.y + zp.y));
  q.z = 6.0 * c.z - (((c.y + c.w) + (ym.z + yp.z)) + (zm.z + zp.z));
  q.w = 6.0 * c.w - (((c.z + xr) + (ym.w + yp.w)) + (zm.w + zp.w));
  return q;
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
struct StripT;  // the strip type of a precision
template <>
struct StripT<float> {
  using V = float4;
  __device__ static V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static V make(const float (&v)[4]) { return make_float4(v[0], v[1], v[2], v[3]); }
};
template <>
struct StripT<double> {
  using V = dbl4;
  __device__ static V zero() { return dbl4{0.0, 0.0, 0.0, 0.0}; }
  __device__ static V make(const double (&v)[4]) { return dbl4{v[0], v[1], v[2], v[3]}; }
};

// The two cluster sums of a CG iteration (which = 0: p.q, 1: r.r) in the
// precision of the inner solve, on the reduction slots of that precision.
template <int NT>
__device__ __forceinline__ float strip_sum(float v, int which, ResRed& rr, RedSmem&, unsigned rank, unsigned csize) {
  return which ? cluster_sum_f32<NT>(v, rr.gam, rr.wgam, rank, csize)
               : cluster_sum_f32<NT>(v, rr.eta, rr.weta, rank, csize);
}
template <int NT>
__device__ __forceinline__ double strip_sum(double v, int which, ResRed&, RedSmem& sm, unsigned rank,
                                            unsigned csize) {
  return cluster_sum_f64<NT>(v, sm.slots[1 + which][0], sm.wsum[which], rank, csize);
}

}  // namespace

// strip columns a thread marches up z together (FP64 strips take twice the
// registers: one column)
template <typename T>
constexpr int kStripsInFlight = sizeof(T) == 4 ? 2 : 1;

// The inner CG on the strip layout.  Vectors r, p0, p1, d of the slot use the
// pitch-padded layout (z, y, 4*xs + lane); r holds the residual on entry
// (padding lanes zero), gamma0 = r.r reduced.  Returns m; d holds the
// correction when m > 0.  T is the inner precision (float: the mixed-
// precision solve, double: the plain FP64 one).  The two sums of an
// iteration are cluster sums in T pre-reduced inside each CTA, and every
// thread forms the same scalars alpha, beta and the stop test from them (no
// broadcast).
template <int NT, typename T>
__device__ int strip_cg(const CgVecs<T>& v, const StripGeo& g, T gamma0, T inner_rtol, int inner_maxit, ResRed& rr,
                        RedSmem& sm, unsigned rank, unsigned csize) {
  using V = typename StripT<T>::V;
  constexpr int SF = kStripsInFlight<T>;
  if (!(gamma0 > T(0)) || inner_maxit <= 0) return 0;
  const int lane = threadIdx.x & 31;
  const int wbase = threadIdx.x - lane;
  const T stop = inner_rtol * sqrt(gamma0);
  T gamma = gamma0, beta = T(0);
  int m = 0;
  T* po = v.p0;
  T* pn = v.p1;
  bool first = true;
  for (;;) {
    // ---------------- pass A: p_new at the strip and its neighbours, q = A_ii p_new, eta = p.q
    // (within a pass the vectors are distinct: pass A reads r and p_old and writes
    // p_new, so the next planes' loads may move ahead of this plane's store).
    // Each thread marches SF strip columns up z together (FP32: 2), so that
    // many independent loads are in flight per plane step.
    const T* __restrict__ rA = v.r;
    const T* __restrict__ poA = po;
    T* __restrict__ pnA = pn;
    auto pnew = [&](long long i) -> V {  // i: element index of a strip start
      const V r = ld4(rA + i);
      return first ? r : fma4(beta, ld4(poA + i), r);
    };
    auto pnew_s = [&](long long i) -> T { return first ? rA[i] : fma_t(beta, poA[i], rA[i]); };
    T eta_loc = T(0);
    for (int s0 = wbase; s0 < g.nstrips; s0 += SF * NT) {
      StripPos s[SF];
      V zm[SF], c[SF];
#pragma unroll
      for (int u = 0; u < SF; ++u) {
        s[u] = strip_pos(g, s0 + u * NT + lane, lane);
        zm[u] = (s[u].has && g.z0 > 0 && g.z0 < g.z1) ? pnew((long long)(g.z0 - 1) * g.plane + s[u].off) : StripT<T>::zero();
        c[u] = (s[u].has && g.z0 < g.z1) ? pnew((long long)g.z0 * g.plane + s[u].off) : StripT<T>::zero();
      }
      for (int z = g.z0; z < g.z1; ++z) {
        const long long base = (long long)z * g.plane;
        V zp[SF], ym[SF], yp[SF];
#pragma unroll
        for (int u = 0; u < SF; ++u) {
          zp[u] = (s[u].has && z + 1 < g.bz) ? pnew(base + g.plane + s[u].off) : StripT<T>::zero();
          ym[u] = (s[u].has && s[u].y > 0) ? pnew(base + s[u].off - g.pitch) : StripT<T>::zero();
          yp[u] = (s[u].has && s[u].y + 1 < g.by) ? pnew(base + s[u].off + g.pitch) : StripT<T>::zero();
        }
#pragma unroll
        for (int u = 0; u < SF; ++u) {
          const T l_sh = __shfl_up_sync(0xffffffffu, c[u].w, 1);
          const T r_sh = __shfl_down_sync(0xffffffffu, c[u].x, 1);
          const T xl = s[u].lin ? l_sh : ((s[u].has && s[u].xs > 0) ? pnew_s(base + s[u].off - 1) : T(0));
          const T xr = s[u].rin ? r_sh : ((s[u].has && s[u].xs + 1 < g.spr) ? pnew_s(base + s[u].off + 4) : T(0));
          const V q = msk4(stencil_strip(c[u], zm[u], zp[u], ym[u], yp[u], xl, xr), s[u].msk);
          if (s[u].has) st4(pnA + base + s[u].off, c[u]);
          eta_loc += dot4f(c[u], q);
          zm[u] = c[u];
          c[u] = zp[u];
        }
      }
    }
    const T eta = strip_sum<NT>(eta_loc, 0, rr, sm, rank, csize);
    if (!(eta > T(0))) break;  // curvature breakdown or NaN: keep d from earlier steps
    const T alpha = gamma / eta;
    // ---------------- pass B: q = A_ii p_new again, d += alpha p, r -= alpha q, gamma = r.r
    // (reads p_new; d and r are read and written at the strip itself only)
    const T* __restrict__ pnB = pn;
    T* __restrict__ dB = v.d;
    T* __restrict__ rB = v.r;
    T g_loc = T(0);
    for (int s0 = wbase; s0 < g.nstrips; s0 += SF * NT) {
      StripPos s[SF];
      V zm[SF], c[SF];
#pragma unroll
      for (int u = 0; u < SF; ++u) {
        s[u] = strip_pos(g, s0 + u * NT + lane, lane);
        zm[u] = (s[u].has && g.z0 > 0 && g.z0 < g.z1) ? ld4(pnB + (long long)(g.z0 - 1) * g.plane + s[u].off) : StripT<T>::zero();
        c[u] = (s[u].has && g.z0 < g.z1) ? ld4(pnB + (long long)g.z0 * g.plane + s[u].off) : StripT<T>::zero();
      }
      for (int z = g.z0; z < g.z1; ++z) {
        const long long base = (long long)z * g.plane;
        V zp[SF], ym[SF], yp[SF], dd[SF],
            ro[SF];
#pragma unroll
        for (int u = 0; u < SF; ++u) {
          const long long i = base + s[u].off;
          zp[u] = (s[u].has && z + 1 < g.bz) ? ld4(pnB + i + g.plane) : StripT<T>::zero();
          ym[u] = (s[u].has && s[u].y > 0) ? ld4(pnB + i - g.pitch) : StripT<T>::zero();
          yp[u] = (s[u].has && s[u].y + 1 < g.by) ? ld4(pnB + i + g.pitch) : StripT<T>::zero();
          dd[u] = (s[u].has && !first) ? ld4(dB + i) : StripT<T>::zero();
          ro[u] = s[u].has ? ld4(rB + i) : StripT<T>::zero();
        }
#pragma unroll
        for (int u = 0; u < SF; ++u) {
          const long long i = base + s[u].off;
          const T l_sh = __shfl_up_sync(0xffffffffu, c[u].w, 1);
          const T r_sh = __shfl_down_sync(0xffffffffu, c[u].x, 1);
          const T xl = s[u].lin ? l_sh : ((s[u].has && s[u].xs > 0) ? pnB[i - 1] : T(0));
          const T xr = s[u].rin ? r_sh : ((s[u].has && s[u].xs + 1 < g.spr) ? pnB[i + 4] : T(0));
          const V q = msk4(stencil_strip(c[u], zm[u], zp[u], ym[u], yp[u], xl, xr), s[u].msk);
          if (s[u].has) {
            st4(dB + i, fma4(alpha, c[u], dd[u]));
            const V r = fma4(-alpha, q, ro[u]);
            st4(rB + i, r);
            g_loc += dot4f(r, r);
          }
          zm[u] = c[u];
          c[u] = zp[u];
        }
      }
    }
    const T gnew = strip_sum<NT>(g_loc, 1, rr, sm, rank, csize);
    m += 1;
    if (sqrt(gnew) <= stop || m >= inner_maxit) break;
    beta = gnew / gamma;
    gamma = gnew;
    first = false;
    T* tp = po;
    po = pn;
    pn = tp;
  }
  return m;
}

// One synchronous outer sweep with the vectorised streaming CG (contract of
// sweep_kernel in ms_kernels.cu; T = float: mixed precision, double: FP64).
template <int NT, typename T>
__global__ void __launch_bounds__(NT, 1) strip_sweep_kernel(const SweepArgs a) {
  using V = typename StripT<T>::V;
  __shared__ RedSmem sm;
  __shared__ ResRed rred;
  __shared__ int s_task[2];
  if (*a.all_done) return;
  const unsigned rank = cl_rank(), csize = cl_size(), slot = cl_id();
  const int tid = threadIdx.x, lane = tid & 31, wbase = tid - lane;
  const int k = *a.k_dev;
  const double* __restrict__ xin = (k & 1) ? a.xbuf1 : a.xbuf0;
  double* __restrict__ xout = (k & 1) ? a.xbuf0 : a.xbuf1;
  const bool residual_only = (k >= a.outer_maxit);
  const CgVecs<T> v = slot_vecs<T>(a.scratch, a.vec_stride, slot);
  const Geo G = a.g;
  const long long nxy = (long long)G.nx * G.ny;
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
    const StripGeo g = strip_geo(tk.bx, tk.by, tk.bz, rank, csize);
    if ((long long)g.plane * tk.bz > a.vec_stride) {  // host sizes the slots for the padded layout
      if (tid == 0) atomicOr(a.err, kErrGeometry);
      continue;
    }
    const double scale = inner_scale<T>(a.inv_bnorm[tk.rhs]), unscale = 1.0 / scale;
    const long long rb = (long long)tk.rhs * G.npts;
    const double* __restrict__ xr = xin + rb;
    const double* __restrict__ fr = a.f ? a.f + rb : nullptr;
    const double* __restrict__ br = a.bnd ? a.bnd + (long long)tk.rhs * G.nbnd : nullptr;
    // ---- 1. block residual in FP64, scaled and rounded to T strips (padding lanes 0)
    double red0[2] = {0.0, 0.0};
    {
      double s_loc = 0.0;
      T g_loc = T(0);
      for (int s0 = wbase; s0 < g.nstrips; s0 += NT) {
        const StripPos s = strip_pos(g, s0 + lane, lane);
        if (!s.has) continue;
        const int gy = tk.oy + s.y, gx0 = tk.ox + 4 * s.xs;
        for (int z = g.z0; z < g.z1; ++z) {
          const int gz = tk.oz + z;
          T rv[4];
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            rv[l] = T(0);
            if (s.msk & (1u << l)) {
              const long long gi = (long long)gz * nxy + (long long)gy * G.nx + gx0 + l;
              double si, so;
              nbr_sums(G, xr, br, gx0 + l, gy, gz, gi, si, so);
              const double bh = fr ? fr[gi] + so : so;
              const double rr = bh - (6.0 * xr[gi] - si);
              if (owns(tk, 4 * s.xs + l, s.y, z)) s_loc += rr * rr;  // the global norm counts owned points
              rv[l] = (T)(rr * scale);
            }
          }
          const V r = StripT<T>::make(rv);
          st4(v.r + (long long)z * g.plane + s.off, r);
          g_loc += dot4f(r, r);
        }
      }
      red0[0] = s_loc;
      red0[1] = (double)g_loc;
    }
    cluster_reduce<NT, 2>(red0, sm.slots[0], sm.wsum, rank, csize, [&](double (&tt)[2]) {
      sm.tot[0] = tt[0];
      sm.tot[1] = tt[1];
    });
    if (rank == 0 && tid == 0) a.partial[t] = sm.tot[0];
    if (residual_only) continue;
    // ---- 2. inner CG
    const int m = strip_cg<NT, T>(v, g, (T)sm.tot[1], (T)sweep_inner_rtol(a, tk.rhs), a.inner_maxit, rred, sm, rank,
                                  csize);
    // ---- 3. outer update into the other buffer (owned points only)
    double* __restrict__ xo = xout + rb;
    for (int s0 = wbase; s0 < g.nstrips; s0 += NT) {
      const StripPos s = strip_pos(g, s0 + lane, lane);
      if (!s.has) continue;
      const int gy = tk.oy + s.y, gx0 = tk.ox + 4 * s.xs;
      for (int z = g.z0; z < g.z1; ++z) {
        const long long gi0 = (long long)(tk.oz + z) * nxy + (long long)gy * G.nx + gx0;
        const V d = m > 0 ? ld4(v.d + (long long)z * g.plane + s.off) : StripT<T>::zero();
        const T dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int l = 0; l < 4; ++l)
          if ((s.msk & (1u << l)) && owns(tk, 4 * s.xs + l, s.y, z)) xo[gi0 + l] = xr[gi0 + l] + (double)dv[l] * unscale;
      }
    }
    if (rank == 0 && tid == 0 && m > 0) {
      atomicAdd(a.inner_count + 2 * tk.rhs, (unsigned long long)m);
      atomicAdd(a.inner_count + 2 * tk.rhs + 1, (unsigned long long)m * (unsigned long long)tk.bx * tk.by * tk.bz);
    }
    if (rank == 0 && tid == 0 && a.tr.rec) trace_push(a.tr, *a.k_dev, tk.block, tk.rhs, m, a.partial[t]);
  }
}

// ---------------------------------------------------------------- launchers
template <int NT, typename T>
static cudaError_t prep_strip(int cluster, void** fn) {
  auto kern = strip_sweep_kernel<NT, T>;
  if (cluster > 8) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  *fn = (void*)kern;
  return cudaSuccess;
}

// prec: 1 mixed (FP32 inner solve), 0 FP64
static cudaError_t strip_fn(int prec, int threads, int cluster, void** fn) {
  if (prec == 1) {
    if (threads == 256) return prep_strip<256, float>(cluster, fn);
    if (threads == 512) return prep_strip<512, float>(cluster, fn);
    if (threads == 1024) return prep_strip<1024, float>(cluster, fn);
  } else {
    if (threads == 256) return prep_strip<256, double>(cluster, fn);
    if (threads == 512) return prep_strip<512, double>(cluster, fn);
    if (threads == 1024) return prep_strip<1024, double>(cluster, fn);
  }
  return cudaErrorInvalidValue;
}

static void strip_cfg(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at, int threads, int cluster, int slots,
                      cudaStream_t s) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3((unsigned)(cluster * slots), 1, 1);
  cfg->blockDim = dim3((unsigned)threads, 1, 1);
  cfg->stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg->attrs = at;
  cfg->numAttrs = 1;
}

cudaError_t strip_max_clusters(int prec, int threads, int cluster, int* out) {
  void* fn = nullptr;
  cudaError_t e = strip_fn(prec, threads, cluster, &fn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  strip_cfg(&cfg, at, threads, cluster, 64, nullptr);
  return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

cudaError_t launch_strip_sweep(int prec, int threads, int cluster, int slots, const SweepArgs& a, cudaStream_t s) {
  void* fn = nullptr;
  cudaError_t e = strip_fn(prec, threads, cluster, &fn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  strip_cfg(&cfg, at, threads, cluster, slots, s);
  void* args[] = {(void*)&a};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace ms
