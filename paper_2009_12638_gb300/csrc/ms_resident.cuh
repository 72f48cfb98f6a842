// ms_resident.cuh -- the inner CG (sections 2.2 and 3 of the paper) with the
// whole block state on chip: one thread-block cluster per block, no global
// memory traffic inside the inner loop.
//
// Layout.  The block (bx*by*bz, FP32) is cut into z-slabs, one per CTA
// (every CTA owns >= 1 plane).  A thread owns KC "strips" -- 4 consecutive x
// points of one (y) row -- in every plane of its slab (<= ZS planes), and
// keeps r and d of those points in registers as float4.  p lives in shared
// memory as nzs+2 planes (own planes plus one halo plane below and above),
// each with a zero row above/below and zero columns left/right, so the
// stencil needs no branches: zero padding is the block's Dirichlet-0 face
// (A_ii is A restricted to the block).
//
// Halo planes without a third barrier.  p_new = r + beta p_old needs the
// neighbour CTA's r; after pass B each CTA pushes its first/last plane of r
// into its neighbours' r-halo planes (DSMEM stores, made visible by the
// gamma reduction's cluster barrier).  Every CTA then forms p_new on its own
// planes AND on its halo planes with the same fused multiply-add the owner
// uses, so the copies agree bit for bit.
//
// Per CG iteration: pass A (stencil from shared memory, eta = p.q), cluster
// sum, pass B (stencil again, d += alpha p, r -= alpha q, gamma = r.r, r
// halo push), cluster sum, pass C (p = r + beta p on own and halo planes).

#pragma once
#include "ms_cg.cuh"
#include "ms_device.cuh"
#include "ms_resident_variants.h"

namespace ms {

struct ResGeo {
  int bx, by, bz;
  int spr;      // strips per row = ceil(bx / 4)
  int nstrips;  // spr * by
  int rp;       // smem row pitch in floats: 4 zero floats + 4*spr (the next row's zeros pad the right end)
  int ps;       // smem plane stride in floats: (by + 2) * rp
  int z0, nzs;  // own planes
};

__device__ __forceinline__ ResGeo make_res_geo(int bx, int by, int bz, unsigned rank, unsigned csize) {
  ResGeo g;
  g.bx = bx;
  g.by = by;
  g.bz = bz;
  g.spr = (bx + 3) >> 2;
  g.nstrips = g.spr * by;
  g.rp = 4 * g.spr + 4;
  g.ps = (by + 2) * g.rp + 4;
  g.z0 = (int)(((long long)bz * rank) / csize);
  g.nzs = (int)(((long long)bz * (rank + 1)) / csize) - g.z0;
  return g;
}

__device__ __forceinline__ void st_cluster_v4(float* local, unsigned rank, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(cl_map(local, rank)), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

__device__ __forceinline__ float4 mask4(float4 v, unsigned m) {
  return make_float4((m & 1u) ? v.x : 0.f, (m & 2u) ? v.y : 0.f, (m & 4u) ? v.z : 0.f, (m & 8u) ? v.w : 0.f);
}

__device__ __forceinline__ float dot4(float4 a, float4 b) { return (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w); }

// 7-point stencil q = 6p - sum(nbrs) on the 4 points of a strip.  y and z
// neighbours come from shared memory / registers; the x neighbours at the
// strip ends come from the adjacent lanes (which hold the adjacent strips of
// the same row) by warp shuffle, or from shared memory (zero padding at a
// row end) for the first and last lane.  All 32 lanes must call it.
__device__ __forceinline__ float4 stencil4(const float* c_ptr, int rp, float4 c, float4 zm, float4 zp,
                                           bool left_lane, bool right_lane) {
  const float4 ym = lds4(c_ptr - rp);
  const float4 yp = lds4(c_ptr + rp);
  const float xl_s = __shfl_up_sync(0xffffffffu, c.w, 1);
  const float xr_s = __shfl_down_sync(0xffffffffu, c.x, 1);
  const float xl = left_lane ? xl_s : c_ptr[-1];
  const float xr = right_lane ? xr_s : c_ptr[4];
  float4 q;
  q.x = 6.f * c.x - (((xl + c.y) + (ym.x + yp.x)) + (zm.x + zp.x));
  q.y = 6.f * c.y - (((c.x + c.z) + (ym.y + yp.y)) + (zm.y + zp.y));
  q.z = 6.f * c.z - (((c.y + c.w) + (ym.z + yp.z)) + (zm.z + zp.z));
  q.w = 6.f * c.w - (((c.z + xr) + (ym.w + yp.w)) + (zm.w + zp.w));
  return q;
}

// Per-thread strip bookkeeping for one task.  Threads without a strip keep
// off = 0 (a harmless in-bounds smem address) and msk = 0: they run every
// loop (shuffles need all lanes) but store nothing.
template <int KC>
struct Strips {
  int off[KC];       // smem offset (floats) of the strip in plane 0 (the lower halo plane)
  unsigned msk[KC];  // lanes with x < bx (0 = no strip)
  unsigned nb[KC];   // bit 0: left strip is held by lane-1; bit 1: right strip by lane+1
  int st[KC];        // strip id (row-major over the plane), -1 if none
};

template <int NT, int KC>
__device__ __forceinline__ Strips<KC> make_strips(const ResGeo& g) {
  Strips<KC> s;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int st = threadIdx.x + k * NT;
    if (st < g.nstrips) {
      const int y = st / g.spr, xs = st - y * g.spr;
      s.off[k] = (y + 1) * g.rp + 4 + 4 * xs;
      const int rem = g.bx - 4 * xs;
      s.msk[k] = rem >= 4 ? 0xFu : ((1u << rem) - 1u);
      s.nb[k] = ((lane > 0 && xs > 0) ? 1u : 0u) | ((lane < 31 && xs + 1 < g.spr) ? 2u : 0u);
      s.st[k] = st;
    } else {
      s.off[k] = 0;
      s.msk[k] = 0u;
      s.nb[k] = 0u;
      s.st[k] = -1;
    }
  }
  return s;
}

// Inner CG on the resident state.  On entry r4 holds r (padding lanes 0),
// the r-halo planes hold the neighbours' boundary r (pushed before the
// cluster barrier of the residual reduction), p planes are zero.  Returns
// m; d4 holds the correction when m > 0.  Scalars are FP32 and computed
// identically by every thread of the cluster.
// DS: d lives in shared memory (compact planes after the r-halo planes,
// float4 per strip, index z * nstrips + strip) instead of registers, which
// halves the registers a thread needs and lets a CTA run 1024 threads.
template <int NT, int KC, int ZS, bool DS>
__device__ __forceinline__ float4* d_slot(float* sp, const ResGeo& g, int z, int st) {
  return reinterpret_cast<float4*>(sp + (long long)(ZS + 4) * g.ps) + (long long)z * g.nstrips + st;
}

// Single-reduction CG (Chronopoulos and Gear's rearrangement of the same
// method: identical iterates in exact arithmetic, one cluster reduction per
// iteration instead of two).  With w = A r, gamma = r.r and delta = w.r
// summed together, beta = gamma_new / gamma, eta = p.A p = delta - beta
// gamma_new / alpha, alpha = gamma_new / eta, and the recurrences
//   p = r + beta p,  s = w + beta s  (s = A p),  d += alpha p,  r -= alpha s.
// Layout: r lives in the shared-memory plane stack (planes 0 and nzs+1 are the
// neighbour CTAs' boundary planes of r), p, s and w in registers, d in shared
// memory (compact planes, as the DS layouts).  Per iteration: one update pass
// (writes r and pushes its first/last plane into the neighbours' halo planes),
// then the stencil w = A r: its interior planes run between the arrive and
// the wait of a split cluster barrier that publishes the pushed planes, its
// two boundary planes after the wait; then the one reduction of (r.r, w.r).
// The stop rules are those of the two-reduction loop: the cap after m
// updates, ||r_m|| <= inner_rtol ||r_0|| after each update, eta <= 0 before it.
// On entry r4 holds r, the residual phase has pushed the neighbours' boundary
// planes of r into the r-halo planes (visible after its cluster barrier), and
// shared memory is otherwise zero.  Returns m; d is in shared memory.
template <int NT, int KC, int ZS>
__device__ int resident_cg_one_reduction(float4 (&r4)[KC][ZS], const ResGeo& g, const Strips<KC>& s, float* sp,
                                         float gamma0, float inner_rtol, int inner_maxit, ResRed& rr, unsigned rank,
                                         unsigned csize) {
  const float* rh_lo = sp + (long long)(ZS + 2) * g.ps;  // residual phase: neighbour below's top plane of r
  const float* rh_hi = rh_lo + g.ps;                     // neighbour above's bottom plane of r
  const bool has_lo = rank > 0, has_hi = rank + 1 < csize;
  if (!(gamma0 > 0.f) || inner_maxit <= 0) return 0;
  // plane count of the slab below (its top halo plane is its plane nzs + 1)
  const int nzs_lo = has_lo ? (int)(((long long)g.bz * rank) / csize) - (int)(((long long)g.bz * (rank - 1)) / csize)
                            : 0;
  auto plane = [&](int z) { return sp + (long long)z * g.ps; };
  auto axpy4 = [](float a, float4 x, float4 y) {  // a x + y, per component
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
  };
  // r into the plane stack: own planes from registers, halo planes from the residual's pushes
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    if (!s.msk[k]) continue;
    const int o = s.off[k];
#pragma unroll
    for (int z = 0; z < ZS; ++z) {
      if (z >= g.nzs) break;
      sts4(plane(z + 1) + o, r4[k][z]);
    }
    if (has_lo) sts4(plane(0) + o, lds4(rh_lo + o));
    if (has_hi) sts4(plane(g.nzs + 1) + o, lds4(rh_hi + o));
  }
  __syncthreads();
  float4(&p4)[KC][ZS] = r4;  // p = r at the first update (beta = 0)
  float4 s4[KC][ZS], w4[KC][ZS];
  // w = A r on own plane z (stack planes z, z+1, z+2), with the r.r and w.r terms
  auto stencil_plane = [&](int k, int z, float& gl, float& dl) {
    const float* cp = plane(z + 1) + s.off[k];
    const float4 c = lds4(cp);
    const float4 w = mask4(stencil4(cp, g.rp, c, lds4(cp - g.ps), lds4(cp + g.ps), s.nb[k] & 1u, s.nb[k] & 2u),
                           s.msk[k]);
    w4[k][z] = w;
    gl += dot4(c, c);
    dl += dot4(w, c);
  };
  // prologue: w = A r, gamma = r.r, delta = w.r (every plane: the halos are in place)
  float gam = 0.f, del = 0.f;
#pragma unroll
  for (int k = 0; k < KC; ++k) {
#pragma unroll
    for (int z = 0; z < ZS; ++z) {
      if (z >= g.nzs) break;
      stencil_plane(k, z, gam, del);
    }
  }
  cluster_sum2_f32<NT>(gam, del, rr.eta, rr.gam, rr.weta, rr.wgam, rank, csize);
  if (!(del > 0.f)) return 0;  // eta = p.A p with p = r
#pragma unroll
  for (int k = 0; k < KC; ++k)
#pragma unroll
    for (int z = 0; z < ZS; ++z) s4[k][z] = w4[k][z];  // s = A p = w (beta = 0 below)
  const float stop = inner_rtol * sqrtf(gamma0);
  float gamma = gam, alpha = gam / del, beta = 0.f;
  int m = 0;
  for (;;) {
    // ---------------- update: p, s, d, r; r's boundary planes to the neighbours
    const bool last = m + 1 >= inner_maxit;  // after this update nothing reads r again
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      if (!s.msk[k]) continue;
#pragma unroll
      for (int z = 0; z < ZS; ++z) {
        if (z >= g.nzs) break;
        float* rp = plane(z + 1) + s.off[k];
        const float4 r = lds4(rp);
        const float4 p = axpy4(beta, p4[k][z], r);
        p4[k][z] = p;
        float4* dp = d_slot<NT, KC, ZS, true>(sp, g, z, s.st[k]);
        const float4 d = m == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : *dp;
        *dp = axpy4(alpha, p, d);
        if (last) continue;
        const float4 sv = axpy4(beta, s4[k][z], w4[k][z]);
        s4[k][z] = sv;
        const float4 rn = axpy4(-alpha, sv, r);
        sts4(rp, rn);
        if (z == 0 && has_lo) st_cluster_v4(plane(nzs_lo + 1) + s.off[k], rank - 1, rn);
        if (z == g.nzs - 1 && has_hi) st_cluster_v4(plane(0) + s.off[k], rank + 1, rn);
      }
    }
    m += 1;
    if (last) break;
    // ---------------- w = A r: interior planes while the halo planes travel
    cl_arrive();
    __syncthreads();
    float gl = 0.f, dl = 0.f;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
#pragma unroll
      for (int z = 1; z < ZS - 1; ++z) {
        if (z >= g.nzs - 1) break;
        stencil_plane(k, z, gl, dl);
      }
    }
    cl_wait();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
#pragma unroll
      for (int z = 0; z < ZS; ++z) {  // planes 0 and nzs - 1 (compile-time indices into w4)
        if (z >= g.nzs) break;
        if (z == 0 || z == g.nzs - 1) stencil_plane(k, z, gl, dl);
      }
    }
    cluster_sum2_f32<NT>(gl, dl, rr.eta, rr.gam, rr.weta, rr.wgam, rank, csize);
    if (sqrtf(gl) <= stop) break;
    beta = gl / gamma;
    const float eta = dl - beta * gl / alpha;
    if (!(eta > 0.f)) break;  // curvature breakdown or NaN: keep d from earlier steps
    alpha = gl / eta;
    gamma = gl;
  }
  // callers read d (own strips) and then clear shared memory for the next task:
  // every remote store of this solve precedes a cluster barrier that every CTA has
  // passed (the last update pushes nothing), and no thread may clear while another
  // still reads r
  __syncthreads();
  return m;
}

// QR: q = A_ii p of pass A stays in registers for pass B (no second stencil),
// and the update d += alpha p moves to the next pass C, which reads p_old
// anyway (the last one runs after the loop).  The FMAs and their order are
// those of the QR = 0 path, so both give bit-identical results; QR costs
// 4 registers per strip-plane and saves pass B's shared-memory reads.
template <int NT, int KC, int ZS, bool DS, bool QR>
__device__ int resident_cg_two_reductions(float4 (&r4)[KC][ZS], float4 (&d4)[DS ? 1 : KC][DS ? 1 : ZS],
                                          const ResGeo& g, const Strips<KC>& s, float* sp, float gamma0,
                                          float inner_rtol, int inner_maxit, ResRed& rr, unsigned rank,
                                          unsigned csize) {
  float* rh_lo = sp + (long long)(ZS + 2) * g.ps;  // neighbour below's top plane of r
  float* rh_hi = rh_lo + g.ps;                     // neighbour above's bottom plane of r
  float* p_lo = sp;                                // p halo plane below (plane 0)
  float* p_hi = sp + (long long)(g.nzs + 1) * g.ps;
  const bool has_lo = rank > 0, has_hi = rank + 1 < csize;
  if (!(gamma0 > 0.f) || inner_maxit <= 0) return 0;
  const float stop = inner_rtol * sqrtf(gamma0);
  float gamma = gamma0, beta = 0.f, alpha = 0.f;
  float4 q4[QR ? KC : 1][QR ? ZS : 1];
  int m = 0;
  float gnew = 0.f;
  // d = alpha p + d on one strip-plane (d = alpha p when first == true)
  auto add_d = [&](int k, int z, float4 p, bool first) {
    if constexpr (DS) {
      float4* dp = d_slot<NT, KC, ZS, DS>(sp, g, z, s.st[k]);
      const float4 d = first ? make_float4(0.f, 0.f, 0.f, 0.f) : *dp;
      *dp = make_float4(fmaf(alpha, p.x, d.x), fmaf(alpha, p.y, d.y), fmaf(alpha, p.z, d.z), fmaf(alpha, p.w, d.w));
    } else {
      const float4 d = first ? make_float4(0.f, 0.f, 0.f, 0.f) : d4[k][z];
      d4[k][z] = make_float4(fmaf(alpha, p.x, d.x), fmaf(alpha, p.y, d.y), fmaf(alpha, p.z, d.z),
                             fmaf(alpha, p.w, d.w));
    }
  };
  auto axpy4 = [](float a, float4 x, float4 y) {  // a x + y, per component
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
  };
  bool pending = false;  // QR: alpha p of the last iteration is not in d yet
  for (;;) {
    // ---------------- pass C: p = r + beta p on own planes and both halo planes
    // (beta = 0 on entry: p = r, halo p = neighbours' r; p planes start zeroed)
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      if (!s.msk[k]) continue;
#pragma unroll
      for (int z = 0; z < ZS; ++z) {
        if (z >= g.nzs) break;
        float* pp = sp + (long long)(z + 1) * g.ps + s.off[k];
        const float4 po = lds4(pp);
        if constexpr (QR) {
          if (m > 0) add_d(k, z, po, m == 1);
        }
        sts4(pp, axpy4(beta, po, r4[k][z]));
      }
    }
    pending = false;
    // halo planes: the thread's own strips (strip tid + k NT sits at the same
    // offset in every plane), which cover every strip of a plane
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      if (!s.msk[k]) continue;
      const int o = s.off[k];
      if (has_lo) sts4(p_lo + o, axpy4(beta, lds4(p_lo + o), lds4(rh_lo + o)));
      if (has_hi) sts4(p_hi + o, axpy4(beta, lds4(p_hi + o), lds4(rh_hi + o)));
    }
    __syncthreads();
    // ---------------- pass A: q = A_ii p, eta = p.q
    float eta_loc = 0.f;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const float* base = sp + s.off[k];
      const bool lft = s.nb[k] & 1u, rgt = s.nb[k] & 2u;
      float4 zm = lds4(base);
      float4 c = lds4(base + g.ps);
#pragma unroll
      for (int z = 0; z < ZS; ++z) {
        if (z >= g.nzs) break;
        const float* cp = base + (long long)(z + 1) * g.ps;
        const float4 zp = lds4(cp + g.ps);
        const float4 q = mask4(stencil4(cp, g.rp, c, zm, zp, lft, rgt), s.msk[k]);
        if constexpr (QR) q4[k][z] = q;
        eta_loc += dot4(c, q);
        zm = c;
        c = zp;
      }
    }
    // eta needs no cluster barrier: it publishes only its own value (the r
    // halo pushes of pass B are made visible by the gamma sum's barrier), and
    // no CTA pushes r into a neighbour before that neighbour's warps have
    // finished pass C, whose halo reads feed (through p) every eta partial
    // the neighbour's word carries
    const float eta = cluster_sum_tagged_f32<NT>(eta_loc, rr, rank, csize);
    // curvature breakdown or NaN: the solve stops with d from the earlier
    // steps.  No CTA leaves on this total: once a tagged wait ran out anywhere,
    // CTAs may hold different totals (a CTA that ran on with a wrong alpha
    // sends wrong partials), and a CTA that left early could end its launch
    // while the others still push halo data into its shared memory.  The exit
    // is taken at the gamma sum below, whose cluster barrier gives every CTA
    // the same total: this CTA runs pass B with alpha = 0 (r and d unchanged)
    // and contributes NaN, and every CTA leaves after that sum
    const bool brk = !(eta > 0.f);
    alpha = brk ? 0.f : gamma / eta;
    // ---------------- pass B: (QR = false: d += alpha p,) r -= alpha q, gamma = r.r, push boundary r
    float g_loc = 0.f;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const float* base = sp + s.off[k];
      const bool lft = s.nb[k] & 1u, rgt = s.nb[k] & 2u;
      float4 zm, c;
      if constexpr (!QR) {
        zm = lds4(base);
        c = lds4(base + g.ps);
      }
#pragma unroll
      for (int z = 0; z < ZS; ++z) {
        if (z >= g.nzs) break;
        float4 q;
        if constexpr (QR) {
          q = q4[k][z];
        } else {
          const float* cp = base + (long long)(z + 1) * g.ps;
          const float4 zp = lds4(cp + g.ps);
          q = mask4(stencil4(cp, g.rp, c, zm, zp, lft, rgt), s.msk[k]);
          if (DS ? (s.msk[k] != 0u) : true) add_d(k, z, c, m == 0);
          zm = c;
          c = zp;
        }
        const float4 r = axpy4(-alpha, q, r4[k][z]);
        r4[k][z] = r;
        g_loc += dot4(r, r);
        if (s.msk[k]) {
          if (z == 0 && has_lo) st_cluster_v4(rh_hi + s.off[k], rank - 1, r);
          if (z == g.nzs - 1 && has_hi) st_cluster_v4(rh_lo + s.off[k], rank + 1, r);
        }
      }
    }
    pending = QR && !brk;
    gnew = cluster_sum_f32<NT>(brk ? __uint_as_float(0x7fc00000u) : g_loc, rr.gam, rr.wgam, rank, csize);
    m += 1;
    // (NaN: a breakdown in some CTA, not counted below; for any other value the
    // test is sqrt(gnew) <= stop)
    if (!(sqrtf(gnew) > stop) || m >= inner_maxit) break;
    beta = gnew / gamma;
    gamma = gnew;
  }
  if ((__float_as_uint(gnew) & 0x7fffffffu) > 0x7f800000u) {  // left at a breakdown: that step does not count
    m -= 1;
    pending = false;
  }
  if constexpr (QR) {
    // the last d += alpha p (own strips only: p was written by this thread)
    if (pending) {
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        if (!s.msk[k]) continue;
#pragma unroll
        for (int z = 0; z < ZS; ++z) {
          if (z >= g.nzs) break;
          add_d(k, z, lds4(sp + (long long)(z + 1) * g.ps + s.off[k]), m == 1);
        }
      }
    }
    // callers clear shared memory for the next task as soon as this returns:
    // no thread may do so while another is still reading its p above
    __syncthreads();
  }
  return m;
}

// The inner CG of one task on the resident state: QR = 0 two stencils per
// iteration, QR = 1 q = A p kept in registers (bit-identical to QR = 0),
// QR = 2 the single-reduction CG (d in shared memory: DS = true).
template <int NT, int KC, int ZS, bool DS, int QR>
__device__ __forceinline__ int resident_cg(float4 (&r4)[KC][ZS], float4 (&d4)[DS ? 1 : KC][DS ? 1 : ZS],
                                           const ResGeo& g, const Strips<KC>& s, float* sp, float gamma0,
                                           float inner_rtol, int inner_maxit, ResRed& rr, unsigned rank,
                                           unsigned csize) {
  if constexpr (QR == 2) {
    static_assert(DS, "the single-reduction CG keeps d in shared memory");
    return resident_cg_one_reduction<NT, KC, ZS>(r4, g, s, sp, gamma0, inner_rtol, inner_maxit, rr, rank, csize);
  } else {
    return resident_cg_two_reductions<NT, KC, ZS, DS, QR == 1>(r4, d4, g, s, sp, gamma0, inner_rtol, inner_maxit,
                                                                rr, rank, csize);
  }
}

}  // namespace ms
