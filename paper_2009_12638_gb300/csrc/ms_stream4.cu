// ms_stream4.cu -- streaming engine, FP32, vectorised: the inner CG of one
// block per thread-block cluster with the CG vectors in the cluster's global
// scratch slot (L2-resident), for blocks too large to keep on chip.
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
  unsigned magic;  // st / spr == __umulhi(st, magic)
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
  g.magic = (unsigned)((0x100000000ULL + (unsigned long long)g.spr - 1) / (unsigned long long)g.spr);
  return g;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
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
  s.y = (int)__umulhi((unsigned)stc, g.magic);
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

}  // namespace

constexpr int kStripsInFlight = 2;  // strip columns a thread marches up z together

// The inner CG on the strip layout.  Vectors r, p0, p1, d of the slot use the
// pitch-padded layout (z, y, 4*xs + lane); r holds the residual on entry
// (padding lanes zero), gamma0 = r.r reduced.  Returns m; d holds the
// correction when m > 0.  The two sums of an iteration are FP32 cluster sums
// pre-reduced inside each CTA (cluster_sum_f32), and every thread forms the
// same FP32 scalars alpha, beta and the stop test from them (no broadcast).
template <int NT>
__device__ int strip_cg(const CgVecs<float>& v, const StripGeo& g, float gamma0, float inner_rtol, int inner_maxit,
                        ResRed& rr, unsigned rank, unsigned csize) {
  if (!(gamma0 > 0.f) || inner_maxit <= 0) return 0;
  const int lane = threadIdx.x & 31;
  const int wbase = threadIdx.x - lane;
  const float stop = inner_rtol * sqrtf(gamma0);
  float gamma = gamma0, beta = 0.f;
  int m = 0;
  float* po = v.p0;
  float* pn = v.p1;
  bool first = true;
  for (;;) {
    // ---------------- pass A: p_new at the strip and its neighbours, q = A_ii p_new, eta = p.q
    // (within a pass the vectors are distinct: pass A reads r and p_old and writes
    // p_new, so the next planes' loads may move ahead of this plane's store).
    // Each thread marches kStripsInFlight strip columns up z together, so twice
    // as many independent loads are in flight per plane step.
    const float* __restrict__ rA = v.r;
    const float* __restrict__ poA = po;
    float* __restrict__ pnA = pn;
    auto pnew = [&](long long i) -> float4 {  // i: float index of a strip start
      const float4 r = ld4(rA + i);
      return first ? r : fma4(beta, ld4(poA + i), r);
    };
    auto pnew_s = [&](long long i) -> float { return first ? rA[i] : fmaf(beta, poA[i], rA[i]); };
    float eta_loc = 0.f;
    for (int s0 = wbase; s0 < g.nstrips; s0 += kStripsInFlight * NT) {
      StripPos s[kStripsInFlight];
      float4 zm[kStripsInFlight], c[kStripsInFlight];
#pragma unroll
      for (int u = 0; u < kStripsInFlight; ++u) {
        s[u] = strip_pos(g, s0 + u * NT + lane, lane);
        zm[u] = (s[u].has && g.z0 > 0 && g.z0 < g.z1) ? pnew((long long)(g.z0 - 1) * g.plane + s[u].off) : zero4();
        c[u] = (s[u].has && g.z0 < g.z1) ? pnew((long long)g.z0 * g.plane + s[u].off) : zero4();
      }
      for (int z = g.z0; z < g.z1; ++z) {
        const long long base = (long long)z * g.plane;
        float4 zp[kStripsInFlight], ym[kStripsInFlight], yp[kStripsInFlight];
#pragma unroll
        for (int u = 0; u < kStripsInFlight; ++u) {
          zp[u] = (s[u].has && z + 1 < g.bz) ? pnew(base + g.plane + s[u].off) : zero4();
          ym[u] = (s[u].has && s[u].y > 0) ? pnew(base + s[u].off - g.pitch) : zero4();
          yp[u] = (s[u].has && s[u].y + 1 < g.by) ? pnew(base + s[u].off + g.pitch) : zero4();
        }
#pragma unroll
        for (int u = 0; u < kStripsInFlight; ++u) {
          const float l_sh = __shfl_up_sync(0xffffffffu, c[u].w, 1);
          const float r_sh = __shfl_down_sync(0xffffffffu, c[u].x, 1);
          const float xl = s[u].lin ? l_sh : ((s[u].has && s[u].xs > 0) ? pnew_s(base + s[u].off - 1) : 0.f);
          const float xr = s[u].rin ? r_sh : ((s[u].has && s[u].xs + 1 < g.spr) ? pnew_s(base + s[u].off + 4) : 0.f);
          const float4 q = msk4(stencil_strip(c[u], zm[u], zp[u], ym[u], yp[u], xl, xr), s[u].msk);
          if (s[u].has) st4(pnA + base + s[u].off, c[u]);
          eta_loc += dot4f(c[u], q);
          zm[u] = c[u];
          c[u] = zp[u];
        }
      }
    }
    const float eta = cluster_sum_f32<NT>(eta_loc, rr.eta, rr.weta, rank, csize);
    if (!(eta > 0.f)) break;  // curvature breakdown or NaN: keep d from earlier steps
    const float alpha = gamma / eta;
    // ---------------- pass B: q = A_ii p_new again, d += alpha p, r -= alpha q, gamma = r.r
    // (reads p_new; d and r are read and written at the strip itself only)
    const float* __restrict__ pnB = pn;
    float* __restrict__ dB = v.d;
    float* __restrict__ rB = v.r;
    float g_loc = 0.f;
    for (int s0 = wbase; s0 < g.nstrips; s0 += kStripsInFlight * NT) {
      StripPos s[kStripsInFlight];
      float4 zm[kStripsInFlight], c[kStripsInFlight];
#pragma unroll
      for (int u = 0; u < kStripsInFlight; ++u) {
        s[u] = strip_pos(g, s0 + u * NT + lane, lane);
        zm[u] = (s[u].has && g.z0 > 0 && g.z0 < g.z1) ? ld4(pnB + (long long)(g.z0 - 1) * g.plane + s[u].off) : zero4();
        c[u] = (s[u].has && g.z0 < g.z1) ? ld4(pnB + (long long)g.z0 * g.plane + s[u].off) : zero4();
      }
      for (int z = g.z0; z < g.z1; ++z) {
        const long long base = (long long)z * g.plane;
        float4 zp[kStripsInFlight], ym[kStripsInFlight], yp[kStripsInFlight], dd[kStripsInFlight],
            ro[kStripsInFlight];
#pragma unroll
        for (int u = 0; u < kStripsInFlight; ++u) {
          const long long i = base + s[u].off;
          zp[u] = (s[u].has && z + 1 < g.bz) ? ld4(pnB + i + g.plane) : zero4();
          ym[u] = (s[u].has && s[u].y > 0) ? ld4(pnB + i - g.pitch) : zero4();
          yp[u] = (s[u].has && s[u].y + 1 < g.by) ? ld4(pnB + i + g.pitch) : zero4();
          dd[u] = (s[u].has && !first) ? ld4(dB + i) : zero4();
          ro[u] = s[u].has ? ld4(rB + i) : zero4();
        }
#pragma unroll
        for (int u = 0; u < kStripsInFlight; ++u) {
          const long long i = base + s[u].off;
          const float l_sh = __shfl_up_sync(0xffffffffu, c[u].w, 1);
          const float r_sh = __shfl_down_sync(0xffffffffu, c[u].x, 1);
          const float xl = s[u].lin ? l_sh : ((s[u].has && s[u].xs > 0) ? pnB[i - 1] : 0.f);
          const float xr = s[u].rin ? r_sh : ((s[u].has && s[u].xs + 1 < g.spr) ? pnB[i + 4] : 0.f);
          const float4 q = msk4(stencil_strip(c[u], zm[u], zp[u], ym[u], yp[u], xl, xr), s[u].msk);
          if (s[u].has) {
            st4(dB + i, fma4(alpha, c[u], dd[u]));
            const float4 r = fma4(-alpha, q, ro[u]);
            st4(rB + i, r);
            g_loc += dot4f(r, r);
          }
          zm[u] = c[u];
          c[u] = zp[u];
        }
      }
    }
    const float gnew = cluster_sum_f32<NT>(g_loc, rr.gam, rr.wgam, rank, csize);
    m += 1;
    if (sqrtf(gnew) <= stop || m >= inner_maxit) break;
    beta = gnew / gamma;
    gamma = gnew;
    first = false;
    float* tp = po;
    po = pn;
    pn = tp;
  }
  return m;
}

// One synchronous outer sweep with the vectorised streaming CG (contract of
// sweep_kernel in ms_kernels.cu; mixed precision only).
template <int NT>
__global__ void __launch_bounds__(NT, 1) strip_sweep_kernel(const SweepArgs a) {
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
  const CgVecs<float> v = slot_vecs<float>(a.scratch, a.vec_stride, slot);
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
    const double scale = inner_scale<float>(a.inv_bnorm[tk.rhs]), unscale = 1.0 / scale;
    const long long rb = (long long)tk.rhs * G.npts;
    const double* __restrict__ xr = xin + rb;
    const double* __restrict__ fr = a.f ? a.f + rb : nullptr;
    const double* __restrict__ br = a.bnd ? a.bnd + (long long)tk.rhs * G.nbnd : nullptr;
    // ---- 1. block residual in FP64, scaled, rounded to FP32 strips (padding lanes 0)
    double red0[2] = {0.0, 0.0};
    {
      double s_loc = 0.0;
      float g_loc = 0.f;
      for (int s0 = wbase; s0 < g.nstrips; s0 += NT) {
        const StripPos s = strip_pos(g, s0 + lane, lane);
        if (!s.has) continue;
        const int gy = tk.oy + s.y, gx0 = tk.ox + 4 * s.xs;
        for (int z = g.z0; z < g.z1; ++z) {
          const int gz = tk.oz + z;
          float rv[4];
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            rv[l] = 0.f;
            if (s.msk & (1u << l)) {
              const long long gi = (long long)gz * nxy + (long long)gy * G.nx + gx0 + l;
              double si, so;
              nbr_sums(G, xr, br, gx0 + l, gy, gz, gi, si, so);
              const double bh = fr ? fr[gi] + so : so;
              const double rr = bh - (6.0 * xr[gi] - si);
              if (owns(tk, 4 * s.xs + l, s.y, z)) s_loc += rr * rr;  // the global norm counts owned points
              rv[l] = (float)(rr * scale);
            }
          }
          const float4 r = make_float4(rv[0], rv[1], rv[2], rv[3]);
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
    const int m = strip_cg<NT>(v, g, (float)sm.tot[1], (float)sweep_inner_rtol(a, tk.rhs), a.inner_maxit, rred, rank,
                               csize);
    // ---- 3. outer update into the other buffer (owned points only)
    double* __restrict__ xo = xout + rb;
    for (int s0 = wbase; s0 < g.nstrips; s0 += NT) {
      const StripPos s = strip_pos(g, s0 + lane, lane);
      if (!s.has) continue;
      const int gy = tk.oy + s.y, gx0 = tk.ox + 4 * s.xs;
      for (int z = g.z0; z < g.z1; ++z) {
        const long long gi0 = (long long)(tk.oz + z) * nxy + (long long)gy * G.nx + gx0;
        const float4 d = m > 0 ? ld4(v.d + (long long)z * g.plane + s.off) : zero4();
        const float dv[4] = {d.x, d.y, d.z, d.w};
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
template <int NT>
static cudaError_t prep_strip(int cluster, void** fn) {
  auto kern = strip_sweep_kernel<NT>;
  if (cluster > 8) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  *fn = (void*)kern;
  return cudaSuccess;
}

static cudaError_t strip_fn(int threads, int cluster, void** fn) {
  if (threads == 256) return prep_strip<256>(cluster, fn);
  if (threads == 512) return prep_strip<512>(cluster, fn);
  if (threads == 1024) return prep_strip<1024>(cluster, fn);
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

cudaError_t strip_max_clusters(int threads, int cluster, int* out) {
  void* fn = nullptr;
  cudaError_t e = strip_fn(threads, cluster, &fn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  strip_cfg(&cfg, at, threads, cluster, 64, nullptr);
  return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

cudaError_t launch_strip_sweep(int threads, int cluster, int slots, const SweepArgs& a, cudaStream_t s) {
  void* fn = nullptr;
  cudaError_t e = strip_fn(threads, cluster, &fn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  strip_cfg(&cfg, at, threads, cluster, slots, s);
  void* args[] = {(void*)&a};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace ms
