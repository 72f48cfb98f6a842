// ms_device.cuh -- device building blocks shared by the sweep kernels:
// thread-block-cluster primitives (DSMEM stores, cluster barrier), the
// deterministic cluster-wide sum, and the stencil pieces of the residual.
#pragma once
#include <cuda_runtime.h>

#include "ms_internal.h"

namespace ms {

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_count() {
  unsigned r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}

// Full cluster barrier.  Release on arrive / acquire on wait make every
// global and shared write issued before it by any CTA of the cluster visible
// to every CTA of the cluster after it.
__device__ __forceinline__ void cl_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned cl_map(const void* local, unsigned rank) {
  unsigned la = (unsigned)__cvta_generic_to_shared(local), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
  return ra;
}
__device__ __forceinline__ void cl_store(double* local, unsigned rank, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(cl_map(local, rank)), "d"(v) : "memory");
}
__device__ __forceinline__ void cl_store(int* local, unsigned rank, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(cl_map(local, rank)), "r"(v) : "memory");
}

// One record of the solve trace (called by one thread per block solve, only
// when tr.rec is set).  Callers read sweep and block_rr back from memory
// inside their `if (tr.rec)` so that no register holds them through the
// inner solve.
__device__ __forceinline__ void trace_push(const TraceArgs& tr, int sweep, int block, int rhs, int inner_its,
                                           double block_rr) {
  const unsigned long long i = atomicAdd(tr.head, 1ull);
  unsigned long long now;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
  ms_trace_rec& r = tr.rec[i % (unsigned long long)tr.cap];
  r.sweep = sweep;
  r.block = block;
  r.rhs = rhs;
  r.inner_its = inner_its;
  r.block_rr = block_rr;
  r.t_ns = now;
}

__device__ __forceinline__ double warp_sum_to_lane0(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic cluster-wide sum of NV values per thread (TA = float or
// double accumulators).  Every CTA ends with bit-identical totals: warps sum
// in TA, warp 0 sums the warp totals in FP64, each CTA's total is stored into
// slot[rank] of every CTA (DSMEM), and after the cluster barrier warp 0 of
// every CTA adds the slots in the same tree order.  `finish(tot)` then runs
// on thread 0 alone (FP64 scalar work -- divisions, square roots -- is slow
// on this GPU, so it is never replicated across threads) and may write
// shared memory that every thread reads after this function returns.
// `slots` must not be reused by another reduction before the next cluster
// barrier.  Contains one cluster barrier and two CTA barriers.
template <int NT, int NV, typename TA, typename F>
__device__ __forceinline__ void cluster_reduce(const TA (&v)[NV], double (*slots)[16], double (*wsum)[32],
                                               unsigned rank, unsigned csize, F&& finish) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    TA w = v[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (lane == 0) wsum[a][warp] = (double)w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double w = (lane < NT / 32) ? wsum[a][lane] : 0.0;
      w = warp_sum_to_lane0(w);
      w = __shfl_sync(0xffffffffu, w, 0);
      if (lane < (int)csize) cl_store(&slots[a][rank], (unsigned)lane, w);
    }
  }
  cl_barrier();
  if (warp == 0) {
    double tot[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double w = (lane < (int)csize) ? slots[a][lane] : 0.0;
      tot[a] = warp_sum_to_lane0(w);
    }
    if (lane == 0) finish(tot);
  }
  __syncthreads();
}

__device__ __forceinline__ void st_cluster_f32(float* local, unsigned rank, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(cl_map(local, rank)), "f"(v) : "memory");
}

// Cluster-wide FP32 sum.  Warp totals (xor butterfly: every lane holds the
// same bits) go to `wsum`; after one CTA barrier warp 0 adds them and stores
// the CTA total into slot[rank] of every CTA; after the cluster barrier
// EVERY warp adds the csize slots in the same order, so every thread of the
// cluster holds the bit-identical total.  Pre-reducing inside the CTA keeps
// the remote stores per sum at csize per CTA (instead of one per warp and
// CTA), which shortens the cluster barrier's release.  `slots` and `wsum`
// must not be reused by another sum before the next cluster barrier.
template <int NT>
__device__ __forceinline__ float cluster_sum_f32(float v, float* slots, float* wsum, unsigned rank, unsigned csize) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    float t = lane < NW ? wsum[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane < (int)csize) st_cluster_f32(&slots[rank], (unsigned)lane, t);
  }
  cl_barrier();
  float acc = lane < (int)csize ? slots[lane] : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// cluster_sum_f32 in FP64 (same tree, same slot rules; slots[kMaxCluster] and
// wsum[32] of doubles).
template <int NT>
__device__ __forceinline__ double cluster_sum_f64(double v, double* slots, double* wsum, unsigned rank,
                                                  unsigned csize) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < NW ? wsum[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane < (int)csize) cl_store(&slots[rank], (unsigned)lane, t);
  }
  cl_barrier();
  double acc = lane < (int)csize ? slots[lane] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// The two halves of cl_barrier(), for work in between: every thread of the
// cluster arrives (release: its earlier global and shared writes, DSMEM
// stores included, become visible to the cluster) and later waits (acquire)
// until every thread has arrived.  Each thread alternates arrive and wait;
// no other cluster barrier may sit between them.
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// cluster_sum_f32 for two values at once (one CTA barrier, one cluster
// barrier): a and b are replaced by their cluster-wide totals, bit-identical
// in every thread.  Same slot rules as cluster_sum_f32, for both slot arrays.
template <int NT>
__device__ __forceinline__ void cluster_sum2_f32(float& a, float& b, float* slots_a, float* slots_b, float* wsum_a,
                                                 float* wsum_b, unsigned rank, unsigned csize) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    wsum_a[warp] = a;
    wsum_b[warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    float ta = lane < NW ? wsum_a[lane] : 0.f;
    float tb = lane < NW ? wsum_b[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ta += __shfl_xor_sync(0xffffffffu, ta, o);
      tb += __shfl_xor_sync(0xffffffffu, tb, o);
    }
    if (lane < (int)csize) {
      st_cluster_f32(&slots_a[rank], (unsigned)lane, ta);
      st_cluster_f32(&slots_b[rank], (unsigned)lane, tb);
    }
  }
  cl_barrier();
  float xa = lane < (int)csize ? slots_a[lane] : 0.f;
  float xb = lane < (int)csize ? slots_b[lane] : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    xa += __shfl_xor_sync(0xffffffffu, xa, o);
    xb += __shfl_xor_sync(0xffffffffu, xb, o);
  }
  a = xa;
  b = xb;
}

// Reduction slots of an FP32 CG iteration (resident and vectorised streaming
// engines): CTA totals, one per rank, and this CTA's warp totals, for the
// iteration's two sums (see cluster_sum_f32).
struct ResRed {
  float eta[kMaxCluster], gam[kMaxCluster];
  float weta[32], wgam[32];
  // the tagged sum (cluster_sum_tagged_f32): one word per CTA (total bits |
  // tag << 32), the total handed to the CTA, the tag of the next sum, a flag
  // set once a wait ran out, and where that is reported
  unsigned long long tword[kMaxCluster];
  float ttot;
  unsigned tseq;
  int tstale;
  int* err;
  long long tlimit;  // polls before a wait gives up
};

constexpr long long kTagPollLimit = 1ll << 22;  // ~0.1 s of polling: far beyond any CG step

// Set up the tagged-sum state of a kernel's ResRed (polls: the wait limit, 0 =
// kTagPollLimit).  Called by every thread before the kernel's first cluster
// barrier (no CTA stores a word into another before every CTA has passed it).
__device__ __forceinline__ void res_red_init(ResRed& rr, int* err, long long polls) {
  if (threadIdx.x < kMaxCluster) rr.tword[threadIdx.x] = 0xffffffff00000000ull;  // a tag no sum uses
  if (threadIdx.x == 0) {
    rr.tseq = 0u;
    rr.tstale = 0;
    rr.err = err;
    rr.tlimit = polls > 0 ? polls : kTagPollLimit;
  }
}

// Cluster-wide FP32 sum with the bits of cluster_sum_f32 (the same warp
// butterflies, the same CTA pre-reduction, the CTA totals added in rank
// order), without a cluster barrier.  Warp 0 of each CTA stores its CTA
// total into word [rank] of every CTA as one 64-bit word tagged with this
// sum's number, polls its own CTA's csize words until every one carries that
// tag, and hands the total to the CTA's warps through shared memory (so all
// warps of a CTA always take the same value).  The stores are relaxed: the sum
// publishes nothing but its own value, so a caller that needs earlier writes
// visible to other CTAs uses a cluster barrier.  Words are reused, so two
// tagged sums of a launch must have a cluster barrier between them (no CTA
// stores the next sum's word before every CTA has read this one's); tags never
// repeat within a launch.  The wait is bounded: after rr.tlimit polls the CTA
// records kErrTimeout, takes the words as they are, and waits in no later
// tagged sum of the launch.  Callers keep their control flow independent of
// a total that may then differ between CTAs (see the CG's breakdown test).
template <int NT>
__device__ __forceinline__ float cluster_sum_tagged_f32(float v, ResRed& rr, unsigned rank, unsigned csize) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) rr.weta[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const unsigned tag = rr.tseq;
    float t = lane < NW ? rr.weta[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane < (int)csize) {
      const unsigned long long w = (unsigned long long)__float_as_uint(t) | ((unsigned long long)tag << 32);
      asm volatile("st.relaxed.cluster.shared::cluster.b64 [%0], %1;" ::"r"(cl_map(&rr.tword[rank], (unsigned)lane)),
                   "l"(w)
                   : "memory");
    }
    const unsigned mine = (unsigned)__cvta_generic_to_shared(&rr.tword[lane < (int)csize ? lane : 0]);
    bool stale = rr.tstale != 0;
    unsigned long long w = 0ull;
    for (long long polls = 0;; ++polls) {
      asm volatile("ld.relaxed.cluster.shared::cta.b64 %0, [%1];" : "=l"(w) : "r"(mine) : "memory");
      if (stale || __all_sync(0xffffffffu, lane >= (int)csize || (unsigned)(w >> 32) == tag)) break;
      if (polls >= rr.tlimit) {
        stale = true;
        if (lane == 0) {
          rr.tstale = 1;
          atomicOr(rr.err, kErrTimeout);
        }
        break;
      }
    }
    float acc = lane < (int)csize ? __uint_as_float((unsigned)w) : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      rr.ttot = acc;
      rr.tseq = tag + 1u;
    }
  }
  __syncthreads();
  return rr.ttot;
}

// Shared memory used by the reductions of one cluster, and the CG scalars
// that thread 0 derives from them and every thread reads.
struct RedSmem {
  double slots[3][2][kMaxCluster];  // [phase][value][cta]: residual pair, eta, gamma
  double wsum[2][32];
  double tot[2];                    // totals of the last reduction
  double gamma, gamma0, stop;       // CG state (thread 0 writes)
  float alpha, beta;                // CG step scalars in the inner precision
  double alpha_d, beta_d;           // the same in FP64 (FP64 inner path)
  int m, done;                      // iterations taken, loop exit flag
};

// Sum of the block partials of rhs s over the task list, by one warp: lane l
// adds tasks l, l+32, ... in order, then a fixed shuffle tree.  Deterministic
// and identical wherever it runs (check kernel, persistent decision).  The
// total is returned in every lane.
__device__ __forceinline__ double rhs_partial_sum_warp(const Task* tasks, const double* partial, int ntasks, int s) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int t = lane; t < ntasks; t += 32)
    if (tasks[t].rhs == s) acc += partial[t];
  acc = warp_sum_to_lane0(acc);
  return __shfl_sync(0xffffffffu, acc, 0);
}

// Neighbour sums of interior grid point (gx, gy, gz) of one rhs: `inner`
// gets the neighbours inside the grid, `outer` the Dirichlet values of the
// neighbours on the boundary, read from the packed faces (bnd may be null:
// zero data).  bhat = f + outer is the right-hand side with section 2.1's
// boundary values lifted into it, applied on the fly; (A x) = 6 x - inner.
// XL2: read x through L2 only (ld.global.cg) -- for kernels in which other
// clusters write x while this one reads it.
template <bool XL2 = false>
__device__ __forceinline__ double ldx(const double* x, long long i) {
  if constexpr (XL2) return __ldcg(x + i);
  else return x[i];
}

template <bool XL2 = false>
__device__ __forceinline__ void nbr_sums(const Geo& g, const double* x, const double* __restrict__ bnd, int gx,
                                         int gy, int gz, long long gi, double& inner, double& outer) {
  const long long nxy = (long long)g.nx * g.ny;
  const long long fyz = (long long)g.nz * g.ny, fxz = (long long)g.nz * g.nx;
  double si = 0.0, so = 0.0;
  if (gx > 0) si += ldx<XL2>(x, gi - 1);
  else if (bnd) so += bnd[(long long)gz * g.ny + gy];
  if (gx < g.nx - 1) si += ldx<XL2>(x, gi + 1);
  else if (bnd) so += bnd[fyz + (long long)gz * g.ny + gy];
  if (gy > 0) si += ldx<XL2>(x, gi - g.nx);
  else if (bnd) so += bnd[2 * fyz + (long long)gz * g.nx + gx];
  if (gy < g.ny - 1) si += ldx<XL2>(x, gi + g.nx);
  else if (bnd) so += bnd[2 * fyz + fxz + (long long)gz * g.nx + gx];
  if (gz > 0) si += ldx<XL2>(x, gi - nxy);
  else if (bnd) so += bnd[2 * fyz + 2 * fxz + (long long)gy * g.nx + gx];
  if (gz < g.nz - 1) si += ldx<XL2>(x, gi + nxy);
  else if (bnd) so += bnd[2 * fyz + 2 * fxz + nxy + (long long)gy * g.nx + gx];
  inner = si;
  outer = so;
}

}  // namespace ms
