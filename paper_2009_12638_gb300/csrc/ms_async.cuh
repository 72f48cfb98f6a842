// ms_async.cuh -- the asynchronous outer iteration's protocol, shared by
// the streaming (ms_async.cu) and resident (ms_resident.cu) async kernels:
// task choice, seqlocked halo refresh, face publication and the stale
// global-residual monitor (sections 2.1, 2.3 and 3 of the paper).
//
// Ownership: task t = (block, rhs) belongs to cluster t % nclusters for the
// whole launch; only its owner writes its x, faces, halo cache, partial and
// sweep count.  Readers of a neighbour's face never wait: they take the
// newest complete version (two slots per face, per-slot seqlock counters)
// or keep the halo they hold.
#pragma once
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


// Per-thread async state; meaningful in thread 0 of cluster rank 0, which
// takes every control decision and broadcasts it (DSMEM + cluster barrier).
struct AsyncCtl {
  int par;                       // broadcast buffer parity
  int next;                      // round-robin cursor over owned tasks
  int owned;                     // tasks owned by this cluster
  unsigned* s1v;                 // [6] seqlock snapshot of the faces being fetched (shared memory)
  unsigned* vvv;                 // [6] versions being fetched (shared memory)
  unsigned long long t_start;    // launch start (globaltimer, ns)
};

// snap: 12 unsigned of shared memory for the seqlock snapshot (thread 0 of rank 0 uses it)
__device__ __forceinline__ AsyncCtl async_ctl_init(const AsyncArgs& a, unsigned cid, unsigned ncl, unsigned* snap) {
  AsyncCtl c;
  c.s1v = snap;
  c.vvv = snap + 6;
  c.par = 0;
  c.next = (int)cid;
  c.owned = (int)cid < a.ntasks ? (a.ntasks - (int)cid + (int)ncl - 1) / (int)ncl : 0;
  c.t_start = globaltimer();
  return c;
}

// Picks the next runnable owned task (round-robin) or decides to stop; the
// result (task index, or -1 to leave the loop) is identical in every CTA.
// bc is the cluster broadcast area [2][32]; c.par selects the half used by
// this visit (the caller flips it at the end of the visit).
__device__ __forceinline__ int async_pick(const AsyncArgs& a, AsyncCtl& c, int (*bc)[32], unsigned rank,
                                          unsigned csize, unsigned cid, unsigned ncl) {
  if (rank == 0 && threadIdx.x == 0) {
    int t = -1;
    const unsigned long long now = globaltimer();
    if (ld_rlx_s32(a.stop)) {
      t = -1;
    } else if (a.time_budget_ns && now - c.t_start > a.time_budget_ns) {
      atomicOr(a.err, kErrTimeout);
      st_rlx_s32(a.stop, 1);
    } else if (a.slice_ns && now - c.t_start > a.slice_ns) {
      t = -1;  // end of this launch's time slice: state is kept, the host relaunches
    } else {
      for (int j = 0; j < c.owned; ++j) {
        const int cand = c.next;
        c.next += (int)ncl;
        if (c.next >= a.ntasks) c.next = (int)cid;
        if (a.sweeps[cand] < a.outer_maxit && !ld_rlx_s32(a.rhs_stop + a.tasks[cand].rhs)) {
          t = cand;
          break;
        }
      }
    }
    for (unsigned j = 0; j < csize; ++j) cl_store(&bc[c.par][1], j, t);
  }
  cl_barrier();
  return bc[c.par][1];
}

// Halo refresh: for each face with a neighbouring block, copy the neighbour's
// newest published face into the spare halo slot (all threads of the cluster)
// and switch to it if the seqlock shows the copy is consistent; otherwise the
// halo in use stays.  The slot in use per face is left in bc[par][20..25]
// (see async_halo).  Three cluster barriers.
template <int NT>
__device__ __forceinline__ void async_halo_refresh(const AsyncArgs& a, const Task& tk, int t, int (*bc)[32],
                                                   AsyncCtl& c, unsigned rank, unsigned csize) {
  const long long fs = a.face_stride;
  const int par = c.par;
  if (rank == 0 && threadIdx.x == 0) {
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
            c.s1v[f] = s1;
            c.vvv[f] = vv;
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
  const unsigned cl_threads = csize * NT, cl_tid = rank * NT + threadIdx.x;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int nb = bc[par][2 + f];
    if (nb < 0) continue;
    const int nel = face_size(f, tk.bx, tk.by, tk.bz);
    const double* src = a.faces + (((long long)nb * 6 + (f ^ 1)) * 2 + bc[par][8 + f]) * fs;
    double* dst = a.halo + (((long long)t * 6 + f) * 2 + (bc[par][14 + f] ^ 1)) * fs;
    for (unsigned e = cl_tid; e < (unsigned)nel; e += cl_threads) dst[e] = __ldcg(src + e);
  }
  __threadfence();
  cl_barrier();
  if (rank == 0 && threadIdx.x == 0) {
    for (int f = 0; f < 6; ++f) {
      const int nb = bc[par][2 + f];
      int cur = bc[par][14 + f];
      if (nb >= 0) {
        const unsigned s2 = ld_acq_u32(a.face_seq + (nb * 6 + (f ^ 1)) * 2 + bc[par][8 + f]);
        if (s2 == c.s1v[f]) {  // consistent copy: switch to it
          cur ^= 1;
          a.halo_cur[t * 6 + f] = cur;
          a.halo_ver[t * 6 + f] = c.vvv[f];
        }
      }
      for (unsigned j = 0; j < csize; ++j) cl_store(&bc[par][20 + f], j, cur);
    }
  }
  cl_barrier();
}

// The halo face f in use after async_halo_refresh (cur = bc[par] + 20).
__device__ __forceinline__ const double* async_halo(const AsyncArgs& a, int t, const int* cur, int f) {
  return a.halo + (((long long)t * 6 + f) * 2 + cur[f]) * a.face_stride;
}

// Neighbour sums of block point (x, y, z) (block coordinates) of task tk:
// inside the block from x (in place), across a block face from the halo in
// use, at the domain boundary from the packed Dirichlet faces.
__device__ __forceinline__ void async_nbr_sums(const AsyncArgs& a, const Task& tk, int t, const int* cur,
                                               const double* xr, const double* __restrict__ br, int x, int y, int z,
                                               long long gi, double& si, double& so) {
  const Geo& g = a.g;
  const long long nxy = (long long)g.nx * g.ny;
  const long long fyz = (long long)g.nz * g.ny, fxz = (long long)g.nz * g.nx;
  const int gx = tk.ox + x, gy = tk.oy + y, gz = tk.oz + z;
  si = 0.0;
  so = 0.0;
  if (x > 0) si += xr[gi - 1];
  else if (gx > 0) si += async_halo(a, t, cur, 0)[z * tk.by + y];
  else if (br) so += br[(long long)gz * g.ny + gy];
  if (x < tk.bx - 1) si += xr[gi + 1];
  else if (gx < g.nx - 1) si += async_halo(a, t, cur, 1)[z * tk.by + y];
  else if (br) so += br[fyz + (long long)gz * g.ny + gy];
  if (y > 0) si += xr[gi - g.nx];
  else if (gy > 0) si += async_halo(a, t, cur, 2)[z * tk.bx + x];
  else if (br) so += br[2 * fyz + (long long)gz * g.nx + gx];
  if (y < tk.by - 1) si += xr[gi + g.nx];
  else if (gy < g.ny - 1) si += async_halo(a, t, cur, 3)[z * tk.bx + x];
  else if (br) so += br[2 * fyz + fxz + (long long)gz * g.nx + gx];
  if (z > 0) si += xr[gi - nxy];
  else if (gz > 0) si += async_halo(a, t, cur, 4)[y * tk.bx + x];
  else if (br) so += br[2 * fyz + 2 * fxz + (long long)gy * g.nx + gx];
  if (z < tk.bz - 1) si += xr[gi + nxy];
  else if (gz < g.nz - 1) si += async_halo(a, t, cur, 5)[y * tk.bx + x];
  else if (br) so += br[2 * fyz + 2 * fxz + nxy + (long long)gy * g.nx + gx];
}

// Face publication, part 1: mark the slots about to be written (odd seq) and
// broadcast them (bc[par] + 26, -1 where there is no neighbouring block).
__device__ __forceinline__ void async_publish_begin(const AsyncArgs& a, const Task& tk, int t, int (*bc)[32],
                                                    const AsyncCtl& c, unsigned rank, unsigned csize) {
  if (rank == 0 && threadIdx.x == 0) {
    for (int f = 0; f < 6; ++f) {
      int slot = -1;
      if (nbr_task(a, tk, f) >= 0) {
        const unsigned vv = a.face_ver[t * 6 + f];
        slot = (int)((vv + 1u) & 1u);
        unsigned* sp = a.face_seq + (t * 6 + f) * 2 + slot;
        st_rlx_u32(sp, *sp + 1u);  // odd: slot being written
      }
      for (unsigned j = 0; j < csize; ++j) cl_store(&bc[c.par][26 + f], j, slot);
    }
    __threadfence();
  }
  cl_barrier();
  __threadfence();  // order the odd marks before this thread's face stores
}

// Store the new value of block point (x, y, z) into every face slot it belongs to.
__device__ __forceinline__ void async_face_store(const AsyncArgs& a, const Task& tk, int t, const int* fslot, int x,
                                                 int y, int z, double v) {
  const long long fs = a.face_stride;
  if (x == 0 && fslot[0] >= 0) a.faces[(((long long)t * 6 + 0) * 2 + fslot[0]) * fs + z * tk.by + y] = v;
  if (x == tk.bx - 1 && fslot[1] >= 0) a.faces[(((long long)t * 6 + 1) * 2 + fslot[1]) * fs + z * tk.by + y] = v;
  if (y == 0 && fslot[2] >= 0) a.faces[(((long long)t * 6 + 2) * 2 + fslot[2]) * fs + z * tk.bx + x] = v;
  if (y == tk.by - 1 && fslot[3] >= 0) a.faces[(((long long)t * 6 + 3) * 2 + fslot[3]) * fs + z * tk.bx + x] = v;
  if (z == 0 && fslot[4] >= 0) a.faces[(((long long)t * 6 + 4) * 2 + fslot[4]) * fs + y * tk.bx + x] = v;
  if (z == tk.bz - 1 && fslot[5] >= 0) a.faces[(((long long)t * 6 + 5) * 2 + fslot[5]) * fs + y * tk.bx + x] = v;
}

// Face publication, part 2 (after every thread stored its face values):
// complete the slots (even seq, release), bump the versions and the task's
// sweep count, record the inner iterations (and the trace record, with the
// block residual this visit started from, read back from the partials).
__device__ __forceinline__ void async_publish_end(const AsyncArgs& a, const Task& tk, int t, const int* fslot,
                                                  unsigned rank, int m) {
  __threadfence();
  cl_barrier();
  if (rank == 0 && threadIdx.x == 0) {
    for (int f = 0; f < 6; ++f) {
      if (fslot[f] < 0) continue;
      unsigned* sp = a.face_seq + (t * 6 + f) * 2 + fslot[f];
      st_rel_u32(sp, *sp + 1u);  // even: slot complete
      st_rel_u32(a.face_ver + t * 6 + f, a.face_ver[t * 6 + f] + 1u);
    }
    if (a.tr.rec) trace_push(a.tr, a.sweeps[t], tk.block, tk.rhs, m, a.partial[t]);
    a.sweeps[t] += 1;
    if (m > 0) {
      atomicAdd(a.inner_count + 2 * tk.rhs, (unsigned long long)m);
      atomicAdd(a.inner_count + 2 * tk.rhs + 1, (unsigned long long)m * (unsigned long long)tk.bx * tk.by * tk.bz);
    }
  }
}

// Stale global estimate per rhs (warp 0 of cluster rank 0): section 3's
// sqrt(sum_i ||r_i||^2) / ||bhat|| from the latest published block partials;
// a rhs whose estimate is below tol stops; all stopped -> the launch stops.
__device__ __forceinline__ void async_monitor(const AsyncArgs& a, unsigned rank) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (rank != 0 || warp != 0) return;
  int all = 1;
  for (int r = 0; r < a.g.nrhs; ++r) {
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

}  // namespace ms
