// ms_internal.h -- types shared by the host orchestration (ms_api.cu) and the
// device kernels (ms_kernels.cu, ms_async.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ms.h"

struct ms_grid;

namespace ms {

constexpr int kMaxCluster = 16;

// One unit of outer work: block `block` of right-hand side `rhs`.
// (ox, oy, oz) is the block origin in the grid, (bx, by, bz) its edge lengths.
// One (block, rhs) pair.  (ox, oy, oz) + (bx, by, bz) is the box the inner
// CG solves on: the block itself, or with overlapping blocks the block
// extended by the overlap on every face (clipped to the grid).  The block's
// own points are [wx0, wx1) x [wy0, wy1) x [wz0, wz1) in box coordinates:
// only they count towards the global residual and only they are updated.
struct Task {
  int ox, oy, oz, bx, by, bz, rhs, block;
  int wx0, wx1, wy0, wy1, wz0, wz1;
};

__host__ __device__ inline bool owns(const Task& t, int lx, int ly, int lz) {
  return lx >= t.wx0 && lx < t.wx1 && ly >= t.wy0 && ly < t.wy1 && lz >= t.wz0 && lz < t.wz1;
}

struct Geo {
  int nx, ny, nz, nrhs;
  long long npts;  // nx*ny*nz
  long long nbnd;  // packed boundary doubles per rhs
};

// rhs_state values
constexpr int kActive = 0;
constexpr int kConverged = 1;
constexpr int kStopped = 2;

// Solve trace (opts.trace): a ring of ms_trace_rec in device memory.  Every
// block solve takes the next ticket from `head` and writes record
// ticket % cap; rec == nullptr = no trace.
struct TraceArgs {
  ms_trace_rec* rec;
  unsigned long long* head;
  int cap;
};

// device error word bits
constexpr int kErrGeometry = 1;
constexpr int kErrTimeout = 2;

// Arguments of one synchronous outer sweep.  The sweep index k is read from
// device memory (k_dev) so that a captured graph of sweeps can be replayed.
struct SweepArgs {
  Geo g;
  const double* f;    // [nrhs][npts] or null
  const double* bnd;  // [nrhs][nbnd] or null
  double* xbuf0;      // x^k for even k
  double* xbuf1;      // x^k for odd k
  const Task* tasks;
  int ntasks;
  unsigned int* counter;  // dynamic task queue head, reset by the check kernel
  const int* rhs_state;   // [nrhs]
  const int* all_done;
  double* partial;  // [ntasks] block sum of squares of b - A x^k
  void* scratch;    // per cluster slot: r, p0, p1, d (vec_stride elements each)
  long long vec_stride;
  double inner_rtol;
  int inner_maxit;
  int outer_maxit;
  const int* k_dev;
  unsigned long long* inner_count;  // [nrhs][2]: inner iterations, inner lattice updates
  const double* inv_bnorm;          // [nrhs] 1/||bhat|| (1 if bhat = 0): FP32 inner scaling
  int* err;
  const double* inner_rtol_rhs;  // [nrhs] per-rhs inner tolerance (opts.inner_adapt) or null: inner_rtol
  int inner_method;              // 0 CG, 1 restarted GMRES (scalar streaming engine)
  int gmres_restart;             // GMRES basis size per cycle (slot holds gmres_restart + 3 vectors)
  TraceArgs tr;                  // solve trace (rec == nullptr: none)
  long long sum_polls = 0;       // polls of a tagged cluster sum before it gives up (0 = default)
};

__host__ __device__ inline double sweep_inner_rtol(const SweepArgs& a, int rhs) {
  return a.inner_rtol_rhs ? a.inner_rtol_rhs[rhs] : a.inner_rtol;
}

// Runtime adaptation of the inner tolerance (opts.inner_adapt), per rhs, run
// by the check kernel after every sweep.  A ladder of relative inner
// tolerances; rounds of 3 x kAdaptWindow sweeps run the centre rung, the next
// looser and the next tighter one (at an end of the ladder, where that
// neighbour does not exist, the rung kAdaptEdgeProbe steps inward instead, so
// that a search walked to an end by the first rounds can leave it); each
// sweep's decrease of log(rho) is charged to the rung it ran with, against
// its work (inner lattice updates plus kAdaptSweepCost x points for the
// residual and update), except the first kAdaptSkip sweeps of a window, whose
// decrease still reflects the residual the previous rung left.  Every rung
// keeps its charges across rounds, scaled by kAdaptMemory at each round's end,
// so that a rung's rate rests on more than one window; of the round's three
// rungs the one with the largest decrease per work becomes the centre of the
// next round.  Every input is deterministic (residuals and iteration counts,
// no clocks).
constexpr int kAdaptRungs = 11;
constexpr int kAdaptStart = 3;        // rung of the first sweeps (0.3)
constexpr int kAdaptWindow = 8;       // sweeps per rung and round
constexpr int kAdaptSkip = 2;         // sweeps at the start of a window that are not charged
constexpr int kAdaptEdgeProbe = 4;    // inward distance of the probe at an end of the ladder
constexpr double kAdaptMemory = 0.5;  // weight of a rung's earlier charges after each round
constexpr int kAdaptWarmup = 4;       // sweeps before the first round
constexpr double kAdaptSweepCost = 12.0;  // residual + update, in inner iterations per point
__host__ __device__ inline double adapt_rung_rtol(int r) {
  constexpr double ladder[kAdaptRungs] = {0.8, 0.6, 0.45, 0.3, 0.2, 0.12, 0.07, 0.04, 0.02, 0.01, 1e-3};
  return ladder[r < 0 ? 0 : (r >= kAdaptRungs ? kAdaptRungs - 1 : r)];
}
struct AdaptState {
  int c;                       // centre rung of the current round
  int rs;                      // first sweep of the current round
  int cur;                     // rung of the next sweep
  double lr_prev;              // log(rho_{k-1})
  double cum_prev, cum_prev2;  // cumulative work at checks k-1 and k-2
  double acc_d[3], acc_w[3];   // round sums per window: log-residual decrease, work
  double mem_d[kAdaptRungs];   // per rung: charges of earlier rounds, scaled by kAdaptMemory per round
  double mem_w[kAdaptRungs];
};

struct CheckArgs {
  int nrhs;
  int ntasks;
  const Task* tasks;
  const double* partial;
  const double* inv_bnorm;  // [nrhs]
  int* rhs_state;
  int* k_final;  // [nrhs]
  int* all_done;
  unsigned int* counter;
  int* k_dev;
  double* hist;  // [nrhs][outer_maxit+1] or null
  double* thist;  // [outer_maxit+1] or null: ms since the first stop test, per stop test
  double outer_tol;
  int outer_maxit;
  unsigned long long time_budget_ns;  // 0 = none: else active rhs stop (kErrTimeout) once spent
  unsigned long long* t_start;        // device start time, set by the first check of the solve
  int* err;
  int use_cond;                       // set the WHILE condition of the enclosing graph
  cudaGraphConditionalHandle cond;
  AdaptState* adapt;                        // [nrhs] or null (no adaptation)
  double* inner_rtol_rhs;                   // [nrhs] written for the next sweep when adapt != null
  const unsigned long long* inner_count;    // [nrhs][2] cumulative inner iterations / lattice updates
  double npts;                              // points per rhs
};

// Synchronous solve as one persistent "dataflow" launch (ms_resident.cu):
// tickets are handed out sweep-major; ticket j is task j % ntasks of sweep
// k0 + j / ntasks.  A task runs once the stop decision of the previous
// sweep is known and its block and the six neighbouring blocks finished the
// previous sweep.  All counters are relative to the first sweep k0.
struct FlowArgs {
  SweepArgs s;
  CheckArgs c;                   // bookkeeping of the stop decisions (hist, states, k_final)
  int k0;                        // first sweep of this launch
  int px, py, pz, nblocks;
  const int* task_of;            // [nrhs][nblocks] -> task index
  unsigned long long* ticket;    // ticket counter
  int* res_cnt;                  // [outer_maxit + 2 - k0] residuals counted per sweep
  int* done_rel;                 // [ntasks] sweeps completed since k0
  int* decided_rel;              // last sweep (relative) whose stop decision is made, -1 before any
  long long spin_limit;          // polls before a wait gives up (kErrTimeout), summed over the launch
  int slow_block, slow_ns;       // resilience test: this block sleeps slow_ns per task (-1 = none)
};

// Asynchronous persistent solve (see ms_async.cu).  Task t = (block, rhs) is
// owned by cluster t % nclusters for the whole launch.
struct AsyncArgs {
  Geo g;
  const double* f;
  const double* bnd;
  double* x;          // [nrhs][npts], updated in place (each block only by its owner)
  const Task* tasks;  // [ntasks]
  int ntasks;
  int px, py, pz, nblocks;
  const int* task_of;      // [nrhs][nblocks] -> task index
  long long face_stride;   // doubles per face slot (max face size)
  double* faces;           // [ntasks][6][2][face_stride] published boundary layers of x
  unsigned int* face_seq;  // [ntasks][6][2] seqlock counters (odd while a slot is written)
  unsigned int* face_ver;  // [ntasks][6] number of publishes; latest slot = ver & 1
  double* halo;            // [ntasks][6][2][face_stride] neighbour values in use / being fetched
  int* halo_cur;           // [ntasks][6] which halo slot is in use
  unsigned int* halo_ver;  // [ntasks][6] neighbour version held
  double* partial;         // [ntasks] latest ||r_i||^2 of the task (racy, may be stale)
  int* sweeps;             // [ntasks] local sweeps done
  const double* inv_bnorm; // [nrhs]
  int* rhs_stop;           // [nrhs] set when the stale estimate of that rhs is below tol
  int* stop;               // all work stops (all rhs stopped, or time budget spent)
  void* scratch;
  long long vec_stride;
  double inner_rtol;
  int inner_maxit;
  int outer_maxit;
  double outer_tol;
  int slow_block;
  int slow_ns;
  unsigned long long* inner_count;  // [nrhs][2]: iterations, lattice updates
  unsigned long long time_budget_ns;  // 0 = none; when spent the launch stops with kErrTimeout
  unsigned long long slice_ns;        // the launch returns (no error) after this long; the host relaunches
  int* err;
  TraceArgs tr;                       // solve trace (rec == nullptr: none)
  long long sum_polls = 0;            // polls of a tagged cluster sum before it gives up (0 = default)
};

struct ResidArgs {
  Geo g;
  const double* f;
  const double* bnd;
  const double* x;
  double* part;  // [nrhs][nblk][2]: sum r^2, sum bhat^2
  int nblk;
};

// One global FP64 CG solve on the whole grid (ms_gcg.cu).
struct GcgArgs {
  Geo g;
  const double* f;    // [nrhs][npts] or null
  const double* bnd;  // [nrhs][nbnd] or null
  double* x;          // in: x0, out: solution
  double* r;          // [nrhs][npts] workspace
  double* p;
  double* q;
  double* part_rr;  // [2][nrhs][nb]: r.r partials, by iteration parity
  double* part_pq;  // [nrhs][nb]
  int nb;           // CTAs per rhs
  const double* norms;  // [nrhs][2]; norms[2s+1] = ||bhat||^2
  double tol;
  int maxit;
  int* state;    // [nrhs] kActive / kConverged / kStopped
  int* k_final;  // [nrhs] iterations done when the rhs stopped
  int* k_dev;    // iteration counter
  int* stop_all;
  unsigned long long* t_start;
  long long budget_ns;  // 0 = no time budget
  int use_cond;
  cudaGraphConditionalHandle cond;
};
int gcg_blocks(const Geo& g);
cudaError_t launch_gcg_init(const GcgArgs& a, cudaStream_t s);
cudaError_t launch_gcg_iteration(const GcgArgs& a, cudaStream_t s);

// handle accessors for entry points defined outside ms_api.cu
Geo grid_geo(const ms_grid* g);
int grid_fail(ms_grid* g, int code, const char* fmt, ...);

// launchers (ms_kernels.cu / ms_async.cu)
cudaError_t launch_sweep(int prec, int threads, int cluster, int slots, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_check(const CheckArgs& a, cudaStream_t s);
cudaError_t sweep_max_clusters(int prec, int threads, int cluster, int* out);
cudaError_t launch_async(int prec, int threads, int cluster, int slots, const AsyncArgs& a, cudaStream_t s);
cudaError_t async_max_clusters(int prec, int threads, int cluster, int* out);
cudaError_t launch_resid(const ResidArgs& a, double* out /*[nrhs][2]*/, double* inv_bnorm /*[nrhs] or null*/,
                         cudaStream_t s);
cudaError_t launch_face_gather(const Geo& g, const double* lam, double* grad, cudaStream_t s);
// ||bhat||^2 per rhs and 1/||bhat|| (visits only the points next to the boundary when f is null);
// part: [nrhs][nblk] scratch
cudaError_t launch_bhat_sq(const Geo& g, const double* f, const double* bnd, double* part, int nblk, double* out,
                           double* inv_bnorm, cudaStream_t s);
// out[s] = fixed-order sum of the block partials of rhs s
cudaError_t launch_task_sums(const Task* tasks, const double* partial, int ntasks, int nrhs, double* out,
                             cudaStream_t s);
cudaError_t launch_async_init(const AsyncArgs& a, cudaStream_t s);
cudaError_t launch_async_rearm(const AsyncArgs& a, cudaStream_t s);
// on-chip (resident) FP32 inner CG, sync mode (ms_resident.cu)
int res_variant_count();
void res_variant_info(int v, int* nt, int* kc, int* zs, int* ds, int* qr);
cudaError_t res_max_clusters(int variant, int cluster, size_t smem_bytes, int* out, bool async_mode);
cudaError_t launch_res_async(int variant, int cluster, int slots, size_t smem_bytes, const AsyncArgs& a,
                             cudaStream_t s);
cudaError_t launch_res_flow(int variant, int cluster, int slots, size_t smem_bytes, const FlowArgs& a,
                            cudaStream_t s);
cudaError_t res_flow_max_clusters(int variant, int cluster, size_t smem_bytes, int* out);
// vectorised FP32 streaming engine, sync mode (ms_stream4.cu)
cudaError_t strip_max_clusters(int prec, int threads, int cluster, int* out);  // prec 1 mixed, 0 FP64
cudaError_t launch_strip_sweep(int prec, int threads, int cluster, int slots, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_res_sweep(int variant, int cluster, int slots, size_t smem_bytes, const SweepArgs& a,
                             cudaStream_t s);

}  // namespace ms
