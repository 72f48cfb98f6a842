// ms_api.cu -- host side of libms: the C ABI declared in include/ms.h.
//
// Owns the grid handle, the block partition, the device workspace and the
// solve loop.  All device work is ordered on the caller's stream; the library
// allocates its own workspace once per handle and grows it on demand.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ms.h"
#include "ms_internal.h"
#include "ms_gmres.cuh"
#include "ms_tune.h"

using namespace ms;

namespace {

thread_local std::string g_create_error;

constexpr size_t kTuneRounds = 2;  // timed sweeps per autotuning candidate

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  // grow (never shrink); contents are not preserved
  cudaError_t reserve(size_t want) {
    if (want <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

// small per-solve device state, one allocation
struct Ctl {
  unsigned int counter;
  int all_done;
  int k_dev;
  int err;
  int stop;
  int pad[3];
  unsigned long long t_start;
};

}  // namespace

struct ms_grid {
  int nx, ny, nz, nrhs;
  int px = 1, py = 1, pz = 1;
  std::vector<int> cx, cy, cz;
  std::string err;
  int device = 0;
  // workspace
  DevBuf xalt;     // second x buffer [nrhs][npts]
  DevBuf scratch;  // per-slot CG vectors
  DevBuf tasks;    // Task[ntasks]
  DevBuf partial;  // double[ntasks]
  DevBuf ctl;      // Ctl + per-rhs arrays
  DevBuf hist;     // [nrhs][outer_maxit+1]
  DevBuf rpart;    // residual partials
  DevBuf host_io;  // device copies for ms_solve_host: f, bnd, x
  DevBuf async_ws; // face buffers, halos, seq counters (async mode)
  DevBuf flow_ws;  // tickets, per-task progress, per-sweep counters (persistent sync mode)
  DevBuf gcg_ws;   // global CG: r, p, q, partial sums, control words
  DevBuf thist;    // [outer_maxit+1] stop-test times (opts.time_hist)
  DevBuf trace_ws; // trace ring (opts.trace): head counter, then trace_cap records
  TraceArgs trace{nullptr, nullptr, 0};  // the current solve's trace ring (rec == nullptr: none)
  Tuner tuner;
  long long npts() const { return (long long)nx * ny * nz; }
  long long nbnd() const { return ms_boundary_size(nx, ny, nz); }
  Geo geo() const { return Geo{nx, ny, nz, nrhs, npts(), nbnd()}; }
};

static int fail(ms_grid* g, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (g) g->err = buf;
  else g_create_error = buf;
  return code;
}

namespace ms {
Geo grid_geo(const ms_grid* g) { return g->geo(); }
int grid_fail(ms_grid* g, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (g) g->err = buf;
  else g_create_error = buf;
  return code;
}
}  // namespace ms

#define MS_CUDA(g, expr)                                                                        \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      cudaGetLastError(); /* clear a non-sticky error so later calls do not report it */       \
      return fail((g), e_ == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA, "%s: %s (%s)", \
                  #expr, cudaGetErrorName(e_), cudaGetErrorString(e_));                         \
    }                                                                                           \
  } while (0)

extern "C" long long ms_boundary_size(int nx, int ny, int nz) {
  return 2LL * nz * ny + 2LL * nz * nx + 2LL * ny * nx;
}

extern "C" void ms_default_opts(ms_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->mode = MS_MODE_SYNC;
  o->precision = MS_PREC_MIXED;
  o->inner_rtol = 1e-6;
  o->inner_maxit = 50;
  o->outer_tol = 1e-8;
  o->outer_maxit = 100000;
  o->time_limit_ms = 0.0;
  o->cluster = 0;
  o->threads = 0;
  o->slots = 0;
  o->check_every = 0;
  o->use_graph = 1;
  o->slow_block = -1;
  o->slow_ns = 0;
  o->res_hist = nullptr;
  o->profile = 0;
  o->persistent = 1;
  o->engine = 0;
  o->variant = -1;
  o->inner_adapt = 0;
  o->overlap = 0;
  o->inner_method = 0;
  o->gmres_restart = 10;
  o->time_hist = nullptr;
  o->wait_polls = 0;
  o->trace_cap = 0;
  o->trace = nullptr;
  o->sum_polls = 0;
}

static std::vector<int> equal_cuts(int n, int p) {
  std::vector<int> c(p + 1, 0);
  int q = n / p, rem = n % p;
  for (int a = 0; a < p; ++a) c[a + 1] = c[a] + q + (a < rem ? 1 : 0);
  return c;
}

extern "C" int ms_create_grid(int nx, int ny, int nz, int nrhs, ms_grid** out) {
  if (!out) return fail(nullptr, MS_ERR_ARG, "ms_create_grid: out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || nrhs < 1)
    return fail(nullptr, MS_ERR_ARG, "ms_create_grid: sizes must be >= 1 (got %d %d %d nrhs %d)", nx, ny, nz, nrhs);
  const double total = (double)nx * ny * nz * nrhs;
  if (total > 9.0e15) return fail(nullptr, MS_ERR_ARG, "ms_create_grid: grid too large");
  if ((long long)nx * ny > 0x7fffffffLL || (long long)nx * nz > 0x7fffffffLL || (long long)ny * nz > 0x7fffffffLL)
    return fail(nullptr, MS_ERR_ARG, "ms_create_grid: a face exceeds 2^31 points");
  ms_grid* g = new ms_grid();
  g->nx = nx;
  g->ny = ny;
  g->nz = nz;
  g->nrhs = nrhs;
  g->cx = {0, nx};
  g->cy = {0, ny};
  g->cz = {0, nz};
  cudaGetDevice(&g->device);
  *out = g;
  return MS_OK;
}

static bool valid_cuts(const int* c, int p, int n) {
  if (c[0] != 0 || c[p] != n) return false;
  for (int a = 0; a < p; ++a)
    if (c[a + 1] <= c[a]) return false;
  return true;
}

extern "C" int ms_partition(ms_grid* g, int px, int py, int pz, const int* cx, const int* cy, const int* cz) {
  if (!g) return MS_ERR_ARG;
  if (px < 1 || py < 1 || pz < 1) return fail(g, MS_ERR_ARG, "ms_partition: block counts must be >= 1");
  if (px > g->nx || py > g->ny || pz > g->nz)
    return fail(g, MS_ERR_ARG, "ms_partition: more blocks than points along an axis (edge < 1)");
  std::vector<int> ax = cx ? std::vector<int>(cx, cx + px + 1) : equal_cuts(g->nx, px);
  std::vector<int> ay = cy ? std::vector<int>(cy, cy + py + 1) : equal_cuts(g->ny, py);
  std::vector<int> az = cz ? std::vector<int>(cz, cz + pz + 1) : equal_cuts(g->nz, pz);
  if (!valid_cuts(ax.data(), px, g->nx) || !valid_cuts(ay.data(), py, g->ny) || !valid_cuts(az.data(), pz, g->nz))
    return fail(g, MS_ERR_ARG, "ms_partition: cuts must rise strictly from 0 to n (every edge >= 1)");
  const long long nb = (long long)px * py * pz;
  if (nb * g->nrhs > 0x3fffffffLL) return fail(g, MS_ERR_ARG, "ms_partition: too many blocks");
  g->px = px;
  g->py = py;
  g->pz = pz;
  g->cx = ax;
  g->cy = ay;
  g->cz = az;
  return MS_OK;
}

extern "C" int ms_get_cuts(ms_grid* g, int* cx, int* cy, int* cz) {
  if (!g || !cx || !cy || !cz) return g ? fail(g, MS_ERR_ARG, "ms_get_cuts: NULL output") : MS_ERR_ARG;
  std::copy(g->cx.begin(), g->cx.end(), cx);
  std::copy(g->cy.begin(), g->cy.end(), cy);
  std::copy(g->cz.begin(), g->cz.end(), cz);
  return MS_OK;
}

// Tasks: every (block, rhs), largest blocks first (longest-processing-time
// order for the dynamic queue), ties in (rhs, block id) order.
// Tasks of the partition; with overlap o > 0 every box is the block extended
// by o points on each face (clipped to the grid), the owned range marking the
// block itself (section 3.2's overlapping blocks).
static std::vector<Task> build_tasks(const ms_grid* g, long long* max_pts, int overlap = 0) {
  std::vector<Task> ts;
  long long mx = 0;
  auto ext = [&](int lo, int hi, int n, int* o0, int* len, int* w0, int* w1) {
    const int e0 = std::max(0, lo - overlap), e1 = std::min(n, hi + overlap);
    *o0 = e0;
    *len = e1 - e0;
    *w0 = lo - e0;
    *w1 = hi - e0;
  };
  for (int s = 0; s < g->nrhs; ++s)
    for (int bk = 0; bk < g->pz; ++bk)
      for (int bj = 0; bj < g->py; ++bj)
        for (int bi = 0; bi < g->px; ++bi) {
          Task t;
          ext(g->cx[bi], g->cx[bi + 1], g->nx, &t.ox, &t.bx, &t.wx0, &t.wx1);
          ext(g->cy[bj], g->cy[bj + 1], g->ny, &t.oy, &t.by, &t.wy0, &t.wy1);
          ext(g->cz[bk], g->cz[bk + 1], g->nz, &t.oz, &t.bz, &t.wz0, &t.wz1);
          t.rhs = s;
          t.block = bi + g->px * (bj + g->py * bk);
          mx = std::max(mx, (long long)t.bx * t.by * t.bz);
          ts.push_back(t);
        }
  std::stable_sort(ts.begin(), ts.end(), [](const Task& a, const Task& b) {
    return (long long)a.bx * a.by * a.bz > (long long)b.bx * b.by * b.bz;
  });
  *max_pts = mx;
  return ts;
}

static int check_opts(ms_grid* g, const ms_opts& o) {
  if (o.mode != MS_MODE_SYNC && o.mode != MS_MODE_ASYNC) return fail(g, MS_ERR_ARG, "opts.mode must be SYNC or ASYNC");
  if (o.precision != MS_PREC_FP64 && o.precision != MS_PREC_MIXED)
    return fail(g, MS_ERR_ARG, "opts.precision must be FP64 or MIXED");
  if (!(o.inner_rtol >= 0.0) || o.inner_maxit < 0 || !(o.outer_tol >= 0.0) || o.outer_maxit < 0)
    return fail(g, MS_ERR_ARG, "opts: tolerances must be >= 0 and iteration caps >= 0");
  if (o.cluster < 0 || o.cluster > kMaxCluster) return fail(g, MS_ERR_ARG, "opts.cluster must be 0..16");
  if (o.threads != 0 && o.threads != 256 && o.threads != 512 && o.threads != 1024)
    return fail(g, MS_ERR_ARG, "opts.threads must be 0, 256, 512 or 1024");
  if (o.slots < 0 || o.check_every < 0) return fail(g, MS_ERR_ARG, "opts.slots and opts.check_every must be >= 0");
  if (o.time_limit_ms < 0.0) return fail(g, MS_ERR_ARG, "opts.time_limit_ms must be >= 0");
  if (o.engine < 0 || o.engine > 2) return fail(g, MS_ERR_ARG, "opts.engine must be 0 (auto), 1 or 2");
  if (o.variant < -1 || o.variant >= ms::res_variant_count())
    return fail(g, MS_ERR_ARG, "opts.variant must be -1 (tuned) or 0..%d", ms::res_variant_count() - 1);
  if (o.inner_adapt != 0 && o.inner_adapt != 1) return fail(g, MS_ERR_ARG, "opts.inner_adapt must be 0 or 1");
  if (o.overlap < 0) return fail(g, MS_ERR_ARG, "opts.overlap must be >= 0");
  if (o.wait_polls < 0) return fail(g, MS_ERR_ARG, "opts.wait_polls must be >= 0 (0 = default)");
  if (o.trace_cap < 0) return fail(g, MS_ERR_ARG, "opts.trace_cap must be >= 0");
  if (o.sum_polls < 0) return fail(g, MS_ERR_ARG, "opts.sum_polls must be >= 0 (0 = default)");
  if (o.inner_method != 0 && o.inner_method != 1) return fail(g, MS_ERR_ARG, "opts.inner_method must be 0 (CG) or 1 (GMRES)");
  if (o.inner_method == 1 && (o.gmres_restart < 1 || o.gmres_restart > kGmresMaxRestart))
    return fail(g, MS_ERR_ARG, "opts.gmres_restart must be 1..%d", kGmresMaxRestart);
  if (o.inner_method == 1 && (o.mode != MS_MODE_SYNC || o.engine == 2 || o.variant >= 0))
    return fail(g, MS_ERR_ARG, "opts.inner_method GMRES runs in the synchronous mode on the streaming engine");
  if (o.overlap > 0 && o.mode != MS_MODE_SYNC)
    return fail(g, MS_ERR_ARG, "opts.overlap needs the synchronous mode (the asynchronous faces are one layer deep)");
  if (o.overlap > 0 && o.engine == 2)
    return fail(g, MS_ERR_ARG, "opts.overlap runs on the streaming engine (engine 0 or 1)");
  if (o.inner_adapt && o.mode != MS_MODE_SYNC)
    return fail(g, MS_ERR_ARG, "opts.inner_adapt needs the synchronous mode (its controller runs between sweeps)");
  if (o.variant >= 0 && (o.precision != MS_PREC_MIXED || o.engine == 1))
    return fail(g, MS_ERR_ARG, "opts.variant selects a resident-engine layout: it needs precision MIXED and engine 0 or 2");
  return MS_OK;
}

// Per-rhs bookkeeping arrays live after Ctl in the ctl buffer.
struct CtlLayout {
  size_t off_state, off_kfinal, off_inner, off_invb, off_norm, off_adapt, off_rtol, bytes;
};
static CtlLayout ctl_layout(int nrhs) {
  CtlLayout L;
  size_t o = 256;
  L.off_state = o;
  o += ((size_t)nrhs * sizeof(int) + 255) / 256 * 256;
  L.off_kfinal = o;
  o += ((size_t)nrhs * sizeof(int) + 255) / 256 * 256;
  L.off_inner = o;
  o += ((size_t)nrhs * 2 * sizeof(unsigned long long) + 255) / 256 * 256;
  L.off_invb = o;
  o += ((size_t)nrhs * sizeof(double) + 255) / 256 * 256;
  L.off_norm = o;
  o += ((size_t)nrhs * 2 * sizeof(double) + 255) / 256 * 256;
  L.off_adapt = o;
  o += ((size_t)nrhs * sizeof(AdaptState) + 255) / 256 * 256;
  L.off_rtol = o;
  o += ((size_t)nrhs * sizeof(double) + 255) / 256 * 256;
  L.bytes = o;
  return L;
}

static int resid_blocks(long long npts) {
  long long b = (npts + 255) / 256;
  return (int)std::max(1LL, std::min(b, 152LL * 8));
}

// true residual norms of x: out[2s] = ||bhat - A x||^2, out[2s+1] = ||bhat||^2 (device), inv_bnorm optional
static int run_resid(ms_grid* g, const double* f, const double* bnd, const double* x, double* out_dev,
                     double* invb_dev, cudaStream_t st) {
  const int nblk = resid_blocks(g->npts());
  MS_CUDA(g, g->rpart.reserve((size_t)g->nrhs * nblk * 2 * sizeof(double)));
  ResidArgs ra{g->geo(), f, bnd, x, g->rpart.as<double>(), nblk};
  MS_CUDA(g, launch_resid(ra, out_dev, invb_dev, st));
  return MS_OK;
}

static int solve_device(ms_grid* g, const double* f, const double* bnd, double* x, const ms_opts& o, ms_stats* st,
                        cudaStream_t stream);

extern "C" int ms_solve(ms_grid* g, const double* f, const double* bnd, double* x, const ms_opts* opts,
                        ms_stats* stats, void* stream) {
  if (!g) return MS_ERR_ARG;
  if (!x) return fail(g, MS_ERR_ARG, "ms_solve: x is NULL");
  ms_opts o;
  if (opts) o = *opts;
  else ms_default_opts(&o);
  int rc = check_opts(g, o);
  if (rc != MS_OK) return rc;
  cudaGetLastError();  // a stale non-sticky error from unrelated work must not fail this solve
  return solve_device(g, f, bnd, x, o, stats, (cudaStream_t)stream);
}

extern "C" int ms_solve_host(ms_grid* g, const double* f_host, const double* bnd_host, double* x_host,
                             const ms_opts* opts, ms_stats* stats, void* stream) {
  if (!g) return MS_ERR_ARG;
  if (!x_host) return fail(g, MS_ERR_ARG, "ms_solve_host: x is NULL");
  ms_opts o;
  if (opts) o = *opts;
  else ms_default_opts(&o);
  int rc = check_opts(g, o);
  if (rc != MS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t fx = (size_t)g->nrhs * g->npts() * sizeof(double);
  const size_t fb = (size_t)g->nrhs * g->nbnd() * sizeof(double);
  const size_t offb = (fx + 255) / 256 * 256, offx = offb + (fb + 255) / 256 * 256;
  MS_CUDA(g, g->host_io.reserve(offx + fx));
  char* base = g->host_io.as<char>();
  double* fd = f_host ? reinterpret_cast<double*>(base) : nullptr;
  double* bd = bnd_host ? reinterpret_cast<double*>(base + offb) : nullptr;
  double* xd = reinterpret_cast<double*>(base + offx);
  if (fd) MS_CUDA(g, cudaMemcpyAsync(fd, f_host, fx, cudaMemcpyHostToDevice, s));
  if (bd) MS_CUDA(g, cudaMemcpyAsync(bd, bnd_host, fb, cudaMemcpyHostToDevice, s));
  MS_CUDA(g, cudaMemcpyAsync(xd, x_host, fx, cudaMemcpyHostToDevice, s));
  rc = solve_device(g, fd, bd, xd, o, stats, s);
  if (rc != MS_OK && rc != MS_ERR_NOT_CONVERGED) return rc;
  MS_CUDA(g, cudaMemcpyAsync(x_host, xd, fx, cudaMemcpyDeviceToHost, s));
  MS_CUDA(g, cudaStreamSynchronize(s));
  return rc;
}

extern "C" int ms_residual(ms_grid* g, const double* f, const double* bnd, const double* x, double* rel_out,
                           void* stream) {
  if (!g) return MS_ERR_ARG;
  if (!x || !rel_out) return fail(g, MS_ERR_ARG, "ms_residual: x and rel_out must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  CtlLayout L = ctl_layout(g->nrhs);
  MS_CUDA(g, g->ctl.reserve(L.bytes));
  double* norms = reinterpret_cast<double*>(g->ctl.as<char>() + L.off_norm);
  int rc = run_resid(g, f, bnd, x, norms, nullptr, s);
  if (rc != MS_OK) return rc;
  std::vector<double> h(2 * (size_t)g->nrhs);
  MS_CUDA(g, cudaMemcpyAsync(h.data(), norms, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  MS_CUDA(g, cudaStreamSynchronize(s));
  for (int r = 0; r < g->nrhs; ++r)
    rel_out[r] = h[2 * r + 1] > 0.0 ? std::sqrt(h[2 * r]) / std::sqrt(h[2 * r + 1]) : std::sqrt(h[2 * r]);
  return MS_OK;
}

extern "C" int ms_face_gather(ms_grid* g, const double* lam, double* grad_bnd, void* stream) {
  if (!g) return MS_ERR_ARG;
  if (!lam || !grad_bnd) return fail(g, MS_ERR_ARG, "ms_face_gather: NULL argument");
  MS_CUDA(g, launch_face_gather(g->geo(), lam, grad_bnd, (cudaStream_t)stream));
  return MS_OK;
}

extern "C" int ms_norms(ms_grid* g, const double* f, const double* bnd, const double* x, double* rr_out,
                        double* bb_out, void* stream) {
  if (!g) return MS_ERR_ARG;
  if (!x || (!rr_out && !bb_out))
    return fail(g, MS_ERR_ARG, "ms_norms: x and at least one of rr_out, bb_out must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  CtlLayout L = ctl_layout(g->nrhs);
  MS_CUDA(g, g->ctl.reserve(L.bytes));
  double* norms = reinterpret_cast<double*>(g->ctl.as<char>() + L.off_norm);
  int rc = run_resid(g, f, bnd, x, norms, nullptr, s);
  if (rc != MS_OK) return rc;
  // norms is [nrhs][2] (sum r^2, sum bhat^2): strided copies into the caller's arrays
  if (rr_out)
    MS_CUDA(g, cudaMemcpy2DAsync(rr_out, sizeof(double), norms, 2 * sizeof(double), sizeof(double), g->nrhs,
                                 cudaMemcpyDeviceToDevice, s));
  if (bb_out)
    MS_CUDA(g, cudaMemcpy2DAsync(bb_out, sizeof(double), norms + 1, 2 * sizeof(double), sizeof(double), g->nrhs,
                                 cudaMemcpyDeviceToDevice, s));
  return MS_OK;
}

// One synchronous outer sweep outside ms_solve's loop: ||bhat|| (the FP32
// scaling; only the points next to the boundary are visited when f is null),
// one launch of the sweep kernel that ms_solve would use for this problem (its
// tuned shape when a solve of the same problem measured one, else the model's
// first choice) reading x^k from x_in and writing x^{k+1} to x_out, and the
// squared residual of x^k summed from the kernel's block partials.
extern "C" int ms_sweep(ms_grid* g, const double* f, const double* bnd, const double* x_in, double* x_out,
                        double* rr_out, const ms_opts* opts, ms_stats* st, void* stream_ptr) {
  if (!g) return MS_ERR_ARG;
  if (!x_in || !x_out) return fail(g, MS_ERR_ARG, "ms_sweep: x_in and x_out must be non-NULL");
  const long long npts = g->npts();
  const size_t xbytes = (size_t)g->nrhs * npts * sizeof(double);
  {
    const char* a = reinterpret_cast<const char*>(x_in);
    const char* b = reinterpret_cast<const char*>(x_out);
    if (a < b + xbytes && b < a + xbytes) return fail(g, MS_ERR_ARG, "ms_sweep: x_in and x_out overlap");
  }
  ms_opts o;
  if (opts) o = *opts;
  else ms_default_opts(&o);
  int rc = check_opts(g, o);
  if (rc != MS_OK) return rc;
  if (o.mode != MS_MODE_SYNC || o.inner_adapt)
    return fail(g, MS_ERR_ARG, "ms_sweep: one synchronous sweep (mode SYNC, inner_adapt 0)");
  cudaGetLastError();
  cudaStream_t stream = (cudaStream_t)stream_ptr;
  const int prec = o.precision == MS_PREC_MIXED ? 1 : 0;
  const size_t esz = prec ? sizeof(float) : sizeof(double);
  long long maxpts = 0;
  std::vector<Task> tasks = build_tasks(g, &maxpts, o.overlap);
  const int ntasks = (int)tasks.size();
  const bool gmres = o.inner_method == 1;
  const int eff_engine = o.variant >= 0 ? 2 : ((o.overlap > 0 || gmres) ? 1 : o.engine);
  std::vector<LaunchShape> all;
  rc = list_shapes(g->tuner, prec, MS_MODE_SYNC, eff_engine, tasks, maxpts, o.cluster, o.threads, o.slots, o.variant,
                   &all);
  if (rc == 0 && gmres) {
    all.erase(std::remove_if(all.begin(), all.end(), [](const LaunchShape& c) { return c.variant != -1; }), all.end());
    if (all.empty()) rc = (int)cudaErrorInvalidConfiguration;
  }
  if (rc != 0) return fail(g, MS_ERR_CUDA, "ms_sweep: no launchable shape (%s)", cudaGetErrorString((cudaError_t)rc));
  LaunchShape shape = all.front();
  {
    const std::vector<long long> sig = signature(prec, MS_MODE_SYNC, eff_engine + 10 * o.inner_method, tasks);
    auto it = g->tuner.best.find(sig);
    const bool requested = o.cluster || o.threads || o.slots || o.variant >= 0;
    if (!requested && it != g->tuner.best.end()) shape = it->second;
  }
  long long padded = maxpts;
  for (const Task& t : tasks) padded = std::max(padded, (long long)t.bz * t.by * 4 * ((t.bx + 3) / 4));
  const long long vec_stride = (padded + 31) / 32 * 32;
  const CtlLayout L = ctl_layout(g->nrhs);
  if (shape.variant < 0) {
    const int nvec = gmres ? o.gmres_restart + 3 : 4;
    MS_CUDA(g, g->scratch.reserve((size_t)shape.slots * nvec * vec_stride * esz));
  }
  MS_CUDA(g, g->tasks.reserve(tasks.size() * sizeof(Task)));
  MS_CUDA(g, g->partial.reserve((size_t)ntasks * sizeof(double)));
  MS_CUDA(g, g->ctl.reserve(L.bytes));
  char* ctlb = g->ctl.as<char>();
  Ctl* ctl = reinterpret_cast<Ctl*>(ctlb);
  double* invb = reinterpret_cast<double*>(ctlb + L.off_invb);
  unsigned long long* inner = reinterpret_cast<unsigned long long*>(ctlb + L.off_inner);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  struct EvGuard {
    cudaEvent_t* a;
    cudaEvent_t* b;
    ~EvGuard() {
      if (*a) cudaEventDestroy(*a);
      if (*b) cudaEventDestroy(*b);
    }
  } evg{&ev0, &ev1};
  if (st) {
    MS_CUDA(g, cudaEventCreate(&ev0));
    MS_CUDA(g, cudaEventCreate(&ev1));
    MS_CUDA(g, cudaEventRecord(ev0, stream));
  }
  MS_CUDA(g, cudaMemcpyAsync(g->tasks.p, tasks.data(), tasks.size() * sizeof(Task), cudaMemcpyHostToDevice, stream));
  MS_CUDA(g, cudaMemsetAsync(ctlb, 0, L.bytes, stream));  // every rhs active, sweep counter k = 0
  // scratch: per-CTA parts of ||bhat||^2, then ||bhat||^2 and the residual shares per rhs
  const int nblk = resid_blocks(g->npts());
  MS_CUDA(g, g->rpart.reserve(((size_t)g->nrhs * nblk + 2 * (size_t)g->nrhs) * sizeof(double)));
  double* bpart = g->rpart.as<double>();
  double* bb_dev = bpart + (size_t)g->nrhs * nblk;
  double* rr_dev = bb_dev + g->nrhs;
  MS_CUDA(g, launch_bhat_sq(g->geo(), f, bnd, bpart, nblk, bb_dev, invb, stream));
  SweepArgs sa;
  sa.g = g->geo();
  sa.f = f;
  sa.bnd = bnd;
  sa.xbuf0 = const_cast<double*>(x_in);  // read only: sweep k = 0 reads buffer 0 and writes buffer 1
  sa.xbuf1 = x_out;
  sa.tasks = g->tasks.as<Task>();
  sa.ntasks = ntasks;
  sa.counter = &ctl->counter;
  sa.rhs_state = reinterpret_cast<int*>(ctlb + L.off_state);
  sa.all_done = &ctl->all_done;
  sa.partial = g->partial.as<double>();
  sa.scratch = g->scratch.p;
  sa.vec_stride = vec_stride;
  sa.inner_rtol = o.inner_rtol;
  sa.inner_maxit = o.inner_maxit;
  sa.outer_maxit = 1;  // k = 0 < 1: a full sweep, not the residual-only one
  sa.k_dev = &ctl->k_dev;
  sa.inner_count = inner;
  sa.inv_bnorm = invb;
  sa.err = &ctl->err;
  sa.inner_rtol_rhs = nullptr;
  sa.inner_method = o.inner_method;
  sa.gmres_restart = o.gmres_restart;
  sa.tr = TraceArgs{nullptr, nullptr, 0};
  sa.sum_polls = o.sum_polls;
  if (shape.variant >= 0) MS_CUDA(g, launch_res_sweep(shape.variant, shape.cluster, shape.slots, shape.smem, sa, stream));
  else if (shape.variant == -2) MS_CUDA(g, launch_strip_sweep(prec, shape.threads, shape.cluster, shape.slots, sa, stream));
  else MS_CUDA(g, launch_sweep(prec, shape.threads, shape.cluster, shape.slots, sa, stream));
  // the residual share of x^k: the sweep's block partials (owned points), in fixed order
  MS_CUDA(g, launch_task_sums(sa.tasks, sa.partial, ntasks, g->nrhs, rr_dev, stream));
  if (rr_out)
    MS_CUDA(g, cudaMemcpyAsync(rr_out, rr_dev, g->nrhs * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  if (!st) return MS_OK;
  MS_CUDA(g, cudaEventRecord(ev1, stream));
  std::vector<double> hn(2 * (size_t)g->nrhs);
  std::vector<unsigned long long> hin(2 * (size_t)g->nrhs);
  int herr = 0;
  for (int r = 0; r < g->nrhs; ++r) {
    MS_CUDA(g, cudaMemcpyAsync(&hn[2 * r], rr_dev + r, sizeof(double), cudaMemcpyDeviceToHost, stream));
    MS_CUDA(g, cudaMemcpyAsync(&hn[2 * r + 1], bb_dev + r, sizeof(double), cudaMemcpyDeviceToHost, stream));
  }
  MS_CUDA(g, cudaMemcpyAsync(hin.data(), inner, hin.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             stream));
  MS_CUDA(g, cudaMemcpyAsync(&herr, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  MS_CUDA(g, cudaStreamSynchronize(stream));
  if (herr & kErrGeometry) return fail(g, MS_ERR_CUDA, "ms_sweep: device error word 0x%x", herr);
  float ms_el = 0.f;
  MS_CUDA(g, cudaEventElapsedTime(&ms_el, ev0, ev1));
  long long box_pts = 0, inner_total = 0, inner_lups = 0;
  for (const Task& t : tasks)
    if (t.rhs == 0) box_pts += (long long)t.bx * t.by * t.bz;
  double relmax = 0.0;
  for (int r = 0; r < g->nrhs; ++r) {
    const double rel = hn[2 * r + 1] > 0.0 ? std::sqrt(hn[2 * r]) / std::sqrt(hn[2 * r + 1]) : std::sqrt(hn[2 * r]);
    relmax = std::max(relmax, rel);
    inner_total += (long long)hin[2 * r];
    inner_lups += (long long)hin[2 * r + 1];
    if (st->per_rhs_outer_its) st->per_rhs_outer_its[r] = 1;
    if (st->per_rhs_rel) st->per_rhs_rel[r] = rel;
  }
  st->status = MS_OK;
  st->outer_its = 1;
  st->inner_its = inner_total;
  st->lups = inner_lups + (long long)g->nrhs * box_pts;
  st->rel_residual = relmax;  // of x_in, against this grid's own ||bhat||
  st->time_ms = ms_el;
  st->launches = 2;
  st->cluster = shape.cluster;
  st->threads = shape.threads;
  st->slots = shape.slots;
  st->sweep_ms = 0.0;
  st->sweep_launches = 0;
  st->engine = shape.variant >= 0 ? 2 : 1;
  st->variant = shape.variant;
  st->inner_rtol_final = o.inner_rtol;
  if (herr & kErrTimeout) {  // a bounded wait of the sweep ran out: its result is not to be used
    st->status = MS_ERR_TIMEOUT;
    return fail(g, MS_ERR_TIMEOUT, "ms_sweep: a bounded device wait ran out (device error word 0x%x)", herr);
  }
  return MS_OK;
}

extern "C" int ms_gcg_solve(ms_grid* g, const double* f, const double* bnd, double* x, const ms_opts* opts,
                            ms_stats* st, void* stream) {
  if (!g) return MS_ERR_ARG;
  if (!x) return fail(g, MS_ERR_ARG, "ms_gcg_solve: x is NULL");
  ms_opts o;
  if (opts) o = *opts;
  else ms_default_opts(&o);
  if (!(o.outer_tol >= 0.0) || o.outer_maxit < 0 || !(o.time_limit_ms >= 0.0))
    return fail(g, MS_ERR_ARG, "ms_gcg_solve: outer_tol, outer_maxit and time_limit_ms must be >= 0");
  cudaGetLastError();  // a stale non-sticky error from unrelated work must not fail this solve
  cudaStream_t s = (cudaStream_t)stream;
  const Geo G = g->geo();
  const int nb = gcg_blocks(G);
  const size_t vec = (size_t)G.nrhs * G.npts * sizeof(double);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t r = off;
    off += (bytes + 255) / 256 * 256;
    return r;
  };
  const size_t o_r = take(vec), o_p = take(vec), o_q = take(vec);
  const size_t o_ctl = off;  // everything after this is zeroed per solve
  const size_t o_rr = take(2 * (size_t)G.nrhs * nb * sizeof(double)), o_pq = take((size_t)G.nrhs * nb * sizeof(double));
  const size_t o_norm = take(2 * (size_t)G.nrhs * sizeof(double)), o_state = take((size_t)G.nrhs * sizeof(int));
  const size_t o_kf = take((size_t)G.nrhs * sizeof(int)), o_k = take(sizeof(int)), o_stop = take(sizeof(int));
  const size_t o_t = take(sizeof(unsigned long long));
  MS_CUDA(g, g->gcg_ws.reserve(off));
  char* w = g->gcg_ws.as<char>();
  MS_CUDA(g, cudaMemsetAsync(w + o_ctl, 0, off - o_ctl, s));  // state = kActive, counters 0
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  struct Ev {
    cudaEvent_t* a;
    cudaEvent_t* b;
    ~Ev() {
      if (*a) cudaEventDestroy(*a);
      if (*b) cudaEventDestroy(*b);
    }
  } evg{&ev0, &ev1};
  MS_CUDA(g, cudaEventCreate(&ev0));
  MS_CUDA(g, cudaEventCreate(&ev1));
  MS_CUDA(g, cudaEventRecord(ev0, s));
  double* norms = reinterpret_cast<double*>(w + o_norm);
  int rc = run_resid(g, f, bnd, x, norms, nullptr, s);  // norms[2s+1] = ||bhat||^2
  if (rc != MS_OK) return rc;
  GcgArgs a;
  a.g = G;
  a.f = f;
  a.bnd = bnd;
  a.x = x;
  a.r = reinterpret_cast<double*>(w + o_r);
  a.p = reinterpret_cast<double*>(w + o_p);
  a.q = reinterpret_cast<double*>(w + o_q);
  a.part_rr = reinterpret_cast<double*>(w + o_rr);
  a.part_pq = reinterpret_cast<double*>(w + o_pq);
  a.nb = nb;
  a.norms = norms;
  a.tol = o.outer_tol;
  a.maxit = o.outer_maxit;
  a.state = reinterpret_cast<int*>(w + o_state);
  a.k_final = reinterpret_cast<int*>(w + o_kf);
  a.k_dev = reinterpret_cast<int*>(w + o_k);
  a.stop_all = reinterpret_cast<int*>(w + o_stop);
  a.t_start = reinterpret_cast<unsigned long long*>(w + o_t);
  a.budget_ns = o.time_limit_ms > 0.0 ? (long long)(o.time_limit_ms * 1.0e6) : 0;
  a.use_cond = 0;
  a.cond = 0;
  MS_CUDA(g, launch_gcg_init(a, s));
  // the iterations: ONE graph launch, a conditional WHILE node over [p, q, x kernels]
  {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t ce = cudaGraphCreate(&graph, 0);
    cudaGraphConditionalHandle cond = 0;
    if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (ce == cudaSuccess) {
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      cudaStream_t cs = nullptr;
      ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (ce == cudaSuccess) {
        GcgArgs ab = a;
        ab.use_cond = 1;
        ab.cond = cond;
        ce = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        const cudaError_t c1 = ce == cudaSuccess ? launch_gcg_iteration(ab, cs) : ce;
        const cudaError_t c2 = ce == cudaSuccess ? cudaStreamEndCapture(cs, &body) : cudaSuccess;
        if (ce == cudaSuccess) ce = c1 != cudaSuccess ? c1 : c2;
        cudaStreamDestroy(cs);
      }
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    MS_CUDA(g, ce);
  }
  // true residual of the returned x
  rc = run_resid(g, f, bnd, x, norms, nullptr, s);
  if (rc != MS_OK) return rc;
  MS_CUDA(g, cudaEventRecord(ev1, s));
  std::vector<int> h_state(G.nrhs), h_kf(G.nrhs);
  std::vector<double> h_norm(2 * (size_t)G.nrhs);
  int h_k = 0;
  MS_CUDA(g, cudaMemcpyAsync(h_state.data(), a.state, G.nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
  MS_CUDA(g, cudaMemcpyAsync(h_kf.data(), a.k_final, G.nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
  MS_CUDA(g, cudaMemcpyAsync(h_norm.data(), norms, h_norm.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  MS_CUDA(g, cudaMemcpyAsync(&h_k, a.k_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  MS_CUDA(g, cudaStreamSynchronize(s));
  float ms_el = 0.f;
  MS_CUDA(g, cudaEventElapsedTime(&ms_el, ev0, ev1));
  int status = MS_OK;
  long long its_total = 0;
  int its_max = 0;
  double relmax = 0.0;
  for (int r = 0; r < G.nrhs; ++r) {
    if (h_state[r] == kStopped) status = MS_ERR_NOT_CONVERGED;  // iteration cap or time budget
    its_total += h_kf[r];
    its_max = std::max(its_max, h_kf[r]);
    const double rel = h_norm[2 * r + 1] > 0.0 ? std::sqrt(h_norm[2 * r]) / std::sqrt(h_norm[2 * r + 1])
                                               : std::sqrt(h_norm[2 * r]);
    relmax = std::max(relmax, rel);
    if (st && st->per_rhs_outer_its) st->per_rhs_outer_its[r] = h_kf[r];
    if (st && st->per_rhs_rel) st->per_rhs_rel[r] = rel;
  }
  if (status == MS_ERR_NOT_CONVERGED && a.budget_ns > 0) {
    int h_stop = 0;
    MS_CUDA(g, cudaMemcpy(&h_stop, a.stop_all, sizeof(int), cudaMemcpyDeviceToHost));
    if (h_stop) status = MS_ERR_TIMEOUT;
  }
  if (st) {
    st->status = status;
    st->outer_its = its_max;
    st->inner_its = its_total;
    st->lups = its_total * G.npts + 3LL * G.nrhs * G.npts;  // iterations + initial residual + two true residuals
    st->rel_residual = relmax;
    st->time_ms = ms_el;
    st->launches = 3 + 3 * (h_k + 1) + 2;
    st->cluster = 1;
    st->threads = 256;
    st->slots = nb;
    st->sweep_ms = 0.0;
    st->sweep_launches = 0;
    st->engine = 0;
    st->variant = -1;
    st->inner_rtol_final = 0.0;
  }
  return status;
}

extern "C" int ms_resident_variant(int v, int* count, int* threads, int* strips, int* planes, int* d_smem,
                                   int* q_regs, int* one_reduction) {
  const int n = ms::res_variant_count();
  if (count) *count = n;
  if (v < 0 || v >= n) return MS_ERR_ARG;
  int nt, kc, zs, ds, qr;
  ms::res_variant_info(v, &nt, &kc, &zs, &ds, &qr);
  if (threads) *threads = nt;
  if (strips) *strips = kc;
  if (planes) *planes = zs;
  if (d_smem) *d_smem = ds;
  if (q_regs) *q_regs = qr == 1 ? 1 : 0;
  if (one_reduction) *one_reduction = qr == 2 ? 1 : 0;
  return MS_OK;
}

extern "C" int ms_destroy(ms_grid* g) {
  if (!g) return MS_OK;
  cudaDeviceSynchronize();
  g->xalt.release();
  g->scratch.release();
  g->tasks.release();
  g->partial.release();
  g->ctl.release();
  g->hist.release();
  g->rpart.release();
  g->host_io.release();
  g->async_ws.release();
  g->flow_ws.release();
  g->gcg_ws.release();
  g->thist.release();
  g->trace_ws.release();
  g->tuner.release();
  delete g;
  return MS_OK;
}

extern "C" const char* ms_last_error(ms_grid* g) {
  if (!g) return g_create_error.c_str();
  return g->err.c_str();
}

// ------------------------------------------------------------------ solve
int solve_async(ms_grid* g, const double* f, const double* bnd, double* x, const ms_opts& o, ms_stats* st,
                cudaStream_t stream, const LaunchShape& shape, const std::vector<Task>& tasks, long long maxpts,
                double* invb_dev, int* rc_out);

static int solve_device(ms_grid* g, const double* f, const double* bnd, double* x, const ms_opts& o, ms_stats* st,
                        cudaStream_t stream) {
  const int prec = o.precision == MS_PREC_MIXED ? 1 : 0;
  const size_t esz = prec ? sizeof(float) : sizeof(double);
  long long maxpts = 0;
  std::vector<Task> tasks = build_tasks(g, &maxpts, o.overlap);
  const int ntasks = (int)tasks.size();
  const long long npts = g->npts();
  const size_t xbytes = (size_t)g->nrhs * npts * sizeof(double);

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  MS_CUDA(g, cudaEventCreate(&ev0));
  MS_CUDA(g, cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};

  // launch shape: an explicit request, a shape measured earlier for this
  // problem, or -- sync mode -- candidates measured on the first sweeps
  std::vector<LaunchShape> all;
  // overlapping blocks run on the streaming engines (the resident layouts keep
  // no owned range); the GMRES inner solver on the scalar streaming engine only
  const bool gmres = o.inner_method == 1;
  const int eff_engine = o.variant >= 0 ? 2 : ((o.overlap > 0 || gmres) ? 1 : o.engine);
  int rc = list_shapes(g->tuner, prec, o.mode, eff_engine, tasks, maxpts, o.cluster, o.threads, o.slots, o.variant,
                       &all);
  if (rc == 0 && gmres) {
    all.erase(std::remove_if(all.begin(), all.end(), [](const LaunchShape& c) { return c.variant != -1; }), all.end());
    if (all.empty()) rc = (int)cudaErrorInvalidConfiguration;
  }
  if (rc != 0) return fail(g, MS_ERR_CUDA, "ms_solve: no launchable shape (%s)", cudaGetErrorString((cudaError_t)rc));
  LaunchShape shape = all.front();
  std::vector<LaunchShape> cands;
  const std::vector<long long> sig = signature(prec, o.mode, eff_engine + 10 * o.inner_method, tasks);
  {
    auto it = g->tuner.best.find(sig);
    const bool requested = o.cluster || o.threads || o.slots || o.variant >= 0;
    if (!requested && it != g->tuner.best.end()) {
      shape = it->second;
    } else if (!requested && o.mode == MS_MODE_SYNC) {
      int nres = 0;
      bool have_streaming = false;
      for (const LaunchShape& c : all) {
        if (c.variant >= 0 && nres < 6) {
          cands.push_back(c);
          ++nres;
        } else if (c.variant < 0 && (!have_streaming || prec == 0)) {
          cands.push_back(c);
          have_streaming = true;
        }
      }
      // sweep 0 (heuristic shape) + kTuneRounds sweeps per candidate must fit in the sweep budget
      if (cands.size() < 2 || (long long)o.outer_maxit < 2 * (long long)(kTuneRounds * cands.size() + 1))
        cands.clear();
    }
  }

  // workspace (vectors sized for the largest block, in the pitch-padded strip layout when larger)
  long long padded = maxpts;
  for (const Task& t : tasks) padded = std::max(padded, (long long)t.bz * t.by * 4 * ((t.bx + 3) / 4));
  const long long vec_stride = (padded + 31) / 32 * 32;
  CtlLayout L = ctl_layout(g->nrhs);
  {
    int streaming_slots = shape.variant < 0 ? shape.slots : 0;  // scalar and vectorised streaming
    for (const LaunchShape& c : cands)
      if (c.variant < 0) streaming_slots = std::max(streaming_slots, c.slots);
    const int nvec = gmres ? o.gmres_restart + 3 : 4;  // CG: r, p0, p1, d; GMRES: r, d, m + 1 basis vectors
    if (streaming_slots > 0) MS_CUDA(g, g->scratch.reserve((size_t)streaming_slots * nvec * vec_stride * esz));
  }
  MS_CUDA(g, g->tasks.reserve(tasks.size() * sizeof(Task)));
  MS_CUDA(g, g->partial.reserve((size_t)ntasks * sizeof(double)));
  MS_CUDA(g, g->ctl.reserve(L.bytes));
  char* ctlb = g->ctl.as<char>();
  Ctl* ctl = reinterpret_cast<Ctl*>(ctlb);
  int* rhs_state = reinterpret_cast<int*>(ctlb + L.off_state);
  int* k_final = reinterpret_cast<int*>(ctlb + L.off_kfinal);
  unsigned long long* inner = reinterpret_cast<unsigned long long*>(ctlb + L.off_inner);
  double* invb = reinterpret_cast<double*>(ctlb + L.off_invb);
  double* norms = reinterpret_cast<double*>(ctlb + L.off_norm);
  AdaptState* adapt = o.inner_adapt ? reinterpret_cast<AdaptState*>(ctlb + L.off_adapt) : nullptr;
  double* rtol_rhs = reinterpret_cast<double*>(ctlb + L.off_rtol);

  MS_CUDA(g, cudaEventRecord(ev0, stream));
  MS_CUDA(g, cudaMemcpyAsync(g->tasks.p, tasks.data(), tasks.size() * sizeof(Task), cudaMemcpyHostToDevice, stream));
  MS_CUDA(g, cudaMemsetAsync(ctlb, 0, L.bytes, stream));
  std::vector<AdaptState> h_adapt;
  std::vector<double> h_rtol;
  if (adapt) {
    AdaptState a0{};
    a0.c = kAdaptStart;
    a0.rs = kAdaptWarmup;
    a0.cur = kAdaptStart;
    h_adapt.assign(g->nrhs, a0);
    h_rtol.assign(g->nrhs, adapt_rung_rtol(kAdaptStart));
    MS_CUDA(g, cudaMemcpyAsync(adapt, h_adapt.data(), h_adapt.size() * sizeof(AdaptState), cudaMemcpyHostToDevice,
                               stream));
    MS_CUDA(g, cudaMemcpyAsync(rtol_rhs, h_rtol.data(), h_rtol.size() * sizeof(double), cudaMemcpyHostToDevice,
                               stream));
  }
  // solve trace: a ring of records in device memory, copied to opts.trace at the end
  g->trace = TraceArgs{nullptr, nullptr, 0};
  if (o.trace && o.trace_cap > 0) {
    MS_CUDA(g, g->trace_ws.reserve(256 + (size_t)o.trace_cap * sizeof(ms_trace_rec)));
    MS_CUDA(g, cudaMemsetAsync(g->trace_ws.p, 0, sizeof(unsigned long long), stream));
    g->trace = TraceArgs{reinterpret_cast<ms_trace_rec*>(g->trace_ws.as<char>() + 256),
                         g->trace_ws.as<unsigned long long>(), o.trace_cap};
  }
  // ||bhat|| per rhs (and the residual of x^0, unused here)
  rc = run_resid(g, f, bnd, x, norms, invb, stream);
  if (rc != MS_OK) return rc;
  int launches = 2;

  int status = MS_OK;
  int outer_max = 0;
  std::vector<int> h_kfinal(g->nrhs, 0), h_state(g->nrhs, 0);
  if (o.mode == MS_MODE_ASYNC) {
    int arc = MS_OK;
    rc = solve_async(g, f, bnd, x, o, st, stream, shape, tasks, maxpts, invb, &arc);
    if (rc != MS_OK) return rc;
    status = arc;
    launches += st ? st->launches : 0;
    if (st) st->launches = 0;
  } else {
    MS_CUDA(g, g->xalt.reserve(xbytes));
    double* hist_dev = nullptr;
    if (o.res_hist) {
      MS_CUDA(g, g->hist.reserve((size_t)g->nrhs * (o.outer_maxit + 1) * sizeof(double)));
      hist_dev = g->hist.as<double>();
    }
    double* thist_dev = nullptr;
    if (o.time_hist) {
      MS_CUDA(g, g->thist.reserve((size_t)(o.outer_maxit + 1) * sizeof(double)));
      thist_dev = g->thist.as<double>();
      MS_CUDA(g, cudaMemsetAsync(thist_dev, 0, (size_t)(o.outer_maxit + 1) * sizeof(double), stream));
    }
    SweepArgs sa;
    sa.g = g->geo();
    sa.f = f;
    sa.bnd = bnd;
    sa.xbuf0 = x;
    sa.xbuf1 = g->xalt.as<double>();
    sa.tasks = g->tasks.as<Task>();
    sa.ntasks = ntasks;
    sa.counter = &ctl->counter;
    sa.rhs_state = rhs_state;
    sa.sum_polls = o.sum_polls;
    sa.all_done = &ctl->all_done;
    sa.partial = g->partial.as<double>();
    sa.scratch = g->scratch.p;
    sa.vec_stride = vec_stride;
    sa.inner_rtol = o.inner_rtol;
    sa.inner_maxit = o.inner_maxit;
    sa.outer_maxit = o.outer_maxit;
    sa.k_dev = &ctl->k_dev;
    sa.inner_count = inner;
    sa.inv_bnorm = invb;
    sa.err = &ctl->err;
    sa.inner_rtol_rhs = adapt ? rtol_rhs : nullptr;
    sa.inner_method = o.inner_method;
    sa.gmres_restart = o.gmres_restart;
    sa.tr = g->trace;
    CheckArgs ca;
    ca.nrhs = g->nrhs;
    ca.ntasks = ntasks;
    ca.tasks = sa.tasks;
    ca.partial = sa.partial;
    ca.inv_bnorm = invb;
    ca.rhs_state = rhs_state;
    ca.k_final = k_final;
    ca.all_done = &ctl->all_done;
    ca.counter = &ctl->counter;
    ca.k_dev = &ctl->k_dev;
    ca.hist = hist_dev;
    ca.thist = thist_dev;
    ca.outer_tol = o.outer_tol;
    ca.outer_maxit = o.outer_maxit;
    ca.time_budget_ns = o.time_limit_ms > 0.0 ? (unsigned long long)(o.time_limit_ms * 1.0e6) : 0ull;
    ca.t_start = &ctl->t_start;
    ca.err = &ctl->err;
    ca.use_cond = 0;
    ca.cond = 0;
    ca.adapt = adapt;
    ca.inner_rtol_rhs = rtol_rhs;
    ca.inner_count = inner;
    ca.npts = (double)g->npts();

    int chunk = o.check_every > 0 ? o.check_every : 4;
    int* h_flags = nullptr;  // all_done, err
    MS_CUDA(g, cudaMallocHost(&h_flags, 4 * sizeof(int)));
    struct HostGuard {
      int* p;
      ~HostGuard() { cudaFreeHost(p); }
    } hg{h_flags};
    // optional per-sweep timing: one event pair per sweep of a chunk
    std::vector<cudaEvent_t> pev;
    struct EvVec {
      std::vector<cudaEvent_t>* v;
      ~EvVec() {
        for (cudaEvent_t e : *v) cudaEventDestroy(e);
      }
    } pevg{&pev};
    double sweep_ms = 0.0;
    int sweeps_timed = 0;
    auto t_start = std::chrono::steady_clock::now();
    long long launched = 0;  // sweeps launched
    if (!cands.empty()) {
      // autotuning: sweep 0 with the model's favourite (x^0 leaves some blocks
      // trivial), then kTuneRounds rounds of one real sweep per candidate,
      // timed with CUDA events; a candidate's time is its fastest sweep (one
      // sweep alone can be distorted, e.g. by the previous candidate's tail)
      const size_t nc = cands.size();
      std::vector<cudaEvent_t> tev(2 * kTuneRounds * nc);
      struct TevGuard {
        std::vector<cudaEvent_t>* v;
        ~TevGuard() {
          for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
        }
      } tevg{&tev};
      for (auto& e : tev) MS_CUDA(g, cudaEventCreate(&e));
      auto sweep_with = [&](const LaunchShape& sh) -> cudaError_t {
        if (sh.variant >= 0) return launch_res_sweep(sh.variant, sh.cluster, sh.slots, sh.smem, sa, stream);
        if (sh.variant == -2) return launch_strip_sweep(prec, sh.threads, sh.cluster, sh.slots, sa, stream);
        return launch_sweep(prec, sh.threads, sh.cluster, sh.slots, sa, stream);
      };
      MS_CUDA(g, sweep_with(cands[0]));
      MS_CUDA(g, launch_check(ca, stream));
      for (size_t j = 0; j < kTuneRounds * nc; ++j) {
        MS_CUDA(g, cudaEventRecord(tev[2 * j], stream));
        MS_CUDA(g, sweep_with(cands[j % nc]));
        MS_CUDA(g, cudaEventRecord(tev[2 * j + 1], stream));
        MS_CUDA(g, launch_check(ca, stream));
      }
      launched += 1 + (long long)(kTuneRounds * nc);
      launches += 2 * (1 + (int)(kTuneRounds * nc));
      MS_CUDA(g, cudaMemcpyAsync(h_state.data(), rhs_state, g->nrhs * sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaMemcpyAsync(h_flags, &ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaMemcpyAsync(h_flags + 1, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaStreamSynchronize(stream));
      if (h_flags[1] & kErrGeometry) return fail(g, MS_ERR_CUDA, "ms_solve: device error word 0x%x", h_flags[1]);
      if (h_flags[1] & kErrTimeout) status = MS_ERR_TIMEOUT;  // the time limit ran out during the tuning sweeps
      float best_t = 1e30f;
      const bool verbose = std::getenv("MS_TUNE_VERBOSE") != nullptr;
      for (size_t i = 0; i < nc; ++i) {
        float t = 1e30f;
        for (size_t rnd = 0; rnd < kTuneRounds; ++rnd) {
          float tr = 0.f;
          MS_CUDA(g, cudaEventElapsedTime(&tr, tev[2 * (rnd * nc + i)], tev[2 * (rnd * nc + i) + 1]));
          t = std::min(t, tr);
        }
        if (verbose)
          std::fprintf(stderr, "ms tune: variant %d cluster %d threads %d slots %d smem %zu est %.3g -> %.3f ms\n",
                       cands[i].variant, cands[i].cluster, cands[i].threads, cands[i].slots, cands[i].smem,
                       cands[i].est, t);
        if (t < best_t) {
          best_t = t;
          shape = cands[i];
        }
      }
      // keep the measurement only if every rhs was still being solved throughout
      bool clean = true;
      for (int r = 0; r < g->nrhs; ++r)
        if (h_state[r] != kActive) clean = false;
      if (clean) g->tuner.best[sig] = shape;
      if (h_flags[0]) chunk = 0;  // finished during tuning
    }
    auto sweep_launch = [&](const LaunchShape& sh, cudaStream_t cs) -> cudaError_t {
      if (sh.variant >= 0) return launch_res_sweep(sh.variant, sh.cluster, sh.slots, sh.smem, sa, cs);
      if (sh.variant == -2) return launch_strip_sweep(prec, sh.threads, sh.cluster, sh.slots, sa, cs);
      return launch_sweep(prec, sh.threads, sh.cluster, sh.slots, sa, cs);
    };
    // Persistent dataflow launch or per-sweep graph.  In auto mode the
    // persistent launch is a candidate where the per-sweep schedule would idle
    // clusters in its last round (tasks not a multiple of the clusters in
    // flight); which of the two is faster depends on the variant (the
    // persistent kernel holds more state), so the first solve of a problem
    // runs the persistent launch, the next one the graph, each timed, and
    // later solves take the faster.
    const double rounds = (double)ntasks / std::max(1, shape.slots);
    const double tail_waste = 1.0 - rounds / std::ceil(rounds);
    std::vector<long long> mode_key = sig;
    mode_key.insert(mode_key.end(), {shape.variant, shape.cluster, shape.threads, shape.slots});
    Tuner::ModeMs* mm = nullptr;
    bool use_flow = o.persistent == 2;
    // the persistent kernel's in-kernel stop decision has no controller, and its
    // six-neighbour dependencies do not cover the diagonal neighbours an overlapping box reads
    if (o.inner_adapt || o.overlap > 0) use_flow = false;
    else if (o.persistent == 1 && shape.variant >= 0 && tail_waste > 0.05) {
      mm = &g->tuner.mode_ms[mode_key];
      use_flow = mm->flow < 0.0 || (mm->sweep >= 0.0 && mm->flow < mm->sweep);
    }
    struct PhaseEvGuard {
      cudaEvent_t a = nullptr, b = nullptr;
      ~PhaseEvGuard() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
      }
    } pguard;  // timing of the main phase (auto mode choice)
    if (mm) {
      MS_CUDA(g, cudaEventCreate(&pguard.a));
      MS_CUDA(g, cudaEventCreate(&pguard.b));
    }
    const cudaEvent_t pa = pguard.a, pb = pguard.b;
    auto record_phase = [&](double Tuner::ModeMs::*field, long long sweeps) -> cudaError_t {
      if (!mm || sweeps < 10 || status != MS_OK) return cudaSuccess;
      float t = 0.f;
      cudaError_t e = cudaEventElapsedTime(&t, pa, pb);
      if (e == cudaSuccess) (*mm).*field = (double)t / (double)sweeps;
      return e;
    };
    if (chunk != 0 && shape.variant >= 0 && use_flow && !o.profile && launched <= (long long)o.outer_maxit) {
      // The rest of the solve is ONE persistent launch (dataflow between sweeps).
      MS_CUDA(g, cudaMemcpyAsync(&h_flags[2], &ctl->k_dev, sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaStreamSynchronize(stream));
      const int k0 = h_flags[2];
      const int nblocks = g->px * g->py * g->pz;
      std::vector<int> task_of((size_t)g->nrhs * nblocks, -1);
      for (int i = 0; i < ntasks; ++i) task_of[(size_t)tasks[i].rhs * nblocks + tasks[i].block] = i;
      const size_t nres = (size_t)std::max(1, o.outer_maxit + 2 - k0);
      size_t off = 0;
      auto take = [&](size_t bytes) {
        const size_t r = off;
        off += (bytes + 255) / 256 * 256;
        return r;
      };
      const size_t o_ticket = take(sizeof(unsigned long long)), o_dec = take(sizeof(int));
      const size_t o_done = take((size_t)ntasks * sizeof(int)), o_res = take(nres * sizeof(int));
      const size_t o_tof = take(task_of.size() * sizeof(int));
      MS_CUDA(g, g->flow_ws.reserve(off));
      char* fw = g->flow_ws.as<char>();
      MS_CUDA(g, cudaMemsetAsync(fw, 0, o_tof, stream));
      MS_CUDA(g, cudaMemsetAsync(fw + o_dec, 0xFF, sizeof(int), stream));  // decided_rel = -1
      MS_CUDA(g, cudaMemcpyAsync(fw + o_tof, task_of.data(), task_of.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 stream));
      FlowArgs fa;
      fa.s = sa;
      fa.c = ca;
      fa.k0 = k0;
      fa.px = g->px;
      fa.py = g->py;
      fa.pz = g->pz;
      fa.nblocks = nblocks;
      fa.task_of = reinterpret_cast<const int*>(fw + o_tof);
      fa.ticket = reinterpret_cast<unsigned long long*>(fw + o_ticket);
      fa.res_cnt = reinterpret_cast<int*>(fw + o_res);
      fa.done_rel = reinterpret_cast<int*>(fw + o_done);
      fa.decided_rel = reinterpret_cast<int*>(fw + o_dec);
      fa.spin_limit = o.wait_polls > 0 ? (long long)o.wait_polls : 1LL << 24;
      fa.slow_block = o.slow_block;
      fa.slow_ns = o.slow_ns;
      int occ = 0;
      MS_CUDA(g, res_flow_max_clusters(shape.variant, shape.cluster, shape.smem, &occ));
      const int fslots = std::max(1, std::min(occ, ntasks));
      if (pa) MS_CUDA(g, cudaEventRecord(pa, stream));
      MS_CUDA(g, launch_res_flow(shape.variant, shape.cluster, fslots, shape.smem, fa, stream));
      if (pb) MS_CUDA(g, cudaEventRecord(pb, stream));
      MS_CUDA(g, cudaMemcpyAsync(h_flags, &ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaMemcpyAsync(h_flags + 1, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaMemcpyAsync(h_flags + 2, &ctl->k_dev, sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaStreamSynchronize(stream));
      launches += 1;
      launched += h_flags[2] - k0;
      if (h_flags[1] & kErrGeometry) return fail(g, MS_ERR_CUDA, "ms_solve: device error word 0x%x", h_flags[1]);
      if (h_flags[1] & kErrTimeout) status = MS_ERR_TIMEOUT;
      MS_CUDA(g, record_phase(&Tuner::ModeMs::flow, h_flags[2] - k0));
      chunk = 0;
    }
    if (chunk != 0 && o.use_graph && !o.profile && launched <= (long long)o.outer_maxit) {
      // The rest of the solve is ONE graph launch: a WHILE node whose body is
      // [sweep, check]; the check kernel clears the condition on the device
      // once every rhs has stopped (converged, outer_maxit, or time budget).
      int k_before = 0;
      MS_CUDA(g, cudaMemcpyAsync(&h_flags[2], &ctl->k_dev, sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaStreamSynchronize(stream));
      k_before = h_flags[2];
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      cudaError_t ce = cudaGraphCreate(&graph, 0);
      cudaGraphConditionalHandle cond = 0;
      if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
      if (ce == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaStream_t cs = nullptr;
        ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (ce == cudaSuccess) {
          CheckArgs cb = ca;
          cb.use_cond = 1;
          cb.cond = cond;
          ce = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
          cudaError_t c1 = ce == cudaSuccess ? sweep_launch(shape, cs) : ce;
          cudaError_t c2 = c1 == cudaSuccess ? launch_check(cb, cs) : c1;
          cudaError_t c3 = ce == cudaSuccess ? cudaStreamEndCapture(cs, &body) : cudaSuccess;
          if (ce == cudaSuccess) ce = c2 != cudaSuccess ? c2 : c3;
          cudaStreamDestroy(cs);
        }
      }
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
      if (ce == cudaSuccess && pa) ce = cudaEventRecord(pa, stream);
      if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, stream);
      if (ce == cudaSuccess && pb) ce = cudaEventRecord(pb, stream);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_flags, &ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, stream);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_flags + 1, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, stream);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_flags + 2, &ctl->k_dev, sizeof(int), cudaMemcpyDeviceToHost, stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      MS_CUDA(g, ce);
      launches += 2 * (h_flags[2] - k_before);
      launched += h_flags[2] - k_before;
      if (h_flags[1] & kErrGeometry) return fail(g, MS_ERR_CUDA, "ms_solve: device error word 0x%x", h_flags[1]);
      if (h_flags[1] & kErrTimeout) status = MS_ERR_TIMEOUT;
      MS_CUDA(g, record_phase(&Tuner::ModeMs::sweep, h_flags[2] - k_before));
      chunk = 0;
    }
    // plain launches (graphs disabled, or per-sweep event timing requested)
    for (;;) {
      if (chunk == 0) break;
      const long long remaining = (long long)o.outer_maxit + 1 - launched;
      if (remaining <= 0) break;
      const int n = (int)std::min<long long>(chunk, remaining);
      if (o.profile) {
        while ((int)pev.size() < 2 * n) {
          cudaEvent_t e;
          MS_CUDA(g, cudaEventCreate(&e));
          pev.push_back(e);
        }
      }
      for (int i = 0; i < n; ++i) {
        if (o.profile) MS_CUDA(g, cudaEventRecord(pev[2 * i], stream));
        MS_CUDA(g, sweep_launch(shape, stream));
        if (o.profile) MS_CUDA(g, cudaEventRecord(pev[2 * i + 1], stream));
        MS_CUDA(g, launch_check(ca, stream));
      }
      launched += n;
      launches += 2 * n;
      MS_CUDA(g, cudaMemcpyAsync(h_flags, &ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaMemcpyAsync(h_flags + 1, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
      MS_CUDA(g, cudaStreamSynchronize(stream));
      if (h_flags[1] & kErrGeometry) return fail(g, MS_ERR_CUDA, "ms_solve: device error word 0x%x", h_flags[1]);
      if (o.profile) {
        for (int i = 0; i < n; ++i) {
          float t = 0.f;
          MS_CUDA(g, cudaEventElapsedTime(&t, pev[2 * i], pev[2 * i + 1]));
          sweep_ms += t;
          sweeps_timed += 1;
        }
      }
      if (h_flags[1] & kErrTimeout) {
        status = MS_ERR_TIMEOUT;
        break;
      }
      if (h_flags[0]) break;
      if (o.time_limit_ms > 0.0) {
        double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        if (el > o.time_limit_ms) {
          status = MS_ERR_TIMEOUT;
          break;
        }
      }
      if (chunk < 16 && o.check_every == 0) chunk *= 2;
    }
    MS_CUDA(g, cudaMemcpyAsync(h_kfinal.data(), k_final, g->nrhs * sizeof(int), cudaMemcpyDeviceToHost, stream));
    MS_CUDA(g, cudaMemcpyAsync(h_state.data(), rhs_state, g->nrhs * sizeof(int), cudaMemcpyDeviceToHost, stream));
    MS_CUDA(g, cudaStreamSynchronize(stream));
    if (status == MS_ERR_TIMEOUT) {
      // stopped mid-solve: the latest complete iterate is x^k, k = sweeps launched (<= outer_maxit)
      int kk = 0;
      MS_CUDA(g, cudaMemcpy(&kk, &ctl->k_dev, sizeof(int), cudaMemcpyDeviceToHost));
      for (int r = 0; r < g->nrhs; ++r)
        if (h_state[r] == kActive) h_kfinal[r] = kk;
    }
    // move odd-k results into the caller's buffer
    for (int r = 0; r < g->nrhs; ++r) {
      if (h_kfinal[r] & 1)
        MS_CUDA(g, cudaMemcpyAsync(x + (size_t)r * npts, g->xalt.as<double>() + (size_t)r * npts,
                                   npts * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      outer_max = std::max(outer_max, h_kfinal[r]);
      if (h_state[r] == kStopped && status == MS_OK) status = MS_ERR_NOT_CONVERGED;
    }
    if (st) {
      st->sweep_ms = sweep_ms;
      st->sweep_launches = sweeps_timed;
    }
    if (o.res_hist) {
      MS_CUDA(g, cudaMemcpyAsync(o.res_hist, hist_dev, (size_t)g->nrhs * (o.outer_maxit + 1) * sizeof(double),
                                 cudaMemcpyDeviceToHost, stream));
    }
    if (o.time_hist) {
      MS_CUDA(g, cudaMemcpyAsync(o.time_hist, thist_dev, (size_t)(o.outer_maxit + 1) * sizeof(double),
                                 cudaMemcpyDeviceToHost, stream));
    }
  }
  MS_CUDA(g, cudaEventRecord(ev1, stream));
  // final true residual
  rc = run_resid(g, f, bnd, x, norms, nullptr, stream);
  if (rc != MS_OK) return rc;
  launches += 2;
  std::vector<double> hn(2 * (size_t)g->nrhs);
  std::vector<unsigned long long> hin(2 * (size_t)g->nrhs);
  MS_CUDA(g, cudaMemcpyAsync(hn.data(), norms, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  MS_CUDA(g, cudaMemcpyAsync(hin.data(), inner, hin.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             stream));
  MS_CUDA(g, cudaStreamSynchronize(stream));
  MS_CUDA(g, cudaGetLastError());
  long long trace_count = 0;
  if (g->trace.rec) {
    // the ring in ticket order: the oldest record sits at count % cap once it wrapped
    unsigned long long head = 0;
    MS_CUDA(g, cudaMemcpy(&head, g->trace.head, sizeof head, cudaMemcpyDeviceToHost));
    const unsigned long long cap = (unsigned long long)o.trace_cap;
    const unsigned long long n = std::min(head, cap), first = head > cap ? head % cap : 0;
    const size_t rs = sizeof(ms_trace_rec);
    if (n > 0) {
      MS_CUDA(g, cudaMemcpy(o.trace, g->trace.rec + first, (size_t)(n - first) * rs, cudaMemcpyDeviceToHost));
      if (first > 0) MS_CUDA(g, cudaMemcpy(o.trace + (n - first), g->trace.rec, (size_t)first * rs, cudaMemcpyDeviceToHost));
    }
    trace_count = (long long)head;
    g->trace = TraceArgs{nullptr, nullptr, 0};
  }
  if (st) {
    st->trace_count = trace_count;
    float ms_el = 0.f;
    cudaEventElapsedTime(&ms_el, ev0, ev1);
    double relmax = 0.0;
    long long inner_total = 0, inner_lups = 0;
    for (int r = 0; r < g->nrhs; ++r) {
      const double rel = hn[2 * r + 1] > 0.0 ? std::sqrt(hn[2 * r]) / std::sqrt(hn[2 * r + 1]) : std::sqrt(hn[2 * r]);
      relmax = std::max(relmax, rel);
      inner_total += (long long)hin[2 * r];
      inner_lups += (long long)hin[2 * r + 1];
      if (st->per_rhs_rel) st->per_rhs_rel[r] = rel;
      if (o.mode == MS_MODE_SYNC && st->per_rhs_outer_its) st->per_rhs_outer_its[r] = h_kfinal[r];
    }
    // residual passes: sync mode forms one per sweep k = 0..K (the last one
    // decides the stop), async mode one per block visit (st->lups on entry)
    long long resid_lups = 0;
    if (o.mode == MS_MODE_SYNC) {
      long long box_pts = 0;  // residual points per rhs and sweep (the boxes, overlap included)
      for (const Task& t : tasks)
        if (t.rhs == 0) box_pts += (long long)t.bx * t.by * t.bz;
      for (int r = 0; r < g->nrhs; ++r) resid_lups += ((long long)h_kfinal[r] + 1) * box_pts;
    } else {
      resid_lups = st->lups;
    }
    st->status = status;
    if (o.mode == MS_MODE_SYNC) st->outer_its = outer_max;
    st->inner_its = inner_total;
    st->lups = resid_lups + inner_lups;
    st->rel_residual = relmax;
    st->time_ms = ms_el;
    st->launches = launches;
    st->cluster = shape.cluster;
    st->threads = shape.threads;
    st->slots = shape.slots;
    st->engine = shape.variant >= 0 ? 2 : 1;
    st->variant = shape.variant;
    st->inner_rtol_final = o.inner_rtol;
    if (adapt) {
      std::vector<double> hr(g->nrhs);
      MS_CUDA(g, cudaMemcpy(hr.data(), rtol_rhs, hr.size() * sizeof(double), cudaMemcpyDeviceToHost));
      st->inner_rtol_final = *std::max_element(hr.begin(), hr.end());
    }
  }
  return status;
}

// ------------------------------------------------------------------ async solve
// One persistent launch runs until the stale estimate says every rhs is below
// tol (or caps are hit); the host then checks the true residual and, for any
// rhs still above tol, re-arms it and relaunches from the current state.
int solve_async(ms_grid* g, const double* f, const double* bnd, double* x, const ms_opts& o, ms_stats* st,
                cudaStream_t stream, const LaunchShape& shape, const std::vector<Task>& tasks, long long maxpts,
                double* invb_dev, int* rc_out) {
  const int prec = o.precision == MS_PREC_MIXED ? 1 : 0;
  const int ntasks = (int)tasks.size();
  const int nblocks = g->px * g->py * g->pz;
  long long face_stride = 0;
  for (const Task& t : tasks)
    face_stride = std::max({face_stride, (long long)t.bz * t.by, (long long)t.bz * t.bx, (long long)t.by * t.bx});
  face_stride = (face_stride + 31) / 32 * 32;
  std::vector<int> task_of((size_t)g->nrhs * nblocks, -1);
  for (int i = 0; i < ntasks; ++i) task_of[(size_t)tasks[i].rhs * nblocks + tasks[i].block] = i;

  // workspace layout (256-byte aligned pieces)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o2 = off;
    off += (bytes + 255) / 256 * 256;
    return o2;
  };
  const size_t o_taskof = take(task_of.size() * sizeof(int));
  const size_t o_faces = take((size_t)ntasks * 12 * face_stride * sizeof(double));
  const size_t o_halo = take((size_t)ntasks * 12 * face_stride * sizeof(double));
  const size_t o_seq = take((size_t)ntasks * 12 * sizeof(unsigned));
  const size_t o_ver = take((size_t)ntasks * 6 * sizeof(unsigned));
  const size_t o_hcur = take((size_t)ntasks * 6 * sizeof(int));
  const size_t o_hver = take((size_t)ntasks * 6 * sizeof(unsigned));
  const size_t o_part = take((size_t)ntasks * sizeof(double));
  const size_t o_sweeps = take((size_t)ntasks * sizeof(int));
  const size_t o_rstop = take((size_t)g->nrhs * sizeof(int));
  const size_t o_flags = take(4 * sizeof(int));
  MS_CUDA(g, g->async_ws.reserve(off));
  char* w = g->async_ws.as<char>();
  MS_CUDA(g, cudaMemsetAsync(w + o_seq, 0, o_part - o_seq, stream));  // seq, ver, hcur, hver
  MS_CUDA(g, cudaMemsetAsync(w + o_rstop, 0, off - o_rstop, stream));
  MS_CUDA(g, cudaMemcpyAsync(w + o_taskof, task_of.data(), task_of.size() * sizeof(int), cudaMemcpyHostToDevice,
                             stream));
  CtlLayout L = ctl_layout(g->nrhs);
  char* ctlb = g->ctl.as<char>();
  Ctl* ctl = reinterpret_cast<Ctl*>(ctlb);
  unsigned long long* inner = reinterpret_cast<unsigned long long*>(ctlb + L.off_inner);

  AsyncArgs a;
  a.sum_polls = o.sum_polls;
  a.g = g->geo();
  a.f = f;
  a.bnd = bnd;
  a.x = x;
  a.tasks = g->tasks.as<Task>();
  a.ntasks = ntasks;
  a.px = g->px;
  a.py = g->py;
  a.pz = g->pz;
  a.nblocks = nblocks;
  a.task_of = reinterpret_cast<const int*>(w + o_taskof);
  a.face_stride = face_stride;
  a.faces = reinterpret_cast<double*>(w + o_faces);
  a.face_seq = reinterpret_cast<unsigned*>(w + o_seq);
  a.face_ver = reinterpret_cast<unsigned*>(w + o_ver);
  a.halo = reinterpret_cast<double*>(w + o_halo);
  a.halo_cur = reinterpret_cast<int*>(w + o_hcur);
  a.halo_ver = reinterpret_cast<unsigned*>(w + o_hver);
  a.partial = reinterpret_cast<double*>(w + o_part);
  a.sweeps = reinterpret_cast<int*>(w + o_sweeps);
  a.inv_bnorm = invb_dev;
  a.rhs_stop = reinterpret_cast<int*>(w + o_rstop);
  a.stop = reinterpret_cast<int*>(w + o_flags);
  a.scratch = g->scratch.p;
  a.vec_stride = (maxpts + 31) / 32 * 32;
  a.inner_rtol = o.inner_rtol;
  a.inner_maxit = o.inner_maxit;
  a.outer_maxit = o.outer_maxit;
  a.outer_tol = o.outer_tol;
  a.slow_block = o.slow_block;
  a.slow_ns = o.slow_ns;
  a.inner_count = inner;
  a.time_budget_ns = o.time_limit_ms > 0.0 ? (unsigned long long)(o.time_limit_ms * 1.0e6) : 0ull;
  a.slice_ns = 2000000000ull;  // no single launch runs longer than ~2 s
  a.err = &ctl->err;
  a.tr = g->trace;
  MS_CUDA(g, launch_async_init(a, stream));

  CtlLayout L2 = L;
  double* norms = reinterpret_cast<double*>(ctlb + L2.off_norm);
  std::vector<double> hn(2 * (size_t)g->nrhs);
  std::vector<int> rstop(g->nrhs), sweeps(ntasks);
  int launches = 1;
  int status = MS_ERR_NOT_CONVERGED;
  auto t_start = std::chrono::steady_clock::now();
  for (int rel = 0; rel < 100000; ++rel) {
    MS_CUDA(g, shape.variant >= 0 ? launch_res_async(shape.variant, shape.cluster, shape.slots, shape.smem, a, stream)
                                  : launch_async(prec, shape.threads, shape.cluster, shape.slots, a, stream));
    launches += 1;
    int rc = run_resid(g, f, bnd, x, norms, nullptr, stream);
    if (rc != MS_OK) return rc;
    launches += 2;
    int herr = 0;
    MS_CUDA(g, cudaMemcpyAsync(hn.data(), norms, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
    MS_CUDA(g, cudaMemcpyAsync(sweeps.data(), a.sweeps, sweeps.size() * sizeof(int), cudaMemcpyDeviceToHost, stream));
    MS_CUDA(g, cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    MS_CUDA(g, cudaStreamSynchronize(stream));
    if (herr & kErrGeometry) return fail(g, MS_ERR_CUDA, "ms_solve: device error word 0x%x", herr);
    bool all_ok = true;
    for (int r = 0; r < g->nrhs; ++r) {
      const double relr = hn[2 * r + 1] > 0.0 ? std::sqrt(hn[2 * r]) / std::sqrt(hn[2 * r + 1]) : std::sqrt(hn[2 * r]);
      rstop[r] = relr < o.outer_tol ? 1 : 0;
      if (!rstop[r]) all_ok = false;
    }
    if (all_ok) {
      status = MS_OK;
      break;
    }
    if (herr & kErrTimeout) {
      status = MS_ERR_TIMEOUT;
      break;
    }
    int min_sweeps = o.outer_maxit;
    for (int i = 0; i < ntasks; ++i)
      if (!rstop[tasks[i].rhs]) min_sweeps = std::min(min_sweeps, sweeps[i]);
    if (min_sweeps >= o.outer_maxit) {
      status = MS_ERR_NOT_CONVERGED;
      break;
    }
    if (o.time_limit_ms > 0.0) {
      double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
      if (el > o.time_limit_ms) {
        status = MS_ERR_TIMEOUT;
        break;
      }
      a.time_budget_ns = (unsigned long long)((o.time_limit_ms - el) * 1.0e6) + 1ull;
    }
    // re-arm the rhs whose true residual is still above tol
    MS_CUDA(g, cudaMemcpyAsync(a.rhs_stop, rstop.data(), rstop.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
    MS_CUDA(g, cudaMemsetAsync(a.stop, 0, sizeof(int), stream));
    MS_CUDA(g, launch_async_rearm(a, stream));
    launches += 1;
  }
  *rc_out = status;
  if (st) {
    int mx = 0;
    std::vector<int> per(g->nrhs, 0);
    for (int i = 0; i < ntasks; ++i) {
      mx = std::max(mx, sweeps[i]);
      per[tasks[i].rhs] = std::max(per[tasks[i].rhs], sweeps[i]);
    }
    st->outer_its = mx;
    if (st->per_rhs_outer_its)
      for (int r = 0; r < g->nrhs; ++r) st->per_rhs_outer_its[r] = per[r];
    long long lups = 0;
    for (int i = 0; i < ntasks; ++i) lups += (long long)sweeps[i] * tasks[i].bx * tasks[i].by * tasks[i].bz;
    st->lups = lups;  // residual passes; inner lattice updates are added by the caller
    st->launches = launches;
  }
  return MS_OK;
}
