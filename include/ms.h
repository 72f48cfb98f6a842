/*
 * ms.h -- C ABI of libms: two-stage multisplitting (outer block Jacobi,
 * inner conjugate gradients) for the 3D Laplace 7-point stencil on one
 * NVIDIA GB300 GPU (sm_103a).
 *
 * Method: Brown, Bull and Bethune, "A highly scalable approach to solving
 * linear systems using two-stage multisplitting".
 *   - model problem, section 2.1: Laplace's equation on a box, 7-point
 *     stencil, Dirichlet boundary; A = 6 I - adjacency (the section 2.1
 *     Jacobi listing averages the six neighbours with weight 1/6);
 *   - stop rule, section 2.1: ||A x - b||_2 < tol on the global residual,
 *     here relative to ||b||_2;
 *   - outer stage, section 3: block Jacobi
 *     X_i = A_ii^{-1} (B_i - sum_{j != i} A_ij X_j), right-hand side
 *     assembled from neighbour halos only;
 *   - inner stage, sections 2.2 and 3: a Krylov solve (CG) of each block
 *     system, independent per block;
 *   - synchronous or asynchronous halo exchange, sections 2.1 and 3 (the
 *     asynchronous mode uses the latest complete neighbour data and a
 *     possibly stale global residual, Listing 1);
 *   - global residual from block partial sums, section 3.
 *
 * Conventions shared by every call:
 *   - interior grid nx*ny*nz per right-hand side (rhs), point (i,j,k) with
 *     0 <= i < nx stored x-fastest; a field with nrhs right-hand sides is a
 *     C-contiguous array [nrhs][nz][ny][nx] of double;
 *   - Dirichlet data per rhs is packed as the six faces
 *     x-(nz*ny), x+(nz*ny), y-(nz*nx), y+(nz*nx), z-(ny*nx), z+(ny*nx), each
 *     row-major in the order written (edges and corners are never used by a
 *     7-point stencil and are not stored); a boundary array is
 *     [nrhs][ms_boundary_size(nx,ny,nz)] doubles;
 *   - unless a function says otherwise, array arguments are DEVICE pointers
 *     on the current CUDA device, owned by the caller, never retained after
 *     the call returns; `stream` is a cudaStream_t (NULL = legacy default
 *     stream) on which all work of the call is ordered;
 *   - functions return an ms_status; nothing throws or aborts across the ABI.
 *     After a failure, ms_last_error(grid) (or ms_last_error(NULL) for a
 *     failed ms_create_grid) describes it.  A grid handle must not be used
 *     from two host threads at once.
 */
#ifndef MS_H
#define MS_H

#if defined(__GNUC__)
#define MS_API __attribute__((visibility("default")))
#else
#define MS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ms_grid ms_grid;

typedef enum {
  MS_OK = 0,
  MS_ERR_ARG = 1,            /* invalid argument; nothing was launched */
  MS_ERR_CUDA = 2,           /* a CUDA call failed (message has the CUDA error) */
  MS_ERR_OOM = 3,            /* device workspace could not be allocated */
  MS_ERR_NOT_CONVERGED = 4,  /* outer_maxit sweeps done, residual still >= outer_tol */
  MS_ERR_TIMEOUT = 5         /* time_limit_ms reached, or a bounded device wait ran out */
} ms_status;

typedef enum { MS_MODE_SYNC = 0, MS_MODE_ASYNC = 1 } ms_mode;

/* FP64: inner CG vectors and arithmetic in double.
 * MIXED: inner CG vectors and arithmetic in float; the outer residual
 * b - A x, the global norm, the solution accumulation and the halo values
 * stay double (two-stage iterative refinement). */
typedef enum { MS_PREC_FP64 = 0, MS_PREC_MIXED = 1 } ms_precision;

/* One record of the solve trace (opts.trace): one block solve of one sweep.
 * The paper's observable is the residual against time (sections 3.2 and 4);
 * the trace gives it per block, which is what separates the synchronous and
 * asynchronous modes (in the latter every block runs its own sweep count). */
typedef struct {
  int sweep;               /* sync: outer sweep k (the block solve that forms x^{k+1});
                              async: the block's own sweep count before this visit */
  int block;               /* block id bx + px*(by + py*bz) */
  int rhs;                 /* right-hand side */
  int inner_its;           /* inner iterations of this block solve */
  double block_rr;         /* ||r_i||^2 of the block residual this solve started from (FP64) */
  unsigned long long t_ns; /* device clock (%globaltimer, ns) when the block solve ended */
} ms_trace_rec;

typedef struct {
  int mode;              /* ms_mode, default MS_MODE_SYNC */
  int precision;         /* ms_precision, default MS_PREC_MIXED */
  double inner_rtol;     /* inner CG stop: ||r_m|| <= inner_rtol ||r_0||, default 1e-6 */
  int inner_maxit;       /* inner CG iteration cap per block and sweep, default 50 */
  double outer_tol;      /* stop when ||b - A x|| / ||b|| < outer_tol, default 1e-8 */
  int outer_maxit;       /* outer sweep cap (async: per block), default 100000 */
  double time_limit_ms;  /* host wall-clock cap for the solve, 0 = none */
  int cluster;           /* CTAs cooperating on one block (thread-block cluster), 0 = tuned */
  int threads;           /* threads per CTA (128, 256, 512 or 1024), 0 = tuned */
  int slots;             /* blocks in flight at once (clusters launched), 0 = tuned */
  int check_every;       /* sync mode: sweeps between host convergence polls, 0 = auto */
  int use_graph;         /* sync mode: replay sweeps from a captured CUDA graph (default 1) */
  int slow_block;        /* resilience test (asynchronous mode and the persistent synchronous launch):
                            this block id sleeps slow_ns per visit; -1 = none */
  int slow_ns;           /*   bounded __nanosleep budget per visit of slow_block */
  double* res_hist;      /* HOST, optional: [nrhs][outer_maxit+1] relative residual per sweep
                            (sync mode; entries after each rhs stops are left untouched) */
  int profile;           /* sync mode: time every sweep kernel with CUDA events (stats.sweep_ms) */
  int persistent;        /* sync mode, resident engine: 2 = all sweeps in one persistent launch, a
                            task starts as soon as its neighbours finished the previous sweep and
                            that sweep's stop decision is made; 0 = one launch per sweep;
                            1 (default) = persistent when more than 5% of the per-sweep schedule's
                            last round would idle */
  int engine;            /* inner-CG engine: 0 auto, 1 streaming (CG vectors in a global scratch slot
                            per cluster, any block size, FP32 or FP64), 2 resident (CG vectors in
                            registers and shared memory of the cluster; MIXED + SYNC, blocks that fit) */
  int variant;           /* resident engine: -1 (default) = chosen by the autotuner; v >= 0 = row v of
                            the variant table (ms_resident_variant), for tests and profiling */
  int inner_adapt;       /* sync mode: 1 = choose the inner tolerance at run time (default 0 = use
                            inner_rtol).  Runtime adaptation of the inner solve, the paper's closing
                            suggestion (sections 3.2 and 5): after every sweep a per-rhs controller
                            charges the sweep's decrease of log(residual) to the relative inner
                            tolerance it ran with, against its work (inner lattice updates plus the
                            residual and update), tries the neighbouring tolerances of a ladder
                            (0.8 ... 1e-3) in rounds of 8 sweeps each (the first 2 of a window not
                            charged; at an end of the ladder the rung 4 steps inward instead of the
                            missing neighbour; each rung's charges kept across rounds, halved per
                            round) and keeps the most efficient; inner_maxit still caps every inner
                            solve.  Deterministic (no clocks). */
  int overlap;           /* sync mode: overlapping blocks (section 3.2), o >= 0 points per face
                            (default 0).  Block i solves on its box extended by o points on every
                            face (clipped to the grid) with zero Dirichlet data outside the box;
                            x^{k+1} takes block i's result on the points block i owns (a
                            multisplitting with weight 1 on owned points, 0 on overlapped ones);
                            the global residual counts every point once.  Runs on the streaming
                            engine (engine 0 or 1). */
  int inner_method;      /* sync mode: 0 (default) = CG; 1 = restarted GMRES(gmres_restart), the inner
                            method of the paper's own runs (section 3.2), classical Gram-Schmidt
                            Arnoldi; inner_rtol tests its residual estimate, inner_maxit caps its
                            Arnoldi steps.  Runs on the scalar streaming engine (engine 0 or 1). */
  int gmres_restart;     /* GMRES basis vectors per cycle, 1..50 (default 10) */
  double* time_hist;     /* HOST, optional (sync mode): [outer_maxit+1] device time in ms, measured from
                            the first stop test, at which the stop test of x^k ran -- with res_hist the
                            residual-versus-time curve the paper plots */
  int wait_polls;        /* persistent synchronous launch: polls a cluster may spend, summed over the
                            launch, in its bounded waits for a neighbour's progress flag or a stop
                            decision; when they run out the solve ends with MS_ERR_TIMEOUT and x holds
                            the last complete iterate.  0 (default) = 2^24 polls (backing off to
                            ~1 us each) */
  int trace_cap;         /* records the trace ring holds (0 = no trace) */
  ms_trace_rec* trace;   /* HOST, optional [trace_cap]: per block solve records, written by the kernels
                            into a device ring and copied here after the solve in the order they were
                            taken (when more than trace_cap were taken, the last trace_cap) */
  int sum_polls;         /* resident engine: polls a CTA may spend in one cluster-wide sum that has no
                            cluster barrier (each CTA's total arrives as a tagged word) before it gives
                            up; the solve then ends with MS_ERR_TIMEOUT (ms_sweep: with stats).
                            0 (default) = 2^22 polls, far beyond any CG step; small values exist to
                            test that bounded wait */
} ms_opts;

typedef struct {
  int status;            /* ms_status of the solve */
  int outer_its;         /* sync: max over rhs of sweeps K with x = x^K; async: max sweeps of any block */
  long long inner_its;   /* total inner CG iterations over all blocks, rhs and sweeps */
  long long lups;        /* stencil lattice updates: inner iterations x block points + residual points */
  double rel_residual;   /* max over rhs of the true final ||b - A x|| / ||b|| (absolute if ||b|| = 0) */
  double time_ms;        /* device time of the solve on `stream` (CUDA events) */
  int launches;          /* solver kernel launches (sweep, check and residual kernels) */
  int cluster, threads, slots; /* launch shape used */
  int* per_rhs_outer_its;      /* HOST, optional [nrhs]: filled if non-NULL */
  double* per_rhs_rel;         /* HOST, optional [nrhs]: filled if non-NULL */
  double sweep_ms;             /* with opts.profile: summed device time of the sweep kernels */
  int sweep_launches;          /* with opts.profile: sweep kernels timed */
  int engine;                  /* inner-CG engine used: 1 streaming, 2 resident */
  int variant;                 /* launch variant used: >= 0 resident table row, -1 scalar streaming,
                                  -2 vectorised (float4) streaming */
  double inner_rtol_final;     /* the inner tolerance of the last sweep (opts.inner_adapt: max over
                                  rhs of the controller's choice; else opts.inner_rtol) */
  long long trace_count;       /* with opts.trace: records taken (min(trace_count, trace_cap) returned) */
} ms_stats;

/* Number of doubles in one rhs's packed boundary array. */
MS_API long long ms_boundary_size(int nx, int ny, int nz);

/* Fill *opts with the defaults listed above. */
MS_API void ms_default_opts(ms_opts* opts);

/* Create a grid of nx*ny*nz interior points with nrhs right-hand sides
 * (section 2.1 model problem).  *out receives a handle owned by the caller
 * (free with ms_destroy).  Sizes must be >= 1.  Partitioned as one block
 * until ms_partition is called. */
MS_API int ms_create_grid(int nx, int ny, int nz, int nrhs, ms_grid** out);

/* Block layout (section 3: the matrix split into blocks by a domain
 * decomposition): px*py*pz blocks with per-axis cut arrays cx[0..px],
 * cy[0..py], cz[0..pz] (HOST int arrays, strictly increasing from 0 to n;
 * copied).  A NULL cut array means an equal split with the remainder given
 * to the leading blocks.  Block id = bx + px*(by + py*bz).  Fails with
 * MS_ERR_ARG if an edge is < 1. */
MS_API int ms_partition(ms_grid* grid, int px, int py, int pz, const int* cx, const int* cy, const int* cz);

/* Copy the current cut arrays to HOST arrays of length px+1, py+1, pz+1. */
MS_API int ms_get_cuts(ms_grid* grid, int* cx, int* cy, int* cz);

/* Solve A x = bhat for every rhs, bhat = f + lift(bnd) (section 2.1 problem,
 * section 3 method, Listing 1 loop).
 *   f:   [nrhs][nz][ny][nx] interior source, or NULL for zero;
 *   bnd: [nrhs][ms_boundary_size] Dirichlet faces, or NULL for zero;
 *   x:   [nrhs][nz][ny][nx], in: initial guess x^0, out: solution;
 *   opts: HOST, NULL = defaults; stats: HOST, may be NULL.
 * Each rhs stops independently at the first x^K with relative residual
 * < outer_tol (sync mode; tested on x^k before sweep k+1).  Blocks until the
 * solve is finished (the result is ready on `stream`'s timeline when it
 * returns).  Returns MS_ERR_NOT_CONVERGED if any rhs hit outer_maxit, with x
 * holding the last iterate. */
MS_API int ms_solve(ms_grid* grid, const double* f, const double* bnd, double* x, const ms_opts* opts, ms_stats* stats,
             void* stream);

/* ms_solve with HOST arrays (pageable or pinned): copies f, bnd and x to
 * device workspace, solves, copies x back, all on `stream`. */
MS_API int ms_solve_host(ms_grid* grid, const double* f_host, const double* bnd_host, double* x_host,
                  const ms_opts* opts, ms_stats* stats, void* stream);

/* True relative residual ||bhat - A x||_2 / ||bhat||_2 per rhs (section 2.1
 * stop-rule norm), computed from scratch in FP64.  rel_out: HOST [nrhs];
 * where ||bhat|| = 0 the absolute norm is returned.  Synchronises `stream`. */
MS_API int ms_residual(ms_grid* grid, const double* f, const double* bnd, const double* x, double* rel_out, void* stream);

/* Adjoint helper: since bhat = f + lift(g), d bhat_q / d g_p = 1 for the
 * interior point q next to boundary point p.  Writes grad_bnd[s][p] =
 * lam[s][q(p)] for every packed boundary point p ([nrhs][ms_boundary_size],
 * device).  lam is [nrhs][nz][ny][nx] (device). */
MS_API int ms_face_gather(ms_grid* grid, const double* lam, double* grad_bnd, void* stream);

/* The raw sums behind ms_residual, per rhs, left on the device:
 *   rr_out DEVICE [nrhs] or NULL: sum over this grid's points of (bhat - A x)^2;
 *   bb_out DEVICE [nrhs] or NULL: sum of bhat^2 (bhat = f + lift(bnd));
 * at least one must be non-NULL; FP64, summed in a fixed order (the result
 * does not depend on the stream or the launch).  Section 3 assembles the
 * global residual from per-block partial sums; a grid that is one shard of a
 * larger problem (its neighbours' values given as Dirichlet data in bnd)
 * returns its share of the global sums, to be added over the shards.  Ready
 * on `stream`'s timeline; no host synchronisation. */
MS_API int ms_norms(ms_grid* grid, const double* f, const double* bnd, const double* x, double* rr_out,
                    double* bb_out, void* stream);

/* One synchronous outer sweep (section 3: X_i <- X_i + A_ii^{-1}(B_i - A X)_i
 * for every block i, all blocks reading the same x^k), for callers that run
 * the outer loop themselves -- a grid that is one shard of a problem split
 * over several GPUs, whose neighbouring shards' boundary planes enter as the
 * Dirichlet data in bnd (section 3's halo swap between block groups):
 *   f, bnd: as ms_solve (device; may be NULL);
 *   x_in:   [nrhs][nz][ny][nx] x^k (device, read only);
 *   x_out:  [nrhs][nz][ny][nx] receives x^{k+1} (device; must not overlap x_in);
 *   rr_out: DEVICE [nrhs] or NULL: sum of (bhat - A x^k)^2 over this grid (the
 *           residual the stop rule of section 2.1 tests on x^k), formed from
 *           the sweep's own block partials in a fixed order (ms_norms gives the
 *           same sum up to rounding);
 *   opts:   HOST or NULL; precision, inner_rtol, inner_maxit, overlap,
 *           inner_method, gmres_restart and the launch-shape fields are used;
 *           mode must be MS_MODE_SYNC and inner_adapt 0;
 *   stats:  HOST or NULL.  NULL: nothing waits for the GPU (the results are
 *           ready on `stream`'s timeline).  Non-NULL: synchronises `stream` and
 *           fills inner_its, lups, time_ms, the launch shape, outer_its = 1 and
 *           rel_residual = that of x^k against this grid's own ||bhat||;
 *           returns MS_ERR_TIMEOUT (stats->status too) if a bounded device
 *           wait of the sweep ran out (opts.sum_polls), the result then not
 *           to be used.
 * Returns MS_OK, MS_ERR_ARG (NULL or overlapping buffers, invalid options,
 * a mode other than sync), MS_ERR_CUDA or MS_ERR_TIMEOUT (above).
 * The launch shape is the one a solve of the same problem measured (ms_solve
 * caches it per handle), else the model's first choice.  The inner solves use
 * the same kernels and FP32 scaling as ms_solve, so a sweep here equals a
 * sweep of ms_solve on the same data.  Besides the sweep kernel, the call
 * reads f (when given) or only the points next to the boundary, for ||bhat||
 * and the FP32 scaling. */
MS_API int ms_sweep(ms_grid* grid, const double* f, const double* bnd, const double* x_in, double* x_out,
                    double* rr_out, const ms_opts* opts, ms_stats* stats, void* stream);

/* The largest nrhs ms_residual_noalloc accepts (its scratch has a fixed size). */
#define MS_NOALLOC_MAX_RHS 1024

/* ms_residual without any device allocation.  (The paper has no counterpart:
 * this is an interface for callers, not a step of the method.)
 *
 * For callers that cannot call cudaMalloc where they need the residual:
 * latency-critical loops that cannot absorb cudaMalloc's implicit device
 * synchronisation, or applications whose device memory is owned by their own
 * pool allocator and that may not allocate behind its back.  ms_residual
 * allocates a per-handle workspace on first use; this function uses instead
 * a fixed 1 MiB array of partial sums compiled into the library (a static
 * device array that every GPU loading the library holds until the process
 * exits).
 *   f, bnd, x: as ms_residual (device; f and bnd may be NULL);
 *   rel_out:   DEVICE [nrhs] doubles, ||bhat - A x||_2 / ||bhat||_2 per rhs
 *              (the absolute norm where ||bhat|| = 0), ready on `stream`'s
 *              timeline when the call returns (no synchronisation).
 * Limits and caveats:
 *   - nrhs must be <= MS_NOALLOC_MAX_RHS, else MS_ERR_ARG with a message;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and caches it; make
 *     that first call before any stream capture on that device;
 *   - the cached address is not looked up again: after cudaDeviceReset on a
 *     device, do not call this function on that device again in the same
 *     process (the address may have changed);
 *   - every call on a device shares the one array: calls whose work can
 *     overlap on the GPU (unordered streams) race on it and must be
 *     serialised by the caller.  Each call writes all the scratch it reads,
 *     so no clearing is needed between calls. */
MS_API int ms_residual_noalloc(ms_grid* grid, const double* f, const double* bnd, const double* x, double* rel_out,
                               void* stream);

/* Row v of the resident engine's variant table (no counterpart in the paper:
 * the table lists the on-chip layouts of one block's CG state that the
 * autotuner chooses from).  threads: threads per CTA; strips: 4-point x-strips
 * a thread owns per plane; planes: z-planes a CTA holds at most; d_smem: the
 * correction d lives in shared memory (else registers); q_regs: A p is kept
 * in registers between the two halves of a CG iteration (one stencil per
 * iteration instead of two, bit-identical results); one_reduction: the
 * single-reduction CG (Chronopoulos and Gear's rearrangement of CG: one
 * cluster-wide reduction of r.r and r.A r per iteration instead of two, the
 * same iterates in exact arithmetic; p, A p and A r in registers, r and d in
 * shared memory).  Any output pointer may be NULL.  Returns MS_OK, or
 * MS_ERR_ARG if v is outside [0, count); *count (if non-NULL) always receives
 * the number of rows.  Host only, no device work. */
MS_API int ms_resident_variant(int v, int* count, int* threads, int* strips, int* planes, int* d_smem, int* q_regs,
                               int* one_reduction);

/* One global conjugate-gradient solve of A x = f + lift(bnd) on the whole
 * grid, in FP64, with no block splitting: the single-matrix Krylov method the
 * multisplitting solve is compared against on the same GPU.  CG is the inner
 * method of sections 2.2 and 3 applied to A itself; the stop rule is the one
 * of section 2.1, ||r_k|| < outer_tol ||bhat|| (strict, absolute if
 * ||bhat|| = 0), on the CG recurrence residual, tested before iteration k
 * (k = 0 included).  Arguments as for ms_solve (device pointers, x = x0 in,
 * solution out, stream = cudaStream_t or NULL); of opts only outer_tol,
 * outer_maxit (iteration cap) and time_limit_ms (device-side budget, applied
 * from the next iteration) are used, every other field is ignored and the
 * arithmetic is FP64 throughout.  Workspace: three vectors of nrhs x npts
 * doubles, kept by the grid handle.  stats: outer_its = iterations (max over
 * rhs), inner_its = iterations summed over rhs, lups = iterations x points +
 * the three residual evaluations, rel_residual = the true final relative
 * residual (max over rhs), engine = 0, variant = -1.  Returns MS_OK, or
 * MS_ERR_NOT_CONVERGED / MS_ERR_TIMEOUT (x holds the last iterate), or
 * MS_ERR_ARG / MS_ERR_CUDA / MS_ERR_OOM. */
MS_API int ms_gcg_solve(ms_grid* grid, const double* f, const double* bnd, double* x, const ms_opts* opts,
                        ms_stats* stats, void* stream);

/* Free the handle and its device workspace.  Synchronises the device work
 * the handle issued.  NULL is accepted. */
MS_API int ms_destroy(ms_grid* grid);

/* Message for the last failure on this handle (or of ms_create_grid when
 * grid is NULL).  Valid until the next call on the handle. */
MS_API const char* ms_last_error(ms_grid* grid);

#ifdef __cplusplus
}
#endif
#endif
