/*
 * ms_oracle.c -- plain, slow, FP64 CPU oracle for two-stage multisplitting
 * (outer block Jacobi, inner conjugate gradients) on the 3D Laplace 7-point
 * stencil, after Brown, Bull and Bethune, "A highly scalable approach to
 * solving linear systems using two-stage multisplitting".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header or constant with
 * the CUDA library, and the CUDA library never calls it.
 *
 * Every loop is written in the most direct order: points in lexicographic
 * order (x fastest), blocks in id order, sums serial in FP64.  Build with
 * -O2 -ffp-contract=off so that no multiply-add is fused.
 *
 * Conventions (readings of the paper, where it is silent):
 *   - interior point (i,j,k), 0 <= i < nx, x fastest: idx = (k*ny + j)*nx + i
 *   - A u = 6 u(i,j,k) - sum of the six face neighbours that lie inside the
 *     interior (section 2.1: the Jacobi listing averages the six neighbours
 *     with weight 1/6, which is point Jacobi for exactly this matrix).
 *   - Dirichlet data g lives on the six faces of the box and is packed per
 *     right-hand side as x-(nz*ny), x+(nz*ny), y-(nz*nx), y+(nz*nx),
 *     z-(ny*nx), z+(ny*nx); edges and corners are never referenced.
 *   - the right-hand side is bhat = f + lift(g): every interior point adds the
 *     boundary values of its neighbours that lie on the boundary.
 *   - block Jacobi, section 3: X_i <- A_ii^{-1}(B_i - sum_{j != i} A_ij X_j),
 *     written in correction form x^{k+1}_i = x^k_i + delta_i with
 *     A_ii delta_i = r_i, r = bhat - A x^k (identical in exact arithmetic).
 *   - inner CG starts from delta = 0, stops when the recurrence residual
 *     satisfies ||r_m|| <= inner_rtol ||r_0|| or after inner_maxit steps,
 *     or on curvature eta <= 0.
 *   - outer stop, section 2.1 and Listing 1: ||bhat - A x^k|| / ||bhat|| <
 *     outer_tol tested on x^k before sweep k+1, including k = 0; the global
 *     norm is sqrt(sum over blocks of the block sums of squares) (section 3).
 *     When ||bhat|| = 0 the absolute norm is used.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ms_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

int or_get_max_threads(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

static long long idx3(int i, int j, int k, int nx, int ny) {
  return ((long long)k * ny + j) * nx + i;
}

long long or_boundary_size(int nx, int ny, int nz) {
  return 2LL * nz * ny + 2LL * nz * nx + 2LL * ny * nx;
}

/* y = A u on the whole interior grid, with u taken as zero outside it. */
void or_apply_A(int nx, int ny, int nz, const double* u, double* y) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double nb = 0.0;
        if (i > 0) nb += u[idx3(i - 1, j, k, nx, ny)];
        if (i < nx - 1) nb += u[idx3(i + 1, j, k, nx, ny)];
        if (j > 0) nb += u[idx3(i, j - 1, k, nx, ny)];
        if (j < ny - 1) nb += u[idx3(i, j + 1, k, nx, ny)];
        if (k > 0) nb += u[idx3(i, j, k - 1, nx, ny)];
        if (k < nz - 1) nb += u[idx3(i, j, k + 1, nx, ny)];
        y[idx3(i, j, k, nx, ny)] = 6.0 * u[idx3(i, j, k, nx, ny)] - nb;
      }
}

/* bhat = f + lift(g).  f may be NULL (zero source), bnd may be NULL (g = 0). */
void or_lift(int nx, int ny, int nz, const double* f, const double* bnd, double* bhat) {
  long long n = (long long)nx * ny * nz;
  for (long long p = 0; p < n; ++p) bhat[p] = f ? f[p] : 0.0;
  if (!bnd) return;
  const double* gxm = bnd;
  const double* gxp = gxm + (long long)nz * ny;
  const double* gym = gxp + (long long)nz * ny;
  const double* gyp = gym + (long long)nz * nx;
  const double* gzm = gyp + (long long)nz * nx;
  const double* gzp = gzm + (long long)ny * nx;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double add = 0.0;
        if (i == 0) add += gxm[(long long)k * ny + j];
        if (i == nx - 1) add += gxp[(long long)k * ny + j];
        if (j == 0) add += gym[(long long)k * nx + i];
        if (j == ny - 1) add += gyp[(long long)k * nx + i];
        if (k == 0) add += gzm[(long long)j * nx + i];
        if (k == nz - 1) add += gzp[(long long)j * nx + i];
        bhat[idx3(i, j, k, nx, ny)] += add;
      }
}

/* r = bhat - A x */
void or_residual(int nx, int ny, int nz, const double* bhat, const double* x, double* r) {
  long long n = (long long)nx * ny * nz;
  or_apply_A(nx, ny, nz, x, r);
  for (long long p = 0; p < n; ++p) r[p] = bhat[p] - r[p];
}

static double dot(long long n, const double* a, const double* b) {
  double s = 0.0;
  for (long long p = 0; p < n; ++p) s += a[p] * b[p];
  return s;
}

/*
 * Inner stage: CG on the block system A_ii d = r (section 2.2 and section 3),
 * with A_ii the stencil restricted to a bx*by*bz block and zero outside it.
 * r is overwritten with the CG recurrence residual; d receives the
 * correction.  work holds 2*n doubles (p and q).  Returns the number of CG
 * iterations taken.
 */
int or_block_cg(int bx, int by, int bz, double* r, double* d, double* work, double inner_rtol, int inner_maxit) {
  long long n = (long long)bx * by * bz;
  double* p = work;
  double* q = work + n;
  for (long long t = 0; t < n; ++t) {
    d[t] = 0.0;
    p[t] = r[t];
  }
  double gamma = dot(n, r, r);
  double gamma0 = gamma;
  int m = 0;
  if (gamma0 == 0.0) return 0;
  while (m < inner_maxit) {
    or_apply_A(bx, by, bz, p, q); /* q = A_ii p */
    double eta = dot(n, p, q);
    if (eta <= 0.0) break;
    double alpha = gamma / eta;
    for (long long t = 0; t < n; ++t) d[t] += alpha * p[t];
    for (long long t = 0; t < n; ++t) r[t] -= alpha * q[t];
    double gamma_new = dot(n, r, r);
    m += 1;
    if (sqrt(gamma_new) <= inner_rtol * sqrt(gamma0)) break;
    double beta = gamma_new / gamma;
    for (long long t = 0; t < n; ++t) p[t] = r[t] + beta * p[t];
    gamma = gamma_new;
  }
  return m;
}

/*
 * Inner stage alternative: restarted GMRES(restart) on the block system
 * A_ii d = r, from d = 0 -- the Krylov method of the paper's own runs
 * (PETSc's GMRES, section 3.2), written from its textbook definition:
 * Arnoldi with classical Gram-Schmidt (every projection of a step from the
 * same vector w = A v_j, as in PETSc's default), Givens rotations on the
 * Hessenberg column, |g_{j+1}| as the residual norm of the current iterate,
 * d += V y at the end of a cycle, and the true residual r - A d recomputed
 * at every restart.  Stops when the residual estimate is <= inner_rtol ||r||
 * or after inner_maxit Arnoldi steps (the iteration count, one stencil
 * application each, as for CG).  On return r holds the true residual
 * r - A d.  Returns the number of Arnoldi steps.
 */
int or_block_gmres(int bx, int by, int bz, double* r, double* d, double inner_rtol, int inner_maxit, int restart) {
  long long n = (long long)bx * by * bz;
  if (restart < 1) restart = 1;
  int m1 = restart + 1;
  double* V = (double*)malloc(sizeof(double) * n * m1);  /* basis vectors, column j at V + j*n */
  double* w = (double*)malloc(sizeof(double) * n);
  double* H = (double*)calloc((size_t)m1 * restart, sizeof(double)); /* H[i*restart + j] */
  double* cs = (double*)malloc(sizeof(double) * restart);
  double* sn = (double*)malloc(sizeof(double) * restart);
  double* g = (double*)malloc(sizeof(double) * m1);
  double* y = (double*)malloc(sizeof(double) * restart);
  for (long long t = 0; t < n; ++t) d[t] = 0.0;
  double beta0 = sqrt(dot(n, r, r));
  int total = 0;
  if (beta0 > 0.0 && inner_maxit > 0) {
    double stop = inner_rtol * beta0;
    for (;;) {
      /* residual of the current iterate: r - A d (r itself in the first cycle) */
      or_apply_A(bx, by, bz, d, w);
      for (long long t = 0; t < n; ++t) w[t] = r[t] - w[t];
      double beta = sqrt(dot(n, w, w));
      if (beta <= stop || beta == 0.0) break;
      for (long long t = 0; t < n; ++t) V[t] = w[t] / beta;
      for (int i = 0; i < m1; ++i) g[i] = 0.0;
      g[0] = beta;
      int k = 0;
      int finished = 0;
      for (int j = 0; j < restart; ++j) {
        or_apply_A(bx, by, bz, V + (long long)j * n, w);
        /* classical Gram-Schmidt: every h_ij from the same w */
        for (int i = 0; i <= j; ++i) H[i * restart + j] = dot(n, w, V + (long long)i * n);
        for (int i = 0; i <= j; ++i) {
          double h = H[i * restart + j];
          for (long long t = 0; t < n; ++t) w[t] -= h * V[(long long)i * n + t];
        }
        double hn = sqrt(dot(n, w, w));
        H[(j + 1) * restart + j] = hn;
        if (hn > 0.0)
          for (long long t = 0; t < n; ++t) V[(long long)(j + 1) * n + t] = w[t] / hn;
        /* earlier rotations on column j, then the rotation that zeroes H[j+1][j] */
        for (int i = 0; i < j; ++i) {
          double a = H[i * restart + j], b = H[(i + 1) * restart + j];
          H[i * restart + j] = cs[i] * a + sn[i] * b;
          H[(i + 1) * restart + j] = -sn[i] * a + cs[i] * b;
        }
        double a = H[j * restart + j], b = H[(j + 1) * restart + j];
        double rho = sqrt(a * a + b * b);
        cs[j] = rho > 0.0 ? a / rho : 1.0;
        sn[j] = rho > 0.0 ? b / rho : 0.0;
        H[j * restart + j] = rho;
        H[(j + 1) * restart + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        total += 1;
        k = j + 1;
        if (fabs(g[j + 1]) <= stop || total >= inner_maxit || hn == 0.0) {
          finished = 1;
          break;
        }
      }
      /* y = R^{-1} g (upper triangular k x k), d += V y */
      for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int c = i + 1; c < k; ++c) s -= H[i * restart + c] * y[c];
        y[i] = H[i * restart + i] != 0.0 ? s / H[i * restart + i] : 0.0;
      }
      for (int i = 0; i < k; ++i)
        for (long long t = 0; t < n; ++t) d[t] += y[i] * V[(long long)i * n + t];
      if (finished && (fabs(g[k]) <= stop || total >= inner_maxit)) break;
      if (total >= inner_maxit) break;
    }
  }
  /* true residual of the final iterate */
  or_apply_A(bx, by, bz, d, w);
  for (long long t = 0; t < n; ++t) r[t] -= w[t];
  free(V);
  free(w);
  free(H);
  free(cs);
  free(sn);
  free(g);
  free(y);
  return total;
}

static int check_cuts(int n, int p, const int* c) {
  if (p < 1 || c[0] != 0 || c[p] != n) return 0;
  for (int a = 0; a < p; ++a)
    if (c[a + 1] <= c[a]) return 0;
  return 1;
}

/* Copy block (ox..ox+bx, ...) of a grid array into a compact block array, and back. */
static void gather_block(int nx, int ny, const double* g, int ox, int oy, int oz, int bx, int by, int bz, double* b) {
  for (int k = 0; k < bz; ++k)
    for (int j = 0; j < by; ++j)
      for (int i = 0; i < bx; ++i) b[idx3(i, j, k, bx, by)] = g[idx3(ox + i, oy + j, oz + k, nx, ny)];
}

/*
 * One outer block-Jacobi sweep (section 3): given x^k and its residual r^k
 * (whole grid), every block solves A_ii d_i = r_i by CG and
 * x^{k+1}_i = x^k_i + d_i.  All blocks read the same x^k (strict Jacobi).
 * Returns the total number of inner iterations over the blocks.
 */
static long long outer_sweep(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy,
                             const int* cz, const double* r_grid, double* x, double inner_rtol, int inner_maxit,
                             int* inner_per_block) {
  int nblocks = px * py * pz;
  long long total = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads) reduction(+ : total)
#endif
  for (int b = 0; b < nblocks; ++b) {
    int bi = b % px, bj = (b / px) % py, bk = b / (px * py);
    int ox = cx[bi], oy = cy[bj], oz = cz[bk];
    int bx = cx[bi + 1] - ox, by = cy[bj + 1] - oy, bz = cz[bk + 1] - oz;
    long long n = (long long)bx * by * bz;
    double* rb = (double*)malloc(sizeof(double) * n);
    double* db = (double*)malloc(sizeof(double) * n);
    double* wk = (double*)malloc(sizeof(double) * 2 * n);
    gather_block(nx, ny, r_grid, ox, oy, oz, bx, by, bz, rb);
    int m = or_block_cg(bx, by, bz, rb, db, wk, inner_rtol, inner_maxit);
    if (inner_per_block) inner_per_block[b] = m;
    total += m;
    /* blocks are disjoint, so this update touches only block b's points */
    for (int k = 0; k < bz; ++k)
      for (int j = 0; j < by; ++j)
        for (int i = 0; i < bx; ++i) x[idx3(ox + i, oy + j, oz + k, nx, ny)] += db[idx3(i, j, k, bx, by)];
    free(rb);
    free(db);
    free(wk);
  }
  return total;
}

/* Global norm from block partial sums, section 3: sqrt(sum_i ||r_i||^2). */
static double global_norm(int nx, int ny, int px, int py, int pz, const int* cx, const int* cy, const int* cz,
                          const double* r) {
  double s = 0.0;
  for (int b = 0; b < px * py * pz; ++b) {
    int bi = b % px, bj = (b / px) % py, bk = b / (px * py);
    double sb = 0.0;
    for (int k = cz[bk]; k < cz[bk + 1]; ++k)
      for (int j = cy[bj]; j < cy[bj + 1]; ++j)
        for (int i = cx[bi]; i < cx[bi + 1]; ++i) {
          double v = r[idx3(i, j, k, nx, ny)];
          sb += v * v;
        }
    s += sb;
  }
  return sqrt(s);
}

int or_solve(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy, const int* cz,
             const double* f, const double* bnd, double* x, double inner_rtol, int inner_maxit, double outer_tol,
             int outer_maxit, int* outer_its, long long* inner_its, double* res_hist, double* final_rel) {
  if (nx < 1 || ny < 1 || nz < 1) return OR_ERR_ARG;
  if (!check_cuts(nx, px, cx) || !check_cuts(ny, py, cy) || !check_cuts(nz, pz, cz)) return OR_ERR_ARG;
  if (inner_maxit < 0 || outer_maxit < 0) return OR_ERR_ARG;
  long long n = (long long)nx * ny * nz;
  double* bhat = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  if (!bhat || !r) {
    free(bhat);
    free(r);
    return OR_ERR_ARG;
  }
  or_lift(nx, ny, nz, f, bnd, bhat);
  double bnorm = sqrt(dot(n, bhat, bhat));
  double scale = bnorm > 0.0 ? 1.0 / bnorm : 1.0;
  long long inner_total = 0;
  int status = OR_ERR_NOT_CONVERGED;
  int k = 0;
  double rho = 0.0;
  for (;;) {
    or_residual(nx, ny, nz, bhat, x, r);
    rho = global_norm(nx, ny, px, py, pz, cx, cy, cz, r) * scale;
    if (res_hist) res_hist[k] = rho;
    if (rho < outer_tol) {
      status = OR_OK;
      break;
    }
    if (k == outer_maxit) break;
    inner_total += outer_sweep(nx, ny, nz, px, py, pz, cx, cy, cz, r, x, inner_rtol, inner_maxit, NULL);
    k += 1;
  }
  if (outer_its) *outer_its = k;
  if (inner_its) *inner_its = inner_total;
  if (final_rel) *final_rel = rho;
  free(bhat);
  free(r);
  return status;
}

/*
 * Multisplitting with overlapping blocks (section 3.2: blocks may overlap by
 * o elements in each dimension; the first multisplitting work the paper cites
 * shows overlapping blocks still converge).  Block i is extended by o points
 * on every face (clipped to the grid); it solves A_ee d = r_e by CG on the
 * extended box, with zero Dirichlet data outside that box, r_e = bhat - A x^k
 * on the box.  The paper leaves the weighting of overlapping contributions
 * open; the weighting used here gives every point weight 1 in the block that
 * owns it and 0 in the blocks that only overlap it (a multisplitting with
 * diagonal 0/1 weights summing to the identity), so
 * x^{k+1} = x^k + d_i on the points block i owns.  With o = 0 this is exactly
 * or_solve.  The stop rule and the global norm are those of or_solve.
 */
static long long overlap_sweep(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy,
                               const int* cz, int o, const double* r_grid, double* x, double inner_rtol,
                               int inner_maxit, int gmres_restart) {
  int nblocks = px * py * pz;
  long long total = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads) reduction(+ : total)
#endif
  for (int b = 0; b < nblocks; ++b) {
    int bi = b % px, bj = (b / px) % py, bk = b / (px * py);
    /* owned box [cx[bi], cx[bi+1]) x ...; extended box clipped to the grid */
    int ex0 = cx[bi] - o < 0 ? 0 : cx[bi] - o, ex1 = cx[bi + 1] + o > nx ? nx : cx[bi + 1] + o;
    int ey0 = cy[bj] - o < 0 ? 0 : cy[bj] - o, ey1 = cy[bj + 1] + o > ny ? ny : cy[bj + 1] + o;
    int ez0 = cz[bk] - o < 0 ? 0 : cz[bk] - o, ez1 = cz[bk + 1] + o > nz ? nz : cz[bk + 1] + o;
    int ex = ex1 - ex0, ey = ey1 - ey0, ez = ez1 - ez0;
    long long n = (long long)ex * ey * ez;
    double* rb = (double*)malloc(sizeof(double) * n);
    double* db = (double*)malloc(sizeof(double) * n);
    double* wk = (double*)malloc(sizeof(double) * 2 * n);
    gather_block(nx, ny, r_grid, ex0, ey0, ez0, ex, ey, ez, rb);
    int m = gmres_restart > 0 ? or_block_gmres(ex, ey, ez, rb, db, inner_rtol, inner_maxit, gmres_restart)
                              : or_block_cg(ex, ey, ez, rb, db, wk, inner_rtol, inner_maxit);
    total += m;
    /* owned points only: the owned boxes are disjoint, and every x read this
       sweep went into r_grid before any update */
    for (int k = cz[bk]; k < cz[bk + 1]; ++k)
      for (int j = cy[bj]; j < cy[bj + 1]; ++j)
        for (int i = cx[bi]; i < cx[bi + 1]; ++i)
          x[idx3(i, j, k, nx, ny)] += db[idx3(i - ex0, j - ey0, k - ez0, ex, ey)];
    free(rb);
    free(db);
    free(wk);
  }
  return total;
}

/* Overlap o >= 0 and inner method (gmres_restart = 0: CG, > 0: GMRES(restart)). */
int or_solve_ex(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy, const int* cz,
                int overlap, int gmres_restart, const double* f, const double* bnd, double* x, double inner_rtol,
                int inner_maxit, double outer_tol, int outer_maxit, int* outer_its, long long* inner_its,
                double* res_hist, double* final_rel) {
  if (nx < 1 || ny < 1 || nz < 1 || overlap < 0 || gmres_restart < 0) return OR_ERR_ARG;
  if (!check_cuts(nx, px, cx) || !check_cuts(ny, py, cy) || !check_cuts(nz, pz, cz)) return OR_ERR_ARG;
  if (inner_maxit < 0 || outer_maxit < 0) return OR_ERR_ARG;
  long long n = (long long)nx * ny * nz;
  double* bhat = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  if (!bhat || !r) {
    free(bhat);
    free(r);
    return OR_ERR_ARG;
  }
  or_lift(nx, ny, nz, f, bnd, bhat);
  double bnorm = sqrt(dot(n, bhat, bhat));
  double scale = bnorm > 0.0 ? 1.0 / bnorm : 1.0;
  long long inner_total = 0;
  int status = OR_ERR_NOT_CONVERGED;
  int k = 0;
  double rho = 0.0;
  for (;;) {
    or_residual(nx, ny, nz, bhat, x, r);
    rho = global_norm(nx, ny, px, py, pz, cx, cy, cz, r) * scale;
    if (res_hist) res_hist[k] = rho;
    if (rho < outer_tol) {
      status = OR_OK;
      break;
    }
    if (k == outer_maxit) break;
    inner_total +=
        overlap_sweep(nx, ny, nz, px, py, pz, cx, cy, cz, overlap, r, x, inner_rtol, inner_maxit, gmres_restart);
    k += 1;
  }
  if (outer_its) *outer_its = k;
  if (inner_its) *inner_its = inner_total;
  if (final_rel) *final_rel = rho;
  free(bhat);
  free(r);
  return status;
}

int or_solve_overlap(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy, const int* cz,
                     int overlap, const double* f, const double* bnd, double* x, double inner_rtol, int inner_maxit,
                     double outer_tol, int outer_maxit, int* outer_its, long long* inner_its, double* res_hist,
                     double* final_rel) {
  return or_solve_ex(nx, ny, nz, px, py, pz, cx, cy, cz, overlap, 0, f, bnd, x, inner_rtol, inner_maxit, outer_tol,
                     outer_maxit, outer_its, inner_its, res_hist, final_rel);
}

/*
 * Asynchronous block Jacobi with bounded delays (sections 2.1 and 2.3; the
 * asynchronous halo swap of section 3 uses "the latest received" data).
 * Block b in sweep k assembles its residual from its own x_b^k and, for
 * each neighbouring block, the neighbour's values from sweep
 * max(0, k - delay[k][b][face]) (face 0..5 = x-, x+, y-, y+, z-, z+).
 * The delays are inputs (drawn by the caller's seeded generator).
 * The stop test is the true global residual of x^k, as in or_solve.
 * A ring of max_delay+2 iterates holds x^{k-max_delay} .. x^{k+1}.  Returns OR_OK or
 * OR_ERR_NOT_CONVERGED.
 */
int or_solve_delayed(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy, const int* cz,
                     const double* f, const double* bnd, double* x, double inner_rtol, int inner_maxit,
                     double outer_tol, int outer_maxit, int max_delay, const int* delays, int* outer_its,
                     double* final_rel) {
  if (nx < 1 || ny < 1 || nz < 1 || max_delay < 0) return OR_ERR_ARG;
  if (!check_cuts(nx, px, cx) || !check_cuts(ny, py, cy) || !check_cuts(nz, pz, cz)) return OR_ERR_ARG;
  long long n = (long long)nx * ny * nz;
  int nblocks = px * py * pz;
  int depth = max_delay + 2; /* x^{k-max_delay} .. x^{k+1} */
  double* bhat = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  double* hist = (double*)malloc(sizeof(double) * n * depth); /* hist[k % depth] = x^k */
  double* xv = (double*)malloc(sizeof(double) * n);           /* x as seen by one block */
  or_lift(nx, ny, nz, f, bnd, bhat);
  double bnorm = sqrt(dot(n, bhat, bhat));
  double scale = bnorm > 0.0 ? 1.0 / bnorm : 1.0;
  memcpy(hist, x, sizeof(double) * n);
  int status = OR_ERR_NOT_CONVERGED;
  int k = 0;
  double rho = 0.0;
  for (;;) {
    double* xk = hist + (long long)(k % depth) * n;
    or_residual(nx, ny, nz, bhat, xk, r);
    rho = global_norm(nx, ny, px, py, pz, cx, cy, cz, r) * scale;
    if (rho < outer_tol) {
      status = OR_OK;
      break;
    }
    if (k == outer_maxit) break;
    double* xnext = hist + (long long)((k + 1) % depth) * n;
    memcpy(xnext, xk, sizeof(double) * n);
    for (int b = 0; b < nblocks; ++b) {
      int bi = b % px, bj = (b / px) % py, bk = b / (px * py);
      int lo[3] = {cx[bi], cy[bj], cz[bk]};
      int hi[3] = {cx[bi + 1], cy[bj + 1], cz[bk + 1]};
      /* the view of x this block sees: its own x^k, and per face the
         neighbour's x from the delayed sweep on the halo layer */
      memcpy(xv, xk, sizeof(double) * n);
      for (int face = 0; face < 6; ++face) {
        int axis = face / 2;
        int d = delays[((long long)k * nblocks + b) * 6 + face];
        if (d > max_delay) d = max_delay;
        int ks = k - d < 0 ? 0 : k - d;
        if (ks < k - max_delay) ks = k - max_delay;
        const double* xs = hist + (long long)(ks % depth) * n;
        int layer = (face % 2 == 0) ? lo[axis] - 1 : hi[axis];
        int nn[3] = {nx, ny, nz};
        if (layer < 0 || layer >= nn[axis]) continue; /* domain boundary */
        int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
        for (int u = lo[a1]; u < hi[a1]; ++u)
          for (int v = lo[a2]; v < hi[a2]; ++v) {
            int c[3];
            c[axis] = layer;
            c[a1] = u;
            c[a2] = v;
            long long p = idx3(c[0], c[1], c[2], nx, ny);
            xv[p] = xs[p];
          }
      }
      /* block residual from that view, restricted to block b */
      long long bn = (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
      double* rb = (double*)malloc(sizeof(double) * bn);
      double* db = (double*)malloc(sizeof(double) * bn);
      double* wk = (double*)malloc(sizeof(double) * 2 * bn);
      int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
      for (int kk = 0; kk < bz; ++kk)
        for (int jj = 0; jj < by; ++jj)
          for (int ii = 0; ii < bx; ++ii) {
            int gi = lo[0] + ii, gj = lo[1] + jj, gk = lo[2] + kk;
            double nb = 0.0;
            if (gi > 0) nb += xv[idx3(gi - 1, gj, gk, nx, ny)];
            if (gi < nx - 1) nb += xv[idx3(gi + 1, gj, gk, nx, ny)];
            if (gj > 0) nb += xv[idx3(gi, gj - 1, gk, nx, ny)];
            if (gj < ny - 1) nb += xv[idx3(gi, gj + 1, gk, nx, ny)];
            if (gk > 0) nb += xv[idx3(gi, gj, gk - 1, nx, ny)];
            if (gk < nz - 1) nb += xv[idx3(gi, gj, gk + 1, nx, ny)];
            long long p = idx3(gi, gj, gk, nx, ny);
            rb[idx3(ii, jj, kk, bx, by)] = bhat[p] - (6.0 * xv[p] - nb);
          }
      or_block_cg(bx, by, bz, rb, db, wk, inner_rtol, inner_maxit);
      for (int kk = 0; kk < bz; ++kk)
        for (int jj = 0; jj < by; ++jj)
          for (int ii = 0; ii < bx; ++ii)
            xnext[idx3(lo[0] + ii, lo[1] + jj, lo[2] + kk, nx, ny)] += db[idx3(ii, jj, kk, bx, by)];
      free(rb);
      free(db);
      free(wk);
    }
    k += 1;
  }
  memcpy(x, hist + (long long)(k % depth) * n, sizeof(double) * n);
  if (outer_its) *outer_its = k;
  if (final_rel) *final_rel = rho;
  free(bhat);
  free(r);
  free(hist);
  free(xv);
  return status;
}
