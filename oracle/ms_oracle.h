/*
 * ms_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure).
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * use this header; the CUDA library has its own, unrelated one.
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOT_CONVERGED 4

void or_set_threads(int n);
int or_get_max_threads(void);
long long or_boundary_size(int nx, int ny, int nz);
void or_apply_A(int nx, int ny, int nz, const double* u, double* y);
void or_lift(int nx, int ny, int nz, const double* f, const double* bnd, double* bhat);
void or_residual(int nx, int ny, int nz, const double* bhat, const double* x, double* r);
int or_block_cg(int bx, int by, int bz, double* r, double* d, double* work, double inner_rtol, int inner_maxit);
int or_solve(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy, const int* cz,
             const double* f, const double* bnd, double* x, double inner_rtol, int inner_maxit, double outer_tol,
             int outer_maxit, int* outer_its, long long* inner_its, double* res_hist, double* final_rel);
int or_block_gmres(int bx, int by, int bz, double* r, double* d, double inner_rtol, int inner_maxit, int restart);
int or_solve_ex(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy, const int* cz,
                int overlap, int gmres_restart, const double* f, const double* bnd, double* x, double inner_rtol,
                int inner_maxit, double outer_tol, int outer_maxit, int* outer_its, long long* inner_its,
                double* res_hist, double* final_rel);
int or_solve_overlap(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy, const int* cz,
                     int overlap, const double* f, const double* bnd, double* x, double inner_rtol, int inner_maxit,
                     double outer_tol, int outer_maxit, int* outer_its, long long* inner_its, double* res_hist,
                     double* final_rel);
int or_solve_delayed(int nx, int ny, int nz, int px, int py, int pz, const int* cx, const int* cy, const int* cz,
                     const double* f, const double* bnd, double* x, double inner_rtol, int inner_maxit,
                     double outer_tol, int outer_maxit, int max_delay, const int* delays, int* outer_its,
                     double* final_rel);

#ifdef __cplusplus
}
#endif
#endif
