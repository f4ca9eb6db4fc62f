/* ffp_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure
 * only; see ffp_oracle.c).  All arrays are host FP64, length N = nx*ny*nz,
 * index a = x + nx*(y + ny*z).  Band convention: cx[a] = A[a, a+1],
 * cy[a] = A[a, a+nx], cz[a] = A[a, a+nx*ny], zero where the neighbour does
 * not exist.  Return 0 on success, negative on error. */
#ifndef FFP_ORACLE_H
#define FFP_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif
int or_assemble(int nx, int ny, int nz, double lx, double ly, double lz,
                const double *kappa, const unsigned char *bc,
                double *d, double *cx, double *cy, double *cz);
int or_spmv(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
            const double *cz, const double *x, double *y);
/* classic = 0: the Schur terms use X = 2 beta - beta P beta (Sec. II-A as
 * printed); classic = 1: X = beta. */
int or_setup(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
             const double *cz, const double *t, int classic,
             double *Pd, double *Px, double *Py, double *Td, double *To, double *M);
int or_apply(int nx, int ny, int nz, const double *l3, const double *l2, const double *l1,
             const double *M, const double *r, double *z);
int or_pcg(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
           const double *cz, const double *l2, const double *l1, const double *M,
           const double *Dilu, const double *b, double *x, double rtol, int maxit, int flexible,
           int *iters_out, double *relres_out, double *alpha_hist, double *beta_hist,
           double *res_hist);
int or_ilu0_setup(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
                  const double *cz, double *D);
int or_ilu0_solve(int nx, int ny, int nz, const double *cx, const double *cy, const double *cz,
                  const double *D, const double *r, double *z);
int or_combo_apply(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
                   const double *cz, const double *l2, const double *l1, const double *M,
                   const double *Dilu, const double *r, double *z);
#ifdef __cplusplus
}
#endif
#endif
