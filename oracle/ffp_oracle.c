/*
 * ffp_oracle.c -- plain, slow, FP64 CPU oracle for the nested twisted
 * frequency-filtering preconditioner (NTD) and its PCG driver.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA library against an
 * obviously correct restatement of the paper.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * Paper: "Multithreaded Filtering Preconditioner for Diffusion Equation on
 * Structured Grid" (arXiv 1909.09771).  Passages followed:
 *   - model problem and linear system: Sec. I, Eq. (1)-(2)
 *   - nested block-tridiagonal structure of A: Sec. II (matrix A, D^_i, D-_i)
 *   - twisted bands L1..L3 / U1..U3: Sec. II-A
 *   - exact twisted block LU and the beta-approximated recurrences for P_i
 *     (level 3), T_i (level 2) and the scalar pivots M_i (level 1):
 *     Sec. II-A, recurrences for P_i, T_i, M_i and the definitions of beta
 *   - band storage l1,l2,l3 (u = l by symmetry): Sec. II-A, band list
 *   - solve: Sec. II-B, Algorithms 1-7 (SOLVE, LowerSolve, LowerSolveUpperHalf,
 *     LowerSolveLowerHalf, UpperSolve, UpperSolveUpperHalf,
 *     UpperSolveLowerHalf), entry SOLVE(1, N, x, y, n^2, 3)
 *   - PCG conventions: Sec. III, "Parameters for conjugate gradient"
 *
 * Readings where the paper is silent or garbled (each is repeated in the
 * design notes):
 *   R1  beta at level 3 needs P_{i-1}^{-1}; it is applied through the nested
 *       approximate inverse of plane i-1, i.e. the level-2 SOLVE of that plane.
 *       At level 2 the inverse of the tridiagonal T_{k-1} is exact.
 *   R2  the beta used when building block i is formed from the neighbouring
 *       block it is eliminated from (i-1 in the top half, i+1 in the bottom
 *       half) with w = (coupling between the two blocks) .* t restricted to
 *       block i.
 *   R4  "D_nz" at every level means the last block of that level.
 *   R5  twist block index m = floor((nblocks-1)/2), 0-based, at every level,
 *       the same in setup and solve.
 *   R6  Algorithm 4 couples to the already-solved block below (x(i+bs:..)).
 *   R7  Algorithm 6 couples to the final x of the block below, not x'.
 *   R8  UpperSolve consumes the LowerSolve output y.
 *   R9  level 1 is an exact (twisted) tridiagonal solve; recursion bottoms out
 *       at a division by the scalar pivot M_a ("level 0").
 *   R10 block sizes per level: nx*ny (planes), nx (lines), 1 (cells).
 *   R12 finite-volume assembly with harmonic-mean face coefficients; a
 *       Dirichlet face sits half a cell from the centre.
 *   R15 |w_a| < 1e-300 -> beta_a = 1/(diagonal entry).
 *   R16 a non-positive or non-finite pivot / diagonal is a breakdown (-3).
 *   R17 stop on the recursive residual, then verify the true residual and
 *       continue from it if it is not below rtol.
 *   R19 flexible CG (Notay) beta for inexact applies.
 *
 * Built with gcc -O2 -ffp-contract=off (no FMA contraction): every
 * operation rounds exactly as written.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "ffp_oracle.h"

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_ALLOC (-2)
#define OR_ERR_BREAKDOWN (-3)
#define OR_ERR_NOT_CONVERGED (-4)

/* ------------------------------------------------------------------ */
/* Operator assembly (Eq. (2), finite-volume reading R12)              */
/* ------------------------------------------------------------------ */

static double harmonic(double ka, double kb) { return 2.0 * ka * kb / (ka + kb); }

int or_assemble(int nx, int ny, int nz, double lx, double ly, double lz,
                const double *kappa, const unsigned char *bc,
                double *d, double *cx, double *cy, double *cz)
{
    if (nx < 1 || ny < 1 || nz < 1 || !kappa || !bc || !d || !cx || !cy || !cz) return OR_ERR_ARG;
    const double hx = lx / nx, hy = ly / ny, hz = lz / nz;
    const double ax = hy * hz / hx, ay = hx * hz / hy, az = hx * hy / hz; /* area / distance */
    const long nxy = (long)nx * ny;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long a = x + (long)nx * (y + (long)ny * z);
                const double ka = kappa[a];
                if (!(ka > 0.0) || !isfinite(ka)) return OR_ERR_ARG;
                double diag = 0.0;
                /* face x- */
                if (x > 0) diag += harmonic(ka, kappa[a - 1]) * ax;
                else if (bc[0] == 0) diag += 2.0 * ka * ax;
                /* face x+ */
                if (x + 1 < nx) { double c = harmonic(ka, kappa[a + 1]) * ax; cx[a] = -c; diag += c; }
                else { cx[a] = 0.0; if (bc[1] == 0) diag += 2.0 * ka * ax; }
                /* face y- */
                if (y > 0) diag += harmonic(ka, kappa[a - nx]) * ay;
                else if (bc[2] == 0) diag += 2.0 * ka * ay;
                /* face y+ */
                if (y + 1 < ny) { double c = harmonic(ka, kappa[a + nx]) * ay; cy[a] = -c; diag += c; }
                else { cy[a] = 0.0; if (bc[3] == 0) diag += 2.0 * ka * ay; }
                /* face z- */
                if (z > 0) diag += harmonic(ka, kappa[a - nxy]) * az;
                else if (bc[4] == 0) diag += 2.0 * ka * az;
                /* face z+ */
                if (z + 1 < nz) { double c = harmonic(ka, kappa[a + nxy]) * az; cz[a] = -c; diag += c; }
                else { cz[a] = 0.0; if (bc[5] == 0) diag += 2.0 * ka * az; }
                d[a] = diag;
            }
    return OR_OK;
}

/* y = A x for the 7-point band storage (Sec. II, "only store the bands"). */
int or_spmv(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
            const double *cz, const double *x, double *y)
{
    const long nxy = (long)nx * ny, n = nxy * nz;
    for (long a = 0; a < n; ++a) {
        const int ix = (int)(a % nx), iy = (int)((a / nx) % ny), iz = (int)(a / nxy);
        double s = d[a] * x[a];
        if (ix > 0) s += cx[a - 1] * x[a - 1];
        if (ix + 1 < nx) s += cx[a] * x[a + 1];
        if (iy > 0) s += cy[a - nx] * x[a - nx];
        if (iy + 1 < ny) s += cy[a] * x[a + nx];
        if (iz > 0) s += cz[a - nxy] * x[a - nxy];
        if (iz + 1 < nz) s += cz[a] * x[a + nxy];
        y[a] = s;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* NTD solve: Algorithms 1-7 of Sec. II-B, generic over the 3 levels.  */
/* ------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
    const double *l[4]; /* l[1]=l1 (x-band of T), l[2]=l2 (y-band of P), l[3]=l3 (z-band of A) */
    const double *M;    /* level-1 twisted pivots */
    int classic;        /* setup only: X = beta in the Schur terms instead of 2 beta - beta P beta */
} ntd_ctx;

static long block_size(const ntd_ctx *c, int level)
{
    /* R10: planes, lines, cells */
    if (level == 3) return (long)c->nx * c->ny;
    if (level == 2) return c->nx;
    return 1;
}

static void ntd_solve(const ntd_ctx *c, long start, long len, int level, const double *b, double *x);

/* LowerSolve (Algorithm 2) with its two halves (Algorithms 3 and 4):
 * solves (P + L) y = b on the range [start, start+len) made of blocks of
 * size block_size(level); the block solves recurse one level down. */
static void lower_solve(const ntd_ctx *c, long start, long len, int level, const double *b, double *y)
{
    const long bs = block_size(c, level);
    const long nb = len / bs;
    const long mid = (nb - 1) / 2;              /* twist block (R5) */
    const double *L = c->l[level];
    double *rhs = (double *)malloc(sizeof(double) * bs);
    /* Algorithm 3: first block to the block above the twist */
    for (long q = 0; q < mid; ++q) {
        const long i = start + q * bs;
        for (long e = 0; e < bs; ++e) rhs[e] = b[i + e];
        if (q > 0)
            for (long e = 0; e < bs; ++e) rhs[e] -= L[i - bs + e] * y[i - bs + e];
        ntd_solve(c, i, bs, level - 1, rhs - i, y);
    }
    /* Algorithm 4: last block up to the block below the twist (R6) */
    for (long q = nb - 1; q > mid; --q) {
        const long i = start + q * bs;
        for (long e = 0; e < bs; ++e) rhs[e] = b[i + e];
        if (q < nb - 1)
            for (long e = 0; e < bs; ++e) rhs[e] -= L[i + e] * y[i + bs + e];
        ntd_solve(c, i, bs, level - 1, rhs - i, y);
    }
    /* twist block: couplings from both sides, then its own solve */
    {
        const long cur = start + mid * bs;
        for (long e = 0; e < bs; ++e) rhs[e] = b[cur + e];
        if (mid > 0)
            for (long e = 0; e < bs; ++e) rhs[e] -= L[cur - bs + e] * y[cur - bs + e];
        if (mid < nb - 1)
            for (long e = 0; e < bs; ++e) rhs[e] -= L[cur + e] * y[cur + bs + e];
        ntd_solve(c, cur, bs, level - 1, rhs - cur, y);
    }
    free(rhs);
}

/* UpperSolve (Algorithm 5) with its halves (Algorithms 6 and 7): solves
 * (I + P^{-1} U) x = y where U = L^T (symmetric bands). */
static void upper_solve(const ntd_ctx *c, long start, long len, int level, const double *y, double *x)
{
    const long bs = block_size(c, level);
    const long nb = len / bs;
    const long mid = (nb - 1) / 2;
    const double *U = c->l[level];
    double *bp = (double *)malloc(sizeof(double) * bs);
    double *xp = (double *)malloc(sizeof(double) * bs);
    const long cur = start + mid * bs;
    for (long e = 0; e < bs; ++e) x[cur + e] = y[cur + e];     /* x(mid) = y(mid) (R8) */
    /* Algorithm 6: from the block above the twist up to the first block (R7) */
    for (long q = mid - 1; q >= 0; --q) {
        const long i = start + q * bs;
        for (long e = 0; e < bs; ++e) bp[e] = U[i + e] * x[i + bs + e];
        ntd_solve(c, i, bs, level - 1, bp - i, xp - i);
        for (long e = 0; e < bs; ++e) x[i + e] = y[i + e] - xp[e];
    }
    /* Algorithm 7: from the block below the twist down to the last block */
    for (long q = mid + 1; q < nb; ++q) {
        const long i = start + q * bs;
        for (long e = 0; e < bs; ++e) bp[e] = U[i - bs + e] * x[i - bs + e];
        ntd_solve(c, i, bs, level - 1, bp - i, xp - i);
        for (long e = 0; e < bs; ++e) x[i + e] = y[i + e] - xp[e];
    }
    free(bp);
    free(xp);
}

/* SOLVE (Algorithm 1).  b and x are indexed with global indices. Level 0 is
 * the scalar pivot division that closes the level-1 twisted tridiagonal solve
 * (R9). */
static void ntd_solve(const ntd_ctx *c, long start, long len, int level, const double *b, double *x)
{
    if (level == 0) {
        x[start] = b[start] / c->M[start];
        return;
    }
    double *y = (double *)malloc(sizeof(double) * len);
    lower_solve(c, start, len, level, b, y - start);
    upper_solve(c, start, len, level, y - start, x);
    free(y);
}

int or_apply(int nx, int ny, int nz, const double *l3, const double *l2, const double *l1,
             const double *M, const double *r, double *z)
{
    ntd_ctx c;
    c.nx = nx; c.ny = ny; c.nz = nz;
    c.l[0] = NULL; c.l[1] = l1; c.l[2] = l2; c.l[3] = l3;
    c.M = M;
    c.classic = 0;
    const long n = (long)nx * ny * nz;
    ntd_solve(&c, 0, n, 3, r, z);     /* SOLVE(1, N, x, y, n^2, 3) */
    return OR_OK;
}

/* Nested solve on one plane (level 2) or one line (level 1). */
static void solve_block(const ntd_ctx *c, long start, int level, const double *b, double *x)
{
    ntd_solve(c, start, block_size(c, level + 1), level, b, x);
}

/* ------------------------------------------------------------------ */
/* Setup (Sec. II-A)                                                   */
/* ------------------------------------------------------------------ */

static int bad(double v) { return !(v > 0.0) || !isfinite(v); }

/* Level 1: twisted pivots of the tridiagonal T on the line starting at s
 * (recurrence for M_i).  Td = diagonal, To = x-band (To[a] couples a,a+1). */
static int factor_line(int nx, long s, const double *Td, const double *To, double *M)
{
    const int m = (nx - 1) / 2;
    for (int a = 0; a < m; ++a) {                          /* top half, forward */
        double v = Td[s + a];
        if (a > 0) v -= To[s + a - 1] * To[s + a - 1] / M[s + a - 1];
        if (bad(v)) return OR_ERR_BREAKDOWN;
        M[s + a] = v;
    }
    for (int a = nx - 1; a > m; --a) {                     /* bottom half, backward */
        double v = Td[s + a];
        if (a < nx - 1) v -= To[s + a] * To[s + a] / M[s + a + 1];
        if (bad(v)) return OR_ERR_BREAKDOWN;
        M[s + a] = v;
    }
    {                                                      /* twist cell: both */
        double v = Td[s + m];
        if (m > 0) v -= To[s + m - 1] * To[s + m - 1] / M[s + m - 1];
        if (m < nx - 1) v -= To[s + m] * To[s + m] / M[s + m + 1];
        if (bad(v)) return OR_ERR_BREAKDOWN;
        M[s + m] = v;
    }
    return OR_OK;
}

/* beta = (X^{-1} w) ./ w  with the R15 guard. */
static double beta_of(double xinvw, double w, double diag)
{
    if (fabs(w) < 1e-300) return 1.0 / diag;
    return xinvw / w;
}

/* Level-2 Schur term: the approximate -Lbar (2b - b T_s b) Ubar added to
 * the line block k, computed from the already factored line s (s = k-1 in
 * the top half, k+1 in the bottom half).  p = y-coupling between lines s and
 * k (length nx); t = filter on line k.  Adds into (dk, ok). */
static void line_schur(const ntd_ctx *c, int nx, long ls, const double *Td, const double *To,
                       const double *p, const double *t, double *dk, double *ok,
                       double *w, double *v, double *beta)
{
    for (int a = 0; a < nx; ++a) w[a] = p[a] * (t ? t[a] : 1.0);
    solve_block(c, ls, 1, w - ls, v - ls);                 /* v = T_s^{-1} w (exact) */
    for (int a = 0; a < nx; ++a) beta[a] = beta_of(v[a], w[a], Td[ls + a]);
    /* X = 2 beta - beta T_s beta  (tridiagonal) ; Schur term = -p X p.  With
     * c->classic, X = beta (diagonal), the approximation the recurrences'
     * 2 beta - beta T beta is presented as improving on. */
    for (int a = 0; a < nx; ++a) {
        const double xd = 2.0 * beta[a] - beta[a] * Td[ls + a] * beta[a];
        dk[a] -= p[a] * (c->classic ? beta[a] : xd) * p[a];
        if (a + 1 < nx && !c->classic) {
            const double xo = -beta[a] * To[ls + a] * beta[a + 1];
            ok[a] -= p[a] * xo * p[a + 1];
        }
    }
}

/* Level 2: factor plane z whose 5-point matrix has bands (Pd, Px, Py):
 * the T_k recurrence over lines with the twist at line my, then the level-1
 * pivots of every T_k. Writes Td, To (= l1) and M for the plane. */
static int factor_plane(const ntd_ctx *c, int z, const double *Pd, const double *Px,
                        const double *Py, const double *t, double *Td, double *To, double *M)
{
    const int nx = c->nx, ny = c->ny;
    const long p0 = (long)z * nx * ny;
    const int my = (ny - 1) / 2;
    double *w = (double *)malloc(sizeof(double) * nx * 4);
    double *v = w + nx, *beta = w + 2 * nx, *pc = w + 3 * nx;
    int st = OR_OK;
#define LINE(k) (p0 + (long)(k) * nx)
    /* top half: T_0 = Dbar_0 ; T_k = Dbar_k - L (2b - b T_{k-1} b) U */
    for (int k = 0; k < my && st == OR_OK; ++k) {
        const long s = LINE(k);
        for (int a = 0; a < nx; ++a) { Td[s + a] = Pd[s + a]; To[s + a] = Px[s + a]; }
        if (k > 0) {
            for (int a = 0; a < nx; ++a) pc[a] = Py[s - nx + a];
            line_schur(c, nx, s - nx, Td, To, pc, t ? t + s : NULL, Td + s, To + s, w, v, beta);
        }
        st = factor_line(nx, s, Td, To, M);
    }
    /* bottom half: T_{ny-1} = Dbar_{ny-1} ; T_k from T_{k+1} */
    for (int k = ny - 1; k > my && st == OR_OK; --k) {
        const long s = LINE(k);
        for (int a = 0; a < nx; ++a) { Td[s + a] = Pd[s + a]; To[s + a] = Px[s + a]; }
        if (k < ny - 1) {
            for (int a = 0; a < nx; ++a) pc[a] = Py[s + a];
            line_schur(c, nx, s + nx, Td, To, pc, t ? t + s : NULL, Td + s, To + s, w, v, beta);
        }
        st = factor_line(nx, s, Td, To, M);
    }
    /* twist line: both corrections */
    if (st == OR_OK) {
        const long s = LINE(my);
        for (int a = 0; a < nx; ++a) { Td[s + a] = Pd[s + a]; To[s + a] = Px[s + a]; }
        if (my > 0) {
            for (int a = 0; a < nx; ++a) pc[a] = Py[s - nx + a];
            line_schur(c, nx, s - nx, Td, To, pc, t ? t + s : NULL, Td + s, To + s, w, v, beta);
        }
        if (my < ny - 1) {
            for (int a = 0; a < nx; ++a) pc[a] = Py[s + a];
            line_schur(c, nx, s + nx, Td, To, pc, t ? t + s : NULL, Td + s, To + s, w, v, beta);
        }
        st = factor_line(nx, s, Td, To, M);
    }
    for (long e = p0; e < p0 + (long)nx * ny && st == OR_OK; ++e)
        if (bad(Td[e])) st = OR_ERR_BREAKDOWN;
#undef LINE
    free(w);
    return st;
}

/* Level-3 Schur term for plane k from the already factored plane s (s = k-1
 * top half, k+1 bottom half): - C (2b - b P_s b) C with C = diag(cz between
 * s and k), b = (B_{P,s}^{-1} w) ./ w, w = C t_k (R1, R2).  Adds into the
 * plane-k bands (dk, xk, yk). */
static void plane_schur(const ntd_ctx *c, long ps, const double *Pd, const double *Px,
                        const double *Py, const double *C, const double *t,
                        double *dk, double *xk, double *yk, double *w, double *v, double *beta)
{
    const int nx = c->nx, ny = c->ny;
    const long nxy = (long)nx * ny;
    for (long e = 0; e < nxy; ++e) w[e] = C[e] * (t ? t[e] : 1.0);
    solve_block(c, ps, 2, w - ps, v - ps);                 /* v = B_{P,s}^{-1} w */
    for (long e = 0; e < nxy; ++e) beta[e] = beta_of(v[e], w[e], Pd[ps + e]);
    for (long e = 0; e < nxy; ++e) {
        const int ix = (int)(e % nx), iy = (int)(e / nx);
        const double xd = 2.0 * beta[e] - beta[e] * Pd[ps + e] * beta[e];
        dk[e] -= C[e] * (c->classic ? beta[e] : xd) * C[e];
        if (c->classic) continue;                         /* X = beta: diagonal only */
        if (ix + 1 < nx) {
            const double xo = -beta[e] * Px[ps + e] * beta[e + 1];
            xk[e] -= C[e] * xo * C[e + 1];
        }
        if (iy + 1 < ny) {
            const double xo = -beta[e] * Py[ps + e] * beta[e + nx];
            yk[e] -= C[e] * xo * C[e + nx];
        }
    }
}

int or_setup(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
             const double *cz, const double *t, int classic,
             double *Pd, double *Px, double *Py, double *Td, double *To, double *M)
{
    if (nx < 1 || ny < 1 || nz < 1) return OR_ERR_ARG;
    const long nxy = (long)nx * ny, n = nxy * nz;
    if (t)
        for (long e = 0; e < n; ++e)
            if (!(t[e] > 0.0) || !isfinite(t[e])) return OR_ERR_ARG;
    ntd_ctx c;
    c.nx = nx; c.ny = ny; c.nz = nz;
    c.l[0] = NULL; c.l[1] = To; c.l[2] = Py; c.l[3] = cz;
    c.M = M;
    c.classic = classic ? 1 : 0;
    double *w = (double *)malloc(sizeof(double) * nxy * 3);
    if (!w) return OR_ERR_ALLOC;
    double *v = w + nxy, *beta = w + 2 * nxy;
    const int mz = (nz - 1) / 2;
    int st = OR_OK;
    /* P_i starts as Dhat_i (the plane blocks of A) */
    for (long e = 0; e < n; ++e) { Pd[e] = d[e]; Px[e] = cx[e]; Py[e] = cy[e]; }
#define PL(i) ((long)(i) * nxy)
    /* top half: P_0 = Dhat_0, P_i from P_{i-1} */
    for (int i = 0; i < mz && st == OR_OK; ++i) {
        if (i > 0)
            plane_schur(&c, PL(i - 1), Pd, Px, Py, cz + PL(i - 1), t ? t + PL(i) : NULL,
                        Pd + PL(i), Px + PL(i), Py + PL(i), w, v, beta);
        st = factor_plane(&c, i, Pd, Px, Py, t, Td, To, M);
    }
    /* bottom half: P_{nz-1} = Dhat_{nz-1}, P_i from P_{i+1} */
    for (int i = nz - 1; i > mz && st == OR_OK; --i) {
        if (i < nz - 1)
            plane_schur(&c, PL(i + 1), Pd, Px, Py, cz + PL(i), t ? t + PL(i) : NULL,
                        Pd + PL(i), Px + PL(i), Py + PL(i), w, v, beta);
        st = factor_plane(&c, i, Pd, Px, Py, t, Td, To, M);
    }
    /* twist plane: both Schur terms */
    if (st == OR_OK) {
        if (mz > 0)
            plane_schur(&c, PL(mz - 1), Pd, Px, Py, cz + PL(mz - 1), t ? t + PL(mz) : NULL,
                        Pd + PL(mz), Px + PL(mz), Py + PL(mz), w, v, beta);
        if (mz < nz - 1)
            plane_schur(&c, PL(mz + 1), Pd, Px, Py, cz + PL(mz), t ? t + PL(mz) : NULL,
                        Pd + PL(mz), Px + PL(mz), Py + PL(mz), w, v, beta);
        st = factor_plane(&c, mz, Pd, Px, Py, t, Td, To, M);
    }
#undef PL
    free(w);
    return st;
}


/* ------------------------------------------------------------------ */
/* ILU(0) smoother and the combination preconditioner B_c (Sec. III,   */
/* "Smoothing high frequency components of error", Eq. (com))          */
/* ------------------------------------------------------------------ */

/* ILU(0) of the block-diagonal approximation blkD(A(1:M,1:M), A(M+1:N,M+1:N)),
 * M = floor(N/2).  In natural order the 7-point pattern produces no fill that
 * ILU(0) keeps, so the factorization only changes the pivots:
 *   D_a = A_aa - sum over the lower neighbours b of a in the same block of A_ab^2 / D_b,
 * and B_ILU0 = (D + L) D^{-1} (D + U), L / U the strict lower / upper parts of blkD(A). */
int or_ilu0_setup(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
                  const double *cz, double *D)
{
    const long nxy = (long)nx * ny, n = nxy * nz, M = n / 2;
    for (long a = 0; a < n; ++a) {
        const int ix = (int)(a % nx), iy = (int)((a / nx) % ny), iz = (int)(a / nxy);
        const long lo = (a < M) ? 0 : M;           /* first row of a's block */
        double v = d[a];
        if (ix > 0 && a - 1 >= lo) v -= cx[a - 1] * cx[a - 1] / D[a - 1];
        if (iy > 0 && a - nx >= lo) v -= cy[a - nx] * cy[a - nx] / D[a - nx];
        if (iz > 0 && a - nxy >= lo) v -= cz[a - nxy] * cz[a - nxy] / D[a - nxy];
        if (bad(v)) return OR_ERR_BREAKDOWN;
        D[a] = v;
    }
    return OR_OK;
}

/* z = B_ILU0^{-1} r: forward sweep (D + L) y = r, backward sweep (I + D^{-1} U) z = y. */
int or_ilu0_solve(int nx, int ny, int nz, const double *cx, const double *cy, const double *cz,
                  const double *D, const double *r, double *z)
{
    const long nxy = (long)nx * ny, n = nxy * nz, M = n / 2;
    for (long a = 0; a < n; ++a) {
        const int ix = (int)(a % nx), iy = (int)((a / nx) % ny), iz = (int)(a / nxy);
        const long lo = (a < M) ? 0 : M;
        double v = r[a];
        if (ix > 0 && a - 1 >= lo) v -= cx[a - 1] * z[a - 1];
        if (iy > 0 && a - nx >= lo) v -= cy[a - nx] * z[a - nx];
        if (iz > 0 && a - nxy >= lo) v -= cz[a - nxy] * z[a - nxy];
        z[a] = v / D[a];
    }
    for (long a = n - 1; a >= 0; --a) {
        const int ix = (int)(a % nx), iy = (int)((a / nx) % ny), iz = (int)(a / nxy);
        const long hi = (a < M) ? M : n;             /* one past the last row of a's block */
        double v = 0.0;
        if (ix + 1 < nx && a + 1 < hi) v += cx[a] * z[a + 1];
        if (iy + 1 < ny && a + nx < hi) v += cy[a] * z[a + nx];
        if (iz + 1 < nz && a + nxy < hi) v += cz[a] * z[a + nxy];
        z[a] -= v / D[a];
    }
    return OR_OK;
}

/* B_c^{-1} r = B_NTD^{-1} r + B_ILU0^{-1} r - B_NTD^{-1} A B_ILU0^{-1} r
 *            = y1 + B_NTD^{-1} (r - A y1),  y1 = B_ILU0^{-1} r. */
int or_combo_apply(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
                   const double *cz, const double *l2, const double *l1, const double *M,
                   const double *Dilu, const double *r, double *z)
{
    const long n = (long)nx * ny * nz;
    double *y1 = (double *)malloc(sizeof(double) * n * 2);
    if (!y1) return OR_ERR_ALLOC;
    double *w = y1 + n;
    or_ilu0_solve(nx, ny, nz, cx, cy, cz, Dilu, r, y1);
    or_spmv(nx, ny, nz, d, cx, cy, cz, y1, w);
    for (long e = 0; e < n; ++e) w[e] = r[e] - w[e];
    or_apply(nx, ny, nz, cz, l2, l1, M, w, z);
    for (long e = 0; e < n; ++e) z[e] += y1[e];
    free(y1);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* PCG / flexible CG (Sec. III conventions, readings R17 and R19)      */
/* ------------------------------------------------------------------ */

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long e = 0; e < n; ++e) s += a[e] * b[e];
    return s;
}

int or_pcg(int nx, int ny, int nz, const double *d, const double *cx, const double *cy,
           const double *cz, const double *l2, const double *l1, const double *M,
           const double *Dilu, const double *b, double *x, double rtol, int maxit, int flexible,
           int *iters_out, double *relres_out, double *alpha_hist, double *beta_hist,
           double *res_hist)
{
    const long n = (long)nx * ny * nz;
    double *r = (double *)malloc(sizeof(double) * n * 5);
    if (!r) return OR_ERR_ALLOC;
    double *z = r + n, *p = r + 2 * n, *q = r + 3 * n, *rold = r + 4 * n;
    const double bnorm = sqrt(dot(n, b, b));
    int it = 0, st = OR_OK;
    *iters_out = 0;
    if (bnorm == 0.0) {
        for (long e = 0; e < n; ++e) x[e] = 0.0;
        *relres_out = 0.0;
        free(r);
        return OR_OK;
    }
    /* r = b - A x0 */
    or_spmv(nx, ny, nz, d, cx, cy, cz, x, q);
    for (long e = 0; e < n; ++e) r[e] = b[e] - q[e];
    double rnorm = sqrt(dot(n, r, r));
    double rho = 0.0;
    int fresh = 1;                                        /* (re)start direction */
    while (1) {
        if (rnorm / bnorm < rtol) {
            /* R17: confirm with the true residual */
            or_spmv(nx, ny, nz, d, cx, cy, cz, x, q);
            for (long e = 0; e < n; ++e) r[e] = b[e] - q[e];
            rnorm = sqrt(dot(n, r, r));
            if (rnorm / bnorm < rtol) break;
            fresh = 1;
        }
        if (it >= maxit) { st = OR_ERR_NOT_CONVERGED; break; }
        if (Dilu) or_combo_apply(nx, ny, nz, d, cx, cy, cz, l2, l1, M, Dilu, r, z);
        else or_apply(nx, ny, nz, cz, l2, l1, M, r, z);
        const double rho_new = dot(n, r, z);
        if (fresh) {
            for (long e = 0; e < n; ++e) p[e] = z[e];
            fresh = 0;
            if (beta_hist) beta_hist[it] = 0.0;
        } else {
            double beta;
            if (flexible) beta = (rho_new - dot(n, z, rold)) / rho;
            else beta = rho_new / rho;
            if (beta_hist) beta_hist[it] = beta;
            for (long e = 0; e < n; ++e) p[e] = z[e] + beta * p[e];
        }
        rho = rho_new;
        or_spmv(nx, ny, nz, d, cx, cy, cz, p, q);
        const double pq = dot(n, p, q);
        if (!(pq > 0.0)) { st = OR_ERR_BREAKDOWN; break; }
        const double alpha = rho / pq;
        if (alpha_hist) alpha_hist[it] = alpha;
        if (flexible) for (long e = 0; e < n; ++e) rold[e] = r[e];
        for (long e = 0; e < n; ++e) { x[e] += alpha * p[e]; r[e] -= alpha * q[e]; }
        rnorm = sqrt(dot(n, r, r));
        ++it;
        if (res_hist) res_hist[it - 1] = rnorm / bnorm;
    }
    *iters_out = it;
    /* final true residual */
    or_spmv(nx, ny, nz, d, cx, cy, cz, x, q);
    for (long e = 0; e < n; ++e) r[e] = b[e] - q[e];
    *relres_out = sqrt(dot(n, r, r)) / bnorm;
    free(r);
    return st;
}
