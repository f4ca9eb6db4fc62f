/*
 * ffp.h -- C ABI of the GB300 (sm_103a) library libffp.so: preconditioned
 * conjugate gradients for the variable-coefficient 7-point finite-volume
 * diffusion operator on a structured 3-D grid, preconditioned by the nested
 * twisted frequency-filtering preconditioner (NTD) of arXiv 1909.09771.
 *
 * Conventions (all entry points)
 *   - Grid index a = x + nx*(y + ny*z): x fastest, then y (lines), then z
 *     (planes).  This is the ordering of the nested block-tridiagonal matrix
 *     in Sec. II of the paper (nx cells per line, ny lines per plane, nz planes).
 *   - Every vector argument is a DEVICE pointer to N = nx*ny*nz FP64 values,
 *     owned by the caller; the library never allocates, frees or keeps device
 *     memory beyond the caller's workspace, and never copies to the host
 *     except the small status/scalar block of ffp_pcg_solve.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call enqueues its kernels on that stream; only
 *     ffp_setup (status check) and ffp_pcg_solve (convergence checks)
 *     synchronise it.
 *   - Return value: FFP_OK (0) or a negative FFP_ERR_* code; ffp_strerror()
 *     names it.  On an error the output buffers hold unspecified values.
 *   - Only one GPU (the current device at ffp_setup) is used.
 */
#ifndef FFP_H
#define FFP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FFP_OK 0
#define FFP_ERR_ARG (-1)            /* bad argument: null pointer, n < 1, nx > FFP_MAX_NX,
                                       kappa or t not positive and finite, workspace too small */
#define FFP_ERR_CUDA (-2)           /* a CUDA runtime call failed */
#define FFP_ERR_BREAKDOWN (-3)      /* a non-positive / non-finite pivot or diagonal in setup,
                                       or (p, Ap) <= 0 in CG */
#define FFP_ERR_NOT_CONVERGED (-4)  /* maxit reached, or the true residual stopped falling;
                                       x holds the last iterate */
#define FFP_ERR_TIMEOUT (-5)        /* a bounded wait inside a kernel gave up (results unusable) */
#define FFP_ERR_UNSUPPORTED (-6)    /* the requested option is not available */

#define FFP_MAX_NX 1024             /* longest line (cells along x) the line solvers support */

/* boundary condition per face */
#define FFP_DIRICHLET 0             /* u = 0 on the face (Sec. I Eq. (2)) */
#define FFP_NEUMANN 1               /* du/dn = 0 on the face */

/* filter vector t of the filtering property B t = A t (Sec. I Eq. (3)) */
#define FFP_FILTER_ROWSUM 0         /* t = 1, the rowsum constraint (Sec. I Eq. (4)) */
#define FFP_FILTER_USER 1           /* caller-supplied t, device FP64 [N], every entry > 0 */

/* preconditioner */
#define FFP_PRECOND_NTD 0           /* B_NTD, the nested twisted filtering preconditioner (Sec. II) */
#define FFP_PRECOND_COMBO 1         /* B_c^{-1} = B_NTD^{-1} + B_ILU0^{-1} - B_NTD^{-1} A B_ILU0^{-1},
                                       ILU(0) of blkD(A) split at M = floor(N/2) (Sec. III, Eq. (com)),
                                       the preconditioner of the paper's experiments */

/* Option OR'ed into `precond`: the approximate inverse X of the eliminated
 * block in the Schur terms of the plane and line recurrences (Sec. II-A).  By
 * default X = 2 beta - beta P beta, the form the recurrences print, which the
 * paper presents as an improvement on beta alone.  With FFP_SCHUR_BETA,
 * X = beta = diag((P^{-1} w) ./ w), the classical filtering approximation: the
 * Schur terms then change only the diagonals of P_i and T_k, and the filtering
 * property X w = P^{-1} w holds all the same. */
#define FFP_SCHUR_BETA 16

/* storage and arithmetic precision of the preconditioner factors */
#define FFP_FP64 0                  /* FP64 factors, FP64 apply, standard PCG (flexible CG with B_c) */
#define FFP_FP32 1                  /* FP32 factors, FP32 apply, FP64 flexible CG */
#define FFP_BF16 2                  /* BF16 factors, FP32 apply, FP64 flexible CG */

/* Structured grid on the box [0,lx] x [0,ly] x [0,lz] (lengths <= 0 mean 1). */
typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
} ffp_grid;

/* Boundary flag per face, order x-, x+, y-, y+, z-, z+; FFP_DIRICHLET or FFP_NEUMANN. */
typedef struct {
    unsigned char face[6];
} ffp_bc;

/* Result of ffp_pcg_solve. */
typedef struct {
    int iters;            /* CG iterations (products A p) after the initial residual */
    int status;           /* same value the call returns */
    double rel_res;       /* recursive ||r|| / ||b|| at exit */
    double rel_res_true;  /* ||b - A x|| / ||b|| recomputed at exit */
    double solve_s;       /* wall time of the solve (host clock, after a stream sync) */
    double precond_ms;    /* device time of all preconditioner applies (CUDA events on `stream`) */
    double ntd_ms;        /* device time of their B_NTD sweeps: the three apply kernel launches
                             of each apply, precision conversions excluded */
    int napply;           /* number of preconditioner applies */
    long long launches;   /* kernels this call launched */
    int iters_rec;        /* first iteration at which the recursive ||r|| / ||b|| fell below rtol
                             (-1 if it never did); iters can be larger when the true residual,
                             checked then, was not yet below rtol and the solve went on */
    double spmv_ms;       /* device time of the iterations' q = A p launches (fused with
                             (p, q)), CUDA events on `stream`; 0 in batched solves */
    double lanczos_min;   /* extreme eigenvalues of the Lanczos tridiagonal of B^{-1} A that the
                             CG coefficients define (diagonal 1/alpha_k + beta_k/alpha_{k-1},
                             off-diagonal sqrt(beta_k)/alpha_{k-1}, beta_k the coefficient that */
    double lanczos_max;   /* formed p_k), over the iterations before the first restart; their
                             ratio estimates cond(B^{-1} A).  With flexible CG it is an estimate
                             of the same quantity.  0 when fewer than one iteration ran or in
                             batched solves */
} ffp_stats;

typedef struct ffp_handle ffp_handle;

/* Bytes of device workspace ffp_setup needs for this grid and factor precision
 * (0 on a bad grid).  The workspace holds the operator bands, the factors, the
 * CG vectors and small scratch; its base must be 256-byte aligned. */
size_t ffp_workspace_bytes(const ffp_grid *grid, int precision);

/* Assemble A from kappa and build the NTD preconditioner.
 *
 * Operator (Sec. I Eq. (2), finite-volume reading): face coefficient
 * kappa_f * area / distance, kappa_f the harmonic mean 2 ka kb / (ka + kb)
 * of the two cells; a Dirichlet face contributes 2 kappa * area / h (half a
 * cell to the face); a Neumann face nothing; the diagonal is the sum of the
 * cell's face coefficients.
 *
 * Preconditioner (Sec. II-A): twisted block factorizations at three nested
 * levels -- planes (P_i recurrence with the approximate inverse
 * 2 beta - beta P beta), lines of every plane (T_k recurrence, same form) and
 * cells of every line (exact twisted pivots M_i) -- with the twist block
 * m = floor((n-1)/2) at every level, beta = diag((X^{-1} w) ./ w), w = coupling
 * times t restricted to the block being built; the plane inverse inside the
 * level-3 beta is the nested level-2 solve of that plane.  With
 * FFP_PRECOND_COMBO the ILU(0) pivots of blkD(A) are built too (Sec. III).
 * The factors are computed in FP64 and stored in `precision`.
 *
 *   grid       nx, ny, nz >= 1, nx <= FFP_MAX_NX
 *   kappa      device FP64 [N], > 0 and finite (else FFP_ERR_ARG)
 *   bc         host pointer to the 6 face flags
 *   filter     FFP_FILTER_ROWSUM (t ignored, may be NULL) or FFP_FILTER_USER
 *   t          device FP64 [N] filter vector (entries > 0, else FFP_ERR_ARG)
 *   precision  FFP_FP64, FFP_FP32 or FFP_BF16
 *   precond    FFP_PRECOND_NTD or FFP_PRECOND_COMBO, optionally | FFP_SCHUR_BETA
 *   workspace  device memory of ws_bytes >= ffp_workspace_bytes(grid, precision),
 *              owned by the caller and kept alive until ffp_destroy
 *   out        receives a host handle (freed by ffp_destroy)
 * Synchronises `stream` once to read the setup status.  Returns
 * FFP_ERR_BREAKDOWN if a pivot or diagonal is not positive and finite. */
int ffp_setup(const ffp_grid *grid, const double *kappa, const ffp_bc *bc, int filter,
              const double *t, int precision, int precond, void *workspace, size_t ws_bytes,
              void *stream, ffp_handle **out);

/* y = A x (device FP64 [N] each; x and y must not overlap).  Sec. II: the 7-point
 * band storage of A. */
int ffp_spmv(ffp_handle *h, const double *x, double *y, void *stream);

/* z = B^{-1} r (device FP64 [N] each; r and z must not overlap).
 * B_NTD: Sec. II-B Algorithms 1-7, SOLVE(1, N, x, y, n^2, 3) -- a twisted
 * lower then upper sweep over planes, each plane solved by the same two sweeps
 * over its lines, each line by the twisted tridiagonal solve.
 * B_c (FFP_PRECOND_COMBO): y = B_ILU0^{-1} r, z = y + B_NTD^{-1} (r - A y).
 * Arithmetic in FP64 (FFP_FP64) or FP32 (FFP_FP32, FFP_BF16). */
int ffp_apply(ffp_handle *h, const double *r, double *z, void *stream);

/* Solve A x = b by preconditioned CG (Sec. III: x0 given, stop when
 * ||r|| / ||b|| < rtol, then confirm with the true residual ||b - A x|| / ||b||
 * and continue from it if it is not below rtol; at most maxit iterations).
 * FFP_FP64 with B_NTD runs standard PCG; FP32/BF16 factors or B_c (not
 * symmetric) run flexible CG, beta = (z_new, r_new - r_old) / (z_old, r_old).  All CG vectors, dot
 * products and scalars are FP64.
 *   b      device FP64 [N]
 *   x      device FP64 [N]: in x0, out the solution (b = 0 gives x = 0, 0 iterations)
 *   stats  host pointer or NULL
 * Returns FFP_ERR_NOT_CONVERGED at maxit, or when three confirmations in a row
 * fail to halve the best true residual (rtol below what an FP64 iterate can
 * reach, about eps |A||x| / |b|); FFP_ERR_BREAKDOWN if (p, A p) <= 0. */
int ffp_pcg_solve(ffp_handle *h, const double *b, double *x, double rtol, int maxit,
                  ffp_stats *stats, void *stream);

/* Copy the stored operator and factors out as FP64 device arrays [N] each (any
 * pointer may be NULL): d, cx, cy, cz = bands of A (cx[a] = A[a, a+1], cy[a] =
 * A[a, a+nx], cz[a] = A[a, a+nx*ny], zero where there is no neighbour); the
 * band storage of Sec. II-A in the stored precision: l3 = z-band of A, l2 =
 * y-band of every P_i, l1 = x-band of every T_k, minv = 1 / M (level-1
 * pivots); dinv = 1 / D, the ILU(0) pivots (B_c only, else left untouched). */
int ffp_export(ffp_handle *h, double *d, double *cx, double *cy, double *cz, double *l3,
               double *l2, double *l1, double *minv, double *dinv, void *stream);

/* Allocation-free apply.  The paper has no counterpart: this exists for callers
 * that cannot allocate device memory at the point where they apply the
 * preconditioner -- for example code running under a host framework that owns
 * every device allocation (a fixed memory pool, an inference runtime, a plugin
 * inside another program's CUDA context), or code that must not call
 * cudaMalloc at all in its steady state.  Such a caller can still build the
 * handle once (its workspace is caller memory, allocated however the caller
 * may) and then call this entry point, which calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * It computes z = B_NTD^{-1} r with the same kernels as ffp_apply, using the
 * handle's factors; for a handle built with FFP_PRECOND_COMBO it applies only
 * the nested sweeps B_NTD^{-1}, not the combination B_c.  The two planes of
 * scratch the upper sweeps need live in a fixed array in the library's device
 * image (2 * FFP_NOALLOC_MAX_PLANE FP64 values, 2 MiB), which every GPU that
 * loads the library holds until the process exits.
 *   h       handle from ffp_setup; its device must be the current device
 *   r, z    device FP64 [N], distinct (as for ffp_apply)
 * Returns FFP_ERR_ARG if the grid's planes do not fit the fixed scratch -- if
 * nx * ny > FFP_NOALLOC_MAX_PLANE, or if one plane in the apply's line-block
 * layout takes more than FFP_NOALLOC_MAX_PLANE * 8 bytes.  That plane holds
 * ny * (32 * SP + 32) values of the apply's arithmetic type (FP64 for FP64
 * factors, FP32 otherwise), where S is the smallest of 1, 2, 3, 4, 6, 8, 11,
 * 16, 22, 32 with 16 S >= nx - 1 - floor((nx - 1) / 2) and SP is S rounded up
 * to a multiple of 4 (for example nx = 3, ny = 1000 with FP64 factors needs
 * 1000 * 160 * 8 bytes and is rejected).  It also returns FFP_ERR_ARG if the
 * current device is not the handle's.
 * The first call on a device looks up the array's device address in the
 * device's primary context (the one the CUDA runtime uses) and caches it for
 * the life of the process; make that first call before any stream capture on
 * that device.  cudaDeviceReset destroys that context, and the cached address
 * with it: do not call this entry point again after a reset of its device.
 * All calls share the one array: calls whose kernels overlap on the GPU (on
 * different streams, or from several host threads) race on it and must be
 * serialised by the caller.  Nothing in the array needs clearing: each call
 * writes every scratch entry before reading it. */
#define FFP_NOALLOC_MAX_PLANE 131072
int ffp_apply_noalloc(ffp_handle *h, const double *r, double *z, void *stream);

/* Test hook for the failure path (the paper has no counterpart).  Every wait
 * inside the apply kernels -- a compute warp waiting for its producer to fill a
 * shared-memory stage, a producer waiting for a stage to be released -- gives
 * up after a fixed number of tries, records a timeout flag and lets the kernel
 * run to its end, so a broken hand-off yields FFP_ERR_TIMEOUT from
 * ffp_pcg_solve instead of a hung GPU.  This call lets a test exercise that
 * path without faulting anything:
 *   mode 1      in every following apply of this handle, one producer warp
 *               of the first level-3 half withholds its first "stage full"
 *               signal, so its compute warp's wait runs out (the apply's
 *               result is then unusable); mode 0 restores normal operation
 *   wait_tries  try limit of those waits while set (0 = the library default,
 *               about 4 M tries); a small value makes the timeout quick
 * Returns FFP_ERR_ARG for a null handle or an unknown mode. */
int ffp_debug_stall(ffp_handle *h, int mode, unsigned wait_tries);

/* Free the host handle (no device memory is freed). */
void ffp_destroy(ffp_handle *h);

/* ------------------------------------------------------------------------
 * Batched solves: many independent problems at once.  The paper solves one
 * problem at a time; batching is this library's way of filling one GPU with
 * the independent level-3 chains of many problems.  A batch holds `count`
 * instances, each with its own grid (uneven sizes allowed), kappa, boundary
 * conditions and preconditioner (Sec. II / III, as built by ffp_setup), and
 * `nrhs` right-hand sides per instance; a "pair" is one (instance, right-hand
 * side), numbered i * nrhs + j.  Every pair's result is the one its
 * standalone ffp_setup + ffp_pcg_solve would give with the same arguments
 * (same iterations; the same solution up to rounding of an identical
 * sequence of operations).
 * ------------------------------------------------------------------------ */
typedef struct ffp_batch ffp_batch;

#define FFP_BATCH_MAX_PAIRS 65535  /* count * nrhs (the pair is a grid's y index) */

/* Launch configuration chosen by ffp_batch_tune.  It never changes a result. */
typedef struct {
    int ilu_warps;   /* warps per CTA of the ILU(0) sweeps (1..8; each warp walks one plane at a time) */
    int branches;    /* 1: the slot-count groups run as parallel graph branches; 0: in sequence */
    double ms;       /* mean time (ms) of one preconditioner application to every pair
                        under this configuration, as timed by ffp_batch_tune */
    double ntd_ms;   /* mean time (ms) of the B_NTD sweeps alone (3 launches per group) */
    int from_cache;  /* 1 if read from the tuning cache */
    int rhs_per_cta; /* 1, or 2: two right-hand sides of an instance share one chain of apply
                        CTAs (one stage of factor records, two pairs of compute warps); only in
                        groups where every instance's right-hand sides pair up and the two-RHS
                        kernels are built (FP32/BF16 factors, short lines), else 1 is used */
} ffp_batch_config;

/* Bytes of the one device workspace of a batch (0 for invalid arguments).
 *   grids  host array [count]; precision as for ffp_workspace_bytes */
size_t ffp_batch_workspace_bytes(int count, const ffp_grid *grids, int nrhs, int precision);

/* Assemble and set up every instance, on `stream`, and return a host handle.
 *   grids, bcs  host arrays [count]
 *   kappa       host array [count] of device FP64 [N_i] pointers
 *   t           NULL (rowsum filters), or a host array [count] of device FP64
 *               [N_i] filter pointers, NULL entries meaning rowsum
 *   precision, precond  as for ffp_setup, for every instance
 *   workspace   device memory, 256-byte aligned, >= ffp_batch_workspace_bytes
 * Calls no device allocator; it creates streams and events and pins a little
 * host memory.  Returns FFP_ERR_ARG, FFP_ERR_BREAKDOWN (some instance's setup
 * broke down) or FFP_ERR_CUDA, and then no handle. */
int ffp_batch_setup(int count, const ffp_grid *grids, const double *const *kappa,
                    const ffp_bc *bcs, const double *const *t, int nrhs, int precision,
                    int precond, void *workspace, size_t ws_bytes, void *stream, ffp_batch **out);

/* Choose the launch configuration (ILU(0) warps per CTA, branches, right-hand
 * sides per apply CTA) by timing the batched preconditioner on this batch (it
 * overwrites the pairs' internal vectors, none of the caller's).
 * cache_path: NULL, or a text file of "<key> <ilu_warps> <branches> <ms> <ntd_ms>
 * <rhs_per_cta>" lines; a line whose key (GPU, precision, preconditioner, grids, nrhs)
 * matches is used without timing (ms and ntd_ms are then the cached ones),
 * else the choice is appended.  out may be NULL.  A batch that is never tuned
 * uses ilu_warps 4, branches 1, rhs_per_cta 1. */
int ffp_batch_tune(ffp_batch *B, const char *cache_path, ffp_batch_config *out, void *stream);
int ffp_batch_get_config(const ffp_batch *B, ffp_batch_config *cfg);
int ffp_batch_set_config(ffp_batch *B, const ffp_batch_config *cfg);

/* Groups (pairs of one slot count), pairs, kernels one batched CG iteration
 * launches, and kernels ffp_batch_setup launched.  Any output pointer may be NULL. */
int ffp_batch_info(const ffp_batch *B, int *ngroups, int *npairs, long long *launches_per_iter,
                   long long *setup_launches);

/* Solve every pair: PCG / flexible CG exactly as ffp_pcg_solve, all pairs
 * advancing together, each stopping on its own test.  One iteration of all
 * pairs is one CUDA graph launch, captured on the first solve and kept
 * until the configuration changes.
 *   b, x   host arrays [count * nrhs] of device FP64 [N_i] pointers (x: in x0,
 *          out the solution), indexed by pair
 *   stats  NULL or host array [count * nrhs]
 * The solve is synchronous: it waits for prior work on `stream`, and returns
 * once every pair is done.  It returns FFP_OK if every pair converged, else
 * the first failing pair's status (per-pair status in stats).  Calls on one
 * batch must not overlap. */
int ffp_batch_solve(ffp_batch *B, const double *const *b, double *const *x, double rtol, int maxit,
                    ffp_stats *stats, void *stream);

/* Free the batch's host state, streams, events and graphs (not the workspace). */
void ffp_batch_destroy(ffp_batch *B);

/* ------------------------------------------------------------------------
 * Learned filter.  Sec. I: a preconditioner with B t = A t removes the error
 * component along t, and the components hardest to damp lie along the
 * eigenvectors of the smallest eigenvalues of B^{-1}A, so t should
 * approximate those; the paper itself uses t = 1.  The library can learn t:
 * a 3-D convolutional network maps log10(kappa) to t, trained on targets
 * built from Lanczos Ritz vectors of B_rowsum^{-1} A.  The network is not in
 * the paper.  Its t is passed to ffp_setup as FFP_FILTER_USER; PCG still
 * solves to the same tolerance, so correctness never depends on it.
 *
 * Network: x0 = log10(kappa) / 3; four 3x3x3 convolutions with zero padding,
 * channels 1 -> 16 -> 16 -> 16 -> 1, ReLU after the first three; output s,
 * t = exp(s).  Parameters: FP32 [FFP_NET_PARAMS], per layer the weights
 * w[out][in][dz][dy][dx] then the biases (offsets 0, 432 | 448, 7360 |
 * 7376, 14288 | 14304, 14736).  The convolutions run on the tensor cores:
 * BF16 copies of the weights (`wbf16`, the BF16 bit patterns, kept in step by
 * ffp_net_cast or ffp_net_adam), BF16 features, activations and back-
 * propagated gradients between layers, FP32 accumulation; s and the loss are
 * FP32, the weight-gradient partial sums are folded in FP64.  Batches hold
 * `batch` instances of one grid, instance-major: kappa [batch][N]; nx is at
 * most FFP_NET_MAX_NX (a staged row of the padded grid must fit in shared
 * memory).  Every call returns FFP_ERR_TIMEOUT if one of the kernels' bounded
 * waits ran out.
 * ------------------------------------------------------------------------ */
#define FFP_NET_PARAMS 14737
#define FFP_NET_MAX_NX 1000

/* Workspace bytes for a forward pass (train = 0) or a gradient (train = 1);
 * 0 for a bad grid or batch. */
size_t ffp_net_workspace_bytes(const ffp_grid *grid, int batch, int train);

/* He-normal weights (std sqrt(2 / (27 * in))) from a host generator seeded by
 * `seed`, zero biases, and their BF16 copy.  Synchronises `stream`. */
int ffp_net_init(unsigned long long seed, float *params, unsigned short *wbf16, void *stream);

/* wbf16 = BF16(params) (round to nearest even). */
int ffp_net_cast(const float *params, unsigned short *wbf16, void *stream);

/* t = exp(clamp(s, -30, 30)) [batch][N] FP64 device, s the network's output.
 * Synchronises `stream` (it reads the kernels' timeout flag). */
int ffp_net_forward(const ffp_grid *grid, int batch, const double *kappa, const float *params,
                    const unsigned short *wbf16, void *workspace, size_t ws_bytes, double *t,
                    void *stream);

/* Gradient of L = mean over cells of (s - s_target)^2 w.r.t. every parameter
 * (through the BF16 weights the forward pass used), into grad FP32
 * [FFP_NET_PARAMS] (device); loss: host pointer or NULL.  Synchronises
 * `stream`.  s_target: FP32 [batch][N] device. */
int ffp_net_grad(const ffp_grid *grid, int batch, const double *kappa, const float *s_target,
                 const float *params, const unsigned short *wbf16, void *workspace,
                 size_t ws_bytes, float *grad, double *loss, void *stream);

/* One Adam step (b1 0.9, b2 0.999, eps 1e-8; step = 1, 2, ... for the bias
 * correction) on params with moments m, v (FP32 device, start at zero), and
 * the new BF16 copy. */
int ffp_net_adam(float *params, unsigned short *wbf16, float *m, float *v, const float *grad,
                 int step, double lr, void *stream);

/* Lanczos on B_NTD^{-1} A (self-adjoint in the A-inner product) with full
 * re-orthogonalisation, from start vector v0 (device FP64 [N]), at most m
 * steps (m <= 64): Ritz values theta (host [m], ascending; *steps of them are
 * set) and the A-normalised Ritz vectors of the nvec <= 8 smallest, Y (device
 * FP64 [nvec][N]).  For a handle built with FFP_PRECOND_COMBO the nested
 * sweeps B_NTD^{-1} alone are used.  scratch: device, 256-byte aligned, >=
 * ffp_lanczos_scratch_bytes(grid, m).  Synchronises `stream` at every step.
 * FFP_ERR_BREAKDOWN if v0 has no positive A-norm. */
size_t ffp_lanczos_scratch_bytes(const ffp_grid *grid, int m);
int ffp_lanczos_ritz(ffp_handle *h, const double *v0, int m, int nvec, void *scratch,
                     size_t scratch_bytes, double *theta, double *Y, int *steps, void *stream);

/* Training target of the learned filter from nvec Ritz pairs (theta host
 * [nvec] > 0, Y device [nvec][N]): t* = sqrt(sum_k (theta_0 / theta_k)
 * (y_k / max|y_k|)^2), scaled to max 1 and floored at floor_ (0 < floor_ <=
 * 1), into t (device FP64 [N]); s = log t* minus its mean into s (device FP32
 * [N]).  scratch as for ffp_lanczos_ritz with m = 1 or more.  Synchronises
 * `stream`. */
int ffp_filter_target(const ffp_grid *grid, int nvec, const double *theta, const double *Y,
                      double floor_, double *t, float *s, void *scratch, size_t scratch_bytes,
                      void *stream);

/* Static text for a status code. */
const char *ffp_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* FFP_H */
