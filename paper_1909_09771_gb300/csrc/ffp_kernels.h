// ffp_kernels.h -- host-side launch interface between the C ABI (ffp_api.cu)
// and the kernel translation units.  Internal to libffp.so.
#pragma once

#include <cuda_runtime.h>

#include "ffp_internal.cuh"

namespace ffp {

struct KernelCtx {
    int nx, ny, nz;
    long long n;    // nx*ny*nz
    double lx, ly, lz;
    int prec;       // FFP_FP64 / FFP_FP32 / FFP_BF16
    int precond;    // FFP_PRECOND_NTD / FFP_PRECOND_COMBO
    int slots;      // S of the line solver
    int schur;      // approximate inverse in the Schur terms: 0 = 2 beta - beta P beta, 1 = beta
    Ws ws;
    // test hook (ffp_debug_stall): 1 = the apply withholds one stage signal;
    // try limit of the apply's waits (0 = kWaitTries)
    int dbg_stall;
    unsigned dbg_tries;
};

// ffp_api.cu: bytes per stored factor value, and the workspace layout (base may
// be null to size it; S_force > 0 forces the line slot count)
size_t prec_bytes(int prec);
// ffp_api.cu: the kernel context and device of a handle
const KernelCtx *handle_ctx(const ffp_handle *h);
int handle_device(const ffp_handle *h);
size_t carve_workspace(const ffp_grid *g, int prec, int S_force, char *base, Ws *ws);

// ffp_ops.cu
cudaError_t launch_assemble(const KernelCtx &c, const double *kappa, const unsigned char bc[6],
                            cudaStream_t st);
cudaError_t launch_check_filter(const KernelCtx &c, const double *t, cudaStream_t st);
cudaError_t launch_convert_bands(const KernelCtx &c, cudaStream_t st);  // l3 (and lx, ly for B_c)
cudaError_t launch_resid_vec(const KernelCtx &c, const double *r, const double *y, double *w,
                             cudaStream_t st);                           // w = r - A y
cudaError_t launch_add(const KernelCtx &c, double *z, const double *y, cudaStream_t st);  // z += y
// natural-order FP64 x -> the apply's line-block layout in its arithmetic type (ws.ra
// layout), and back (y = value + add, add optional)
cudaError_t launch_to_lb(const KernelCtx &c, const double *x, void *xb, cudaStream_t st);
cudaError_t launch_from_lb(const KernelCtx &c, const void *xb, double *y, const double *add,
                           cudaStream_t st);
cudaError_t launch_spmv(const KernelCtx &c, const double *x, double *y, cudaStream_t st);
cudaError_t launch_export(const KernelCtx &c, const void *src, double *dst, cudaStream_t st);
// natural-order band from the factor records: 0 = l1, 1 = 1/M, 2 = l2, 3 = l3
cudaError_t launch_export_rec(const KernelCtx &c, int what, double *dst, cudaStream_t st);
// CG building blocks (FP64); each fills ws.red with per-block partial sums and
// finalize() folds them, in a fixed order, into the scalar block ws.scal.
cudaError_t launch_resid(const KernelCtx &c, const double *b, const double *x, cudaStream_t st);
cudaError_t launch_spmv_dot(const KernelCtx &c, cudaStream_t st);
cudaError_t launch_update_xr(const KernelCtx &c, double *x, cudaStream_t st);
cudaError_t launch_dot_rz(const KernelCtx &c, cudaStream_t st);
cudaError_t launch_update_p(const KernelCtx &c, int fresh, cudaStream_t st);
enum FinalizeMode { FIN_RESID = 0, FIN_PQ = 1, FIN_RR = 2, FIN_RZ = 3 };
cudaError_t launch_finalize(const KernelCtx &c, int mode, int fresh, int flexible, cudaStream_t st);

// ffp_setup.cu
cudaError_t launch_setup(const KernelCtx &c, const double *t, cudaStream_t st);

// One instance of the setup kernels.
struct SetupArgs {
    int nx, ny, nz;
    int prec;  // storage precision of the factor records
    int schur; // 0: X = 2 beta - beta P beta (Sec. II-A as printed); 1: X = beta
    const double *d, *cx, *cy, *cz;
    const double *t;  // filter, NULL = rowsum
    void *rec;        // factor line records (rec_len(S) entries per line)
    void *l1n;        // natural-order x-band of T (for export)
    Ws ws;
};

inline void fill_setup_args(const KernelCtx &c, const double *t, SetupArgs *a) {
    a->nx = c.nx; a->ny = c.ny; a->nz = c.nz; a->prec = c.prec; a->schur = c.schur;
    a->d = c.ws.d; a->cx = c.ws.cx; a->cy = c.ws.cy; a->cz = c.ws.cz;
    a->t = t;
    a->rec = c.ws.rec;
    a->l1n = c.ws.l1;
    a->ws = c.ws;
}

// ffp_dispatch.cu: setup of every instance of a device table whose lines all use `slots`
cudaError_t launch_setup_table(int slots, const SetupArgs *table, int count, int nx_max,
                               cudaStream_t st);

// One (instance, right-hand side) pair of the NTD apply.  Vectors r, z, scr are
// in the line-block layout (lb_pos) and the compute type (FP64 for FP64
// factors, FP32 otherwise).
struct ApplyArgs {
    int nx, ny, nz;
    const void *rec;  // factor line records
    const void *l3n;  // natural-order z-band
    const void *r;
    void *z;
    void *scr;        // 2 planes
    int *flags;
    const int *ctl;   // batched solves: the pair is skipped unless *ctl & 1 (null: always run)
    // a second right-hand side of the same instance (the two-RHS form of the batched
    // apply): its vectors, scratch, flags and control word (unused with one RHS)
    const void *r1;
    void *z1;
    void *scr1;
    int *flags1;
    const int *ctl1;
    unsigned wait_tries;  // try limit of every mbarrier wait (kWaitTries; lowered by a test)
    int stall;        // test hook: 1 = the first producer of the first level-3 half withholds
                      // its first "stage full" signal in phase 0, so a compute warp's wait runs out
};

// ffp_dispatch.cu: NTD apply of every entry of a device table (one launch per phase); nr =
// right-hand sides per entry (2: the entry's second pair in r1, z1, scr1, flags1, ctl1)
cudaError_t launch_apply_table(int prec, int slots, const ApplyArgs *table, int n, int nx_max, int nr,
                               cudaStream_t st);
// whether the two-RHS form of the apply is built for this precision and slot count
bool apply_two_rhs_ok(int prec, int slots);

// ffp_dispatch.cu: z = B_NTD^{-1} r (+ add, optional); ev (optional) = two events
// recorded just before and just after the three sweep launches
cudaError_t launch_apply(const KernelCtx &c, const double *r, double *z, cudaStream_t st,
                         const cudaEvent_t *ev = nullptr, const double *add = nullptr);

// ffp_ilu.cu: ILU(0) of blkD(A) (pivots in D64 scratch, 1/D stored) and t = B_ILU0^{-1} r
cudaError_t launch_ilu_setup(const KernelCtx &c, double *D64, cudaStream_t st);

// One instance of the ILU(0) pivot wavefront.
struct IluPivArgs {
    int nx, ny, nz, prec;
    const double *d, *cx, *cy, *cz;
    double *D64;  // FP64 pivots (scratch)
    void *dinv;   // 1/D in storage precision
    int *flags;
};
cudaError_t launch_ilu_setup_table(int slots, const IluPivArgs *table, int count, int ndiag,
                                   int maxlines, cudaStream_t st);
cudaError_t launch_ilu_solve(const KernelCtx &c, const double *r, double *t, cudaStream_t st);
int ilu_slots(int nx);  // lane split of the ILU(0) line sweeps
long long ilu_solve_launches(const KernelCtx &c);  // kernels one launch_ilu_solve launches

// One pair of the ILU(0) solve t = B_ILU0^{-1} r; factors in storage precision.
struct IluArgs {
    int nx, ny, nz;
    const void *dinv, *lx, *ly, *lz;  // 1/D and the x, y, z bands of A
    const void *r;                    // right-hand side, FP64 (FP32 in the column and
    void *t;                          // dataflow forms with FP32/BF16 factors); result
    double *out64;   // column forms, backward sweep: the result also stored here in FP64 (or null)
    const int *ctl;  // table form: the pair is skipped unless *ctl & 1 (null: always run)
    int *ready;      // table form: the pair's ny*nz line ready flags (FP64 values)
    int *err;        // table form: the pair's flags (FL_TIMEOUT)
    unsigned long long *tw;  // column forms with FP32 values: tagged result words [N]
                             // (zeroed at setup), used in place of t
    int *sync;       // column forms with FP32 values: sync head (sync[2] = sweep epoch)
    int item0;       // table form: the pair's first work item (plane)
};
// ILU(0) solves of every pair of a device table whose lines all use `slots`,
// as ticketed column sweeps (one work item = one plane; entry k's items start
// at item0, nitems in all).  sync: sync_bytes of device memory; sync[0],
// sync[1] are the two sweeps' ticket counters and sync[2] the sweep epoch
// (zeroed at setup; FP32 values: every entry's `sync` is this pointer),
// followed by the entries' ready flags (FP64 values).  Before the sweeps the
// counters are reset and the epoch advanced (FP32 values) or the whole region
// zeroed (FP64 values).  warps: warps per CTA (1..8); one warp per item.
cudaError_t launch_ilu_table(int prec, int slots, const IluArgs *table, int npairs, int nitems, int *sync,
                             size_t sync_bytes, int warps, cudaStream_t st);

}  // namespace ffp
