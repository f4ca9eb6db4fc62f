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
    Ws ws;
};

// ffp_ops.cu
cudaError_t launch_assemble(const KernelCtx &c, const double *kappa, const unsigned char bc[6],
                            cudaStream_t st);
cudaError_t launch_check_filter(const KernelCtx &c, const double *t, cudaStream_t st);
cudaError_t launch_convert_bands(const KernelCtx &c, cudaStream_t st);  // l3 (and lx, ly for B_c)
cudaError_t launch_resid_vec(const KernelCtx &c, const double *r, const double *y, double *w,
                             cudaStream_t st);                           // w = r - A y
cudaError_t launch_add(const KernelCtx &c, double *z, const double *y, cudaStream_t st);  // z += y
cudaError_t launch_to_f32(const KernelCtx &c, const double *x, float *y, cudaStream_t st);
cudaError_t launch_from_f32(const KernelCtx &c, const float *x, double *y, cudaStream_t st);
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

// ffp_dispatch.cu: z = B_NTD^{-1} r
cudaError_t launch_apply(const KernelCtx &c, const double *r, double *z, cudaStream_t st);

// ffp_ilu.cu: ILU(0) of blkD(A) (pivots in D64 scratch, 1/D stored) and t = B_ILU0^{-1} r
cudaError_t launch_ilu_setup(const KernelCtx &c, double *D64, cudaStream_t st);
cudaError_t launch_ilu_solve(const KernelCtx &c, const double *r, double *t, cudaStream_t st);

}  // namespace ffp
