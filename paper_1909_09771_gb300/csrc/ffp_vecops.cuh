// ffp_vecops.cuh -- FP64 building blocks of the CG vector kernels, shared by
// the single-instance kernels (ffp_ops.cu) and the batched ones (ffp_batch.cu):
// the 7-point stencil, fixed-order block and warp reductions, and the update
// of the CG scalars from the folded partial sums.
#pragma once
#include "ffp_kernels.h"

namespace ffp {

constexpr int kThreads = 256;

// Blocks of a grid-stride vector kernel over n entries; it also fixes how a
// reduction over the vector is partitioned, hence its rounding.
inline int grid_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b > kRedBlocks) b = kRedBlocks;
    if (b < 1) b = 1;
    return (int)b;
}

struct Geo {
    int nx, ny, nz;
    long long n;
    int nxy;
};

// (A x)_a with the oracle's term order.
__device__ __forceinline__ double stencil(const Geo &g, long long a, const double *__restrict__ d,
                                          const double *__restrict__ cx,
                                          const double *__restrict__ cy,
                                          const double *__restrict__ cz,
                                          const double *__restrict__ x) {
    const int ix = (int)(a % g.nx);
    const int iy = (int)((a / g.nx) % g.ny);
    const int iz = (int)(a / g.nxy);
    double s = d[a] * x[a];
    if (ix > 0) s += cx[a - 1] * x[a - 1];
    if (ix + 1 < g.nx) s += cx[a] * x[a + 1];
    if (iy > 0) s += cy[a - g.nx] * x[a - g.nx];
    if (iy + 1 < g.ny) s += cy[a] * x[a + g.nx];
    if (iz > 0) s += cz[a - g.nxy] * x[a - g.nxy];
    if (iz + 1 < g.nz) s += cz[a] * x[a + g.nxy];
    return s;
}

// Block sum of NV values per thread, written to red[blockIdx.x * NV + v], fixed order.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *red) {
    __shared__ double sh[NV][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += sh[k][w];
            red[blockIdx.x * NV + k] = s;
        }
    }
}

// Sum of red[i*stride + k], i < nblk, by one warp in a fixed order (lane-strided
// partial sums, then a fixed shuffle tree); every lane gets the result.
__device__ __forceinline__ double warp_fold(const double *__restrict__ red, int nblk, int stride,
                                            int k) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < nblk; i += 32) s += red[i * stride + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Fold the partial sums and update the CG scalars (one warp).
__device__ __forceinline__ void finalize_scalars(int mode, int nblk, int fresh, int flexible,
                                                 const double *__restrict__ red, double *scal,
                                                 int *flags) {
    if (mode == FIN_RESID) {
        const double rr = warp_fold(red, nblk, 2, 0);
        const double bb = warp_fold(red, nblk, 2, 1);
        if (threadIdx.x == 0) { scal[SC_TRR] = rr; scal[SC_RR] = rr; scal[SC_BB] = bb; }
    } else if (mode == FIN_PQ) {
        const double pq = warp_fold(red, nblk, 1, 0);
        if (threadIdx.x == 0) {
            scal[SC_PQ] = pq;
            if (!(pq > 0.0) || !isfinite(pq)) flags[FL_PQ] = 1;
            scal[SC_ALPHA] = scal[SC_RHO] / pq;
        }
    } else if (mode == FIN_RR) {
        const double rr = warp_fold(red, nblk, 1, 0);
        if (threadIdx.x == 0) scal[SC_RR] = rr;
    } else {
        const double rz = warp_fold(red, nblk, 2, 0);
        const double zq = warp_fold(red, nblk, 2, 1);
        if (threadIdx.x == 0) {
            double beta = 0.0;
            if (!fresh) {
                if (flexible) beta = -scal[SC_ALPHA] * zq / scal[SC_RHO];  // (z, r_new - r_old) / rho
                else beta = rz / scal[SC_RHO];
            }
            scal[SC_BETA] = beta;
            scal[SC_ZQ] = zq;
            scal[SC_RHO_OLD] = scal[SC_RHO];
            scal[SC_RHO] = rz;
        }
    }
}

}  // namespace ffp
