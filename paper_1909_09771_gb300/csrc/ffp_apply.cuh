// ffp_apply.cu -- z = B^{-1} r for the nested twisted preconditioner
// (Sec. II-B, Algorithms 1-7, entry SOLVE(1, N, x, y, n^2, 3)).
//
// Level 3 (planes) is twisted at plane mz = floor((nz-1)/2):
//   phase 0 (2 CTAs): lower sweep of the top half, planes 0..mz-1, and of the
//                     bottom half, planes nz-1..mz+1 (Algorithms 3 and 4):
//                     y_i = B_{P,i}^{-1} (r_i - l3 .* y_{i-/+1});
//   phase 1 (1 CTA) : the twist plane takes both couplings (Algorithm 2),
//                     y_mz = B_{P,mz}^{-1} (r_mz - l3 .* y_{mz-1} - l3 .* y_{mz+1}),
//                     and z_mz = y_mz (Algorithm 5);
//   phase 2 (2 CTAs): upper sweeps outwards (Algorithms 6 and 7):
//                     z_i = y_i - B_{P,i}^{-1} (l3 .* z_{i+/-1}).
// The three launches on one stream are the level-3 meeting points, so no CTA
// ever waits on another.  Inside a CTA, two warps run the level-2 halves of
// every plane solve (ffp_plane.cuh) and each line is one warp-wide twisted
// tridiagonal solve (level 1).  y is kept in the output z (in place, reading
// UpperSolve's input from the LowerSolve output); phase 2 keeps its plane
// intermediates in a per-CTA scratch plane.
#pragma once
#include "ffp_plane.cuh"
#include "ffp_kernels.h"

namespace ffp {

template <typename F>
struct ApplyArgs {
    int nx, ny, nz;
    const F *l1, *minv, *l2, *l3;
    const double *r;
    double *z;
    double *scr;  // 2 planes
};

// phase 0: plane i of a half; ip = previous plane of the chain (or -1), ic = coupling plane
template <typename F, typename R>
struct LowerPol {
    const double *r;
    double *z;
    const F *l3;
    long base, prev, cpl;  // plane offsets (prev < 0: chain start)
    int nx;
    __device__ __forceinline__ R rhs(int k, int a) const {
        const long e = (long)k * nx + a;
        R v = (R)__ldg(r + base + e);
        if (prev >= 0) v -= ldf<true, F, R>(l3 + cpl + e) * (R)z[prev + e];
        return v;
    }
    __device__ __forceinline__ void put_w(int k, int a, R w) const { z[base + (long)k * nx + a] = (double)w; }
    __device__ __forceinline__ R get_w(int k, int a) const { return (R)z[base + (long)k * nx + a]; }
    __device__ __forceinline__ void put_out(int k, int a, R u) const { z[base + (long)k * nx + a] = (double)u; }
};

template <typename F, typename R>
struct MidPol {
    const double *r;
    double *z;
    const F *l3;
    long base, top, ctop, bot, cbot;  // top/bot < 0: absent
    int nx;
    __device__ __forceinline__ R rhs(int k, int a) const {
        const long e = (long)k * nx + a;
        R v = (R)__ldg(r + base + e);
        if (top >= 0) v -= ldf<true, F, R>(l3 + ctop + e) * (R)z[top + e];
        if (bot >= 0) v -= ldf<true, F, R>(l3 + cbot + e) * (R)z[bot + e];
        return v;
    }
    __device__ __forceinline__ void put_w(int k, int a, R w) const { z[base + (long)k * nx + a] = (double)w; }
    __device__ __forceinline__ R get_w(int k, int a) const { return (R)z[base + (long)k * nx + a]; }
    __device__ __forceinline__ void put_out(int k, int a, R u) const { z[base + (long)k * nx + a] = (double)u; }
};

template <typename F, typename R>
struct UpperPol {
    double *z;
    double *scr;
    const F *l3;
    long base, adj, cpl;
    int nx;
    __device__ __forceinline__ R rhs(int k, int a) const {
        const long e = (long)k * nx + a;
        return ldf<true, F, R>(l3 + cpl + e) * (R)z[adj + e];
    }
    __device__ __forceinline__ void put_w(int k, int a, R w) const { scr[(long)k * nx + a] = (double)w; }
    __device__ __forceinline__ R get_w(int k, int a) const { return (R)scr[(long)k * nx + a]; }
    __device__ __forceinline__ void put_out(int k, int a, R u) const {
        const long e = base + (long)k * nx + a;
        z[e] = (double)((R)z[e] - u);
    }
};

template <int S, typename F>
__global__ void __launch_bounds__(64) apply_kernel(ApplyArgs<F> A, int phase) {
    using R = typename Compute<F>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *gbase = reinterpret_cast<R *>(smem_raw);  // [2 parity][2 warps][nx]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const LineMap L(nx);
    const int cnt = lane_count<S>(L, lane);
    const long nxy = (long)nx * ny;
    const int mz = (nz - 1) / 2;
    if (phase == 0) {
        const int h = blockIdx.x;
        const int nl3 = (h == 0) ? mz : nz - 1 - mz;
        for (int t = 0; t < nl3; ++t) {
            const int i = (h == 0) ? t : nz - 1 - t;
            LowerPol<F, R> pol;
            pol.r = A.r; pol.z = A.z; pol.l3 = A.l3; pol.nx = nx;
            pol.base = i * nxy;
            pol.prev = (t > 0) ? ((h == 0) ? (i - 1) * nxy : (i + 1) * nxy) : -1;
            pol.cpl = (h == 0) ? (long)(i - 1) * nxy : (long)i * nxy;
            plane_solve<S, true, F, R>(L, nx, ny, A.l1 + i * nxy, A.minv + i * nxy, A.l2 + i * nxy,
                                       pol, gbase + (t & 1) * 2 * nx, wid, lane, cnt);
        }
    } else if (phase == 1) {
        MidPol<F, R> pol;
        pol.r = A.r; pol.z = A.z; pol.l3 = A.l3; pol.nx = nx;
        pol.base = mz * nxy;
        pol.top = (mz > 0) ? (mz - 1) * nxy : -1;
        pol.ctop = (mz > 0) ? (mz - 1) * nxy : 0;
        pol.bot = (mz < nz - 1) ? (mz + 1) * nxy : -1;
        pol.cbot = mz * nxy;
        plane_solve<S, true, F, R>(L, nx, ny, A.l1 + mz * nxy, A.minv + mz * nxy, A.l2 + mz * nxy,
                                   pol, gbase, wid, lane, cnt);
    } else {
        const int h = blockIdx.x;
        const int nl3 = (h == 0) ? mz : nz - 1 - mz;
        for (int t = nl3 - 1; t >= 0; --t) {
            const int i = (h == 0) ? t : nz - 1 - t;
            UpperPol<F, R> pol;
            pol.z = A.z; pol.scr = A.scr + h * nxy; pol.l3 = A.l3; pol.nx = nx;
            pol.base = i * nxy;
            pol.adj = (h == 0) ? (i + 1) * nxy : (i - 1) * nxy;
            pol.cpl = (h == 0) ? (long)i * nxy : (long)(i - 1) * nxy;
            plane_solve<S, true, F, R>(L, nx, ny, A.l1 + i * nxy, A.minv + i * nxy, A.l2 + i * nxy,
                                       pol, gbase + (t & 1) * 2 * nx, wid, lane, cnt);
        }
    }
}

template <int S, typename F>
cudaError_t apply_for_slots(const KernelCtx &c, const double *r, double *z, cudaStream_t st) {
    using R = typename Compute<F>::type;
    ApplyArgs<F> a;
    a.nx = c.nx; a.ny = c.ny; a.nz = c.nz;
    a.l1 = (const F *)c.ws.l1; a.minv = (const F *)c.ws.minv;
    a.l2 = (const F *)c.ws.l2; a.l3 = (const F *)c.ws.l3;
    a.r = r; a.z = z; a.scr = c.ws.ascr;
    const size_t smem = sizeof(R) * 4 * (size_t)a.nx;
    const int mz = (a.nz - 1) / 2;
    const bool halves = (mz > 0) || (a.nz - 1 - mz > 0);
    if (halves) apply_kernel<S, F><<<2, 64, smem, st>>>(a, 0);
    apply_kernel<S, F><<<1, 64, smem, st>>>(a, 1);
    if (halves) apply_kernel<S, F><<<2, 64, smem, st>>>(a, 2);
    return cudaGetLastError();
}

}  // namespace ffp
