// ffp_ilu.cu -- ILU(0) smoother of the combination preconditioner
// B_c^{-1} = B_NTD^{-1} + B_ILU0^{-1} - B_NTD^{-1} A B_ILU0^{-1} (Sec. III, Eq. (com)).
//
// ILU(0) is taken of blkD(A(1:M,1:M), A(M+1:N,M+1:N)), M = floor(N/2) (Sec. III,
// "Parallel Solve with Preconditioner").  For the 7-point pattern in natural
// order ILU(0) keeps no fill, so it only changes the pivots:
//   D_a = A_aa - sum over lower neighbours b of a (same block) of A_ab^2 / D_b
// and B_ILU0 = (D + L) D^{-1} (D + U).
//
// GPU schedule: line (y, z) of the grid depends only on lines (y-1, z) and
// (y, z-1), so all lines on a diagonal y + z = s are independent; each launch
// handles one diagonal, one warp per line.  Along a line the recurrence in x
// is first order: an affine map per cell (triangular sweeps) or a Moebius map
// (pivots), evaluated as lane-local composition + a 32-lane scan + lane-local
// substitution, lane l holding cells l*S .. l*S+S-1.
#include <cstring>

#include "ffp_kernels.h"

namespace ffp {

struct IluGeo {
    int nx, ny, nz;
    long long nxy, n, M;  // M = floor(N/2): first row of the second block
};

__device__ __forceinline__ IluGeo ilu_geo(int nx, int ny, int nz) {
    IluGeo g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.nxy = (long long)nx * ny;
    g.n = g.nxy * nz;
    g.M = g.n / 2;
    return g;
}

// line number j on diagonal s -> (y, z); returns false if this warp has no line
__device__ __forceinline__ bool diag_line(const IluGeo &g, int s, int j, int &y, int &z) {
    const int z0 = (s - (g.ny - 1) > 0) ? s - (g.ny - 1) : 0;
    z = z0 + j;
    y = s - z;
    return z < g.nz && y >= 0 && z <= s;
}

// ---------------------------------------------------------------- pivots (FP64)
// D_a = c_a - e_a^2 / D_{a-1} along the line, c_a = d_a - (y, z neighbour terms),
// e_a = A[a-1, a] (0 at x = 0 or across the block split).  Projective scan as
// in twisted_pivots, over one 32-lane chain.
template <int S>
__global__ void __launch_bounds__(128) ilu_pivot_kernel(IluPivArgs P0,
                                                        const IluPivArgs *__restrict__ table, int s) {
    const IluPivArgs &P = table ? table[blockIdx.y] : P0;
    const int nx = P.nx, ny = P.ny, nz = P.nz, prec = P.prec;
    const double *__restrict__ d = P.d;
    const double *__restrict__ cx = P.cx;
    const double *__restrict__ cy = P.cy;
    const double *__restrict__ cz = P.cz;
    double *D64 = P.D64;
    void *dinv = P.dinv;
    int *flags = P.flags;
    const IluGeo g = ilu_geo(nx, ny, nz);
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int y, z;
    if (!diag_line(g, s, j, y, z)) return;
    const long long base = (long long)nx * y + g.nxy * z;
    double c[S], e2[S];
    int cnt = nx - lane * S;
    cnt = cnt < 0 ? 0 : (cnt > S ? S : cnt);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        c[k] = 1.0; e2[k] = 0.0;
        if (k < cnt) {
            const int x = lane * S + k;
            const long long a = base + x;
            const long long lo = (a < g.M) ? 0 : g.M;
            double v = d[a];
            if (y > 0 && a - nx >= lo) v -= cy[a - nx] * cy[a - nx] / D64[a - nx];
            if (z > 0 && a - g.nxy >= lo) v -= cz[a - g.nxy] * cz[a - g.nxy] / D64[a - g.nxy];
            c[k] = v;
            if (x > 0 && a - 1 >= lo) e2[k] = cx[a - 1] * cx[a - 1];
        }
    }
    // lane-local product of [[c, -e^2], [1, 0]] (pads are identity)
    double p11 = 1.0, p12 = 0.0, p21 = 0.0, p22 = 1.0;
#pragma unroll
    for (int k = 0; k < S; ++k)
        if (k < cnt) {
            const double n11 = c[k] * p11 - e2[k] * p21;
            const double n12 = c[k] * p12 - e2[k] * p22;
            p21 = p11; p22 = p12; p11 = n11; p12 = n12;
        }
    scale4(p11, p12, p21, p22);
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const double q11 = __shfl_up_sync(FULL, p11, dd);
        const double q12 = __shfl_up_sync(FULL, p12, dd);
        const double q21 = __shfl_up_sync(FULL, p21, dd);
        const double q22 = __shfl_up_sync(FULL, p22, dd);
        if (lane >= dd) {
            const double n11 = p11 * q11 + p12 * q21;
            const double n12 = p11 * q12 + p12 * q22;
            const double n21 = p21 * q11 + p22 * q21;
            const double n22 = p21 * q12 + p22 * q22;
            p11 = n11; p12 = n12; p21 = n21; p22 = n22;
            scale4(p11, p12, p21, p22);
        }
    }
    double pp = __shfl_up_sync(FULL, p11, 1), qq = __shfl_up_sync(FULL, p21, 1);
    if (lane == 0) { pp = 1.0; qq = 0.0; }
    {
        const double mx = fmax(fabs(pp), fabs(qq));
        if (mx > 0.0 && isfinite(mx)) { const int e = ilogb(mx); pp = scalbn(pp, -e); qq = scalbn(qq, -e); }
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < S; ++k)
        if (k < cnt) {
            const double np = c[k] * pp - e2[k] * qq;
            qq = pp;
            pp = np;
            const double Dv = pp / qq;
            const long long a = base + lane * S + k;
            D64[a] = Dv;
            const double di = qq / pp;
            if (prec == FFP_FP64) static_cast<double *>(dinv)[a] = di;
            else if (prec == FFP_FP32) static_cast<float *>(dinv)[a] = (float)di;
            else static_cast<__nv_bfloat16 *>(dinv)[a] = __double2bfloat16(di);
            bad |= !(Dv > 0.0) || !isfinite(Dv);
        }
    if (bad) atomicOr(flags + FL_BREAKDOWN, 1);
}

// ---------------------------------------------------------------- triangular sweeps
// Typed view of one pair's IluArgs.
template <typename F>
struct IluView {
    int nx, ny, nz;
    const F *dinv, *lx, *ly, *lz;
    const double *r;
    double *t;
    __device__ __forceinline__ explicit IluView(const IluArgs &a)
        : nx(a.nx), ny(a.ny), nz(a.nz), dinv(static_cast<const F *>(a.dinv)),
          lx(static_cast<const F *>(a.lx)), ly(static_cast<const F *>(a.ly)),
          lz(static_cast<const F *>(a.lz)), r(a.r), t(a.t) {}
};

// The pair of this CTA (A0, or table[blockIdx.y]); false if it is skipped.
__device__ __forceinline__ bool ilu_pair(const IluArgs &A0, const IluArgs *table, IluArgs &A) {
    A = table ? table[blockIdx.y] : A0;
    return !A.ctl || (*A.ctl & 1);
}

template <int S, typename F>
__global__ void __launch_bounds__(256) ilu_fwd_kernel(IluArgs A0, const IluArgs *__restrict__ table, int s) {
    using R = typename Compute<F>::type;
    IluArgs a0;
    if (!ilu_pair(A0, table, a0)) return;
    const IluView<F> A(a0);
    const IluGeo g = ilu_geo(A.nx, A.ny, A.nz);
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int y, z;
    if (!diag_line(g, s, j, y, z)) return;
    const long long base = (long long)A.nx * y + g.nxy * z;
    int cnt = A.nx - lane * S;
    cnt = cnt < 0 ? 0 : (cnt > S ? S : cnt);
    R al[S], be[S];
    R Am = R(1), B = R(0);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        al[k] = R(1); be[k] = R(0);
        if (k < cnt) {
            const int x = lane * S + k;
            const long long a = base + x;
            const long long lo = (a < g.M) ? 0 : g.M;
            const R di = ldf<true, F, R>(A.dinv + a);
            R v = (R)__ldg(A.r + a);
            if (y > 0 && a - A.nx >= lo) v -= ldf<true, F, R>(A.ly + a - A.nx) * (R)A.t[a - A.nx];
            if (z > 0 && a - g.nxy >= lo) v -= ldf<true, F, R>(A.lz + a - g.nxy) * (R)A.t[a - g.nxy];
            al[k] = (x > 0 && a - 1 >= lo) ? -di * ldf<true, F, R>(A.lx + a - 1) : R(0);
            be[k] = di * v;
        }
        B = fma(al[k], B, be[k]);
        Am = Am * al[k];
    }
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const R Au = __shfl_up_sync(FULL, Am, dd);
        const R Bu = __shfl_up_sync(FULL, B, dd);
        if (lane >= dd) { B = fma(Am, Bu, B); Am = Am * Au; }
    }
    R c = __shfl_up_sync(FULL, B, 1);
    if (lane == 0) c = R(0);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        c = fma(al[k], c, be[k]);
        if (k < cnt) A.t[base + lane * S + k] = (double)c;
    }
}

// backward: z_a = t_a - dinv_a (lx_a z_{a+1} + ly_a z_{a+nx} + lz_a z_{a+nxy}), in place on t
template <int S, typename F>
__global__ void __launch_bounds__(256) ilu_bwd_kernel(IluArgs A0, const IluArgs *__restrict__ table, int s) {
    using R = typename Compute<F>::type;
    IluArgs a0;
    if (!ilu_pair(A0, table, a0)) return;
    const IluView<F> A(a0);
    const IluGeo g = ilu_geo(A.nx, A.ny, A.nz);
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int y, z;
    if (!diag_line(g, s, j, y, z)) return;
    const long long base = (long long)A.nx * y + g.nxy * z;
    int cnt = A.nx - lane * S;
    cnt = cnt < 0 ? 0 : (cnt > S ? S : cnt);
    R ga[S], de[S];
    R G = R(1), B = R(0);
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
        ga[k] = R(1); de[k] = R(0);
        if (k < cnt) {
            const int x = lane * S + k;
            const long long a = base + x;
            const long long hi = (a < g.M) ? g.M : g.n;
            const R di = ldf<true, F, R>(A.dinv + a);
            R v = R(0);
            if (y + 1 < A.ny && a + A.nx < hi) v += ldf<true, F, R>(A.ly + a) * (R)A.t[a + A.nx];
            if (z + 1 < A.nz && a + g.nxy < hi) v += ldf<true, F, R>(A.lz + a) * (R)A.t[a + g.nxy];
            ga[k] = (x + 1 < A.nx && a + 1 < hi) ? -di * ldf<true, F, R>(A.lx + a) : R(0);
            de[k] = (R)A.t[a] - di * v;
        }
        B = fma(ga[k], B, de[k]);
        G = G * ga[k];
    }
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const R Gd = __shfl_down_sync(FULL, G, dd);
        const R Bd = __shfl_down_sync(FULL, B, dd);
        if (lane + dd < 32) { B = fma(G, Bd, B); G = G * Gd; }
    }
    R c = __shfl_down_sync(FULL, B, 1);
    if (lane == 31) c = R(0);
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
        c = fma(ga[k], c, de[k]);
        if (k < cnt) A.t[base + lane * S + k] = (double)c;
    }
}

// ---------------------------------------------------------------- launchers
static int diag_len(int ny, int nz, int s) {
    const int z0 = (s - (ny - 1) > 0) ? s - (ny - 1) : 0;
    const int z1 = (s < nz - 1) ? s : nz - 1;
    return z1 - z0 + 1;
}

template <int S>
static cudaError_t ilu_setup_s(const KernelCtx &c, double *D64, cudaStream_t st) {
    IluPivArgs a;
    a.nx = c.nx; a.ny = c.ny; a.nz = c.nz; a.prec = c.prec;
    a.d = c.ws.d; a.cx = c.ws.cx; a.cy = c.ws.cy; a.cz = c.ws.cz;
    a.D64 = D64; a.dinv = c.ws.dinv; a.flags = c.ws.flags;
    const int nd = c.ny + c.nz - 1;
    for (int s = 0; s < nd; ++s) {
        const int lines = diag_len(c.ny, c.nz, s);
        ilu_pivot_kernel<S><<<(lines + 3) / 4, 128, 0, st>>>(a, nullptr, s);
    }
    return cudaGetLastError();
}

template <int S>
static cudaError_t ilu_setup_table_s(const IluPivArgs *table, int count, int ndiag, int maxlines,
                                     cudaStream_t st) {
    IluPivArgs none;
    std::memset(&none, 0, sizeof(none));
    for (int s = 0; s < ndiag; ++s)
        ilu_pivot_kernel<S><<<dim3((maxlines + 3) / 4, count), 128, 0, st>>>(none, table, s);
    return cudaGetLastError();
}

cudaError_t launch_ilu_setup_table(int slots, const IluPivArgs *table, int count, int ndiag,
                                   int maxlines, cudaStream_t st) {
    if (count < 1 || ndiag < 1 || maxlines < 1) return cudaErrorInvalidValue;
    switch (slots) {
#define FFP_CASE(SS) case SS: return ilu_setup_table_s<SS>(table, count, ndiag, maxlines, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <int S, typename F>
static cudaError_t ilu_solve_s(const KernelCtx &c, const double *r, double *t, cudaStream_t st) {
    IluArgs a;
    a.nx = c.nx; a.ny = c.ny; a.nz = c.nz;
    a.dinv = c.ws.dinv; a.lx = c.ws.lx; a.ly = c.ws.ly; a.lz = c.ws.l3;
    a.r = r; a.t = t;
    a.ctl = nullptr;
    const int nd = c.ny + c.nz - 1;
    for (int s = 0; s < nd; ++s) {
        const int lines = diag_len(c.ny, c.nz, s);
        ilu_fwd_kernel<S, F><<<(lines + 3) / 4, 128, 0, st>>>(a, nullptr, s);
    }
    for (int s = nd - 1; s >= 0; --s) {
        const int lines = diag_len(c.ny, c.nz, s);
        ilu_bwd_kernel<S, F><<<(lines + 3) / 4, 128, 0, st>>>(a, nullptr, s);
    }
    return cudaGetLastError();
}

template <int S, typename F>
static cudaError_t ilu_table_s(const IluArgs *table, int npairs, int ndiag, int maxlines, int warps,
                               cudaStream_t st) {
    IluArgs none;
    std::memset(&none, 0, sizeof(none));
    const dim3 grid((maxlines + warps - 1) / warps, npairs);
    for (int s = 0; s < ndiag; ++s) ilu_fwd_kernel<S, F><<<grid, 32 * warps, 0, st>>>(none, table, s);
    for (int s = ndiag - 1; s >= 0; --s) ilu_bwd_kernel<S, F><<<grid, 32 * warps, 0, st>>>(none, table, s);
    return cudaGetLastError();
}

int ilu_slots(int nx) {
    const int need = (nx + 31) / 32;
    const int list[] = {1, 2, 3, 4, 6, 8, 11, 16, 22, 32};
    for (int s : list)
        if (s >= need) return s;
    return -1;
}

cudaError_t launch_ilu_setup(const KernelCtx &c, double *D64, cudaStream_t st) {
    switch (ilu_slots(c.nx)) {
#define FFP_CASE(SS) case SS: return ilu_setup_s<SS>(c, D64, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename F>
static cudaError_t ilu_solve_t(const KernelCtx &c, const double *r, double *t, cudaStream_t st) {
    switch (ilu_slots(c.nx)) {
#define FFP_CASE(SS) case SS: return ilu_solve_s<SS, F>(c, r, t, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ilu_solve(const KernelCtx &c, const double *r, double *t, cudaStream_t st) {
    switch (c.prec) {
        case FFP_FP64: return ilu_solve_t<double>(c, r, t, st);
        case FFP_FP32: return ilu_solve_t<float>(c, r, t, st);
        case FFP_BF16: return ilu_solve_t<__nv_bfloat16>(c, r, t, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename F>
static cudaError_t ilu_table_t(int slots, const IluArgs *t, int np, int nd, int ml, int w, cudaStream_t st) {
    switch (slots) {
#define FFP_CASE(SS) case SS: return ilu_table_s<SS, F>(t, np, nd, ml, w, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ilu_table(int prec, int slots, const IluArgs *table, int npairs, int ndiag,
                             int maxlines, int warps, cudaStream_t st) {
    if (npairs < 1 || ndiag < 1 || maxlines < 1 || warps < 1 || warps > 8) return cudaErrorInvalidValue;
    switch (prec) {
        case FFP_FP64: return ilu_table_t<double>(slots, table, npairs, ndiag, maxlines, warps, st);
        case FFP_FP32: return ilu_table_t<float>(slots, table, npairs, ndiag, maxlines, warps, st);
        case FFP_BF16: return ilu_table_t<__nv_bfloat16>(slots, table, npairs, ndiag, maxlines, warps, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ffp
