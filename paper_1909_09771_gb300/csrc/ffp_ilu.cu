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
// (y, z-1).  Along a line the recurrence in x is first order: an affine map
// per cell (triangular sweeps) or a Moebius map (pivots), evaluated as
// lane-local composition + a 32-lane scan + lane-local substitution, lane l
// holding cells l*S .. l*S+S-1.  Three schedules of the sweeps, same
// arithmetic in the same order:
//  * column form (used whenever it fits): the warp of plane z walks its lines
//    in order and takes the z-neighbour line from the warp of plane z -/+ 1;
//    one cooperative launch per sweep for a single instance, one ticketed
//    launch per sweep over all planes of a batch group;
//  * dataflow form: lines in diagonal order over all warps, ready flags;
//  * wavefront form: one launch per diagonal y + z = s, one warp per line
//    (the pivots always use it; the sweeps only as a last resort).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "ffp_vecops.cuh"

namespace ffp {

// y = (float) x; with sync non-null, block 0 also does what ilu_epoch_kernel does
// (the single-instance sweeps that follow in stream order read the new epoch)
__global__ void __launch_bounds__(kThreads) f64_to_f32_kernel(long long n, const double *__restrict__ x,
                                                             float *y, int *sync) {
    if (sync && blockIdx.x == 0 && threadIdx.x == 0) {
        sync[0] = 0;
        sync[1] = 0;
        sync[2] += 2;
    }
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        y[a] = (float)x[a];
}

__global__ void __launch_bounds__(kThreads) f32_to_f64_kernel(long long n, const float *__restrict__ x,
                                                             double *y) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        y[a] = (double)x[a];
}

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
    scale2(pp, qq);
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
// Typed view of one pair's IluArgs; V = type of r and t (FP64, or the FP32
// copies the single-instance dataflow forms work on, so that no FP64 <-> FP32
// conversion sits on their dependency chain; the values are the same).
template <typename F, typename V = double>
struct IluView {
    int nx, ny, nz;
    const F *dinv, *lx, *ly, *lz;
    const V *r;
    V *t;
    __device__ __forceinline__ explicit IluView(const IluArgs &a)
        : nx(a.nx), ny(a.ny), nz(a.nz), dinv(static_cast<const F *>(a.dinv)),
          lx(static_cast<const F *>(a.lx)), ly(static_cast<const F *>(a.ly)),
          lz(static_cast<const F *>(a.lz)), r(static_cast<const V *>(a.r)),
          t(static_cast<V *>(a.t)) {}
};

// Loads of t values other warps of the same launch may have written (dataflow
// form): through L2, never a stale L1 line.
template <bool COH>
__device__ __forceinline__ double ld_t(const double *p) {
    if constexpr (COH) return __ldcg(p);
    else return *p;
}
template <bool COH>
__device__ __forceinline__ float ld_t(const float *p) {
    if constexpr (COH) return __ldcg(p);
    else return *p;
}

// Forward sweep of line (y, z): t = L^{-1} r along x (Sec. III, ILU(0) of blkD(A)).
template <int S, typename F, bool COH>
__device__ __forceinline__ void ilu_fwd_line(const IluView<F> &A, const IluGeo &g, int y, int z,
                                             int lane) {
    using R = typename Compute<F>::type;
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
            if (y > 0 && a - A.nx >= lo) v -= ldf<true, F, R>(A.ly + a - A.nx) * (R)ld_t<COH>(A.t + a - A.nx);
            if (z > 0 && a - g.nxy >= lo) v -= ldf<true, F, R>(A.lz + a - g.nxy) * (R)ld_t<COH>(A.t + a - g.nxy);
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
        if (k < cnt) A.t[base + lane * S + k] = static_cast<typename std::remove_pointer<decltype(A.t)>::type>(c);
    }
}

// Backward sweep of line (y, z): z_a = t_a - dinv_a (lx_a z_{a+1} + ly_a z_{a+nx} +
// lz_a z_{a+nxy}), in place on t.
template <int S, typename F, bool COH>
__device__ __forceinline__ void ilu_bwd_line(const IluView<F> &A, const IluGeo &g, int y, int z,
                                             int lane) {
    using R = typename Compute<F>::type;
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
            if (y + 1 < A.ny && a + A.nx < hi) v += ldf<true, F, R>(A.ly + a) * (R)ld_t<COH>(A.t + a + A.nx);
            if (z + 1 < A.nz && a + g.nxy < hi) v += ldf<true, F, R>(A.lz + a) * (R)ld_t<COH>(A.t + a + g.nxy);
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
        if (k < cnt) A.t[base + lane * S + k] = static_cast<typename std::remove_pointer<decltype(A.t)>::type>(c);
    }
}

// The same two sweeps split for the dataflow form: everything a line reads that
// no other line writes (1/D, the bands, r) is loaded before its predecessors'
// flags are awaited, so only the t reads and the scan stay on the critical path.
template <int S, typename F>
struct IluLinePre {
    using R = typename Compute<F>::type;
    R di[S], cx[S], cy[S], cz[S], rv[S];
};

template <int S, typename F, typename V>
__device__ __forceinline__ void ilu_fwd_pre(const IluView<F, V> &A, const IluGeo &g, int y, int z,
                                            int lane, IluLinePre<S, F> &P) {
    using R = typename Compute<F>::type;
    const long long base = (long long)A.nx * y + g.nxy * z;
    int cnt = A.nx - lane * S;
    cnt = cnt < 0 ? 0 : (cnt > S ? S : cnt);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        P.di[k] = R(0); P.cx[k] = R(0); P.cy[k] = R(0); P.cz[k] = R(0); P.rv[k] = R(0);
        if (k < cnt) {
            const int x = lane * S + k;
            const long long a = base + x;
            const long long lo = (a < g.M) ? 0 : g.M;
            P.di[k] = ldf<true, F, R>(A.dinv + a);
            P.rv[k] = (R)__ldg(A.r + a);
            if (y > 0 && a - A.nx >= lo) P.cy[k] = ldf<true, F, R>(A.ly + a - A.nx);
            if (z > 0 && a - g.nxy >= lo) P.cz[k] = ldf<true, F, R>(A.lz + a - g.nxy);
            if (x > 0 && a - 1 >= lo) P.cx[k] = ldf<true, F, R>(A.lx + a - 1);
        }
    }
}

// same arithmetic, in the same order, as ilu_fwd_line
template <int S, typename F, typename V>
__device__ __forceinline__ void ilu_fwd_fin(const IluView<F, V> &A, const IluGeo &g, int y, int z,
                                            int lane, const IluLinePre<S, F> &P) {
    using R = typename Compute<F>::type;
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
            const R di = P.di[k];
            R v = P.rv[k];
            if (y > 0 && a - A.nx >= lo) v -= P.cy[k] * (R)ld_t<true>(A.t + a - A.nx);
            if (z > 0 && a - g.nxy >= lo) v -= P.cz[k] * (R)ld_t<true>(A.t + a - g.nxy);
            al[k] = (x > 0 && a - 1 >= lo) ? -di * P.cx[k] : R(0);
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
        if (k < cnt) A.t[base + lane * S + k] = static_cast<typename std::remove_pointer<decltype(A.t)>::type>(c);
    }
}

template <int S, typename F, typename V>
__device__ __forceinline__ void ilu_bwd_pre(const IluView<F, V> &A, const IluGeo &g, int y, int z,
                                            int lane, IluLinePre<S, F> &P) {
    using R = typename Compute<F>::type;
    const long long base = (long long)A.nx * y + g.nxy * z;
    int cnt = A.nx - lane * S;
    cnt = cnt < 0 ? 0 : (cnt > S ? S : cnt);
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
        P.di[k] = R(0); P.cx[k] = R(0); P.cy[k] = R(0); P.cz[k] = R(0); P.rv[k] = R(0);
        if (k < cnt) {
            const int x = lane * S + k;
            const long long a = base + x;
            const long long hi = (a < g.M) ? g.M : g.n;
            P.di[k] = ldf<true, F, R>(A.dinv + a);
            if (y + 1 < A.ny && a + A.nx < hi) P.cy[k] = ldf<true, F, R>(A.ly + a);
            if (z + 1 < A.nz && a + g.nxy < hi) P.cz[k] = ldf<true, F, R>(A.lz + a);
            if (x + 1 < A.nx && a + 1 < hi) P.cx[k] = ldf<true, F, R>(A.lx + a);
            P.rv[k] = (R)A.t[a];  // this line's forward value (previous launch)
        }
    }
}

// same arithmetic, in the same order, as ilu_bwd_line
template <int S, typename F, typename V>
__device__ __forceinline__ void ilu_bwd_fin(const IluView<F, V> &A, const IluGeo &g, int y, int z,
                                            int lane, const IluLinePre<S, F> &P) {
    using R = typename Compute<F>::type;
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
            const R di = P.di[k];
            R v = R(0);
            if (y + 1 < A.ny && a + A.nx < hi) v += P.cy[k] * (R)ld_t<true>(A.t + a + A.nx);
            if (z + 1 < A.nz && a + g.nxy < hi) v += P.cz[k] * (R)ld_t<true>(A.t + a + g.nxy);
            ga[k] = (x + 1 < A.nx && a + 1 < hi) ? -di * P.cx[k] : R(0);
            de[k] = P.rv[k] - di * v;
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
        if (k < cnt) A.t[base + lane * S + k] = static_cast<typename std::remove_pointer<decltype(A.t)>::type>(c);
    }
}

// Wavefront form: one launch per diagonal s, one warp per line of it.
template <int S, typename F>
__global__ void __launch_bounds__(256) ilu_fwd_kernel(IluArgs a0, int s) {
    const IluView<F> A(a0);
    const IluGeo g = ilu_geo(A.nx, A.ny, A.nz);
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int y, z;
    if (!diag_line(g, s, j, y, z)) return;
    ilu_fwd_line<S, F, false>(A, g, y, z, threadIdx.x & 31);
}

template <int S, typename F>
__global__ void __launch_bounds__(256) ilu_bwd_kernel(IluArgs a0, int s) {
    const IluView<F> A(a0);
    const IluGeo g = ilu_geo(A.nx, A.ny, A.nz);
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int y, z;
    if (!diag_line(g, s, j, y, z)) return;
    ilu_bwd_line<S, F, false>(A, g, y, z, threadIdx.x & 31);
}

// Dataflow form: one cooperative launch per sweep.  Line (s, j) of diagonal s
// (j-th line, z ascending) is taken by warp (off(s) + j) mod W, so every warp
// meets its lines in diagonal order and waits only on lines of earlier
// diagonals, which earlier work of other warps produces: with every warp
// resident (cooperative launch) the sweep cannot deadlock.  A line waits for
// its two predecessors' ready flags (forward: y-1 and z-1; backward: y+1 and
// z+1), written with release semantics after the line's values; the waits are
// bounded, and a wait that gives up records FL_TIMEOUT and goes on (the
// results are then unusable, the kernel still ends).
constexpr int kFlowSpin = 1 << 22;

// Wait until *f >= want.  Bounded: a wait that gives up records FL_TIMEOUT and
// returns; once that flag is set (by any wait of the same pair) the remaining
// waits give up after at most 1024 polls, so a broken chain costs one timeout,
// not one per line.
__device__ __forceinline__ void flow_wait(const int *f, int want, int *err) {
    for (int it = 0; it < kFlowSpin; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
        if (v >= want) return;
        if ((it & 1023) == 1023 && __ldcg(err + FL_TIMEOUT)) return;
    }
    atomicOr(err + FL_TIMEOUT, 1);
}

__device__ __forceinline__ void flow_signal(int *f, int v) {
    __threadfence();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}

// Ready-flag values: a forward sweep signals 1, the backward sweep after it 2,
// so one zeroing of the flags serves both sweeps of a solve.
constexpr int kFwdReady = 1, kBwdReady = 2;

template <int S, typename F, bool FWD, typename V>
__global__ void __launch_bounds__(256) ilu_flow_kernel(IluArgs a0, int *ready, int *err) {
    const IluView<F, V> A(a0);
    const IluGeo g = ilu_geo(A.nx, A.ny, A.nz);
    const int lane = threadIdx.x & 31;
    const long long W = (long long)gridDim.x * (blockDim.x >> 5);
    const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nd = A.ny + A.nz - 1;
    long long rem = 0;  // (lines in the diagonals before s, in sweep order) mod W
    for (int q = 0; q < nd; ++q) {
        const int s = FWD ? q : nd - 1 - q;
        const int z0 = (s - (A.ny - 1) > 0) ? s - (A.ny - 1) : 0;
        const int z1 = (s < A.nz - 1) ? s : A.nz - 1;
        const int len = z1 - z0 + 1;
        long long j = w - rem;
        if (j < 0) j += W;
        for (; j < len; j += W) {
            const int z = z0 + (int)j, y = s - z;
            IluLinePre<S, F> P;
            if (FWD) {
                ilu_fwd_pre<S, F, V>(A, g, y, z, lane, P);
                if (y > 0) flow_wait(ready + (long long)z * A.ny + y - 1, kFwdReady, err);
                if (z > 0) flow_wait(ready + (long long)(z - 1) * A.ny + y, kFwdReady, err);
                ilu_fwd_fin<S, F, V>(A, g, y, z, lane, P);
            } else {
                ilu_bwd_pre<S, F, V>(A, g, y, z, lane, P);
                if (y + 1 < A.ny) flow_wait(ready + (long long)z * A.ny + y + 1, kBwdReady, err);
                if (z + 1 < A.nz) flow_wait(ready + (long long)(z + 1) * A.ny + y, kBwdReady, err);
                ilu_bwd_fin<S, F, V>(A, g, y, z, lane, P);
            }
            flow_signal(ready + (long long)z * A.ny + y, FWD ? kFwdReady : kBwdReady);
        }
        rem += len;
        while (rem >= W) rem -= W;
    }
}

static int diag_len(int ny, int nz, int s) {
    const int z0 = (s - (ny - 1) > 0) ? s - (ny - 1) : 0;
    const int z1 = (s < nz - 1) ? s : nz - 1;
    return z1 - z0 + 1;
}

// Column form: the warp that owns plane z walks its lines in sweep order, so
// the y-neighbour line is its own previous result (kept in registers) and only
// the z-neighbour comes from another warp (plane z -/+ 1), behind that line's
// ready flag.  The critical path is about ny line solves plus nz flag hand-offs
// instead of ny + nz - 1 hand-offs.  The warp of a plane waits only on the warp
// of the preceding plane, which never waits on it.  out64 (backward sweep, or
// null): the result is also stored there in FP64.
template <int S, typename F, bool FWD, typename V>
__device__ __forceinline__ void ilu_col_plane(const IluView<F, V> &A, const IluGeo &g, int z, int lane,
                                              int *ready, int *err, double *out64) {
    using R = typename Compute<F>::type;
    int cnt = A.nx - lane * S;
    cnt = cnt < 0 ? 0 : (cnt > S ? S : cnt);
    R prev[S];
#pragma unroll
    for (int k = 0; k < S; ++k) prev[k] = R(0);
    const unsigned FULL = 0xffffffffu;
    for (int q = 0; q < A.ny; ++q) {
        const int y = FWD ? q : A.ny - 1 - q;
        const long long base = (long long)A.nx * y + g.nxy * z;
        IluLinePre<S, F> P;
        if (FWD) ilu_fwd_pre<S, F, V>(A, g, y, z, lane, P);
        else ilu_bwd_pre<S, F, V>(A, g, y, z, lane, P);
        if (FWD ? (z > 0) : (z + 1 < A.nz))
            flow_wait(ready + (long long)(FWD ? z - 1 : z + 1) * A.ny + y, FWD ? kFwdReady : kBwdReady, err);
        R c;
        if (FWD) {
            // same arithmetic, in the same order, as ilu_fwd_line
            R al[S], be[S];
            R Am = R(1), B = R(0);
#pragma unroll
            for (int k = 0; k < S; ++k) {
                al[k] = R(1); be[k] = R(0);
                if (k < cnt) {
                    const int x = lane * S + k;
                    const long long a = base + x;
                    const long long lo = (a < g.M) ? 0 : g.M;
                    R v = P.rv[k];
                    if (y > 0 && a - A.nx >= lo) v -= P.cy[k] * prev[k];
                    if (z > 0 && a - g.nxy >= lo) v -= P.cz[k] * (R)ld_t<true>(A.t + a - g.nxy);
                    al[k] = (x > 0 && a - 1 >= lo) ? -P.di[k] * P.cx[k] : R(0);
                    be[k] = P.di[k] * v;
                }
                B = fma(al[k], B, be[k]);
                Am = Am * al[k];
            }
#pragma unroll
            for (int dd = 1; dd < 32; dd <<= 1) {
                const R Au = __shfl_up_sync(FULL, Am, dd);
                const R Bu = __shfl_up_sync(FULL, B, dd);
                if (lane >= dd) { B = fma(Am, Bu, B); Am = Am * Au; }
            }
            c = __shfl_up_sync(FULL, B, 1);
            if (lane == 0) c = R(0);
#pragma unroll
            for (int k = 0; k < S; ++k) {
                c = fma(al[k], c, be[k]);
                prev[k] = c;
                if (k < cnt) A.t[base + lane * S + k] = static_cast<V>(c);
            }
        } else {
            // same arithmetic, in the same order, as ilu_bwd_line
            R ga[S], de[S];
            R G = R(1), B = R(0);
#pragma unroll
            for (int k = S - 1; k >= 0; --k) {
                ga[k] = R(1); de[k] = R(0);
                if (k < cnt) {
                    const int x = lane * S + k;
                    const long long a = base + x;
                    const long long hi = (a < g.M) ? g.M : g.n;
                    R v = R(0);
                    if (y + 1 < A.ny && a + A.nx < hi) v += P.cy[k] * prev[k];
                    if (z + 1 < A.nz && a + g.nxy < hi) v += P.cz[k] * (R)ld_t<true>(A.t + a + g.nxy);
                    ga[k] = (x + 1 < A.nx && a + 1 < hi) ? -P.di[k] * P.cx[k] : R(0);
                    de[k] = P.rv[k] - P.di[k] * v;
                }
                B = fma(ga[k], B, de[k]);
                G = G * ga[k];
            }
#pragma unroll
            for (int dd = 1; dd < 32; dd <<= 1) {
                const R Gd = __shfl_down_sync(FULL, G, dd);
                const R Bd = __shfl_down_sync(FULL, B, dd);
                if (lane + dd < 32) { B = fma(G, Bd, B); G = G * Gd; }
            }
            c = __shfl_down_sync(FULL, B, 1);
            if (lane == 31) c = R(0);
#pragma unroll
            for (int k = S - 1; k >= 0; --k) {
                c = fma(ga[k], c, de[k]);
                prev[k] = c;
                if (k < cnt) {
                    A.t[base + lane * S + k] = static_cast<V>(c);
                    if (out64) out64[base + lane * S + k] = (double)c;
                }
            }
        }
        flow_signal(ready + (long long)z * A.ny + y, FWD ? kFwdReady : kBwdReady);
    }
}

// Tagged column form (FP32 values).  Each cell's result is one 64-bit word:
// the FP32 value in the low half and the sweep's tag in the high half, written
// with one relaxed GPU-scope store.  An aligned 64-bit access is single-copy
// atomic, so a warp that reads a word carrying the tag it waits for also reads
// the value stored with it: the hand-off between planes needs no ready flag,
// no fence and no second load.  The tags come from an epoch that grows by 2
// per solve (forward tag epoch - 1, backward tag epoch); the words are zeroed
// at setup and the epoch starts at 0, so no word an earlier sweep left behind
// carries the tag being waited for.  Per line, everything that does not
// depend on the z-neighbour (the loads, the y-coupling, the products of the
// scan maps) is done before the wait, and the next line's loads are issued
// before it; the arithmetic and its order are those of ilu_fwd_line and
// ilu_bwd_line.
__device__ __forceinline__ void st_tag(unsigned long long *p, float v, unsigned tag) {
    const unsigned long long w = ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v);
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long ld_tag(const unsigned long long *p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

// the loads of line (y, z) that no other warp writes (1/D, the bands, r or this
// cell's forward value)
template <int S, typename F, bool FWD>
__device__ __forceinline__ void colt_load(const IluView<F, float> &A, const unsigned long long *tw,
                                          const IluGeo &g, int y, int z, int lane, IluLinePre<S, F> &P) {
    using R = typename Compute<F>::type;
    const long long base = (long long)A.nx * y + g.nxy * z;
    int cnt = A.nx - lane * S;
    cnt = cnt < 0 ? 0 : (cnt > S ? S : cnt);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        P.di[k] = R(0); P.cx[k] = R(0); P.cy[k] = R(0); P.cz[k] = R(0); P.rv[k] = R(0);
        if (k < cnt) {
            const int x = lane * S + k;
            const long long a = base + x;
            P.di[k] = ldf<true, F, R>(A.dinv + a);
            if (FWD) {
                const long long lo = (a < g.M) ? 0 : g.M;
                P.rv[k] = (R)__ldg(A.r + a);
                if (y > 0 && a - A.nx >= lo) P.cy[k] = ldf<true, F, R>(A.ly + a - A.nx);
                if (z > 0 && a - g.nxy >= lo) P.cz[k] = ldf<true, F, R>(A.lz + a - g.nxy);
                if (x > 0 && a - 1 >= lo) P.cx[k] = ldf<true, F, R>(A.lx + a - 1);
            } else {
                const long long hi = (a < g.M) ? g.M : g.n;
                if (y + 1 < A.ny && a + A.nx < hi) P.cy[k] = ldf<true, F, R>(A.ly + a);
                if (z + 1 < A.nz && a + g.nxy < hi) P.cz[k] = ldf<true, F, R>(A.lz + a);
                if (x + 1 < A.nx && a + 1 < hi) P.cx[k] = ldf<true, F, R>(A.lx + a);
                P.rv[k] = __uint_as_float((unsigned)__ldcg(tw + a));  // forward value (previous launch)
            }
        }
    }
}

template <int S, typename F, bool FWD>
__device__ __forceinline__ void ilu_colt_plane(const IluView<F, float> &A, unsigned long long *tw,
                                               const IluGeo &g, int z, int lane, unsigned tag, int *err,
                                               double *out64) {
    using R = typename Compute<F>::type;
    static_assert(sizeof(R) == 4, "tagged column form: FP32 arithmetic");
    int cnt = A.nx - lane * S;
    cnt = cnt < 0 ? 0 : (cnt > S ? S : cnt);
    const unsigned FULL = 0xffffffffu;
    const long long dz = FWD ? -g.nxy : g.nxy;  // offset of the z-neighbour this sweep reads
    R prev[S];
#pragma unroll
    for (int k = 0; k < S; ++k) prev[k] = R(0);
    // the next line's loads are issued one line ahead where the registers allow
    constexpr bool kAhead = S <= 11;
    IluLinePre<S, F> P, Pn;
    if (kAhead) colt_load<S, F, FWD>(A, tw, g, FWD ? 0 : A.ny - 1, z, lane, P);
    for (int q = 0; q < A.ny; ++q) {
        const int y = FWD ? q : A.ny - 1 - q;
        const long long base = (long long)A.nx * y + g.nxy * z;
        if (!kAhead) colt_load<S, F, FWD>(A, tw, g, y, z, lane, P);
        else if (q + 1 < A.ny) colt_load<S, F, FWD>(A, tw, g, FWD ? q + 1 : A.ny - 2 - q, z, lane, Pn);
        // coupling-free part: v without the z term, the map factors, their scan products
        R al[S], v[S];
        bool hz[S];
        R Am = R(1);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            al[k] = R(1); v[k] = R(0); hz[k] = false;
            if (k < cnt) {
                const int x = lane * S + k;
                const long long a = base + x;
                if (FWD) {
                    const long long lo = (a < g.M) ? 0 : g.M;
                    R vv = P.rv[k];
                    if (y > 0 && a - A.nx >= lo) vv -= P.cy[k] * prev[k];
                    v[k] = vv;
                    hz[k] = z > 0 && a - g.nxy >= lo;
                    al[k] = (x > 0 && a - 1 >= lo) ? -P.di[k] * P.cx[k] : R(0);
                } else {
                    const long long hi = (a < g.M) ? g.M : g.n;
                    R vv = R(0);
                    if (y + 1 < A.ny && a + A.nx < hi) vv += P.cy[k] * prev[k];
                    v[k] = vv;
                    hz[k] = z + 1 < A.nz && a + g.nxy < hi;
                    al[k] = (x + 1 < A.nx && a + 1 < hi) ? -P.di[k] * P.cx[k] : R(0);
                }
            }
        }
        if (FWD) {
#pragma unroll
            for (int k = 0; k < S; ++k) Am = Am * al[k];
        } else {
#pragma unroll
            for (int k = S - 1; k >= 0; --k) Am = Am * al[k];
        }
        R AmL[5];
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            const int dd = 1 << l;
            AmL[l] = Am;
            if (FWD) {
                const R Au = __shfl_up_sync(FULL, Am, dd);
                if (lane >= dd) Am = Am * Au;
            } else {
                const R Ad = __shfl_down_sync(FULL, Am, dd);
                if (lane + dd < 32) Am = Am * Ad;
            }
        }
        // wait for the z-neighbour's words of this sweep
        R tz[S];
#pragma unroll
        for (int k = 0; k < S; ++k) tz[k] = R(0);
        for (int it = 0;; ++it) {
            bool ok = true;
#pragma unroll
            for (int k = 0; k < S; ++k)
                if (hz[k]) {
                    const unsigned long long w = ld_tag(tw + base + lane * S + k + dz);
                    ok &= (unsigned)(w >> 32) == tag;
                    tz[k] = __uint_as_float((unsigned)w);
                }
            if (__all_sync(FULL, ok)) break;
            if (it >= kFlowSpin) {
                if (lane == 0) atomicOr(err + FL_TIMEOUT, 1);
                break;
            }
            if ((it & 1023) == 1023 && __ldcg(err + FL_TIMEOUT)) break;
        }
        R be[S];
        R B = R(0);
        if (FWD) {
#pragma unroll
            for (int k = 0; k < S; ++k) {
                be[k] = R(0);
                if (k < cnt) {
                    R vv = v[k];
                    if (hz[k]) vv -= P.cz[k] * tz[k];
                    be[k] = P.di[k] * vv;
                }
                B = fma(al[k], B, be[k]);
            }
#pragma unroll
            for (int l = 0; l < 5; ++l) {
                const int dd = 1 << l;
                const R Bu = __shfl_up_sync(FULL, B, dd);
                if (lane >= dd) B = fma(AmL[l], Bu, B);
            }
            R c = __shfl_up_sync(FULL, B, 1);
            if (lane == 0) c = R(0);
#pragma unroll
            for (int k = 0; k < S; ++k) {
                c = fma(al[k], c, be[k]);
                prev[k] = c;
                if (k < cnt) st_tag(tw + base + lane * S + k, c, tag);
            }
        } else {
#pragma unroll
            for (int k = S - 1; k >= 0; --k) {
                be[k] = R(0);
                if (k < cnt) {
                    R vv = v[k];
                    if (hz[k]) vv += P.cz[k] * tz[k];
                    be[k] = P.rv[k] - P.di[k] * vv;
                }
                B = fma(al[k], B, be[k]);
            }
#pragma unroll
            for (int l = 0; l < 5; ++l) {
                const int dd = 1 << l;
                const R Bd = __shfl_down_sync(FULL, B, dd);
                if (lane + dd < 32) B = fma(AmL[l], Bd, B);
            }
            R c = __shfl_down_sync(FULL, B, 1);
            if (lane == 31) c = R(0);
#pragma unroll
            for (int k = S - 1; k >= 0; --k) {
                c = fma(al[k], c, be[k]);
                prev[k] = c;
                if (k < cnt) {
                    st_tag(tw + base + lane * S + k, c, tag);
                    if (out64) out64[base + lane * S + k] = (double)c;
                }
            }
        }
        if (kAhead) P = Pn;
    }
}

// Single instance: warp z of a cooperative launch takes plane z, so every
// warp a plane waits on is resident and the sweep cannot deadlock.
template <int S, typename F, bool FWD, typename V>
__global__ void __launch_bounds__(256) ilu_col_kernel(IluArgs a0, int *ready, int *err) {
    const IluView<F, V> A(a0);
    const IluGeo g = ilu_geo(A.nx, A.ny, A.nz);
    const int z = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (z >= A.nz) return;
    if constexpr (sizeof(V) == 4) {
        const unsigned e = (unsigned)__ldcg(a0.sync + 2);
        ilu_colt_plane<S, F, FWD>(A, a0.tw, g, z, threadIdx.x & 31, FWD ? e - 1 : e, err,
                                  FWD ? nullptr : a0.out64);
    } else {
        ilu_col_plane<S, F, FWD, V>(A, g, z, threadIdx.x & 31, ready, err, FWD ? nullptr : a0.out64);
    }
}

// Table form: the work items are the planes of every pair of the table, pair
// after pair (entry k's planes are items item0 .. item0 + nz - 1, in sweep
// order: z ascending forward, descending backward).  A warp takes the next
// item from a ticket counter and walks that plane.  An item waits only on the
// item before it of the same pair, which holds a smaller ticket, so it was
// taken by a warp that is running: the smallest unfinished item never waits,
// and the sweep finishes with any number of resident warps (no cooperative
// launch needed).  Items of pairs whose control word is clear are skipped.
template <int S, typename F, bool FWD, typename V>
__global__ void __launch_bounds__(256) ilu_colq_kernel(const IluArgs *__restrict__ table, int npairs,
                                                       int nitems, int *sync) {
    const int lane = threadIdx.x & 31;
    int *ticket = sync + (FWD ? 0 : 1);
    const unsigned ep = (unsigned)__ldcg(sync + 2);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(ticket, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) return;
        int lo = 0, hi = npairs - 1;  // last entry with item0 <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&table[mid].item0) <= it) lo = mid;
            else hi = mid - 1;
        }
        const IluArgs a = table[lo];
        if (a.ctl && !(*a.ctl & 1)) continue;
        const int q = it - a.item0;
        const IluView<F, V> A(a);
        const IluGeo g = ilu_geo(A.nx, A.ny, A.nz);
        if constexpr (sizeof(V) == 4)
            ilu_colt_plane<S, F, FWD>(A, a.tw, g, FWD ? q : A.nz - 1 - q, lane, FWD ? ep - 1 : ep, a.err,
                                      FWD ? nullptr : a.out64);
        else
            ilu_col_plane<S, F, FWD, V>(A, g, FWD ? q : A.nz - 1 - q, lane, a.ready, a.err,
                                        FWD ? nullptr : a.out64);
    }
}

// Before the tagged sweeps of a solve: reset the ticket counters, advance the epoch.
__global__ void ilu_epoch_kernel(int *sync) {
    if (threadIdx.x == 0) {
        sync[0] = 0;
        sync[1] = 0;
        sync[2] += 2;
    }
}

// Blocks of a cooperative launch of kernel k (CTAs of `warps` warps) with every
// block resident (0: not possible).  Cached per kernel and CTA size.
template <auto K>
static int coop_blocks(int warps) {
    static int cached[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
    if (warps < 1 || warps > 8) return 0;
    if (cached[warps] < 0) {
        int dev = 0, coop = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K, 32 * warps, 0) != cudaSuccess)
            cached[warps] = 0;
        else
            cached[warps] = coop ? per * sms : 0;
    }
    return cached[warps];
}

// Blocks of a cooperative dataflow launch: every block resident (0: not possible).
template <int S, typename F, bool FWD, typename V = typename Compute<F>::type>
static int flow_grid() {
    static int cached = -1;
    if (cached < 0) {
        int dev = 0, coop = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ilu_flow_kernel<S, F, FWD, V>, 256, 0) != cudaSuccess)
            cached = 0;
        else
            cached = coop ? per * sms : 0;
    }
    return cached;
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

// Which form a single-instance ILU(0) solve takes: the column form if its
// cooperative launch fits, else the dataflow form if that fits, else the
// wavefront (one launch per diagonal).
enum { ILU_WAVE = 0, ILU_FLOW = 1, ILU_COL = 2 };

// Warps per CTA of the single-instance column form: the nz plane warps spread
// over every SM (each SM's load pipe serves fewer of them), at most 8.
static int col_warps(int nz) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
    }
    return std::max(1, std::min(8, nz / sms));
}

template <int S, typename F>
static int ilu_form(const KernelCtx &c) {
    using V = typename Compute<F>::type;
    if (!c.ws.ilu_ready || (sizeof(V) == 4 && (!c.ws.ilu_v || !c.ws.ilu_tw))) return ILU_WAVE;
    const int w = col_warps(c.nz), ncol = (c.nz + w - 1) / w;
    if (ncol <= coop_blocks<ilu_col_kernel<S, F, true, V>>(w) && ncol <= coop_blocks<ilu_col_kernel<S, F, false, V>>(w))
        return ILU_COL;
    if (flow_grid<S, F, true>() > 0 && flow_grid<S, F, false>() > 0) return ILU_FLOW;
    return ILU_WAVE;
}

template <int S, typename F>
static cudaError_t ilu_solve_s(const KernelCtx &c, const double *r, double *t, cudaStream_t st) {
    IluArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = c.nx; a.ny = c.ny; a.nz = c.nz;
    a.dinv = c.ws.dinv; a.lx = c.ws.lx; a.ly = c.ws.ly; a.lz = c.ws.l3;
    a.r = r; a.t = t;
    const int nd = c.ny + c.nz - 1;
    // the cooperative forms run on r and t in the arithmetic type V (FP32 copies
    // for FP32/BF16 factors: no conversion on their dependency chain)
    using V = typename Compute<F>::type;
    const int form = ilu_form<S, F>(c);
    if (form != ILU_WAVE) {
        const bool col = form == ILU_COL;
        int *ready = c.ws.ilu_ready, *err = c.ws.flags;
        cudaError_t e = cudaSuccess;
        // FP32/BF16 factors: r -> FP32 copy; the column form works on the tagged
        // words (and its backward sweep stores the FP64 result in t), the dataflow
        // form on an FP32 t in the same memory
        float *rv = static_cast<float *>(c.ws.ilu_v);
        float *tv = reinterpret_cast<float *>(c.ws.ilu_tw);
        if constexpr (sizeof(V) == 4) {
            f64_to_f32_kernel<<<grid_for(c.n), kThreads, 0, st>>>(c.n, r, rv, col ? c.ws.ilu_sync : nullptr);
            a.r = rv;
            if (col) {
                a.t = nullptr;
                a.tw = c.ws.ilu_tw;
                a.sync = c.ws.ilu_sync;
                a.out64 = t;
            } else {
                a.t = tv;
            }
            e = cudaGetLastError();
        }
        void *args[] = {&a, &ready, &err};
        const size_t fb = sizeof(int) * (size_t)c.ny * c.nz;
        const void *kf = col ? (const void *)ilu_col_kernel<S, F, true, V> : (const void *)ilu_flow_kernel<S, F, true, V>;
        const void *kb = col ? (const void *)ilu_col_kernel<S, F, false, V> : (const void *)ilu_flow_kernel<S, F, false, V>;
        const int cw = col ? col_warps(c.nz) : 8, ncol = (c.nz + cw - 1) / cw;
        const int blf = col ? ncol : flow_grid<S, F, true>(), blb = col ? ncol : flow_grid<S, F, false>();
        const bool flagged = !(col && sizeof(V) == 4);
        if (e == cudaSuccess && flagged) e = cudaMemsetAsync(ready, 0, fb, st);
        if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(kf, blf, 32 * cw, args, 0, st);
        if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(kb, blb, 32 * cw, args, 0, st);
        if constexpr (sizeof(V) == 4) {
            if (e == cudaSuccess && !col) {
                f32_to_f64_kernel<<<grid_for(c.n), kThreads, 0, st>>>(c.n, tv, t);
                e = cudaGetLastError();
            }
        }
        return e;
    }
    for (int s = 0; s < nd; ++s) {
        const int lines = diag_len(c.ny, c.nz, s);
        ilu_fwd_kernel<S, F><<<(lines + 3) / 4, 128, 0, st>>>(a, s);
    }
    for (int s = nd - 1; s >= 0; --s) {
        const int lines = diag_len(c.ny, c.nz, s);
        ilu_bwd_kernel<S, F><<<(lines + 3) / 4, 128, 0, st>>>(a, s);
    }
    return cudaGetLastError();
}

// One warp per work item: CTAs are short-lived (one plane each), so they give
// their SM slots back as they finish and higher-priority work queued behind
// them starts without waiting for the whole sweep.
template <int S, typename F>
static cudaError_t ilu_table_s(const IluArgs *table, int npairs, int nitems, int *sync, size_t sync_bytes,
                               int warps, cudaStream_t st) {
    using V = typename Compute<F>::type;
    const int gf = (nitems + warps - 1) / warps, gb = gf;
    if constexpr (sizeof(V) == 4) {
        ilu_epoch_kernel<<<1, 32, 0, st>>>(sync);
    } else {
        const cudaError_t e = cudaMemsetAsync(sync, 0, sync_bytes, st);
        if (e != cudaSuccess) return e;
    }
    ilu_colq_kernel<S, F, true, V><<<gf, 32 * warps, 0, st>>>(table, npairs, nitems, sync);
    ilu_colq_kernel<S, F, false, V><<<gb, 32 * warps, 0, st>>>(table, npairs, nitems, sync);
    return cudaGetLastError();
}

template <typename F>
static long long ilu_launches_t(const KernelCtx &c) {
    const bool f32 = sizeof(typename Compute<F>::type) == 4;
    int form = ILU_WAVE;
    switch (ilu_slots(c.nx)) {
#define FFP_CASE(SS) case SS: form = ilu_form<SS, F>(c); break;
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return 0;
    }
    if (form == ILU_COL) return f32 ? 3 : 2;
    if (form == ILU_FLOW) return f32 ? 4 : 2;
    return 2LL * (c.ny + c.nz - 1);
}

long long ilu_solve_launches(const KernelCtx &c) {
    switch (c.prec) {
        case FFP_FP64: return ilu_launches_t<double>(c);
        case FFP_FP32: return ilu_launches_t<float>(c);
        default: return ilu_launches_t<__nv_bfloat16>(c);
    }
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
static cudaError_t ilu_table_t(int slots, const IluArgs *t, int np, int ni, int *sync, size_t sb, int w,
                               cudaStream_t st) {
    switch (slots) {
#define FFP_CASE(SS) case SS: return ilu_table_s<SS, F>(t, np, ni, sync, sb, w, st);
        FFP_SLOT_LIST(FFP_CASE)
#undef FFP_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ilu_table(int prec, int slots, const IluArgs *table, int npairs, int nitems, int *sync,
                             size_t sync_bytes, int warps, cudaStream_t st) {
    if (npairs < 1 || nitems < 1 || !sync || sync_bytes < 12 || warps < 1 || warps > 8)
        return cudaErrorInvalidValue;
    switch (prec) {
        case FFP_FP64: return ilu_table_t<double>(slots, table, npairs, nitems, sync, sync_bytes, warps, st);
        case FFP_FP32: return ilu_table_t<float>(slots, table, npairs, nitems, sync, sync_bytes, warps, st);
        case FFP_BF16:
            return ilu_table_t<__nv_bfloat16>(slots, table, npairs, nitems, sync, sync_bytes, warps, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ffp
