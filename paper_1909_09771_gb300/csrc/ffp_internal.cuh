// ffp_internal.cuh -- device building blocks shared by the kernels of libffp.so.
//
// Line layout inside a warp (level 1 of the nested preconditioner, Sec. II-A):
// a line of n cells is split at the twist cell m = floor((n-1)/2).  The top
// chain is cells 0..m-1 (eliminated from cell 0 towards m), the bottom chain is
// cells n-1..m+1 (eliminated from n-1 towards m).  Lanes 0-15 hold the top
// chain and lanes 16-31 the bottom chain; within a half, lane j holds the
// chain positions c = j*S .. j*S+S-1 in registers ("slots"), so both chains
// are handled by 16-lane affine scans running side by side, which is the
// two-way parallelism the twist exposes.  Chain position c maps to cell
// a = c (top) or a = n-1-c (bottom).  Slots past the end of a chain are
// identity steps (pads).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/ffp.h"

namespace ffp {

// ---------------------------------------------------------------- storage types
template <typename F> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

__device__ __forceinline__ double to_r(double v, double) { return v; }
__device__ __forceinline__ float to_r(float v, float) { return v; }
__device__ __forceinline__ float to_r(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ float to_r(double v, float) { return (float)v; }

template <typename F> __device__ __forceinline__ F from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}

// Factor loads.  NC = true: through the read-only (non-coherent) path, for
// data no thread writes while the kernel runs; NC = false: coherent loads, for
// buffers the same kernel rewrites (setup scratch).
template <bool NC, typename F, typename R>
__device__ __forceinline__ R ldf(const F *p) {
    if constexpr (NC) return to_r(__ldg(p), R());
    else return to_r(*p, R());
}

// ---------------------------------------------------------------- line geometry
struct LineMap {
    int n;     // cells in the line
    int m;     // twist cell
    int ntop;  // cells in the top chain (= m)
    int nbot;  // cells in the bottom chain (= n-1-m)
    __device__ __forceinline__ explicit LineMap(int n_) : n(n_), m((n_ - 1) / 2) {
        ntop = m;
        nbot = n_ - 1 - m;
    }
};

// Number of valid slots of this lane (slots >= cnt are pads).
template <int S>
__device__ __forceinline__ int lane_count(const LineMap &L, int lane) {
    const int j = lane & 15;
    const int tot = (lane < 16) ? L.ntop : L.nbot;
    int c = tot - j * S;
    return c < 0 ? 0 : (c > S ? S : c);
}

// Cell index of slot s of this lane (only meaningful for valid slots).
template <int S>
__device__ __forceinline__ int slot_cell(const LineMap &L, int lane, int s) {
    const int c = (lane & 15) * S + s;
    return (lane < 16) ? c : L.n - 1 - c;
}

// Coefficients of one twisted tridiagonal factor T = (M + L1) M^{-1} (M + U1)
// as seen from this lane: minv = 1/M per slot, ein = coupling to the chain
// predecessor, eout = coupling towards the twist cell; plus the twist cell.
template <int S, typename R>
struct LineFactor {
    R minv[S], ein[S], eout[S];
    R minv_m;  // 1 / M_m
    R em1;     // T[m-1, m] (0 if m == 0)
    R em;      // T[m, m+1] (0 if m == n-1)
};

// Load the factor of one line from band arrays l1 (x-band, l1[a] couples a and
// a+1, 0 at a = n-1) and minv (1/M), both indexed by cell of this line.
template <int S, bool NC, typename F, typename R>
__device__ __forceinline__ void load_line_factor(const LineMap &L, int lane, int cnt,
                                                 const F *__restrict__ l1,
                                                 const F *__restrict__ minv,
                                                 LineFactor<S, R> &f) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (s < cnt) {
            const int a = slot_cell<S>(L, lane, s);
            const R e_lo = (a > 0) ? ldf<NC, F, R>(l1 + a - 1) : R(0);  // couples a-1, a
            const R e_hi = ldf<NC, F, R>(l1 + a);                       // couples a, a+1
            f.minv[s] = ldf<NC, F, R>(minv + a);
            if (lane < 16) { f.ein[s] = e_lo; f.eout[s] = e_hi; }
            else { f.ein[s] = e_hi; f.eout[s] = e_lo; }
        } else {
            f.minv[s] = R(0); f.ein[s] = R(0); f.eout[s] = R(0);
        }
    }
    f.minv_m = ldf<NC, F, R>(minv + L.m);
    f.em1 = (L.m > 0) ? ldf<NC, F, R>(l1 + L.m - 1) : R(0);
    f.em = ldf<NC, F, R>(l1 + L.m);
}

// ---------------------------------------------------------------- level-1 solve
// Solve T x = b for one line with the twisted factorization of Sec. II-A
// (level 1): lower sweep (M + L1) y = b from both ends towards the twist cell,
// the twist cell takes both couplings, then the upper sweep (I + M^{-1} U1) x = y
// from the twist cell outwards.  Each sweep is a first-order affine recurrence
// along a chain, evaluated as lane-local composition + a 16-lane scan +
// lane-local substitution.  b/x are per-slot registers; bm/xm the twist cell.
// This is the apply's form, associated for a short critical path; the setup's
// form (twisted_solve_split, ffp_plane.cuh) splits the slots over two warps.
// Forward: lane-local prefixes y[s] = pa[s] * c + pb[s] of the affine chain,
// with c the value entering the lane.  Backward: x[s] = Xb[s] + Xa[s] * c +
// Gs[s] * cin, where Xb, Xa, Gs are the lane-local suffix compositions of
// x[s] = y[s] + ga[s] x[s+1] applied to pb, pa and 1, and cin the value
// entering from the lane above.  Xb only needs pb and Xa, Gs only factors, so
// all three are formed while the forward scan runs; the critical path is
// forward compose -> forward scan -> backward scan -> one FMA per slot.
template <int S, typename R>
__device__ __forceinline__ void twisted_solve_fast(const LineFactor<S, R> &f, int cnt, int lane,
                                                   const R (&b)[S], R bm, R (&x)[S], R &xm) {
    const int j = lane & 15;
    const unsigned FULL = 0xffffffffu;
    R pa[S], pb[S], ga[S];
    R A = R(1), B = R(0);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const bool v = s < cnt;
        const R a_ = v ? -f.minv[s] * f.ein[s] : R(1);
        const R be = v ? f.minv[s] * b[s] : R(0);
        B = fma(a_, B, be);
        A = A * a_;
        pa[s] = A;
        pb[s] = B;
        ga[s] = v ? -f.minv[s] * f.eout[s] : R(1);
    }
    // suffix compositions of the backward chain (pads: ga = 1 and no own term)
    R Xa[S], Xb[S], Gs[S];
    {
        R xa = R(0), xb = R(0), gs = R(1);
#pragma unroll
        for (int s = S - 1; s >= 0; --s) {
            const bool v = s < cnt;
            xa = fma(ga[s], xa, v ? pa[s] : R(0));
            xb = fma(ga[s], xb, v ? pb[s] : R(0));
            gs = ga[s] * gs;
            Xa[s] = xa; Xb[s] = xb; Gs[s] = gs;
        }
    }
    // forward scan over the 16 lanes of the chain
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const R Au = __shfl_up_sync(FULL, A, d, 16);
        const R Bu = __shfl_up_sync(FULL, B, d, 16);
        if (j >= d) { B = fma(A, Bu, B); A = A * Au; }
    }
    R c = __shfl_up_sync(FULL, B, 1, 16);
    if (j == 0) c = R(0);
    const R ytop = __shfl_sync(FULL, B, 15);
    const R ybot = __shfl_sync(FULL, B, 31);
    // backward scan: lane map x_first = G * x_in + Bb
    R G = Gs[0];
    R Bb = fma(Xa[0], c, Xb[0]);
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const R Gd = __shfl_down_sync(FULL, G, d, 16);
        const R Bd = __shfl_down_sync(FULL, Bb, d, 16);
        if (j + d < 16) { Bb = fma(G, Bd, Bb); G = G * Gd; }
    }
    const R ym = f.minv_m * (bm - f.em1 * ytop - f.em * ybot);
    const R Gn = __shfl_down_sync(FULL, G, 1, 16);
    const R Bn = __shfl_down_sync(FULL, Bb, 1, 16);
    const R cin = (j == 15) ? ym : fma(Gn, ym, Bn);
#pragma unroll
    for (int s = 0; s < S; ++s) x[s] = fma(Gs[s], cin, fma(Xa[s], c, Xb[s]));
    xm = ym;
}

// The same solve from precomputed multipliers (factor line records): al =
// forward multiplier, ga = backward multiplier (both 1 on pads), mi = 1/M
// (0 on pads), and the twist cell.  Pads need no selects except in the
// backward own terms, which must vanish on pads.
template <int S, typename R>
__device__ __forceinline__ void twisted_solve_pre(const R (&al)[S], const R (&ga)[S],
                                                  const R (&mi)[S], R minv_m, R em1, R em,
                                                  int cnt, int lane, const R (&b)[S], R bm,
                                                  R (&x)[S], R &xm) {
    const int j = lane & 15;
    const unsigned FULL = 0xffffffffu;
    R pa[S], pb[S];
    R A = R(1), B = R(0);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        B = fma(al[s], B, mi[s] * b[s]);
        A = A * al[s];
        pa[s] = A;
        pb[s] = B;
    }
    R Xa[S], Xb[S], Gs[S];
    {
        R xa = R(0), xb = R(0), gs = R(1);
#pragma unroll
        for (int s = S - 1; s >= 0; --s) {
            const bool v = s < cnt;
            xa = fma(ga[s], xa, v ? pa[s] : R(0));
            xb = fma(ga[s], xb, v ? pb[s] : R(0));
            gs = ga[s] * gs;
            Xa[s] = xa; Xb[s] = xb; Gs[s] = gs;
        }
    }
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const R Au = __shfl_up_sync(FULL, A, d, 16);
        const R Bu = __shfl_up_sync(FULL, B, d, 16);
        if (j >= d) { B = fma(A, Bu, B); A = A * Au; }
    }
    R c = __shfl_up_sync(FULL, B, 1, 16);
    if (j == 0) c = R(0);
    const R ytop = __shfl_sync(FULL, B, 15);
    const R ybot = __shfl_sync(FULL, B, 31);
    R G = Gs[0];
    R Bb = fma(Xa[0], c, Xb[0]);
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const R Gd = __shfl_down_sync(FULL, G, d, 16);
        const R Bd = __shfl_down_sync(FULL, Bb, d, 16);
        if (j + d < 16) { Bb = fma(G, Bd, Bb); G = G * Gd; }
    }
    const R ym = minv_m * (bm - em1 * ytop - em * ybot);
    const R Gn = __shfl_down_sync(FULL, G, 1, 16);
    const R Bn = __shfl_down_sync(FULL, Bb, 1, 16);
    const R cin = (j == 15) ? ym : fma(Gn, ym, Bn);
#pragma unroll
    for (int s = 0; s < S; ++s) x[s] = fma(Gs[s], cin, fma(Xa[s], c, Xb[s]));
    xm = ym;
}

// ---------------------------------------------------------------- level-1 pivots
// Twisted pivots of the tridiagonal T (recurrence for M_i, Sec. II-A):
// M[c] = D[c] - ein[c]^2 / M[c-1] along each chain, and at the twist cell
// M_m = D_m - em1^2 / M_{m-1} - em^2 / M_{m+1}.  The continued fraction is
// evaluated projectively: M = p/q with (p, q) <- (D p - e^2 q, p), i.e. a
// product of 2x2 matrices, scanned across the 16 lanes of a chain (scaled by
// powers of two, which leaves p/q unchanged) and then substituted slot by
// slot from the lane's incoming (p, q), in FP64 (the setup's form is
// twisted_pivots_split in ffp_setup.cuh; the ILU(0) pivots use the same scheme).
//
// The scale is 2^-e, e the binary exponent of the largest magnitude.  It is
// read from the IEEE-754 bit patterns with integer operations, so that only
// the exact multiplies by 2^-e use the FP64 pipe (a scarce unit on this GPU);
// the result is that of ilogb/scalbn.  Values that are all zero or not all
// finite are left as they are; the rare case of a largest magnitude that is
// subnormal, or too large for 2^-e to be a normal number, takes ilogb/scalbn.
__device__ __forceinline__ int biased_exp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

template <int N>
__device__ __forceinline__ void scale_pow2(double (&v)[N]) {
    int em = 0;
    bool nonzero = false;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        em = max(em, biased_exp(v[i]));
        nonzero |= (__double2hiint(v[i]) & 0x7fffffff) != 0 || __double2loint(v[i]) != 0;
    }
    if (em == 0x7ff || !nonzero) return;  // a value is not finite, or all are zero
    if (em >= 1 && em <= 2045) {
        const double f = __hiloint2double((2046 - em) << 20, 0);  // 2^-(em - 1023)
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] *= f;
        return;
    }
    double mx = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) mx = fmax(mx, fabs(v[i]));
    const int e = ilogb(mx);
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = scalbn(v[i], -e);
}

__device__ __forceinline__ void scale4(double &a, double &b, double &c, double &d) {
    double v[4] = {a, b, c, d};
    scale_pow2<4>(v);
    a = v[0]; b = v[1]; c = v[2]; d = v[3];
}

__device__ __forceinline__ void scale2(double &a, double &b) {
    double v[2] = {a, b};
    scale_pow2<2>(v);
    a = v[0]; b = v[1];
}


// ---------------------------------------------------------------- factor line records
// The apply reads the stored factors line by line in the warp's own order, so
// they are stored as one record per line (i, k), record index i*ny + k, with
// the multipliers of the twisted line solve precomputed:
//   field 0 alpha[32][SP]  -minv_a * (coupling to the chain predecessor)  (pads 1)
//   field 1 gamma[32][SP]  -minv_a * (coupling towards the twist cell)    (pads 1)
//   field 2 minv[32][SP]   1 / M_a                                        (pads 0)
//   field 3 l2[32][SP]     y-band of P_i: coupling of cell a of line k with line k+1 (pads 0)
//   field 4 l3[32][SP]     z-band of A: coupling of cell a of plane i with plane i+1 (pads 0)
//   mid[8]                the twist cell: 1/M_m, T[m-1,m], T[m,m+1], l2, l3, 0, 0, 0
// Fields are lane-major, [32][SP] (slot_pitch).  A record is a multiple of 16
// bytes, so a warp pulls it with 16-byte asynchronous copies.
enum { REC_ALPHA = 0, REC_GAMMA = 1, REC_MINV = 2, REC_L2 = 3, REC_L3 = 4, REC_NFIELD = 5 };
enum { MID_MINV = 0, MID_EM1 = 1, MID_EM = 2, MID_L2 = 3, MID_L3 = 4, REC_NMID = 8 };

// Slots per lane rounded up to a multiple of 4: a lane's slots of a field are
// contiguous and 16-byte aligned, so a lane reads or writes them with vector
// accesses (lane-major layout [32][SP]).
__host__ __device__ constexpr int slot_pitch(int S) { return (S + 3) & ~3; }

__host__ __device__ __forceinline__ long rec_len(int S) {
    return (long)REC_NFIELD * 32 * slot_pitch(S) + REC_NMID;
}
// offset of slot s of lane `lane` of field f, and of the twist-cell block
__host__ __device__ __forceinline__ long rec_slot(int S, int f, int lane, int s) {
    return ((long)f * 32 + lane) * slot_pitch(S) + s;
}
__host__ __device__ __forceinline__ long rec_mid(int S) { return (long)REC_NFIELD * 32 * slot_pitch(S); }

// Line-block layout of the apply's vectors: every line of nx cells is a block
// of 32 SP + 32 values; position lane * SP + s holds the cell of slot s of that
// lane (the register layout of the line solve), position 32 SP the twist cell,
// every other position 0.  Each block is one contiguous, 16-byte aligned row.
__host__ __device__ __forceinline__ long lb_len(int S) { return 32L * slot_pitch(S) + 32; }

__host__ __device__ __forceinline__ long lb_pos(int nx, int S, int a) {
    const int m = (nx - 1) / 2;
    if (a == m) return 32L * slot_pitch(S);
    int c, lane;
    if (a < m) { c = a; lane = c / S; }
    else { c = nx - 1 - a; lane = 16 + c / S; }
    return (long)lane * slot_pitch(S) + c % S;
}

// Cell of position p of a line block, or -1 for a padding position.
__host__ __device__ __forceinline__ int lb_cell(int nx, int S, int p) {
    const int SP = slot_pitch(S);
    const int m = (nx - 1) / 2;
    if (p >= 32 * SP) return (p == 32 * SP) ? m : -1;
    const int lane = p / SP, s = p - lane * SP;
    if (s >= S) return -1;
    const int j = lane & 15;
    const int tot = (lane < 16) ? m : nx - 1 - m;
    const int c = j * S + s;
    if (c >= tot) return -1;
    return (lane < 16) ? c : nx - 1 - c;
}

// Offset inside a record of field f at cell a of an nx-cell line (the twist
// cell maps to mid + midf).
__host__ __device__ __forceinline__ long rec_cell(int nx, int S, int f, int midf, int a) {
    const int m = (nx - 1) / 2;
    if (a == m) return rec_mid(S) + midf;
    int c, lane;
    if (a < m) { c = a; lane = c / S; }
    else { c = nx - 1 - a; lane = 16 + c / S; }
    return rec_slot(S, f, lane, c % S);
}

// ---------------------------------------------------------------- async copies
// The copies carry no compiler memory clobber so that they interleave with the
// arithmetic that follows them; cp_async_wait (which has one) orders the reads
// of the destination after completion, and callers never read a stage that
// copies are still being issued into.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_dyn(int n) {
    switch (n) {
        case 0: cp_async_wait<0>(); break;
        case 1: cp_async_wait<1>(); break;
        case 2: cp_async_wait<2>(); break;
        case 3: cp_async_wait<3>(); break;
        case 4: cp_async_wait<4>(); break;
        default: cp_async_wait<5>(); break;
    }
}

// ---------------------------------------------------------------- mbarriers
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// arrive (release at CTA scope)
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}
// arrive when all of this thread's earlier cp.async copies have completed (count not incremented)
__device__ __forceinline__ void mbar_arrive_cpasync(unsigned long long *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// One bounded try of the phase with the given parity (acquire at CTA scope).
__device__ __forceinline__ bool mbar_try(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Wait for a phase with an iteration limit: returns false (and the caller
// records a timeout) if the phase does not complete in `tries` tries
// (kWaitTries unless a test lowers it).
constexpr unsigned kWaitTries = 1u << 22;
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          unsigned tries = kWaitTries) {
    for (unsigned it = 0; it < tries; ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------- misc
__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The element-per-lane split used by every line kernel: S = the smallest
// supported slot count with 16 * S >= the longer chain of an nx-cell line.
#define FFP_SLOT_LIST(X) X(1) X(2) X(3) X(4) X(6) X(8) X(11) X(16) X(22) X(32)

inline int slots_for(int nx) {
    if (nx > FFP_MAX_NX) return -1;
    const int nbot = nx - 1 - (nx - 1) / 2;
    const int need = (nbot + 15) / 16;
    const int list[] = {1, 2, 3, 4, 6, 8, 11, 16, 22, 32};
    for (int s : list)
        if (s >= need) return s;
    return -1;
}

// ---------------------------------------------------------------- workspace
struct Ws {
    // operator bands (FP64)
    double *d, *cx, *cy, *cz;
    // factors in storage precision: one record per line (see rec_len), l3 =
    // z-band of A in natural order (for the ILU(0) sweeps), l1 = x-band of T in
    // natural order (kept for ffp_export)
    void *rec, *l3, *l1;
    // combination preconditioner: ILU(0) 1/D and the x, y bands of A in storage precision
    void *dinv, *lx, *ly;
    // combination temporaries
    double *c1, *c2;
    // CG vectors
    double *r, *z, *p, *q;
    // the apply's input and output in the line-block layout (lb_pos), in the
    // apply's arithmetic type (FP64 for FP64 factors, FP32 otherwise)
    void *ra, *za;
    // apply scratch: 2 planes (one per level-3 half), line-block layout, same type
    void *ascr;
    // setup scratch, per half h: P bands ping-pong [h][pp][3], FP64 line factors of the
    // current plane [h][2] (l1, minv), w/v/beta plane [h][2], correction to the twist plane [h][3]
    double *sP[2][2][3];
    double *sF[2][2];
    double *sW[2][2];
    double *sC[2][3];
    // ILU(0) sweeps: ready flag per line [ny * nz] (flagged forms); sync head [32]
    // (ticket counters, sweep epoch); with FP32/BF16 factors the FP32 copy of r [N]
    // and the tagged result words [N] (FP32 value + sweep tag; the dataflow form
    // keeps its FP32 t there), else null
    int *ilu_ready;
    int *ilu_sync;
    void *ilu_v;
    unsigned long long *ilu_tw;
    // reductions
    double *red;   // partial sums [kRedSlots]
    double *scal;  // scalars [kScal]
    int *flags;    // error flags [16]
};

// The CG drivers stop with FFP_ERR_NOT_CONVERGED when this many true-residual
// confirmations in a row fail to halve the best true residual: the tolerance
// lies below what the FP64 iterate can reach (eps |A||x| / |b|).
constexpr int kStallConfirms = 3;

constexpr int kRedBlocks = 1216;  // 8 x 152 SMs
constexpr int kRedSlots = kRedBlocks * 4;
constexpr int kScal = 64;

// scalar slots
enum {
    SC_BB = 0,     // ||b||^2
    SC_RR = 1,     // ||r||^2 (recursive)
    SC_RHO = 2,    // (r, z)
    SC_RHO_OLD = 3,
    SC_PQ = 4,     // (p, A p)
    SC_ALPHA = 5,
    SC_BETA = 6,
    SC_ZQ = 7,     // (z, q)  (flexible CG)
    SC_TRR = 8,    // ||b - A x||^2
};
// flag slots
enum { FL_BREAKDOWN = 0, FL_ARG = 1, FL_PQ = 2, FL_TIMEOUT = 3 };

}  // namespace ffp
