// ffp_setup.cu -- construction of the nested twisted filtering preconditioner
// (Sec. II-A), FP64, stored in the requested precision.
//
// Level 3 (planes), twisted at mz = floor((nz-1)/2):
//   phase 0 (2 CTAs, one per half): P_0 = Dhat_0 (top) / P_{nz-1} = Dhat_{nz-1}
//     (bottom); for each plane of the half, in elimination order:
//       (a) level-2 factorization of P_i (lines, below),
//       (b) w = C t_dst, v = B_{P,i}^{-1} w by the nested plane solve (reading R1),
//           beta = v ./ w,
//       (c) the Schur term C (2 beta - beta P_i beta) C of the next plane dst of
//           the chain: P_dst = Dhat_dst - C X C, or, for the last plane of the
//           half, saved for the twist plane.
//   phase 1 (1 CTA): P_mz = Dhat_mz - (term from mz-1) - (term from mz+1), then
//     its level-2 factorization.
// The batched setup runs phase 0 fused in one launch per instance table.  The
// single-instance setup runs every plane step of phase 0 as two launches, (a)-(b)
// on the two CTAs of the chains and the cell-wise rest of (b)-(c) on the whole GPU
// (setup_plane_kernel, setup_cells_kernel below), with the same arithmetic.
// Level 2 (lines of P_i), twisted at my = floor((ny-1)/2), two warps per half
// that split every line's slots (warps 0/2 and 1/3, see SlotSplit):
//   T_0 = Dbar_0 / T_{ny-1} = Dbar_{ny-1}; T_k = Dbar_k - p X p with
//   X = 2 beta - beta T_prev beta, beta = (T_prev^{-1} w) ./ w, w = p .* t_k,
//   p = y-band of P_i between the two lines; the twist line takes both terms.
// Level 1: twisted pivots M of every T_k (exact), see twisted_pivots().
// Stored: l1 = x-band of T_k, minv = 1/M, l2 = y-band of P_i (l3 = z-band of A
// is converted separately).
#pragma once
#include <algorithm>
#include <cstring>

#include "ffp_plane.cuh"
#include "ffp_kernels.h"

namespace ffp {

#ifdef FFP_STEP_PROFILE
// Setup profile (profiling builds only): clock64 cycles of thread 0 of the first
// level-3 half, accumulated over its planes: [0] level-2 factorization, of which
// [5] line Schur terms, [6] line pivots, [7] line stores; [1] the w vector; [2] the
// nested plane solve; [3] beta = v ./ w; [4] the Schur term of the next plane;
// [8] planes; [9] the whole plane loop.
static __device__ unsigned long long g_setup_prof[16];
__device__ __forceinline__ unsigned long long setup_stamp() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(t)::"memory");
    return t;
}
#define FFP_SPROF(...) __VA_ARGS__
#else
#define FFP_SPROF(...)
#endif

// Store one factor entry in the storage precision.
__device__ __forceinline__ void put_factor(void *base, long idx, double v, int prec) {
    if (prec == FFP_FP64) static_cast<double *>(base)[idx] = v;
    else if (prec == FFP_FP32) static_cast<float *>(base)[idx] = (float)v;
    else static_cast<__nv_bfloat16 *>(base)[idx] = __double2bfloat16(v);
}

struct SetupPol {
    const double *W;
    double *V;
    int nx;
    __device__ __forceinline__ double rhs(int k, int a) const { return W[(long)k * nx + a]; }
    __device__ __forceinline__ void put_w(int k, int a, double w) const { V[(long)k * nx + a] = w; }
    __device__ __forceinline__ double get_w(int k, int a) const { return V[(long)k * nx + a]; }
    __device__ __forceinline__ void put_out(int k, int a, double u) const { V[(long)k * nx + a] = u; }
};

// w = c3 (.) t of one cell of the next plane (t = 1 for rowsum).
__device__ __forceinline__ double w_cell(const double *C, const double *T, long e) {
    return __dmul_rn(C[e], T ? T[e] : 1.0);
}
// beta-hat = (B_P^{-1} w) ./ w of one cell (Sec. II-A), 1/P_ee where w vanishes.
__device__ __forceinline__ double beta_cell(double v, double w, double pd) {
    const bool z = fabs(w) < 1e-300;
    return __ddiv_rn(z ? 1.0 : v, z ? pd : w);
}
// The Schur term C X C at cell e of the next plane dst (X = 2 beta - beta P beta,
// or X = beta with `schur`), from beta-hat at e, e+1 and e+nx: written as the
// term itself (to_mid: the twist plane collects both halves' terms) or as
// P_dst = Dhat_dst - C X C.  The same rounded operations in every setup form.
__device__ __forceinline__ void schur_cell(long e, int ix, int iy, int nx, int ny, int schur, double be,
                                           double be1, double beny, const double *Pd, const double *Px,
                                           const double *Py, const double *C, bool to_mid,
                                           const double *dd, const double *dx, const double *dy,
                                           double *od, double *ox, double *oy) {
    const double xd = schur ? be : __fma_rn(2.0, be, -__dmul_rn(__dmul_rn(be, Pd[e]), be));
    const double cd = __dmul_rn(__dmul_rn(C[e], xd), C[e]);
    double cxo = 0.0, cyo = 0.0;
    if (ix + 1 < nx && !schur) {
        const double xo = __dmul_rn(__dmul_rn(-be, Px[e]), be1);
        cxo = __dmul_rn(__dmul_rn(C[e], xo), C[e + 1]);
    }
    if (iy + 1 < ny && !schur) {
        const double xo = __dmul_rn(__dmul_rn(-be, Py[e]), beny);
        cyo = __dmul_rn(__dmul_rn(C[e], xo), C[e + nx]);
    }
    if (to_mid) {
        od[e] = cd; ox[e] = cxo; oy[e] = cyo;
    } else {
        od[e] = __dsub_rn(dd[e], cd);
        ox[e] = __dsub_rn(dx[e], cxo);
        oy[e] = __dsub_rn(dy[e], cyo);
    }
}

// State of the previous line T_prev as seen by this lane (this part's slots).
template <int S>
struct LineState {
    LineFactor<S, double> f;
    double Td[S], To[S], Tdm, Tom;
};

// twisted_pivots (level 1) with the slots split over the two parts of sp:
// each part multiplies its own slots' 2x2 matrices, the lane's product is
// formed from both, both parts scan it, and part 1 enters its slots with part
// 0's product applied.  minv is valid on this part's slots.
template <int S>
__device__ __forceinline__ void twisted_pivots_split(int cnt, int lane, const double (&D)[S],
                                                     const double (&ein)[S], double Dm, double em1,
                                                     double em, double (&minv)[S], double &minv_m,
                                                     bool &bad, SlotSplit &sp) {
    const int j = lane & 15;
    const unsigned FULL = 0xffffffffu;
    // this part's product E_{s1-1} ... E_{s0}, E = [[D, -e^2], [1, 0]] (pads are identity)
    double p11 = 1.0, p12 = 0.0, p21 = 0.0, p22 = 1.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (sp.mine(s) && s < cnt) {
            const double e2 = ein[s] * ein[s];
            const double n11 = D[s] * p11 - e2 * p21;
            const double n12 = D[s] * p12 - e2 * p22;
            p21 = p11; p22 = p12; p11 = n11; p12 = n12;
        }
    }
    // P0 = part 0's product, P1 = part 1's; the lane's product is P1 P0
    double a11, a12, a21, a22, f11, f12, f21, f22;
    {
        const double mv[4] = {p11, p12, p21, p22};
        double o[4];
        sp.swap<4>(mv, o, lane);
        const double b11 = sp.part ? p11 : o[0], b12 = sp.part ? p12 : o[1];
        const double b21 = sp.part ? p21 : o[2], b22 = sp.part ? p22 : o[3];
        a11 = sp.part ? o[0] : p11; a12 = sp.part ? o[1] : p12;
        a21 = sp.part ? o[2] : p21; a22 = sp.part ? o[3] : p22;
        f11 = b11 * a11 + b12 * a21;
        f12 = b11 * a12 + b12 * a22;
        f21 = b21 * a11 + b22 * a21;
        f22 = b21 * a12 + b22 * a22;
    }
    scale4(f11, f12, f21, f22);
    // inclusive scan: lane j <- (lane j) x (lane j-d)
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const double q11 = __shfl_up_sync(FULL, f11, d, 16);
        const double q12 = __shfl_up_sync(FULL, f12, d, 16);
        const double q21 = __shfl_up_sync(FULL, f21, d, 16);
        const double q22 = __shfl_up_sync(FULL, f22, d, 16);
        if (j >= d) {
            const double n11 = f11 * q11 + f12 * q21;
            const double n12 = f11 * q12 + f12 * q22;
            const double n21 = f21 * q11 + f22 * q21;
            const double n22 = f21 * q12 + f22 * q22;
            f11 = n11; f12 = n12; f21 = n21; f22 = n22;
            scale4(f11, f12, f21, f22);
        }
    }
    // incoming (p, q) = first column of the prefix of lane j-1 ((1, 0) for lane 0);
    // part 1 enters its first slot after part 0's slots
    double pp = __shfl_up_sync(FULL, f11, 1, 16);
    double qq = __shfl_up_sync(FULL, f21, 1, 16);
    if (j == 0) { pp = 1.0; qq = 0.0; }
    scale2(pp, qq);
    if (sp.part) {
        const double np = a11 * pp + a12 * qq, nq = a21 * pp + a22 * qq;
        pp = np;
        qq = nq;
        scale2(pp, qq);
    }
    bool b_ = false;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (!sp.mine(s)) continue;
        if (s < cnt) {
            const double e2 = ein[s] * ein[s];
            const double np = D[s] * pp - e2 * qq;
            qq = pp;
            pp = np;
            const double mi = qq / pp;
            minv[s] = mi;
            b_ |= !(mi > 0.0) || !isfinite(mi);
        } else {
            minv[s] = 0.0;
        }
    }
    // chain ends: 1/M_{m-1} = q/p of the top prefix (lane 15), 1/M_{m+1} of lane 31
    const double t_inv = __shfl_sync(FULL, f21, 15) / __shfl_sync(FULL, f11, 15);
    const double b_inv = __shfl_sync(FULL, f21, 31) / __shfl_sync(FULL, f11, 31);
    const double Mm = Dm - em1 * em1 * t_inv - em * em * b_inv;
    minv_m = 1.0 / Mm;
    b_ |= !(Mm > 0.0) || !isfinite(Mm);
    bad = b_;
}

// beta of the level-2 Schur term from T_prev onto the line with coupling p
// (global, this line's cells) and filter tl (or NULL): returns the terms
// cd = p X p (diagonal) and co = p X p (x-band) per slot of this part and for
// the twist cell.
template <int S>
__device__ __forceinline__ void line_schur(const LineMap &L, int nx, int lane, int cnt,
                                           const LineState<S> &st, const double *p,
                                           const double *tl, double *SB, double *SP,
                                           double (&cd)[S], double (&co)[S], double &cdm,
                                           double &com, SlotSplit &sp, int classic) {
    double w[S], wm, pa[S], pm;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        pa[s] = 0.0; w[s] = 0.0;
        if (sp.mine(s) && s < cnt) {
            const int a = slot_cell<S>(L, lane, s);
            pa[s] = p[a];
            w[s] = pa[s] * (tl ? tl[a] : 1.0);
        }
    }
    pm = p[L.m];
    wm = pm * (tl ? tl[L.m] : 1.0);
    double v[S], vm;
    twisted_solve_split<S, double>(st.f, cnt, lane, w, wm, v, vm, sp);  // v = T_prev^{-1} w
    double be[S], bem;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        be[s] = 0.0;
        if (sp.mine(s) && s < cnt) {
            const bool z = fabs(w[s]) < 1e-300;  // one divide either way
            be[s] = (z ? 1.0 : v[s]) / (z ? st.Td[s] : w[s]);
            const int a = slot_cell<S>(L, lane, s);
            SB[a] = be[s];
            SP[a] = pa[s];
        }
    }
    {
        const bool z = fabs(wm) < 1e-300;
        bem = (z ? 1.0 : vm) / (z ? st.Tdm : wm);
    }
    if (lane == 0 && sp.part == 0) { SB[L.m] = bem; SP[L.m] = pm; }
    sp.sync();
#pragma unroll
    for (int s = 0; s < S; ++s) {
        cd[s] = 0.0; co[s] = 0.0;
        if (sp.mine(s) && s < cnt) {
            const int a = slot_cell<S>(L, lane, s);
            const double xd = classic ? be[s] : 2.0 * be[s] - be[s] * st.Td[s] * be[s];
            cd[s] = pa[s] * xd * pa[s];
            if (a + 1 < nx && !classic) {
                const double xo = -be[s] * st.To[s] * SB[a + 1];
                co[s] = pa[s] * xo * SP[a + 1];
            }
        }
    }
    {
        const double xd = classic ? bem : 2.0 * bem - bem * st.Tdm * bem;
        cdm = pm * xd * pm;
        if (L.m + 1 < nx && !classic) {
            const double xo = -bem * st.Tom * SB[L.m + 1];
            com = pm * xo * SP[L.m + 1];
        } else {
            com = 0.0;
        }
    }
    sp.sync();
}

// Twisted pivots of T = tridiag(To, Td, To) of one line -> line state (this part's slots).
template <int S>
__device__ __forceinline__ void factor_line(const LineMap &L, int lane, int cnt,
                                            const double (&Td)[S], const double (&To)[S],
                                            double Tdm, double Tom, double *SO,
                                            LineState<S> &st, int *flags, SlotSplit &sp) {
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (sp.mine(s) && s < cnt) SO[slot_cell<S>(L, lane, s)] = To[s];
    if (lane == 0 && sp.part == 0) SO[L.m] = Tom;
    sp.sync();
    double ein[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        st.f.ein[s] = 0.0; st.f.eout[s] = 0.0; ein[s] = 0.0;
        if (sp.mine(s) && s < cnt) {
            const int a = slot_cell<S>(L, lane, s);
            const double e_lo = (a > 0) ? SO[a - 1] : 0.0;
            const double e_hi = To[s];
            if (lane < 16) { st.f.ein[s] = e_lo; st.f.eout[s] = e_hi; }
            else { st.f.ein[s] = e_hi; st.f.eout[s] = e_lo; }
            ein[s] = st.f.ein[s];
        }
        st.Td[s] = Td[s];
        st.To[s] = To[s];
    }
    st.f.em1 = (L.m > 0) ? SO[L.m - 1] : 0.0;
    st.f.em = Tom;
    st.Tdm = Tdm;
    st.Tom = Tom;
    bool bad = false;
    twisted_pivots_split<S>(cnt, lane, Td, ein, Tdm, st.f.em1, st.f.em, st.f.minv, st.f.minv_m, bad, sp);
    if (bad) atomicOr(flags + FL_BREAKDOWN, 1);
    sp.sync();
}

// Store line k of the plane (this part's slots; the twist cell by part 0):
// FP64 natural-order copies for the setup's own plane solves (l1d, mid), the
// natural-order l1 (for export) and the line record line0 + k: the line
// solve's multipliers -1/M * coupling (forward and backward), 1/M and the
// twist cell.
template <int S>
__device__ __forceinline__ void store_line(const LineMap &L, int lane, int cnt, int nx, int k,
                                           const LineState<S> &st, double *l1d, double *mid,
                                           void *rec, void *l1n, long line0, int prec,
                                           const SlotSplit &sp) {
    const long o = (long)k * nx;
    const long rb = (line0 + k) * rec_len(S);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (!sp.mine(s)) continue;
        const bool v = s < cnt;
        if (v) {
            const int a = slot_cell<S>(L, lane, s);
            l1d[o + a] = st.To[s];
            mid[o + a] = st.f.minv[s];
            put_factor(l1n, (line0 + k) * nx + a, st.To[s], prec);
        }
        put_factor(rec, rb + rec_slot(S, REC_ALPHA, lane, s), v ? -st.f.minv[s] * st.f.ein[s] : 1.0, prec);
        put_factor(rec, rb + rec_slot(S, REC_GAMMA, lane, s), v ? -st.f.minv[s] * st.f.eout[s] : 1.0, prec);
        put_factor(rec, rb + rec_slot(S, REC_MINV, lane, s), v ? st.f.minv[s] : 0.0, prec);
    }
    if (lane == 0 && sp.part == 0) {
        l1d[o + L.m] = st.Tom;
        mid[o + L.m] = st.f.minv_m;
        put_factor(l1n, (line0 + k) * nx + L.m, st.Tom, prec);
        const long mb = rb + rec_mid(S);
        put_factor(rec, mb + MID_MINV, st.f.minv_m, prec);
        put_factor(rec, mb + MID_EM1, st.f.em1, prec);
        put_factor(rec, mb + MID_EM, st.f.em, prec);
    }
}

// Level-2 factorization of one plane (warps 0-3: half wid = warp & 1 on two
// warps that split the slots).  Pd/Px/Py: bands of P (plane slice, FP64); tp:
// filter on the plane or NULL; outputs the FP64 line factors (l1d, mid) used
// by the nested plane solve and the stored factors.
template <int S>
__device__ void level2_setup(const LineMap &L, int nx, int ny, const double *Pd,
                             const double *Px, const double *Py, const double *tp, double *l1d,
                             double *mid, void *rec, void *l1n, long line0, int prec,
                             double *lbuf, double *meet, int wid, int lane, int cnt,
                             int *flags, SlotSplit &sp, int classic,
                             unsigned long long *prof = nullptr) {
    const int my = (ny - 1) / 2;
    const int nl = (wid == 0) ? my : ny - 1 - my;
    double *SB = lbuf + wid * 3 * nx, *SP = SB + nx, *SO = SP + nx;
    LineState<S> st;
    double Td[S], To[S], Tdm, Tom, cd[S], co[S], cdm, com;
    for (int t = 0; t < nl; ++t) {
        const int k = (wid == 0) ? t : ny - 1 - t;
        const long o = (long)k * nx;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            Td[s] = 1.0; To[s] = 0.0;
            if (sp.mine(s) && s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                Td[s] = Pd[o + a];
                To[s] = Px[o + a];
            }
        }
        Tdm = Pd[o + L.m];
        Tom = Px[o + L.m];
        FFP_SPROF(const unsigned long long q0 = setup_stamp();)
        if (t > 0) {
            const int kc = (wid == 0) ? k - 1 : k;
            line_schur<S>(L, nx, lane, cnt, st, Py + (long)kc * nx, tp ? tp + o : nullptr, SB, SP,
                          cd, co, cdm, com, sp, classic);
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (sp.mine(s)) { Td[s] -= cd[s]; To[s] -= co[s]; }
            Tdm -= cdm;
            Tom -= com;
        }
        FFP_SPROF(const unsigned long long q1 = setup_stamp();)
        factor_line<S>(L, lane, cnt, Td, To, Tdm, Tom, SO, st, flags, sp);
        FFP_SPROF(const unsigned long long q2 = setup_stamp();)
        store_line<S>(L, lane, cnt, nx, k, st, l1d, mid, rec, l1n, line0, prec, sp);
        FFP_SPROF(if (prof) { const unsigned long long q3 = setup_stamp();
                              prof[5] += q1 - q0; prof[6] += q2 - q1; prof[7] += q3 - q2; })
    }
    // twist line: Schur terms from both halves
    {
        const long o = (long)my * nx;
        const int kc = (wid == 0) ? my - 1 : my;
        if (nl > 0) {
            line_schur<S>(L, nx, lane, cnt, st, Py + (long)kc * nx, tp ? tp + o : nullptr, SB, SP,
                          cd, co, cdm, com, sp, classic);
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) { cd[s] = 0.0; co[s] = 0.0; }
            cdm = 0.0; com = 0.0;
        }
        double *MD = meet + wid * 2 * nx, *MO = MD + nx;
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (sp.mine(s) && s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                MD[a] = cd[s];
                MO[a] = co[s];
            }
        if (lane == 0 && sp.part == 0) { MD[L.m] = cdm; MO[L.m] = com; }
        named_barrier(2, 128);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            Td[s] = 1.0; To[s] = 0.0;
            if (sp.mine(s) && s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                Td[s] = Pd[o + a] - meet[a] - meet[2 * nx + a];
                To[s] = Px[o + a] - meet[nx + a] - meet[3 * nx + a];
            }
        }
        Tdm = Pd[o + L.m] - meet[L.m] - meet[2 * nx + L.m];
        Tom = Px[o + L.m] - meet[nx + L.m] - meet[3 * nx + L.m];
        factor_line<S>(L, lane, cnt, Td, To, Tdm, Tom, SO, st, flags, sp);
        if (wid == 0) store_line<S>(L, lane, cnt, nx, my, st, l1d, mid, rec, l1n, line0, prec, sp);
    }
}

template <int S>
__device__ __forceinline__ void setup_body(const SetupArgs &A, int phase) {
    extern __shared__ __align__(16) double sm[];
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const long nxy = (long)nx * ny;
    double *gbuf = sm;                 // plane solve exchange [2][2][nx]
    double *lbuf = sm + 4 * nx;        // level-2 line buffers [2 warps][3][nx]
    double *meet = sm + 10 * nx;       // level-2 twist exchange [2 halves][2][nx]
    double *ex = sm + 14 * nx;         // slot-split exchange [2 halves][512]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // warps 0-3 run the level-2 work: half wid & 1, slot part wid >> 1, so the four
    // warps sit on the four scheduler partitions (pair barriers 3 and 4)
    const int half = wid & 1;
    SlotSplit sp = make_split<S>(wid >> 1, ex + half * 512, 3 + half);
    const LineMap L(nx);
    const int cnt = lane_count<S>(L, lane);
    const int mz = (nz - 1) / 2;
    int *flags = A.ws.flags;
    if (phase == 0) {
        const int h = blockIdx.x;
        const int nl3 = (h == 0) ? mz : nz - 1 - mz;
        double *l1d = A.ws.sF[h][0], *mid = A.ws.sF[h][1];
        double *W = A.ws.sW[h][0], *V = A.ws.sW[h][1];
        FFP_SPROF(const bool sprof = h == 0 && blockIdx.y == 0 && tid == 0;
                  unsigned long long pacc[16] = {0};
                  const unsigned long long pstart = setup_stamp();)
        for (int t = 0; t < nl3; ++t) {
            FFP_SPROF(const unsigned long long s0 = setup_stamp();)
            const int i = (h == 0) ? t : nz - 1 - t;
            const double *Pd, *Px, *Py;
            if (t == 0) {
                Pd = A.d + i * nxy; Px = A.cx + i * nxy; Py = A.cy + i * nxy;
            } else {
                Pd = A.ws.sP[h][t & 1][0]; Px = A.ws.sP[h][t & 1][1]; Py = A.ws.sP[h][t & 1][2];
            }
            for (long e = tid; e < nxy; e += blockDim.x)
                put_factor(A.rec, ((long)i * ny + e / nx) * rec_len(S) +
                                      rec_cell(nx, S, REC_L2, MID_L2, (int)(e % nx)),
                           Py[e], A.prec);
            if (wid < 4)
                level2_setup<S>(L, nx, ny, Pd, Px, Py, A.t ? A.t + i * nxy : nullptr, l1d, mid,
                                A.rec, A.l1n, (long)i * ny, A.prec, lbuf, meet, half, lane, cnt,
                                flags, sp, A.schur FFP_SPROF(, sprof ? pacc : nullptr));
            FFP_SPROF(const unsigned long long s1 = setup_stamp();)
            const int dst = (t == nl3 - 1) ? mz : ((h == 0) ? i + 1 : i - 1);
            const int ic = (i < dst) ? i : dst;
            const double *C = A.cz + ic * nxy;
            for (long e = tid; e < nxy; e += blockDim.x)
                W[e] = w_cell(C, A.t ? A.t + dst * nxy : nullptr, e);
            __syncthreads();
            FFP_SPROF(const unsigned long long s2 = setup_stamp();)
            if (wid < 4) {
                SetupPol pol{W, V, nx};
                plane_solve<S, false, double, double>(L, nx, ny, l1d, mid, Py, pol, gbuf, half, lane,
                                                      cnt, sp);
            }
            __syncthreads();
            FFP_SPROF(const unsigned long long s3 = setup_stamp();)
            for (long e = tid; e < nxy; e += blockDim.x) V[e] = beta_cell(V[e], W[e], Pd[e]);
            __syncthreads();
            FFP_SPROF(const unsigned long long s4 = setup_stamp();)
            const bool to_mid = (dst == mz);
            double *od = to_mid ? A.ws.sC[h][0] : A.ws.sP[h][(t + 1) & 1][0];
            double *ox = to_mid ? A.ws.sC[h][1] : A.ws.sP[h][(t + 1) & 1][1];
            double *oy = to_mid ? A.ws.sC[h][2] : A.ws.sP[h][(t + 1) & 1][2];
            const long g0 = (long)dst * nxy;
            for (long e = tid; e < nxy; e += blockDim.x) {
                const int ix = (int)(e % nx), iy = (int)(e / nx);
                schur_cell(e, ix, iy, nx, ny, A.schur, V[e], ix + 1 < nx ? V[e + 1] : 0.0,
                           iy + 1 < ny ? V[e + nx] : 0.0, Pd, Px, Py, C, to_mid, A.d + g0, A.cx + g0,
                           A.cy + g0, od, ox, oy);
            }
            __syncthreads();
            FFP_SPROF(if (sprof) { const unsigned long long s5 = setup_stamp();
                                   pacc[0] += s1 - s0; pacc[1] += s2 - s1; pacc[2] += s3 - s2;
                                   pacc[3] += s4 - s3; pacc[4] += s5 - s4; pacc[8] += 1; })
        }
        FFP_SPROF(if (sprof) {
            pacc[9] = setup_stamp() - pstart;
            for (int q = 0; q < 16; ++q) g_setup_prof[q] = pacc[q];
        })
    } else {
        double *Pd = A.ws.sP[0][0][0], *Px = A.ws.sP[0][0][1], *Py = A.ws.sP[0][0][2];
        const long g0 = (long)mz * nxy;
        for (long e = tid; e < nxy; e += blockDim.x) {
            double vd = A.d[g0 + e], vx = A.cx[g0 + e], vy = A.cy[g0 + e];
            if (mz > 0) { vd -= A.ws.sC[0][0][e]; vx -= A.ws.sC[0][1][e]; vy -= A.ws.sC[0][2][e]; }
            if (mz < nz - 1) { vd -= A.ws.sC[1][0][e]; vx -= A.ws.sC[1][1][e]; vy -= A.ws.sC[1][2][e]; }
            Pd[e] = vd; Px[e] = vx; Py[e] = vy;
            put_factor(A.rec, ((long)mz * ny + e / nx) * rec_len(S) +
                                  rec_cell(nx, S, REC_L2, MID_L2, (int)(e % nx)),
                       vy, A.prec);
        }
        __syncthreads();
        if (wid < 4)
            level2_setup<S>(L, nx, ny, Pd, Px, Py, A.t ? A.t + g0 : nullptr, A.ws.sF[0][0],
                            A.ws.sF[0][1], A.rec, A.l1n, (long)mz * ny, A.prec, lbuf, meet, half,
                            lane, cnt, flags, sp, A.schur);
    }
}

// Phase 0: one CTA per level-3 half; phase 1: the twist plane.  The instance
// is A0, or table[blockIdx.y] when a table is given.
template <int S>
__global__ void __launch_bounds__(256) setup_kernel(const __grid_constant__ SetupArgs A0,
                                                    const SetupArgs *__restrict__ table, int phase) {
    const SetupArgs &A = table ? table[blockIdx.y] : A0;
    if (phase == 0 && A.nz <= 1) return;  // a single plane has no level-3 halves
    setup_body<S>(A, phase);
}

// ---------------------------------------------------------------- single instance, per plane
// The single-instance setup runs every level-3 plane step as two launches: the
// level-2 factorization and the nested plane solve on one CTA per half (the two
// chains), then the step's cell-wise work -- beta-hat, the next plane's Schur
// term, that plane's l2 records -- spread over the whole GPU.  The arithmetic is
// the fused form's, cell for cell (w_cell, beta_cell, schur_cell); beta-hat of
// the neighbours e+1 and e+nx is recomputed where it is read, so the second
// launch needs no grid-wide barrier, and w is formed where it is read.

struct SetupPolOtf {  // the plane solve's right-hand side w = c3 (.) t, formed on read
    const double *C, *T;
    double *V;
    int nx;
    __device__ __forceinline__ double rhs(int k, int a) const { return w_cell(C, T, (long)k * nx + a); }
    __device__ __forceinline__ void put_w(int k, int a, double w) const { V[(long)k * nx + a] = w; }
    __device__ __forceinline__ double get_w(int k, int a) const { return V[(long)k * nx + a]; }
    __device__ __forceinline__ void put_out(int k, int a, double u) const { V[(long)k * nx + a] = u; }
};

// Plane step t of level-3 half h: the plane i, its operator bands, the plane dst
// the step eliminates towards and the z-coupling plane ic between them.
struct PlaneStep {
    int i, dst, ic, nl3;
    bool to_mid;
    const double *Pd, *Px, *Py;
};
__device__ __forceinline__ PlaneStep plane_step(const SetupArgs &A, int h, int t) {
    const long nxy = (long)A.nx * A.ny;
    const int mz = (A.nz - 1) / 2;
    PlaneStep p;
    p.nl3 = (h == 0) ? mz : A.nz - 1 - mz;
    p.i = (h == 0) ? t : A.nz - 1 - t;
    if (t == 0) {
        p.Pd = A.d + p.i * nxy; p.Px = A.cx + p.i * nxy; p.Py = A.cy + p.i * nxy;
    } else {
        p.Pd = A.ws.sP[h][t & 1][0]; p.Px = A.ws.sP[h][t & 1][1]; p.Py = A.ws.sP[h][t & 1][2];
    }
    p.dst = (t == p.nl3 - 1) ? mz : ((h == 0) ? p.i + 1 : p.i - 1);
    p.ic = (p.i < p.dst) ? p.i : p.dst;
    p.to_mid = (p.dst == mz);
    return p;
}

// Launch 1 of plane step t: one CTA per half (blockIdx.x), 256 threads.
template <int S>
__global__ void __launch_bounds__(256) setup_plane_kernel(const __grid_constant__ SetupArgs A, int t) {
    extern __shared__ __align__(16) double sm[];
    const int h = blockIdx.x;
    const PlaneStep p = plane_step(A, h, t);
    if (A.nz <= 1 || t >= p.nl3) return;
    const int nx = A.nx, ny = A.ny;
    const long nxy = (long)nx * ny;
    double *gbuf = sm, *lbuf = sm + 4 * nx, *meet = sm + 10 * nx, *ex = sm + 14 * nx;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, half = wid & 1;
    SlotSplit sp = make_split<S>(wid >> 1, ex + half * 512, 3 + half);
    const LineMap L(nx);
    const int cnt = lane_count<S>(L, lane);
    FFP_SPROF(const bool sprof = h == 0 && tid == 0; unsigned long long lacc[16] = {0};
              const unsigned long long s0 = setup_stamp();)
    if (t == 0)  // the first plane's l2 records (later planes': launch 2 of the step before)
        for (long e = tid; e < nxy; e += blockDim.x)
            put_factor(A.rec, ((long)p.i * ny + e / nx) * rec_len(S) +
                                  rec_cell(nx, S, REC_L2, MID_L2, (int)(e % nx)),
                       p.Py[e], A.prec);
    double *l1d = A.ws.sF[h][0], *mid = A.ws.sF[h][1];
    if (wid < 4)
        level2_setup<S>(L, nx, ny, p.Pd, p.Px, p.Py, A.t ? A.t + p.i * nxy : nullptr, l1d, mid, A.rec,
                        A.l1n, (long)p.i * ny, A.prec, lbuf, meet, half, lane, cnt, A.ws.flags, sp,
                        A.schur FFP_SPROF(, sprof ? lacc : nullptr));
    __syncthreads();
    FFP_SPROF(const unsigned long long s1 = setup_stamp();)
    if (wid < 4) {
        SetupPolOtf pol{A.cz + p.ic * nxy, A.t ? A.t + p.dst * nxy : nullptr, A.ws.sW[h][1], nx};
        plane_solve<S, false, double, double>(L, nx, ny, l1d, mid, p.Py, pol, gbuf, half, lane, cnt, sp);
    }
    FFP_SPROF(if (sprof) {
        const unsigned long long s2 = setup_stamp();
        atomicAdd(&g_setup_prof[0], s1 - s0);
        atomicAdd(&g_setup_prof[2], s2 - s1);
        for (int q = 5; q < 8; ++q) atomicAdd(&g_setup_prof[q], lacc[q]);
        atomicAdd(&g_setup_prof[8], 1ull);
    })
}

// Launch 2 of plane step t: the cell-wise work, blockIdx.y = half.
template <int S>
__global__ void __launch_bounds__(256) setup_cells_kernel(const __grid_constant__ SetupArgs A, int t) {
    const int h = blockIdx.y;
    const PlaneStep p = plane_step(A, h, t);
    if (A.nz <= 1 || t >= p.nl3) return;
    const int nx = A.nx, ny = A.ny;
    const long nxy = (long)nx * ny;
    const double *C = A.cz + p.ic * nxy, *T = A.t ? A.t + p.dst * nxy : nullptr;
    const double *V = A.ws.sW[h][1];
    double *od = p.to_mid ? A.ws.sC[h][0] : A.ws.sP[h][(t + 1) & 1][0];
    double *ox = p.to_mid ? A.ws.sC[h][1] : A.ws.sP[h][(t + 1) & 1][1];
    double *oy = p.to_mid ? A.ws.sC[h][2] : A.ws.sP[h][(t + 1) & 1][2];
    const long g0 = (long)p.dst * nxy;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nxy; e += (long)gridDim.x * blockDim.x) {
        const int ix = (int)(e % nx), iy = (int)(e / nx);
        const double be = beta_cell(V[e], w_cell(C, T, e), p.Pd[e]);
        const double be1 = ix + 1 < nx ? beta_cell(V[e + 1], w_cell(C, T, e + 1), p.Pd[e + 1]) : 0.0;
        const double beny = iy + 1 < ny ? beta_cell(V[e + nx], w_cell(C, T, e + nx), p.Pd[e + nx]) : 0.0;
        schur_cell(e, ix, iy, nx, ny, A.schur, be, be1, beny, p.Pd, p.Px, p.Py, C, p.to_mid, A.d + g0,
                   A.cx + g0, A.cy + g0, od, ox, oy);
        if (!p.to_mid)  // the next plane's l2 records (the twist plane's: phase 1)
            put_factor(A.rec, ((long)p.dst * ny + iy) * rec_len(S) + rec_cell(nx, S, REC_L2, MID_L2, ix),
                       oy[e], A.prec);
    }
}

#ifdef FFP_STEP_PROFILE
inline cudaError_t setup_profile_read(unsigned long long *host) {
    return cudaMemcpyFromSymbol(host, g_setup_prof, sizeof(g_setup_prof));
}
#endif

template <int S>
cudaError_t setup_table_for_slots(const SetupArgs *table, int count, int nx_max, cudaStream_t st) {
    const size_t smem = sizeof(double) * (14 * (size_t)nx_max + 1024);
    cudaError_t e = cudaFuncSetAttribute(setup_kernel<S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SetupArgs none;
    std::memset(&none, 0, sizeof(none));
    setup_kernel<S><<<dim3(2, count), 256, smem, st>>>(none, table, 0);
    setup_kernel<S><<<dim3(1, count), 256, smem, st>>>(none, table, 1);
    return cudaGetLastError();
}

// Single instance: two launches per level-3 plane step (see above), then the twist plane.
template <int S>
cudaError_t setup_for_slots(const KernelCtx &c, const double *t, cudaStream_t st) {
    SetupArgs a;
    fill_setup_args(c, t, &a);
    const size_t smem = sizeof(double) * (14 * (size_t)a.nx + 1024);
    cudaError_t e = cudaFuncSetAttribute(setup_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(setup_plane_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
#ifdef FFP_STEP_PROFILE
    {
        void *prof = nullptr;
        if (cudaGetSymbolAddress(&prof, g_setup_prof) == cudaSuccess)
            cudaMemsetAsync(prof, 0, sizeof(g_setup_prof), st);
    }
#endif
    const int mz = (a.nz - 1) / 2;
    const int steps = (a.nz > 1) ? (mz > a.nz - 1 - mz ? mz : a.nz - 1 - mz) : 0;
    const long nxy = (long)a.nx * a.ny;
    const int cell_blocks = (int)std::min<long>((nxy + 255) / 256, 304);
    for (int s = 0; s < steps; ++s) {
        setup_plane_kernel<S><<<2, 256, smem, st>>>(a, s);
        setup_cells_kernel<S><<<dim3(cell_blocks, 2), 256, 0, st>>>(a, s);
    }
    setup_kernel<S><<<1, 256, smem, st>>>(a, nullptr, 1);
    return cudaGetLastError();
}

}  // namespace ffp
