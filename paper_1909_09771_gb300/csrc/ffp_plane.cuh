// ffp_plane.cuh -- level-2 solve B_P u = v of one plane (Sec. II-B, Algorithms
// 2-7 applied to the lines of a plane), used by the setup's nested plane
// solves: the CTA runs the two halves of the twisted line factorization side
// by side -- half 0 the lines 0..my-1 (from line 0 towards the twist line
// my = floor((ny-1)/2)), half 1 the lines ny-1..my+1 -- each half on two warps
// that split the slots of every line (SlotSplit), each line solved by the
// warp-wide twisted tridiagonal solve.  At the twist line the halves exchange
// their couplings through shared memory behind one named barrier of the four
// warps and then both solve the twist line (the redundant solve replaces a
// second barrier); half 0 alone writes it.  Every slot is owned by the same
// warp and lane in all sweeps, so a thread re-reads only global memory it
// wrote itself, except twist cells, which are read after a barrier.
#pragma once

#include "ffp_internal.cuh"

namespace ffp {

// Two warps on different scheduler partitions share each level-2 half of the
// setup: part 0 owns slots [0, h) and part 1 slots [h, S) of every lane,
// h = ceil(S/2).  The setup's FP64 work is mostly per slot, and one warp gets
// about one FP64 instruction per 80 cycles on its partition on this GPU, so
// splitting the slots halves that work per warp.  The recurrences along a
// line exchange the two parts' lane-local transfers through shared memory
// behind a 64-thread named barrier; both warps then run the short cross-lane
// scans redundantly.  Every slot's result lives in the warp that owns it.
struct SlotSplit {
    int s0, s1, part;
    double *ex;  // [2 buffers][2 parts][4 values][32 lanes]
    int bar;     // named barrier of the pair
    int buf;     // buffer of the next exchange (alternating: one barrier per exchange
                 // suffices, since a part reuses a buffer only after the other part
                 // has passed the barrier that follows its read of it)
    __device__ __forceinline__ bool mine(int s) const { return s >= s0 && s < s1; }
    __device__ __forceinline__ void sync() const { named_barrier(bar, 64); }
    template <int K>
    __device__ __forceinline__ void swap(const double (&v)[K], double (&o)[K], int lane) {
        double *b = ex + buf * 256;
#pragma unroll
        for (int k = 0; k < K; ++k) b[(part * 4 + k) * 32 + lane] = v[k];
        named_barrier(bar, 64);
#pragma unroll
        for (int k = 0; k < K; ++k) o[k] = b[((1 - part) * 4 + k) * 32 + lane];
        buf ^= 1;
    }
};

template <int S>
__device__ __forceinline__ SlotSplit make_split(int part, double *ex_half, int bar) {
    constexpr int h = (S + 1) / 2;
    SlotSplit sp;
    sp.part = part;
    sp.s0 = part == 0 ? 0 : h;
    sp.s1 = part == 0 ? h : S;
    sp.ex = ex_half;
    sp.bar = bar;
    sp.buf = 0;
    return sp;
}

// twisted_solve with the slots split over the two parts of sp: the same
// recurrences, each part composing its own slots, the lane transfer formed
// from both parts, the scans run by both.  x is valid on this part's slots.
template <int S, typename R>
__device__ __forceinline__ void twisted_solve_split(const LineFactor<S, R> &f, int cnt, int lane,
                                                    const R (&b)[S], R bm, R (&x)[S], R &xm,
                                                    SlotSplit &sp) {
    const int j = lane & 15;
    const unsigned FULL = 0xffffffffu;
    // ---- lower sweep: y[c] = al * y[c-1] + be; part 0's slots come first
    R al[S];
    R A = R(1), B = R(0);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        al[s] = R(1);
        if (sp.mine(s)) {
            const bool v = s < cnt;
            const R a_ = v ? -f.minv[s] * f.ein[s] : R(1);
            const R be = v ? f.minv[s] * b[s] : R(0);
            al[s] = a_;
            x[s] = be;
            B = fma(a_, B, be);
            A = A * a_;
        }
    }
    R A0, B0, AL, BL;
    {
        const double mv[2] = {A, B};
        double ov[2];
        sp.swap<2>(mv, ov, lane);
        const R A1 = sp.part ? A : R(ov[0]), B1 = sp.part ? B : R(ov[1]);
        A0 = sp.part ? R(ov[0]) : A;
        B0 = sp.part ? R(ov[1]) : B;
        AL = A1 * A0;
        BL = fma(A1, B0, B1);
    }
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const R Au = __shfl_up_sync(FULL, AL, d, 16);
        const R Bu = __shfl_up_sync(FULL, BL, d, 16);
        if (j >= d) { BL = fma(AL, Bu, BL); AL = AL * Au; }
    }
    R c = __shfl_up_sync(FULL, BL, 1, 16);
    if (j == 0) c = R(0);
    if (sp.part) c = fma(A0, c, B0);  // the value entering part 1's first slot
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (sp.mine(s)) { c = fma(al[s], c, x[s]); x[s] = c; }
    const R ytop = __shfl_sync(FULL, BL, 15);
    const R ybot = __shfl_sync(FULL, BL, 31);
    const R ym = f.minv_m * (bm - f.em1 * ytop - f.em * ybot);
    // ---- upper sweep: x[c] = y[c] + ga * x[c+1], x[end] = xm; part 1's slots come first
    R ga[S];
    R G = R(1);
    B = R(0);
#pragma unroll
    for (int s = S - 1; s >= 0; --s) {
        ga[s] = R(1);
        if (sp.mine(s)) {
            const bool v = s < cnt;
            const R g_ = v ? -f.minv[s] * f.eout[s] : R(1);
            const R yy = v ? x[s] : R(0);
            ga[s] = g_;
            x[s] = yy;
            B = fma(g_, B, yy);
            G = G * g_;
        }
    }
    R G1, B1, GL, BU;
    {
        const double mv[2] = {G, B};
        double ov[2];
        sp.swap<2>(mv, ov, lane);
        const R G0 = sp.part ? R(ov[0]) : G, B0u = sp.part ? R(ov[1]) : B;
        G1 = sp.part ? G : R(ov[0]);
        B1 = sp.part ? B : R(ov[1]);
        GL = G0 * G1;
        BU = fma(G0, B1, B0u);
    }
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const R Gd = __shfl_down_sync(FULL, GL, d, 16);
        const R Bd = __shfl_down_sync(FULL, BU, d, 16);
        if (j + d < 16) { BU = fma(GL, Bd, BU); GL = GL * Gd; }
    }
    const R Gn = __shfl_down_sync(FULL, GL, 1, 16);
    const R Bn = __shfl_down_sync(FULL, BU, 1, 16);
    c = (j == 15) ? ym : fma(Gn, ym, Bn);
    if (!sp.part) c = fma(G1, c, B1);  // the value entering part 0's last slot
#pragma unroll
    for (int s = S - 1; s >= 0; --s)
        if (sp.mine(s)) { c = fma(ga[s], c, x[s]); x[s] = c; }
    xm = ym;
}

// Pol provides, for line k (0..ny-1) and cell a of the current plane:
//   R rhs(k, a)                the plane right-hand side v
//   void put_w(k, a, R)        store the lower-sweep result
//   R get_w(k, a)              read it back
//   void put_out(k, a, R)      store the final result u
// NC selects read-only loads for the factors (see ldf).
// l1p/mip/l2p point at the plane's slice of the line factors (x-band l1 and
// 1/M per cell) and of the y-band l2 of P.  gbuf holds 2*nx values.
template <int S, bool NC, typename F, typename R, class Pol>
__device__ __forceinline__ void plane_solve(const LineMap &L, int nx, int ny,
                                            const F *__restrict__ l1p,
                                            const F *__restrict__ mip,
                                            const F *__restrict__ l2p, Pol &pol, R *gbuf,
                                            int wid, int lane, int cnt, SlotSplit &sp) {
    // the caller's __syncthreads orders the previous plane's writes (the twist
    // cells by part 0's lane 0 included) before these reads
    const int my = (ny - 1) / 2;
    const int nl = (wid == 0) ? my : ny - 1 - my;
    const bool owner0 = (lane == 0 && sp.part == 0);  // writes this half's twist cells
    LineFactor<S, R> f;
    R b[S], bm;
    R w[S], wm = R(0);
#pragma unroll
    for (int s = 0; s < S; ++s) w[s] = R(0);
    // ---- lower sweep over this warp's half (Algorithms 3 / 4)
    for (int t = 0; t < nl; ++t) {
        const int k = (wid == 0) ? t : ny - 1 - t;
        const int kc = (wid == 0) ? k - 1 : k;  // coupling line between k and its predecessor
        load_line_factor<S, NC, F, R>(L, lane, cnt, l1p + (long)k * nx, mip + (long)k * nx, f);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            b[s] = R(0);
            if (sp.mine(s) && s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                R v = pol.rhs(k, a);
                if (t > 0) v -= ldf<NC, F, R>(l2p + (long)kc * nx + a) * w[s];
                b[s] = v;
            }
        }
        {
            R v = pol.rhs(k, L.m);
            if (t > 0) v -= ldf<NC, F, R>(l2p + (long)kc * nx + L.m) * wm;
            bm = v;
        }
        twisted_solve_split<S, R>(f, cnt, lane, b, bm, w, wm, sp);
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (sp.mine(s) && s < cnt) pol.put_w(k, slot_cell<S>(L, lane, s), w[s]);
        if (owner0) pol.put_w(k, L.m, wm);
    }
    // ---- twist line: couplings from both halves (Algorithm 2, steps 9-11)
    {
        R *g = gbuf + wid * nx;
        const int kc = (wid == 0) ? my - 1 : my;
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (sp.mine(s) && s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                g[a] = (nl > 0) ? ldf<NC, F, R>(l2p + (long)kc * nx + a) * w[s] : R(0);
            }
        if (owner0) g[L.m] = (nl > 0) ? ldf<NC, F, R>(l2p + (long)kc * nx + L.m) * wm : R(0);
    }
    named_barrier(1, 128);
    load_line_factor<S, NC, F, R>(L, lane, cnt, l1p + (long)my * nx, mip + (long)my * nx, f);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        b[s] = R(0);
        if (sp.mine(s) && s < cnt) {
            const int a = slot_cell<S>(L, lane, s);
            b[s] = pol.rhs(my, a) - gbuf[a] - gbuf[nx + a];
        }
    }
    bm = pol.rhs(my, L.m) - gbuf[L.m] - gbuf[nx + L.m];
    R u[S], um;
    twisted_solve_split<S, R>(f, cnt, lane, b, bm, u, um, sp);
    if (wid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (sp.mine(s) && s < cnt) pol.put_out(my, slot_cell<S>(L, lane, s), u[s]);
        if (owner0) pol.put_out(my, L.m, um);
    }
    // ---- upper sweep from the twist line outwards (Algorithms 5-7)
    for (int t = nl - 1; t >= 0; --t) {
        const int k = (wid == 0) ? t : ny - 1 - t;
        const int kc = (wid == 0) ? k : k - 1;  // coupling line between k and the line towards my
        load_line_factor<S, NC, F, R>(L, lane, cnt, l1p + (long)k * nx, mip + (long)k * nx, f);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            b[s] = R(0);
            if (sp.mine(s) && s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                b[s] = ldf<NC, F, R>(l2p + (long)kc * nx + a) * u[s];
            }
        }
        bm = ldf<NC, F, R>(l2p + (long)kc * nx + L.m) * um;
        // the twist cell's lower-sweep value, read by both parts before the barriers
        // inside the solve: part 0's lane 0 overwrites it with the final value after them
        const R wkm = pol.get_w(k, L.m);
        R xp[S], xpm;
        twisted_solve_split<S, R>(f, cnt, lane, b, bm, xp, xpm, sp);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (sp.mine(s) && s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                u[s] = pol.get_w(k, a) - xp[s];
                pol.put_out(k, a, u[s]);
            }
        }
        um = wkm - xpm;
        if (owner0) pol.put_out(k, L.m, um);
    }
}

}  // namespace ffp
