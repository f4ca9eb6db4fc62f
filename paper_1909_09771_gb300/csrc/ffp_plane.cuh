// ffp_plane.cuh -- level-2 solve B_P u = v of one plane (Sec. II-B, Algorithms
// 2-7 applied to the lines of a plane): two warps of the CTA run the two
// halves of the twisted line factorization side by side -- warp 0 the lines
// 0..my-1 (from line 0 towards the twist line my = floor((ny-1)/2)), warp 1
// the lines ny-1..my+1 -- each line solved by the warp-wide twisted
// tridiagonal solve.  At the twist line the two warps exchange their
// couplings through shared memory behind one named barrier and then both
// solve the twist line (the redundant solve replaces a second barrier);
// warp 0 alone writes it.  Every line is owned by the same warp and lane
// mapping in all sweeps, so a thread only ever re-reads global memory it wrote
// itself, except the twist line, which is read only after the next barrier.
#pragma once

#include "ffp_internal.cuh"

namespace ffp {

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
                                            int wid, int lane, int cnt) {
    // lane 0 wrote the twist cell of every line of the previous plane; order
    // those writes before the other lanes read them
    __syncwarp();
    const int my = (ny - 1) / 2;
    const int nl = (wid == 0) ? my : ny - 1 - my;
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
            if (s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                R v = pol.rhs(k, a);
                if (t > 0) v -= ldf<NC, F, R>(l2p + (long)kc * nx + a) * w[s];
                b[s] = v;
            } else {
                b[s] = R(0);
            }
        }
        {
            R v = pol.rhs(k, L.m);
            if (t > 0) v -= ldf<NC, F, R>(l2p + (long)kc * nx + L.m) * wm;
            bm = v;
        }
        twisted_solve<S, R>(f, cnt, lane, b, bm, w, wm);
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (s < cnt) pol.put_w(k, slot_cell<S>(L, lane, s), w[s]);
        if (lane == 0) pol.put_w(k, L.m, wm);
    }
    // ---- twist line: couplings from both halves (Algorithm 2, steps 9-11)
    {
        R *g = gbuf + wid * nx;
        const int kc = (wid == 0) ? my - 1 : my;
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                g[a] = (nl > 0) ? ldf<NC, F, R>(l2p + (long)kc * nx + a) * w[s] : R(0);
            }
        if (lane == 0) g[L.m] = (nl > 0) ? ldf<NC, F, R>(l2p + (long)kc * nx + L.m) * wm : R(0);
    }
    named_barrier(1, 64);
    load_line_factor<S, NC, F, R>(L, lane, cnt, l1p + (long)my * nx, mip + (long)my * nx, f);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (s < cnt) {
            const int a = slot_cell<S>(L, lane, s);
            b[s] = pol.rhs(my, a) - gbuf[a] - gbuf[nx + a];
        } else {
            b[s] = R(0);
        }
    }
    bm = pol.rhs(my, L.m) - gbuf[L.m] - gbuf[nx + L.m];
    R u[S], um;
    twisted_solve<S, R>(f, cnt, lane, b, bm, u, um);
    if (wid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (s < cnt) pol.put_out(my, slot_cell<S>(L, lane, s), u[s]);
        if (lane == 0) pol.put_out(my, L.m, um);
    }
    // ---- upper sweep from the twist line outwards (Algorithms 5-7)
    for (int t = nl - 1; t >= 0; --t) {
        const int k = (wid == 0) ? t : ny - 1 - t;
        const int kc = (wid == 0) ? k : k - 1;  // coupling line between k and the line towards my
        load_line_factor<S, NC, F, R>(L, lane, cnt, l1p + (long)k * nx, mip + (long)k * nx, f);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                b[s] = ldf<NC, F, R>(l2p + (long)kc * nx + a) * u[s];
            } else {
                b[s] = R(0);
            }
        }
        bm = ldf<NC, F, R>(l2p + (long)kc * nx + L.m) * um;
        R xp[S], xpm;
        twisted_solve<S, R>(f, cnt, lane, b, bm, xp, xpm);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (s < cnt) {
                const int a = slot_cell<S>(L, lane, s);
                u[s] = pol.get_w(k, a) - xp[s];
                pol.put_out(k, a, u[s]);
            }
        }
        um = pol.get_w(k, L.m) - xpm;
        if (lane == 0) pol.put_out(k, L.m, um);
    }
}

}  // namespace ffp
