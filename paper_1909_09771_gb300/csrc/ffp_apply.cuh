// ffp_apply.cuh -- z = B_NTD^{-1} r (Sec. II-B, Algorithms 1-7, entry
// SOLVE(1, N, x, y, n^2, 3)).
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
// The three launches on one stream are the level-3 meeting points.  Inside a
// CTA two warps run the level-2 halves of every plane solve: warp 0 the lines
// 0..my-1, warp 1 the lines ny-1..my+1; at the twist line my they exchange
// their couplings through shared memory behind one named barrier and both
// solve it.  Each line is one warp-wide twisted tridiagonal solve (level 1).
//
// Latency hiding.  Every warp walks a fixed sequence of line steps -- per
// plane its lower-sweep lines, the twist line, its upper-sweep lines -- and
// all the data a step reads is known in advance, except what this kernel
// itself writes.  At step g the warp issues the asynchronous copies of step
// g+D into a ring of D+1 shared-memory stages and waits for step g's:
//   * the factor line records (coupling, 1/M, l2, l3 fields and the twist cell)
//     as 16-byte chunks shared by the warp's lanes;
//   * the vector rows of the step (r, y of the neighbouring plane, the lower-
//     sweep result w, ...) as one 8-byte copy per cell, each lane copying the
//     cells it owns.
// A vector row this kernel wrote at step g - delta is fetched only when
// delta > D (it was written before the copy was issued, by the same lane, or
// by lane 0 for the twist cell behind the per-step __syncwarp); rows with
// delta <= D, which occur at the first and last lines of a plane, are loaded
// directly when used.  The twist line's result of the previous plane, which
// the other warp of the pair wrote, is never read back from global memory:
// both warps keep their own copy in shared memory.
#pragma once
#include "ffp_plane.cuh"
#include "ffp_kernels.h"

namespace ffp {

template <typename F>
struct ApplyArgs {
    int nx, ny, nz;
    const F *rec;     // factor line records
    const double *r;  // right-hand side
    double *z;        // output (holds y after the lower sweeps)
    double *scr;      // 2 planes of scratch (phase 2 intermediates)
    int nst;          // stages in the ring (D = nst - 1)
    int vstage;       // 1: vector rows are staged too; 0: loaded directly
    int stage_bytes;
};

// stage layout (bytes): fields [5][32 S] F, mids [4][8] F, vectors [3][S+1][32] double
template <int S, typename F>
struct StageLayout {
    static constexpr int kFld = 32 * S * (int)sizeof(F);
    static constexpr int kMid = 8 * (int)sizeof(F);
    static constexpr int kFields = 5 * kFld;
    static constexpr int kMids = 4 * kMid;
    static constexpr int kVec = (S + 1) * 32 * 8;
    __host__ __device__ static constexpr int bytes(int vstage) {
        return ((kFields + kMids + 15) / 16) * 16 + (vstage ? 3 * kVec : 0);
    }
    __host__ __device__ static constexpr int vec_off() { return ((kFields + kMids + 15) / 16) * 16; }
};

// what one step reads
struct StepPlan {
    bool valid;
    int kind;             // 0 lower, 1 twist, 2 upper
    int t;                // chain position of the line in this warp's half
    int i, k;             // plane, line
    long own, l2r, l3a, l3b;  // record indices (-1: none)
    const double *v[3];   // vector rows to stage (null: none)
};

template <int S, typename F>
struct ApplyWarp {
    using R = typename Compute<F>::type;
    using LY = StageLayout<S, F>;
    const ApplyArgs<F> &A;
    int phase, h, wid, lane, cnt;
    int nl, spp, npl, my, mz, nst, D;
    long nxy;
    unsigned char *ring;  // this warp's stages
    R *tcache;            // this warp's copy of the previous plane's twist line [(S+1)][32]

    __device__ __forceinline__ ApplyWarp(const ApplyArgs<F> &a) : A(a) {}

    // plane of chain position pl, the plane whose output it couples to, and the coupling plane
    __device__ __forceinline__ void plane_of(int pl, int &i, int &other, int &cpl) const {
        const int nz = A.nz;
        if (phase == 1) { i = mz; other = -1; cpl = -1; return; }
        if (phase == 0) {
            i = (h == 0) ? pl : nz - 1 - pl;
            other = (pl > 0) ? ((h == 0) ? i - 1 : i + 1) : -1;
            cpl = (h == 0) ? i - 1 : i;
        } else {
            const int t = npl - 1 - pl;
            i = (h == 0) ? t : nz - 1 - t;
            other = (h == 0) ? i + 1 : i - 1;
            cpl = (h == 0) ? i : i - 1;
        }
    }

    __device__ __forceinline__ StepPlan plan(int g) const {
        StepPlan p;
        p.valid = g < spp * npl;
        p.v[0] = p.v[1] = p.v[2] = nullptr;
        p.own = p.l2r = p.l3a = p.l3b = -1;
        if (!p.valid) return p;
        const int nx = A.nx, ny = A.ny;
        const int pl = g / spp, s = g - pl * spp;
        int i, other, cpl;
        plane_of(pl, i, other, cpl);
        int t, k, kind;
        if (s < nl) { kind = 0; t = s; k = (wid == 0) ? t : ny - 1 - t; }
        else if (s == nl) { kind = 1; t = nl; k = my; }
        else { kind = 2; t = 2 * nl - s; k = (wid == 0) ? t : ny - 1 - t; }
        p.kind = kind; p.t = t; p.i = i; p.k = k;
        p.own = (long)i * ny + k;
        const long row = (long)i * nxy + (long)k * nx;
        if (kind == 0) {
            if (t > 0) p.l2r = (long)i * ny + ((wid == 0) ? k - 1 : k);
        } else if (kind == 1) {
            if (nl > 0) p.l2r = (long)i * ny + ((wid == 0) ? my - 1 : my);
        } else {
            p.l2r = (long)i * ny + ((wid == 0) ? k : k - 1);
        }
        const int D_ = D;
        if (phase == 0) {
            if (kind != 2) {
                if (other >= 0) p.l3a = (long)cpl * ny + k;
                p.v[0] = A.r + row;
                if (kind == 0 && other >= 0 && 2 * t + 1 > D_) p.v[1] = A.z + (long)other * nxy + (long)k * nx;
            } else if (2 * (nl - t) > D_) {
                p.v[0] = A.z + row;
            }
        } else if (phase == 1) {
            if (kind != 2) {
                p.v[0] = A.r + row;
                if (mz > 0) { p.l3a = (long)(mz - 1) * ny + k; p.v[1] = A.z + row - nxy; }
                if (mz < A.nz - 1) { p.l3b = (long)mz * ny + k; p.v[2] = A.z + row + nxy; }
            } else if (2 * (nl - t) > D_) {
                p.v[0] = A.z + row;
            }
        } else {
            if (kind != 2) {
                p.l3a = (long)cpl * ny + k;
                // the first plane's neighbour is the twist plane, written by the previous launch
                if (pl == 0 || (kind == 0 && 2 * t + 1 > D_))
                    p.v[0] = A.z + (long)other * nxy + (long)k * nx;
                if (kind == 1) p.v[1] = A.z + row;  // y_i of the twist line
            } else {
                if (2 * (nl - t) > D_) p.v[0] = A.scr + h * nxy + (long)k * nx;
                p.v[1] = A.z + row;                 // y_i, written by phase 0/1
            }
        }
        return p;
    }

    __device__ __forceinline__ unsigned char *stage(int g) const {
        return ring + (size_t)(g % nst) * A.stage_bytes;
    }

    // issue the copies of step g into its stage and commit one group (empty past the end)
    __device__ __forceinline__ void issue(int g) const {
        const StepPlan p = plan(g);
        if (p.valid) {
            unsigned char *st = stage(g);
            const long RL = rec_len(S);
            const long srcs[5] = {p.own, p.own, p.l2r, p.l3a, p.l3b};
            const int flds[5] = {REC_EOUT, REC_MINV, REC_L2, REC_L3, REC_L3};
            constexpr int CH = LY::kFld / 16;  // 16-byte chunks per field
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                if (srcs[f] < 0) continue;
                const unsigned char *src =
                    reinterpret_cast<const unsigned char *>(A.rec + srcs[f] * RL + (long)flds[f] * 32 * S);
                for (int c = lane; c < CH; c += 32) cp_async16(st + f * LY::kFld + c * 16, src + c * 16);
            }
            // twist-cell blocks of the own, l2, l3a, l3b records
            constexpr int MC = LY::kMid / 16;
            const long ms[4] = {p.own, p.l2r, p.l3a, p.l3b};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (ms[j] < 0) continue;
                const unsigned char *src =
                    reinterpret_cast<const unsigned char *>(A.rec + ms[j] * RL + (long)REC_NFIELD * 32 * S);
                for (int c = lane; c < MC; c += 32) cp_async16(st + LY::kFields + j * LY::kMid + c * 16, src + c * 16);
            }
            if (A.vstage) {
                const LineMap L(A.nx);
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    if (!p.v[v]) continue;
                    double *dst = reinterpret_cast<double *>(st + LY::vec_off() + v * LY::kVec);
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        if (s < cnt) cp_async8(dst + s * 32 + lane, p.v[v] + slot_cell<S>(L, lane, s));
                    cp_async8(dst + S * 32 + lane, p.v[v] + L.m);
                }
            }
        }
        cp_async_commit();
    }

    // staged or direct read of cell (slot s / twist cell) of vector row v of step p
    __device__ __forceinline__ R vec(const unsigned char *st, const StepPlan &p, int v,
                                     const double *row, int s, int a) const {
        if (A.vstage && p.v[v]) {
            const double *src = reinterpret_cast<const double *>(st + LY::vec_off() + v * LY::kVec);
            return (R)src[s * 32 + lane];
        }
        return (R)row[a];
    }

    __device__ __forceinline__ R fld(const unsigned char *st, int f, int s) const {
        const F *src = reinterpret_cast<const F *>(st + f * LY::kFld);
        return to_r(src[s * 32 + lane], R());
    }
    __device__ __forceinline__ R mid(const unsigned char *st, int j, int which) const {
        const F *src = reinterpret_cast<const F *>(st + LY::kFields + j * LY::kMid);
        return to_r(src[which], R());
    }

    // factor of the step's line from the stage (ein = eout of the chain predecessor)
    __device__ __forceinline__ void factor(const unsigned char *st, LineFactor<S, R> &f) const {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            f.eout[s] = fld(st, 0, s);
            f.minv[s] = fld(st, 1, s);
        }
        const R prev = __shfl_up_sync(0xffffffffu, f.eout[S - 1], 1, 16);
#pragma unroll
        for (int s = S - 1; s > 0; --s) f.ein[s] = f.eout[s - 1];
        f.ein[0] = ((lane & 15) == 0) ? R(0) : prev;
        f.minv_m = mid(st, 0, MID_MINV);
        f.em1 = mid(st, 0, MID_EM1);
        f.em = mid(st, 0, MID_EM);
    }
};

template <int S, typename F>
__global__ void __launch_bounds__(64) apply_kernel(ApplyArgs<F> A, int phase) {
    using R = typename Compute<F>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const LineMap L(nx);
    const long nxy = (long)nx * ny;
    // shared memory: [2 warps][nst stages] | twist caches [2][S+1][32] R | gbuf [2 parity][2][nx] R
    const size_t ring_bytes = (size_t)A.nst * A.stage_bytes;
    R *tc = reinterpret_cast<R *>(smem_raw + 2 * ring_bytes);
    R *gbase = tc + 2 * (S + 1) * 32;
    ApplyWarp<S, F> W(A);
    W.phase = phase; W.h = (phase == 1) ? 0 : blockIdx.x; W.wid = wid; W.lane = lane;
    W.cnt = lane_count<S>(L, lane);
    W.my = (ny - 1) / 2; W.mz = (nz - 1) / 2; W.nxy = nxy;
    W.nl = (wid == 0) ? W.my : ny - 1 - W.my;
    W.spp = 2 * W.nl + 1;
    W.npl = (phase == 1) ? 1 : ((blockIdx.x == 0) ? W.mz : nz - 1 - W.mz);
    W.nst = A.nst; W.D = A.nst - 1;
    W.ring = smem_raw + wid * ring_bytes;
    W.tcache = tc + wid * (S + 1) * 32;
    const int cnt = W.cnt, D = W.D, nl = W.nl, my = W.my;
    for (int g = 0; g < D; ++g) W.issue(g);

    R w[S], wm = R(0);   // previous lower-sweep line (lower sweep), then u of the line towards my
    int g = 0;
    for (int pl = 0; pl < W.npl; ++pl) {
        int i, other, cpl;
        W.plane_of(pl, i, other, cpl);
        R *gbuf = gbase + (pl & 1) * 2 * nx;
        const long pbase = (long)i * nxy;
        for (int s = 0; s < W.spp; ++s, ++g) {
            __syncwarp();
            W.issue(g + D);
            cp_async_wait_dyn(D);
            __syncwarp();
            const unsigned char *st = W.stage(g);
            const StepPlan p = W.plan(g);
            LineFactor<S, R> f;
            W.factor(st, f);
            const long row = pbase + (long)p.k * nx;
            R b[S], bm;
            // ---------------------------------------------------------- rhs of the step
            if (p.kind != 2) {
                // plane right-hand side v of this line
#pragma unroll
                for (int q = 0; q <= S; ++q) {
                    const int sidx = (q < S) ? q : S;
                    if (q < S && q >= cnt) { b[q] = R(0); continue; }
                    const int a = (q < S) ? slot_cell<S>(L, lane, q) : L.m;
                    R v;
                    if (phase == 0) {
                        v = W.vec(st, p, 0, A.r + row, sidx, a);
                        if (other >= 0) {
                            R yp;
                            if (p.kind == 1) yp = W.tcache[sidx * 32 + lane];
                            else yp = W.vec(st, p, 1, A.z + (long)other * nxy + (long)p.k * nx, sidx, a);
                            const R c3 = (q < S) ? W.fld(st, 3, q) : W.mid(st, 2, MID_L3);
                            v -= c3 * yp;
                        }
                    } else if (phase == 1) {
                        v = W.vec(st, p, 0, A.r + row, sidx, a);
                        if (W.mz > 0) {
                            const R c3 = (q < S) ? W.fld(st, 3, q) : W.mid(st, 2, MID_L3);
                            v -= c3 * W.vec(st, p, 1, A.z + row - nxy, sidx, a);
                        }
                        if (W.mz < nz - 1) {
                            const R c3 = (q < S) ? W.fld(st, 4, q) : W.mid(st, 3, MID_L3);
                            v -= c3 * W.vec(st, p, 2, A.z + row + nxy, sidx, a);
                        }
                    } else {
                        R za;
                        if (p.kind == 1 && pl > 0) za = W.tcache[sidx * 32 + lane];
                        else za = W.vec(st, p, 0, A.z + (long)other * nxy + (long)p.k * nx, sidx, a);
                        const R c3 = (q < S) ? W.fld(st, 3, q) : W.mid(st, 2, MID_L3);
                        v = c3 * za;
                    }
                    if (q < S) b[q] = v; else bm = v;
                }
                if (p.kind == 0 && p.t > 0) {
#pragma unroll
                    for (int q = 0; q < S; ++q) b[q] -= W.fld(st, 2, q) * w[q];
                    bm -= W.mid(st, 1, MID_L2) * wm;
                }
            } else {
#pragma unroll
                for (int q = 0; q < S; ++q) b[q] = W.fld(st, 2, q) * w[q];
                bm = W.mid(st, 1, MID_L2) * wm;
            }
            if (p.kind == 1) {
                // couplings of the two halves into the twist line (Algorithm 2, steps 9-11)
                R *gw = gbuf + wid * nx;
#pragma unroll
                for (int q = 0; q < S; ++q)
                    if (q < cnt) gw[slot_cell<S>(L, lane, q)] = (nl > 0) ? W.fld(st, 2, q) * w[q] : R(0);
                if (lane == 0) gw[L.m] = (nl > 0) ? W.mid(st, 1, MID_L2) * wm : R(0);
                named_barrier(1, 64);
#pragma unroll
                for (int q = 0; q < S; ++q)
                    if (q < cnt) {
                        const int a = slot_cell<S>(L, lane, q);
                        b[q] = b[q] - gbuf[a] - gbuf[nx + a];
                    }
                bm = bm - gbuf[L.m] - gbuf[nx + L.m];
            }
            // ---------------------------------------------------------- line solve
            R x[S], xm;
            twisted_solve<S, R>(f, cnt, lane, b, bm, x, xm);
            // ---------------------------------------------------------- results
            if (p.kind == 0) {
                double *out = (phase == 2) ? A.scr + W.h * nxy + (long)p.k * nx : A.z + row;
#pragma unroll
                for (int q = 0; q < S; ++q)
                    if (q < cnt) out[slot_cell<S>(L, lane, q)] = (double)x[q];
                if (lane == 0) out[L.m] = (double)xm;
#pragma unroll
                for (int q = 0; q < S; ++q) w[q] = x[q];
                wm = xm;
            } else if (p.kind == 1) {
                // twist line: u_my (kept in registers for the upper sweep)
#pragma unroll
                for (int q = 0; q <= S; ++q) {
                    if (q < S && q >= cnt) continue;
                    const int sidx = (q < S) ? q : S;
                    const int a = (q < S) ? slot_cell<S>(L, lane, q) : L.m;
                    const R u = (q < S) ? x[q] : xm;
                    R fin = u;
                    if (phase == 2) fin = W.vec(st, p, 1, A.z + row, sidx, a) - u;
                    W.tcache[sidx * 32 + lane] = fin;
                    if (wid == 0 && (q < S || lane == 0)) A.z[row + a] = (double)fin;
                }
#pragma unroll
                for (int q = 0; q < S; ++q) w[q] = x[q];
                wm = xm;
            } else {
                const double *wrow = (phase == 2) ? A.scr + W.h * nxy + (long)p.k * nx : A.z + row;
#pragma unroll
                for (int q = 0; q <= S; ++q) {
                    if (q < S && q >= cnt) continue;
                    const int sidx = (q < S) ? q : S;
                    const int a = (q < S) ? slot_cell<S>(L, lane, q) : L.m;
                    const R u = W.vec(st, p, 0, wrow, sidx, a) - ((q < S) ? x[q] : xm);
                    R fin = u;
                    if (phase == 2) fin = W.vec(st, p, 1, A.z + row, sidx, a) - u;
                    if (q < S || lane == 0) A.z[row + a] = (double)fin;
                    if (q < S) w[q] = u; else wm = u;
                }
            }
        }
    }
    cp_async_wait<0>();
}

// shared memory the kernel needs for nst stages
template <int S, typename F>
static size_t apply_smem(int nx, int nst, int vstage) {
    using R = typename Compute<F>::type;
    return 2 * (size_t)nst * StageLayout<S, F>::bytes(vstage) + 2 * (S + 1) * 32 * sizeof(R) +
           4 * (size_t)nx * sizeof(R);
}

template <int S, typename F>
cudaError_t apply_for_slots(const KernelCtx &c, const double *r, double *z, cudaStream_t st) {
    ApplyArgs<F> a;
    a.nx = c.nx; a.ny = c.ny; a.nz = c.nz;
    a.rec = (const F *)c.ws.rec;
    a.r = r; a.z = z; a.scr = c.ws.ascr;
    // deepest ring (up to 5 stages) that fits 220 KB; drop vector staging if 2 do not fit
    const size_t limit = 220 * 1024;
    int vstage = 1, nst = 5;
    while (nst > 2 && apply_smem<S, F>(c.nx, nst, vstage) > limit) --nst;
    if (apply_smem<S, F>(c.nx, nst, vstage) > limit) { vstage = 0; nst = 5; }
    while (nst > 2 && apply_smem<S, F>(c.nx, nst, vstage) > limit) --nst;
    if (apply_smem<S, F>(c.nx, nst, vstage) > limit) return cudaErrorInvalidConfiguration;
    a.nst = nst;
    a.vstage = vstage;
    a.stage_bytes = StageLayout<S, F>::bytes(vstage);
    const size_t smem = apply_smem<S, F>(c.nx, nst, vstage);
    cudaError_t e = cudaFuncSetAttribute(apply_kernel<S, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int mz = (a.nz - 1) / 2;
    const bool halves = (mz > 0) || (a.nz - 1 - mz > 0);
    if (halves) apply_kernel<S, F><<<2, 64, smem, st>>>(a, 0);
    apply_kernel<S, F><<<1, 64, smem, st>>>(a, 1);
    if (halves) apply_kernel<S, F><<<2, 64, smem, st>>>(a, 2);
    return cudaGetLastError();
}

}  // namespace ffp
