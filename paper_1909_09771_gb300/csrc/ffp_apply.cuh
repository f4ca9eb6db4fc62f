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
// Latency hiding (warp specialisation).  Each of the two compute warps walks
// a fixed sequence of line steps -- per plane its lower-sweep lines, the twist
// line, its upper-sweep lines -- and has two producer warps that walk the same
// sequence ahead of it, taking its steps in turn.  The producer copies what step g reads
// into stage g mod NST of a ring in shared memory:
//   * the factor line records (alpha, gamma, 1/M of the line, the l2 field of
//     the line it couples to in the plane, the l3 field of the line it couples
//     to across planes, and their twist cells);
//   * the vector rows of the step -- every vector the sweeps read or write is
//     kept in the line-block layout (lb_pos), the register layout of the line
//     solve, so a row is one contiguous block;
// all as 16-byte cp.async chunks spread over its lanes (coalesced),
// and signals the stage's "full" mbarrier when its copies complete; the
// compute warp waits on it, computes, and releases the stage on its "empty"
// mbarrier.  All the address arithmetic thus stays off the compute warp's
// instruction stream.  The producer refills stage g only after the compute
// warp released step g - NST, so a vector row the kernel wrote at step
// g - delta can be staged when delta >= NST (release/acquire through the
// mbarriers orders the write before the copy); rows with delta < NST occur at
// the first lines of the lower and upper sweeps and are loaded directly.  The
// twist line of the previous plane, which only compute warp 0 writes, is
// never read back from global memory: both compute warps keep their own copy
// in shared memory.  Every mbarrier wait has an iteration limit; on timeout
// the warp records FL_TIMEOUT and runs on without waiting, so the kernel always
// finishes (with unusable results) instead of hanging.
#pragma once
#include <cstring>

#include "ffp_plane.cuh"
#include "ffp_kernels.h"

namespace ffp {

#ifdef FFP_STEP_PROFILE
// Step profile (profiling builds only, see build.py --profile): clock64 stamps
// around the segments of the line steps of compute warp 0 of the first CTA of
// phase 0, accumulated by lane 0 and written out at the end of the launch.
// Slots: lower steps [0] stage wait, [1] right-hand side, [2] line solve,
// [3] store + release, [4] count; upper steps [5..9] likewise; [10] cycles of
// the whole plane loop; [11] stage waits whose first try failed.
static __device__ unsigned long long g_step_prof[16];
__device__ __forceinline__ unsigned long long prof_stamp() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(t)::"memory");
    return t;
}
#define FFP_PROF(...) __VA_ARGS__
#else
#define FFP_PROF(...)
#endif

// Typed view of one (instance, right-hand side) pair's ApplyArgs.  Vectors are
// in the compute type R: FP64 for FP64 factors, FP32 otherwise (the FP32 apply
// converts r to FP32 and z back to FP64 in GPU-wide kernels around the
// sweeps, so no FP64 arithmetic or conversion runs inside them).
template <typename F>
struct ApplyView {
    using R = typename Compute<F>::type;
    int nx, ny, nz;
    const F *rec;  // factor line records
    const F *l3n;  // z-band of A in natural order (the twist-plane phase reads its second
                   // coupling from here)
    const R *r;    // right-hand side
    R *z;          // output (holds y after the lower sweeps)
    R *scr;        // 2 planes of scratch (phase 2 intermediates)
    int *flags;    // error flags (FL_TIMEOUT)
    // the view of right-hand side q (0, or 1 for the second of a two-RHS entry)
    __device__ __forceinline__ ApplyView(const ApplyArgs &a, int q)
        : nx(a.nx), ny(a.ny), nz(a.nz), rec(static_cast<const F *>(a.rec)),
          l3n(static_cast<const F *>(a.l3n)), r(static_cast<const R *>(q ? a.r1 : a.r)),
          z(static_cast<R *>(q ? a.z1 : a.z)), scr(static_cast<R *>(q ? a.scr1 : a.scr)),
          flags(q ? a.flags1 : a.flags) {}
};

constexpr int kSmemBudget = 220 * 1024;

// The S slots of one lane from p (16-byte aligned, lane-major layout) with
// vector loads, converted to the compute type R.
template <int S, typename T, typename R>
__device__ __forceinline__ void ld_slots(const T *p, R (&o)[S]) {
    constexpr int SP = slot_pitch(S);
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < SP / 4; ++q) {
            const float4 v = reinterpret_cast<const float4 *>(p)[q];
            if (4 * q + 0 < S) o[4 * q + 0] = (R)v.x;
            if (4 * q + 1 < S) o[4 * q + 1] = (R)v.y;
            if (4 * q + 2 < S) o[4 * q + 2] = (R)v.z;
            if (4 * q + 3 < S) o[4 * q + 3] = (R)v.w;
        }
    } else if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int q = 0; q < SP / 2; ++q) {
            const double2 v = reinterpret_cast<const double2 *>(p)[q];
            if (2 * q + 0 < S) o[2 * q + 0] = (R)v.x;
            if (2 * q + 1 < S) o[2 * q + 1] = (R)v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < SP / 4; ++q) {
            const uint2 u = reinterpret_cast<const uint2 *>(p)[q];
            const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&u.x);
            const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&u.y);
            if (4 * q + 0 < S) o[4 * q + 0] = (R)__low2float(a);
            if (4 * q + 1 < S) o[4 * q + 1] = (R)__high2float(a);
            if (4 * q + 2 < S) o[4 * q + 2] = (R)__low2float(b);
            if (4 * q + 3 < S) o[4 * q + 3] = (R)__high2float(b);
        }
    }
}

// Store the S slots of one lane (slots >= cnt and the pitch padding as 0) with
// vector stores; p 16-byte aligned.
template <int S, typename R>
__device__ __forceinline__ void st_slots(R *p, const R (&x)[S], int cnt) {
    constexpr int SP = slot_pitch(S);
    auto val = [&](int s) -> R { return (s < S && s < cnt) ? x[s < S ? s : 0] : R(0); };
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int q = 0; q < SP / 4; ++q)
            reinterpret_cast<float4 *>(p)[q] = make_float4(val(4 * q), val(4 * q + 1), val(4 * q + 2), val(4 * q + 3));
    } else {
#pragma unroll
        for (int q = 0; q < SP / 2; ++q)
            reinterpret_cast<double2 *>(p)[q] = make_double2(val(2 * q), val(2 * q + 1));
    }
}

// Compile-time stage layout for phase PH and NR right-hand sides: fields
// [NF][32][SP] F (shared by the right-hand sides), twist-cell blocks [NM][8] F,
// vector row blocks [NR][NV][32 SP + 32] R (SP = slot_pitch(S)).
template <int S, typename F, int PH, int NR = 1>
struct Stage {
    using R = typename Compute<F>::type;
    static constexpr int NF = 5;  // alpha, gamma, minv, l2, l3
    static constexpr int NM = 3;  // twist-cell blocks: own, l2, l3
    static constexpr int NV = (PH == 1) ? 3 : 2;
    static constexpr int SP = slot_pitch(S);
    static constexpr int kFld = 32 * SP * (int)sizeof(F);
    static constexpr int kMid = 8 * (int)sizeof(F);
    static constexpr int kVecOff = ((NF * kFld + NM * kMid + 15) / 16) * 16;
    static constexpr int kVec = (32 * SP + 32) * (int)sizeof(R);
    // twist caches + full/empty mbarriers of both rings
    static constexpr int kExtra = 2 * NR * (S + 1) * 32 * (int)sizeof(R) + 2 * 2 * 5 * 8;
    __host__ __device__ static constexpr int bytes_v(int vst) { return kVecOff + (vst ? NR * NV * kVec : 0); }
    __host__ __device__ static constexpr int total(int nst, int vst, int nx) {
        return 2 * nst * bytes_v(vst) + kExtra + NR * 4 * nx * (int)sizeof(R);
    }
    // vector rows are staged if three stages of them fit beside the longest gbuf
    static constexpr int VST = total(3, 1, FFP_MAX_NX) <= kSmemBudget ? 1 : 0;
    __host__ __device__ static constexpr int pick() {
        int n = 5;
        while (n > 2 && total(n, VST, FFP_MAX_NX) > kSmemBudget) --n;
        return n;
    }
    static constexpr int NST = pick();
    static constexpr int D = NST - 1;  // a staged row must be written >= NST = D + 1 steps earlier
    static constexpr int kBytes = bytes_v(VST);
};

// The two-RHS form is built where its stage ring keeps at least three stages
// with staged rows in every phase.
template <int S, typename F>
__host__ __device__ constexpr bool two_rhs_fits() {
    return Stage<S, F, 0, 2>::VST && Stage<S, F, 1, 2>::VST && Stage<S, F, 2, 2>::VST &&
           Stage<S, F, 0, 2>::NST >= 3 && Stage<S, F, 1, 2>::NST >= 3 && Stage<S, F, 2, 2>::NST >= 3;
}

// One CTA per level-3 half (phases 0, 2) or per twist plane (phase 1) of one
// pair: the pair is A0, or table[blockIdx.y] when a table is given; a pair
// whose control word is given and has bit 0 clear returns at once.
// Warps 0 and 1 compute the two level-2 halves.  Compute warp c has two
// producer warps, 2 + c and 6 + c, which stage its steps in turn (step g by
// producer g mod 2).  A warp runs on scheduler partition warp mod 4, so the
// producers share partitions 2 and 3 and leave partitions 0 and 1 to the
// compute warps; warps 4 and 5 (partitions 0 and 1) only help initialise.
constexpr int kProducers = 2;
constexpr int kApplyThreads = 256;

template <int S, typename F, int PH, int NR>
__global__ void __launch_bounds__(kApplyThreads, 1) apply_kernel(ApplyArgs A0, const ApplyArgs *__restrict__ table) {
    using R = typename Compute<F>::type;
    const ApplyArgs &src = table ? table[blockIdx.y] : A0;
    // a batched entry none of whose pairs iterates now
    if (src.ctl && !(*src.ctl & 1) && (NR == 1 || (src.ctl1 && !(*src.ctl1 & 1)))) return;
    const unsigned wtries = src.wait_tries;
    const int stall = src.stall;
    const ApplyArgs &args = src;   // (the producer's record list below is also named src)
    using SG = Stage<S, F, PH, NR>;
    constexpr int NF = SG::NF, NM = SG::NM, NV = SG::NV, NST = SG::NST, D = SG::D, VST = SG::VST;
    static_assert(SG::total(NST, VST, FFP_MAX_NX) <= kSmemBudget, "stage ring does not fit");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warps 4 and 5 compute the second right-hand side (NR = 2), else only help initialise
    const bool idle = (warp == 4 || warp == 5) && NR == 1;
    const bool producer = (warp & 3) >= 2;
    const int wid = warp & 1;                  // the level-2 half this warp computes or feeds
    const int q = (warp == 4 || warp == 5) ? 1 : 0;   // the right-hand side a compute warp serves
    const ApplyView<F> A(src, producer ? 0 : q);
    const int ppar = (warp >= 6) ? 1 : 0;      // the steps this producer stages (g mod 2)
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int nxy = nx * ny;
    const LineMap L(nx);
    const int cnt = lane_count<S>(L, lane);
    const int h = (PH == 1) ? 0 : (int)blockIdx.x;
    const int my = (ny - 1) / 2, mz = (nz - 1) / 2;
    const int nl = (wid == 0) ? my : ny - 1 - my;
    const int spp = 2 * nl + 1;
    const int npl = (PH == 1) ? 1 : ((h == 0) ? mz : nz - 1 - mz);
    unsigned char *ring = smem_raw + (size_t)wid * NST * SG::kBytes;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem_raw + 2 * (size_t)NST * SG::kBytes);
    unsigned long long *full = bars + wid * 2 * 5, *empty = full + 5;
    R *caches = reinterpret_cast<R *>(bars + 2 * 2 * 5);
    R *tcache = caches + (q * 2 + wid) * (S + 1) * 32;
    R *gbase = caches + 2 * NR * (S + 1) * 32 + q * 4 * A.nx;
    if (threadIdx.x == 0) {
        // bars[c*10 + k] = full[k], bars[c*10 + 5 + k] = empty[k] of level-2 half c
        for (int c = 0; c < 2; ++c)
            for (int k = 0; k < 5; ++k) {
                mbar_init(bars + c * 10 + k, 32);     // full: one cp.async arrival per producer lane
                mbar_init(bars + c * 10 + 5 + k, NR); // empty: one arrival per compute warp of the half
            }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (idle) return;
    bool aborted = false;
    int cell[S];
#pragma unroll
    for (int s = 0; s < S; ++s) cell[s] = (s < cnt) ? slot_cell<S>(L, lane, s) : 0;
    const long RL = rec_len(S);
    const long BL = lb_len(S);  // values per line block of a vector

    // plane of chain position pl, the plane whose output it couples to (-1: none), coupling plane
    auto plane_of = [&](int pl, int &i, int &other, int &cpl) {
        if (PH == 1) { i = mz; other = -1; cpl = -1; return; }
        if (PH == 0) {
            i = (h == 0) ? pl : nz - 1 - pl;
            other = (pl > 0) ? ((h == 0) ? i - 1 : i + 1) : -1;
            cpl = (h == 0) ? i - 1 : i;
        } else {
            const int t = npl - 1 - pl;
            i = (h == 0) ? t : nz - 1 - t;
            other = (h == 0) ? i + 1 : i - 1;
            cpl = (h == 0) ? i : i - 1;
        }
    };
    auto line_of = [&](int t) { return (wid == 0) ? t : ny - 1 - t; };

    // ------------------------------------------------------------------ producer
    // future-step cursor: chain plane fpl, step fs within the plane, global step fg
    int fpl = 0, fs = 0, fg = 0;
    auto issue_next = [&]() {
        if (fpl < npl && fg % kProducers == ppar) {
            const int slot = fg % NST, use = fg / NST;
            if (use > 0 && !aborted && !mbar_wait(empty + slot, (use - 1) & 1, wtries)) {
                aborted = true;
                atomicOr(A.flags + FL_TIMEOUT, 1);
                if (NR == 2) atomicOr(args.flags1 + FL_TIMEOUT, 1);
            }
            unsigned char *st = ring + slot * SG::kBytes;
            int i, other, cpl;
            plane_of(fpl, i, other, cpl);
            const int kind = (fs < nl) ? 0 : ((fs == nl) ? 1 : 2);
            const int t = (kind == 0) ? fs : ((kind == 1) ? nl : 2 * nl - fs);
            const int k = (kind == 1) ? my : line_of(t);
            const long own = (long)i * ny + k;
            long l2r = -1, l3a = -1;
            if (kind == 0) { if (t > 0) l2r = (long)i * ny + ((wid == 0) ? k - 1 : k); }
            else if (kind == 1) { if (nl > 0) l2r = (long)i * ny + ((wid == 0) ? my - 1 : my); }
            else l2r = (long)i * ny + ((wid == 0) ? k : k - 1);
            const long bown = own * BL;
            // the step's vector rows: which vector (1 = r, 2 = z, 3 = scratch) at which block offset
            int vk[3] = {0, 0, 0};
            long vo[3] = {0, 0, 0};
            if (PH == 0) {
                if (kind != 2) {
                    if (other >= 0) l3a = (long)cpl * ny + k;
                    vk[0] = 1; vo[0] = bown;
                    if (kind == 0 && other >= 0 && 2 * t + 1 > D) { vk[1] = 2; vo[1] = ((long)other * ny + k) * BL; }
                } else if (2 * (nl - t) > D) {
                    vk[0] = 2; vo[0] = bown;
                }
            } else if (PH == 1) {
                if (kind != 2) {
                    vk[0] = 1; vo[0] = bown;
                    if (mz > 0) { l3a = (long)(mz - 1) * ny + k; vk[1] = 2; vo[1] = bown - (long)ny * BL; }
                    if (mz < nz - 1) { vk[2] = 2; vo[2] = bown + (long)ny * BL; }
                } else if (2 * (nl - t) > D) {
                    vk[0] = 2; vo[0] = bown;
                }
            } else {
                if (kind != 2) {
                    l3a = (long)cpl * ny + k;
                    // the first plane's neighbour is the twist plane, written by the previous launch
                    if (fpl == 0 || (kind == 0 && 2 * t + 1 > D)) { vk[0] = 2; vo[0] = ((long)other * ny + k) * BL; }
                    if (kind == 1) { vk[1] = 2; vo[1] = bown; }  // y of the twist line
                } else {
                    if (2 * (nl - t) > D) { vk[0] = 3; vo[0] = ((long)h * ny + k) * BL; }
                    vk[1] = 2; vo[1] = bown;                     // y, written by phase 0/1
                }
            }
            // factor records: stage fields [0..2] own alpha, gamma, minv, [3] l2 field of
            // row l2r, [4] l3 field of row l3a (the twist-plane phase's second coupling
            // is read from l3n), as 16-byte chunks spread over the lanes; twist-cell
            // blocks [0] own, [1] l2r, [2] l3a
            const long src[5] = {own, own, own, l2r, l3a};
            const int fld[5] = {REC_ALPHA, REC_GAMMA, REC_MINV, REC_L2, REC_L3};
            constexpr int CH = SG::kFld / 16;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if (src[f] >= 0) {
                    const unsigned char *gp = reinterpret_cast<const unsigned char *>(
                        A.rec + src[f] * RL + rec_slot(S, fld[f], 0, 0));
#pragma unroll
                    for (int c0 = 0; c0 < CH; c0 += 32)
                        if (c0 + lane < CH)
                            cp_async16(st + f * SG::kFld + (c0 + lane) * 16, gp + (c0 + lane) * 16);
                }
            }
            constexpr int MC = SG::kMid / 16;
            if (lane < NM * MC) {
                const int j = lane / MC, c = lane % MC;
                const long msrc = (j == 0) ? own : ((j == 1) ? l2r : l3a);
                if (msrc >= 0)
                    cp_async16(st + NF * SG::kFld + j * SG::kMid + c * 16,
                               reinterpret_cast<const unsigned char *>(A.rec + msrc * RL + rec_mid(S)) +
                                   c * 16);
            }
            if (VST) {
                constexpr int VC = SG::kVec / 16;  // 16-byte chunks of one row block
#pragma unroll
                for (int qq = 0; qq < NR; ++qq) {
                    const ApplyView<F> Aq(args, qq);
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        if (vk[v]) {
                            const R *base = (vk[v] == 1) ? Aq.r : ((vk[v] == 2) ? Aq.z : Aq.scr);
                            unsigned char *dst = st + SG::kVecOff + (qq * NV + v) * SG::kVec;
                            const unsigned char *sp = reinterpret_cast<const unsigned char *>(base + vo[v]);
#pragma unroll
                            for (int c0 = 0; c0 < VC; c0 += 32)
                                if (c0 + lane < VC) cp_async16(dst + (c0 + lane) * 16, sp + (c0 + lane) * 16);
                        }
                    }
                }
            }
            // the test hook withholds the first signal of one producer (the compute warp's
            // wait then runs out; the kernel still ends, with unusable results)
            const bool withhold = PH == 0 && stall == 1 && fg == 0 && wid == 0 && ppar == 0 &&
                                  blockIdx.x == 0;
            if (!withhold) mbar_arrive_cpasync(full + slot);
        }
        ++fg;
        if (++fs == spp) { fs = 0; ++fpl; }
    };
    if (producer) {
        const int total = spp * npl;
        for (int q = 0; q < total; ++q) issue_next();
        cp_async_wait<0>();
        return;
    }

    // ------------------------------------------------------------------ compute
    constexpr int SP = SG::SP;
    // this lane's slots of stage field f; the stage's twist-cell blocks; vector row v
    auto Fp = [&](const unsigned char *st, int f) -> const F * {
        return reinterpret_cast<const F *>(st + f * SG::kFld) + lane * SP;
    };
    auto M_ = [&](const unsigned char *st, int j, int w) -> R {
        return to_r(reinterpret_cast<const F *>(st + NF * SG::kFld + j * SG::kMid)[w], R());
    };
    auto Vp = [&](const unsigned char *st, int v) -> const R * {
        return reinterpret_cast<const R *>(st + SG::kVecOff + (q * NV + v) * SG::kVec);
    };
    // a row block (staged or in global memory): this lane's slots and the twist cell
    auto ldrow = [&](const R *blk, R (&o)[S], R &om) {
        ld_slots<S>(blk + lane * SP, o);
        om = blk[32 * SP];
    };
    // store a row block: valid slots, zero pads, the twist cell from lane 0
    auto put = [&](R *blk, const R (&x)[S], R xm) {
        st_slots<S>(blk + lane * SP, x, cnt);
        blk[32 * SP + lane] = (lane == 0) ? xm : R(0);
    };
#pragma unroll
    for (int s = 0; s <= S; ++s) tcache[s * 32 + lane] = R(0);
    __syncwarp();

    R w[S], wm = R(0);
#pragma unroll
    for (int s = 0; s < S; ++s) w[s] = R(0);
    int slot = 0;
    unsigned phase = 0;
    // wait until the current stage is full
    FFP_PROF(unsigned long long nfail = 0;)
    auto begin = [&]() -> const unsigned char * {
        FFP_PROF(if (!mbar_try(full + slot, phase)) ++nfail;)
        if (!aborted && !mbar_wait(full + slot, phase, wtries)) {
            aborted = true;
            atomicOr(A.flags + FL_TIMEOUT, 1);
        }
        return ring + slot * SG::kBytes;
    };
    // release the current stage to the producer and move to the next
    auto finish = [&]() {
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + slot);
        if (++slot == NST) { slot = 0; phase ^= 1u; }
    };
    // the line solve of a step from its stage
    auto solve = [&](const unsigned char *st, const R (&b)[S], R bm, R (&x)[S], R &xm) {
        R al[S], ga[S], mi[S];
        ld_slots<S>(Fp(st, 0), al);
        ld_slots<S>(Fp(st, 1), ga);
        ld_slots<S>(Fp(st, 2), mi);
        twisted_solve_pre<S, R>(al, ga, mi, M_(st, 0, MID_MINV), M_(st, 0, MID_EM1), M_(st, 0, MID_EM),
                                cnt, lane, b, bm, x, xm);
    };
    // plane right-hand side (b, bm) of a lower or twist step of the line with block
    // offset bk (natural row offset nrow); zrow = the coupled plane's row block;
    // NEAR: that row is read from global memory
    auto rhs = [&](const unsigned char *st, long bk, long nrow, const R *zrow, bool near, bool twist,
                   int pl, int other, R (&b)[S], R &bm) {
        R c3[S];
        ld_slots<S>(Fp(st, 4), c3);
        const R c3m = M_(st, 2, MID_L3);
        R y[S], ym;
        if (PH == 0) {
            if (VST) ldrow(Vp(st, 0), b, bm); else ldrow(A.r + bk, b, bm);
            if (other >= 0) {
                if (twist) {
#pragma unroll
                    for (int s = 0; s < S; ++s) y[s] = tcache[s * 32 + lane];
                    ym = tcache[S * 32 + lane];
                } else if (VST && !near) {
                    ldrow(Vp(st, 1), y, ym);
                } else {
                    ldrow(zrow, y, ym);
                }
#pragma unroll
                for (int s = 0; s < S; ++s) b[s] -= c3[s] * y[s];
                bm -= c3m * ym;
            }
        } else if (PH == 1) {
            if (VST) ldrow(Vp(st, 0), b, bm); else ldrow(A.r + bk, b, bm);
            if (mz > 0) {
                if (VST) ldrow(Vp(st, 1), y, ym); else ldrow(A.z + bk - (long)ny * BL, y, ym);
#pragma unroll
                for (int s = 0; s < S; ++s) b[s] -= c3[s] * y[s];
                bm -= c3m * ym;
            }
            if (mz < nz - 1) {
                // coupling mz <-> mz+1 from the natural-order l3 band
                if (VST) ldrow(Vp(st, 2), y, ym); else ldrow(A.z + bk + (long)ny * BL, y, ym);
#pragma unroll
                for (int s = 0; s < S; ++s) b[s] -= to_r(A.l3n[nrow + cell[s]], R()) * y[s];
                bm -= to_r(A.l3n[nrow + L.m], R()) * ym;
            }
        } else {
            if (twist && pl > 0) {
#pragma unroll
                for (int s = 0; s < S; ++s) y[s] = tcache[s * 32 + lane];
                ym = tcache[S * 32 + lane];
            } else if (VST && (!near || pl == 0)) {
                ldrow(Vp(st, 0), y, ym);
            } else {
                ldrow(zrow, y, ym);
            }
#pragma unroll
            for (int s = 0; s < S; ++s) b[s] = c3[s] * y[s];
            bm = c3m * ym;
        }
    };

    FFP_PROF(const bool prof = PH == 0 && blockIdx.x == 0 && blockIdx.y == 0 && wid == 0 && lane == 0;
             unsigned long long pacc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
             const unsigned long long pstart = prof_stamp();)
    for (int pl = 0; pl < npl; ++pl) {
        int i, other, cpl;
        plane_of(pl, i, other, cpl);
        R *gbuf = gbase + (pl & 1) * 2 * nx;
        const long pbase = (long)i * nxy;                  // natural offset of plane i
        const long pblk = (long)i * ny * BL;               // block offset of plane i
        const long oblk = (other >= 0) ? (long)other * ny * BL : 0;
        R *scrp = A.scr + (long)h * ny * BL;
        // ------------------------------------------------------------ lower sweep
        // steps t < TN read the coupled plane's row directly (written fewer than NST steps ago)
        constexpr int TN = (D + 1) / 2;
        auto lower = [&](int t, bool near) {
            FFP_PROF(const unsigned long long p0 = prof_stamp();)
            const unsigned char *st = begin();
            FFP_PROF(const unsigned long long p1 = prof_stamp();)
            const int k = line_of(t);
            const long bk = pblk + (long)k * BL;
            R b[S], bm;
            rhs(st, bk, pbase + (long)k * nx, A.z + oblk + (long)k * BL, near, false, pl, other, b, bm);
            if (t > 0) {
                R l2[S];
                ld_slots<S>(Fp(st, 3), l2);
#pragma unroll
                for (int s = 0; s < S; ++s) b[s] -= l2[s] * w[s];
                bm -= M_(st, 1, MID_L2) * wm;
            }
            R x[S], xm;
            FFP_PROF(const unsigned long long p2 = prof_stamp();)
            solve(st, b, bm, x, xm);
            FFP_PROF(const unsigned long long p3 = prof_stamp();)
            put((PH == 2) ? scrp + (long)k * BL : A.z + bk, x, xm);
#pragma unroll
            for (int s = 0; s < S; ++s) w[s] = x[s];
            wm = xm;
            finish();
            FFP_PROF(if (prof) { const unsigned long long p4 = prof_stamp();
                                 pacc[0] += p1 - p0; pacc[1] += p2 - p1; pacc[2] += p3 - p2;
                                 pacc[3] += p4 - p3; pacc[4] += 1; })
        };
        {
            int t = 0;
            for (; t < nl && t < TN; ++t) lower(t, true);
            for (; t < nl; ++t) lower(t, false);
        }
        // ------------------------------------------------------------ twist line
        R u[S], um;
        {
            const unsigned char *st = begin();
            const long bk = pblk + (long)my * BL;
            R *gw = gbuf + wid * nx;
            R l2[S];
            ld_slots<S>(Fp(st, 3), l2);
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (s < cnt) gw[cell[s]] = (nl > 0) ? l2[s] * w[s] : R(0);
            if (lane == 0) gw[L.m] = (nl > 0) ? M_(st, 1, MID_L2) * wm : R(0);
            R b[S], bm;
            rhs(st, bk, pbase + (long)my * nx, A.z + oblk + (long)my * BL, false, true, pl, other, b, bm);
            named_barrier(1 + q, 64);
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (s < cnt) b[s] = b[s] - gbuf[cell[s]] - gbuf[nx + cell[s]];
            bm = bm - gbuf[L.m] - gbuf[nx + L.m];
            solve(st, b, bm, u, um);
            // final value of the twist line: u (phases 0, 1) or y - u (phase 2)
            R f[S], fm;
            if (PH == 2) {
                R y[S], ym;
                if (VST) ldrow(Vp(st, 1), y, ym); else ldrow(A.z + bk, y, ym);
#pragma unroll
                for (int s = 0; s < S; ++s) f[s] = y[s] - u[s];
                fm = ym - um;
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) f[s] = u[s];
                fm = um;
            }
#pragma unroll
            for (int s = 0; s < S; ++s) tcache[s * 32 + lane] = f[s];
            tcache[S * 32 + lane] = fm;
            if (wid == 0) put(A.z + bk, f, fm);
            finish();
        }
        // ------------------------------------------------------------ upper sweep
        // the first D/2 steps read the lower-sweep row directly (written < NST steps ago)
        auto upper = [&](int t, bool near) {
            FFP_PROF(const unsigned long long p0 = prof_stamp();)
            const unsigned char *st = begin();
            FFP_PROF(const unsigned long long p1 = prof_stamp();)
            const int k = line_of(t);
            const long bk = pblk + (long)k * BL;
            R l2[S], b[S], bm;
            ld_slots<S>(Fp(st, 3), l2);
#pragma unroll
            for (int s = 0; s < S; ++s) b[s] = l2[s] * u[s];
            bm = M_(st, 1, MID_L2) * um;
            R x[S], xm;
            FFP_PROF(const unsigned long long p2 = prof_stamp();)
            solve(st, b, bm, x, xm);
            FFP_PROF(const unsigned long long p3 = prof_stamp();)
            R wv[S], wvm;
            if (VST && !near) ldrow(Vp(st, 0), wv, wvm);
            else ldrow((PH == 2) ? scrp + (long)k * BL : A.z + bk, wv, wvm);
#pragma unroll
            for (int s = 0; s < S; ++s) u[s] = wv[s] - x[s];
            um = wvm - xm;
            R f[S], fm;
            if (PH == 2) {
                R y[S], ym;
                if (VST) ldrow(Vp(st, 1), y, ym); else ldrow(A.z + bk, y, ym);
#pragma unroll
                for (int s = 0; s < S; ++s) f[s] = y[s] - u[s];
                fm = ym - um;
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) f[s] = u[s];
                fm = um;
            }
            put(A.z + bk, f, fm);
            finish();
            FFP_PROF(if (prof) { const unsigned long long p4 = prof_stamp();
                                 pacc[5] += p1 - p0; pacc[6] += p2 - p1; pacc[7] += p3 - p2;
                                 pacc[8] += p4 - p3; pacc[9] += 1; })
        };
        {
            int t = nl - 1;
            for (; t >= 0 && 2 * (nl - t) <= D; --t) upper(t, true);
            for (; t >= 0; --t) upper(t, false);
        }
    }
    FFP_PROF(if (prof) {
        for (int q = 0; q < 10; ++q) g_step_prof[q] = pacc[q];
        g_step_prof[10] = prof_stamp() - pstart;
        g_step_prof[11] = nfail;
    })
}

#ifdef FFP_STEP_PROFILE
inline cudaError_t step_profile_read(unsigned long long *host) {
    return cudaMemcpyFromSymbol(host, g_step_prof, sizeof(g_step_prof));
}
#endif

template <int S, typename F, int PH, int NR = 1>
static cudaError_t launch_phase(const ApplyArgs &a, const ApplyArgs *table, int nx_max, dim3 grid,
                                cudaStream_t st) {
    using SG = Stage<S, F, PH, NR>;
    const size_t smem = (size_t)SG::total(SG::NST, SG::VST, nx_max);
    cudaError_t e = cudaFuncSetAttribute(apply_kernel<S, F, PH, NR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(apply_kernel<S, F, PH, NR>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    apply_kernel<S, F, PH, NR><<<grid, kApplyThreads, smem, st>>>(a, table);
    return cudaGetLastError();
}

template <int S, typename F>
cudaError_t apply_for_slots(const KernelCtx &c, const double *r, double *z, cudaStream_t st,
                            const cudaEvent_t *ev, const double *add) {
    ApplyArgs a;
    a.nx = c.nx; a.ny = c.ny; a.nz = c.nz;
    a.rec = c.ws.rec;
    a.l3n = c.ws.l3;
    a.scr = c.ws.ascr;
    a.flags = c.ws.flags;
    a.ctl = nullptr;
    a.r1 = nullptr; a.z1 = nullptr; a.scr1 = nullptr; a.flags1 = nullptr; a.ctl1 = nullptr;
    a.wait_tries = c.dbg_tries ? c.dbg_tries : kWaitTries;
    a.stall = c.dbg_stall;
    a.r = c.ws.ra;
    a.z = c.ws.za;
    cudaError_t e = launch_to_lb(c, r, c.ws.ra, st);
    const int mz = (a.nz - 1) / 2;
    const bool halves = (mz > 0) || (a.nz - 1 - mz > 0);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess && halves) e = launch_phase<S, F, 0, 1>(a, nullptr, c.nx, dim3(2), st);
    if (e == cudaSuccess) e = launch_phase<S, F, 1, 1>(a, nullptr, c.nx, dim3(1), st);
    if (e == cudaSuccess && halves) e = launch_phase<S, F, 2, 1>(a, nullptr, c.nx, dim3(2), st);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = launch_from_lb(c, c.ws.za, z, add, st);
    return e;
}

// All entries of a device table at once (vectors already in the compute type);
// nr = right-hand sides per entry (1, or 2 when the two-RHS form fits).
template <int S, typename F, int NR>
static cudaError_t apply_table_nr(const ApplyArgs *table, int n, int nx_max, cudaStream_t st) {
    ApplyArgs none;
    std::memset(&none, 0, sizeof(none));
    cudaError_t e = launch_phase<S, F, 0, NR>(none, table, nx_max, dim3(2, n), st);
    if (e == cudaSuccess) e = launch_phase<S, F, 1, NR>(none, table, nx_max, dim3(1, n), st);
    if (e == cudaSuccess) e = launch_phase<S, F, 2, NR>(none, table, nx_max, dim3(2, n), st);
    return e;
}

template <int S, typename F>
bool two_rhs_supported() { return two_rhs_fits<S, F>(); }

template <int S, typename F>
cudaError_t apply_table_for_slots(const ApplyArgs *table, int n, int nx_max, int nr, cudaStream_t st) {
    if constexpr (two_rhs_fits<S, F>()) {
        if (nr == 2) return apply_table_nr<S, F, 2>(table, n, nx_max, st);
    }
    if (nr != 1) return cudaErrorInvalidValue;
    return apply_table_nr<S, F, 1>(table, n, nx_max, st);
}

}  // namespace ffp
