// ffp_batch.cu -- many independent solves at once (the batched form of the
// PCG of Sec. III with B_NTD or B_c): instances of uneven grid sizes, each with
// its own operator and preconditioner, and several right-hand sides per
// instance.  A "pair" is one (instance, right-hand side).
//
// Every pair computes exactly what its standalone ffp_pcg_solve computes: the
// same kernels (each one has a single-pair form and a table form that takes
// its pair from blockIdx.y), the same line slot count S per instance, the same
// reduction partition per vector, the same control flow.  What changes is how
// the work reaches the GPU:
//  * setup: one launch per setup phase (and per ILU(0) pivot diagonal) covers
//    every instance with the same S, instead of one launch per instance;
//  * solve: the pairs are kept in groups of equal (apply S, ILU S), longest
//    level-3 chain first inside a group (the CTA scheduler takes blockIdx.y in
//    order, so the long chains start first).  One CG iteration of all pairs is
//    one CUDA graph: a branch per group runs the group's ILU(0) column sweeps
//    (one launch per sweep over every plane of the group's pairs), apply
//    phases and vector kernels; the graph is captured once and replayed.
//    Branches run at stream priorities ranked by the group's longest level-3
//    chain, so the kernels of the batch's critical path get SM slots first.
//    Each pair's control word in device memory says whether it iterates this
//    round, whether its direction restarts, or whether its true residual is
//    checked; kernels of pairs that do not take part return at once.  After a
//    replay the host reads every pair's scalar block (one copy) and decides for
//    each pair exactly as the single-instance driver does.
//  * tuning: the ILU(0) warps per CTA and whether the groups run as parallel
//    graph branches or one after another are chosen by timing the
//    preconditioner graph on the batch itself (ffp_batch_tune); neither changes
//    any result.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "ffp_vecops.cuh"

namespace ffp {

struct PairArgs {
    int nx, ny, nz, nxy;
    long long n;
    int nb;                           // blocks of the vector kernels (the standalone solve's)
    const double *d, *cx, *cy, *cz;   // operator bands of the instance
    const double *b;
    double *x;                        // caller's vectors
    double *r, *z, *p, *q, *c1, *c2;  // CG vectors and B_c temporaries
    float *r32;                       // B_c with FP32/BF16 factors: FP32 copy of r (ILU(0) input)
    unsigned long long *tw;           // and the ILU(0) sweeps' tagged result words; else null
    void *ra, *za;                    // apply input and output, line-block layout (lb_pos)
    int S;                            // line slot count of the instance
    double *red, *scal;
    int *flags;
    const int *ctl;                   // control word
};

enum { CTL_ITER = 1, CTL_FRESH = 2, CTL_RESID = 4 };

// The pair of this block; false if it takes no part or the block is past its grid.
__device__ __forceinline__ bool pair_of(const PairArgs *T, int need, PairArgs &P, int &c) {
    P = T[blockIdx.y];
    c = *P.ctl;
    return (c & need) && (int)blockIdx.x < P.nb;
}

__device__ __forceinline__ Geo pgeo(const PairArgs &P) {
    Geo g;
    g.nx = P.nx; g.ny = P.ny; g.nz = P.nz; g.n = P.n; g.nxy = P.nxy;
    return g;
}

// the grid-stride loop of the single-instance kernels, over the pair's own grid
#define FFP_PAIR_LOOP(P, a)                                                       \
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < P.n; \
         a += (long long)P.nb * blockDim.x)

// r = b - A x ; partials (r.r, b.b)
__global__ void __launch_bounds__(kThreads) b_resid(const PairArgs *__restrict__ T) {
    PairArgs P;
    int c;
    if (!pair_of(T, CTL_RESID, P, c)) return;
    const Geo g = pgeo(P);
    double acc[2] = {0.0, 0.0};
    FFP_PAIR_LOOP(P, a) {
        const double ba = P.b[a];
        const double ra = ba - stencil(g, a, P.d, P.cx, P.cy, P.cz, P.x);
        P.r[a] = ra;
        if (P.r32) P.r32[a] = (float)ra;
        acc[0] += ra * ra;
        acc[1] += ba * ba;
    }
    block_sum<2>(acc, P.red);
}

// fold the partials of every pair whose control word has `need` (one warp per pair)
__global__ void b_finalize(const PairArgs *__restrict__ T, int need, int mode, int flexible) {
    const PairArgs &P = T[blockIdx.y];
    const int c = *P.ctl;
    if (!(c & need)) return;
    finalize_scalars(mode, P.nb, (c & CTL_FRESH) ? 1 : 0, flexible, P.red, P.scal, P.flags);
}

// preconditioner input, in the apply's line-block layout and arithmetic type R:
// B_c's r - A c1 (c1 = B_ILU0^{-1} r), or r
template <typename R>
__global__ void __launch_bounds__(kThreads) b_prec_in(const PairArgs *__restrict__ T, int combo) {
    PairArgs P;
    int c;
    if (!pair_of(T, CTL_ITER, P, c)) return;
    const Geo g = pgeo(P);
    R *ra = static_cast<R *>(P.ra);
    const long long L = lb_len(P.S);
    FFP_PAIR_LOOP(P, a) {
        const double v = combo ? P.r[a] - stencil(g, a, P.d, P.cx, P.cy, P.cz, P.c1) : P.r[a];
        const long long line = a / P.nx;
        ra[line * L + lb_pos(P.nx, P.S, (int)(a - line * P.nx))] = (R)v;
    }
}

// preconditioner output: z = the apply's output (+ c1 for B_c)
template <typename R>
__global__ void __launch_bounds__(kThreads) b_prec_out(const PairArgs *__restrict__ T, int combo) {
    PairArgs P;
    int c;
    if (!pair_of(T, CTL_ITER, P, c)) return;
    const R *za = static_cast<const R *>(P.za);
    const long long L = lb_len(P.S);
    FFP_PAIR_LOOP(P, a) {
        const long long line = a / P.nx;
        const double v = (double)za[line * L + lb_pos(P.nx, P.S, (int)(a - line * P.nx))];
        P.z[a] = combo ? v + P.c1[a] : v;
    }
}

// partials (r.z, z.q)
__global__ void __launch_bounds__(kThreads) b_dot_rz(const PairArgs *__restrict__ T) {
    PairArgs P;
    int c;
    if (!pair_of(T, CTL_ITER, P, c)) return;
    double acc[2] = {0.0, 0.0};
    FFP_PAIR_LOOP(P, a) {
        const double za = P.z[a];
        acc[0] += P.r[a] * za;
        acc[1] += za * P.q[a];
    }
    block_sum<2>(acc, P.red);
}

// p = z + beta p (p = z on a restart)
__global__ void __launch_bounds__(kThreads) b_update_p(const PairArgs *__restrict__ T) {
    PairArgs P;
    int c;
    if (!pair_of(T, CTL_ITER, P, c)) return;
    const double beta = P.scal[SC_BETA];
    const bool fresh = (c & CTL_FRESH) != 0;
    FFP_PAIR_LOOP(P, a) P.p[a] = fresh ? P.z[a] : P.z[a] + beta * P.p[a];
}

// q = A p ; partial (p.q)
__global__ void __launch_bounds__(kThreads) b_spmv_dot(const PairArgs *__restrict__ T) {
    PairArgs P;
    int c;
    if (!pair_of(T, CTL_ITER, P, c)) return;
    const Geo g = pgeo(P);
    double acc[1] = {0.0};
    FFP_PAIR_LOOP(P, a) {
        const double qa = stencil(g, a, P.d, P.cx, P.cy, P.cz, P.p);
        P.q[a] = qa;
        acc[0] += P.p[a] * qa;
    }
    block_sum<1>(acc, P.red);
}

// x += alpha p ; r -= alpha q ; partial (r.r)
__global__ void __launch_bounds__(kThreads) b_update_xr(const PairArgs *__restrict__ T) {
    PairArgs P;
    int c;
    if (!pair_of(T, CTL_ITER, P, c)) return;
    const double alpha = P.scal[SC_ALPHA];
    double acc[1] = {0.0};
    FFP_PAIR_LOOP(P, a) {
        P.x[a] += alpha * P.p[a];
        const double ra = P.r[a] - alpha * P.q[a];
        P.r[a] = ra;
        if (P.r32) P.r32[a] = (float)ra;
        acc[0] += ra * ra;
    }
    block_sum<1>(acc, P.red);
}

}  // namespace ffp

// ---------------------------------------------------------------- host side
using namespace ffp;

namespace {

constexpr size_t kPairScal = 8 * (size_t)kScal + 4 * 16;  // scalar block + flags of one pair

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

bool grid_ok(const ffp_grid &g) {
    return g.nx >= 1 && g.ny >= 1 && g.nz >= 1 && g.nx <= FFP_MAX_NX &&
           (long long)g.nx * g.ny * g.nz <= 2000000000LL;
}

// vectors of a pair beyond an instance's first: r z p q c1 c2, the apply input and output
// blocks, apply scratch (line-block layout), partials, and with FP32/BF16 factors the
// FP32 copy of the ILU(0) input and the tagged words of its result
size_t extra_pair_bytes(const ffp_grid &g, int prec) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t ab = (prec == FFP_FP64) ? 8 : 4, lb = (size_t)lb_len(slots_for(g.nx));
    return 6 * al256(8 * n) + 2 * al256(ab * (size_t)g.ny * g.nz * lb) + al256(ab * 2 * (size_t)g.ny * lb) +
           al256(8 * (size_t)kRedSlots) + (prec == FFP_FP64 ? 0 : al256(4 * n) + al256(8 * n));
}

// ints of the ILU(0) sync region: per group 2 ticket counters (padded to 32 ints)
// and one ready flag per line of each of its pairs
constexpr int kSyncHead = 32;

struct Group {
    int p0, np;  // device pair range
    int q0, nq;  // the group's range in the two-RHS entry table; nq = 0: it has none
    int S, Si;   // apply and ILU(0) slot counts
    int nx_max, nb_max;
    int nitems;        // ILU(0) work items (planes) of the group's pairs
    long long chain;   // longest level-3 chain of its pairs, (ny + 1)(nz + 1) line solves
    int *sync;         // the group's ILU(0) sync region
    size_t sync_bytes;
};

long long kernel_count_of(const std::vector<Group> &gs, int combo, int f32) {
    long long k = 0;
    for (const Group &g : gs)
        k += (combo ? (f32 ? 3 : 2) : 0) + 2 + 3 + 7;
    return k;
}

}  // namespace

struct ffp_batch {
    int device;
    int count, nrhs, npairs, prec, precond;
    std::vector<KernelCtx> inst;
    std::vector<int> order;        // order[k] = caller's pair index (i * nrhs + j) at device slot k
    std::vector<PairArgs> pairs;   // host copy of the device pair table (device order)
    std::vector<Group> groups;
    int nb_max;
    PairArgs *dpairs;
    ApplyArgs *dapply;
    ApplyArgs *dapply2;            // two-RHS entries (pairs (i, 2j) and (i, 2j + 1))
    IluArgs *dilu;
    SetupArgs *dsetup;
    IluPivArgs *dpiv;
    int *dsync;                    // ILU(0) sync regions of all groups
    int *dctl;
    char *dscal;                   // scalar blocks of all pairs, contiguous
    int *hctl;                     // pinned
    char *hscal;                   // pinned
    ffp_batch_config cfg;
    cudaStream_t gs;
    std::vector<cudaStream_t> side;
    cudaEvent_t fork, tev[2];
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t g_iter, g_resid;
    long long iter_launches, resid_launches, setup_launches;
};

namespace {

// Workspace layout; base == nullptr only sizes it.  Pair (i, 0) uses the CG
// vectors of instance i's own workspace; pairs (i, j > 0) get their own.
size_t batch_layout(int count, const ffp_grid *grids, int nrhs, int prec, char *base, ffp_batch *B,
                    std::vector<void *> *ascr) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += al256(bytes);
        return p;
    };
    const int np = count * nrhs;
    char *t_pairs = take(sizeof(PairArgs) * np);
    char *t_apply = take(sizeof(ApplyArgs) * np);
    char *t_apply2 = take(sizeof(ApplyArgs) * np);
    char *t_ilu = take(sizeof(IluArgs) * np);
    char *t_setup = take(sizeof(SetupArgs) * count);
    char *t_piv = take(sizeof(IluPivArgs) * count);
    char *t_ctl = take(4 * (size_t)np);
    size_t sync_ints = 0;
    for (int i = 0; i < count; ++i) sync_ints += (size_t)nrhs * ((size_t)grids[i].ny * grids[i].nz + kSyncHead);
    char *t_sync = take(4 * sync_ints);
    char *t_scal = take(kPairScal * np);
    if (B) {
        B->dpairs = (PairArgs *)t_pairs; B->dapply = (ApplyArgs *)t_apply; B->dilu = (IluArgs *)t_ilu;
        B->dapply2 = (ApplyArgs *)t_apply2;
        B->dsetup = (SetupArgs *)t_setup; B->dpiv = (IluPivArgs *)t_piv; B->dctl = (int *)t_ctl;
        B->dsync = (int *)t_sync;
        B->dscal = t_scal;
    }
    for (int i = 0; i < count; ++i) {
        const size_t wsb = carve_workspace(&grids[i], prec, 0, nullptr, nullptr);
        char *wbase = take(wsb);
        if (B) carve_workspace(&grids[i], prec, 0, wbase, &B->inst[i].ws);
        const ffp_grid &g = grids[i];
        const size_t n = (size_t)g.nx * g.ny * g.nz;
        const size_t ab = (prec == FFP_FP64) ? 8 : 4, lb = (size_t)lb_len(slots_for(g.nx));
        for (int j = 0; j < nrhs; ++j) {
            const int up = i * nrhs + j;  // caller's pair index
            if (j == 0) {
                if (B) {
                    const Ws &w = B->inst[i].ws;
                    PairArgs &P = B->pairs[up];
                    P.r = w.r; P.z = w.z; P.p = w.p; P.q = w.q; P.c1 = w.c1; P.c2 = w.c2;
                    P.ra = w.ra; P.za = w.za; P.red = w.red;
                    P.r32 = (float *)w.ilu_v;
                    P.tw = w.ilu_tw;
                    (*ascr)[up] = w.ascr;
                }
                continue;
            }
            char *pb = take(extra_pair_bytes(g, prec));
            if (B) {
                PairArgs &P = B->pairs[up];
                size_t o = 0;
                auto sub = [&](size_t bytes) { char *p = pb + o; o += al256(bytes); return p; };
                P.r = (double *)sub(8 * n); P.z = (double *)sub(8 * n); P.p = (double *)sub(8 * n);
                P.q = (double *)sub(8 * n); P.c1 = (double *)sub(8 * n); P.c2 = (double *)sub(8 * n);
                P.ra = sub(ab * (size_t)g.ny * g.nz * lb);
                P.za = sub(ab * (size_t)g.ny * g.nz * lb);
                (*ascr)[up] = sub(ab * 2 * (size_t)g.ny * lb);
                P.red = (double *)sub(8 * (size_t)kRedSlots);
                if (prec != FFP_FP64) {
                    P.r32 = (float *)sub(4 * n);
                    P.tw = (unsigned long long *)sub(8 * n);
                }
            }
        }
    }
    return off;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? FFP_OK : FFP_ERR_CUDA; }

// The preconditioner z = B^{-1} r of a group's pairs with CTL_ITER, as in the
// single-instance driver: B_c^{-1} r = c1 + B_NTD^{-1} (r - A c1), c1 = B_ILU0^{-1} r.
cudaError_t group_precond(const ffp_batch *B, const Group &g, cudaStream_t s) {
    const int combo = B->precond == FFP_PRECOND_COMBO, f32 = B->prec != FFP_FP64;
    const PairArgs *T = B->dpairs + g.p0;
    const dim3 gv(g.nb_max, g.np);
    cudaError_t e = cudaSuccess;
    if (combo)
        e = launch_ilu_table(B->prec, g.Si, B->dilu + g.p0, g.np, g.nitems, g.sync, g.sync_bytes,
                             B->cfg.ilu_warps, s);
    if (e == cudaSuccess) {
        if (f32) b_prec_in<float><<<gv, kThreads, 0, s>>>(T, combo);
        else b_prec_in<double><<<gv, kThreads, 0, s>>>(T, combo);
        e = (B->cfg.rhs_per_cta == 2 && g.nq > 0)
                ? launch_apply_table(B->prec, g.S, B->dapply2 + g.q0, g.nq, g.nx_max, 2, s)
                : launch_apply_table(B->prec, g.S, B->dapply + g.p0, g.np, g.nx_max, 1, s);
    }
    if (e == cudaSuccess) {
        if (f32) b_prec_out<float><<<gv, kThreads, 0, s>>>(T, combo);
        else b_prec_out<double><<<gv, kThreads, 0, s>>>(T, combo);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// One CG iteration of a group's pairs with CTL_ITER (the single-pair order:
// preconditioner, (r,z), p, (p,Ap), x and r).
cudaError_t group_iteration(const ffp_batch *B, const Group &g, cudaStream_t s) {
    const int flexible = (B->prec != FFP_FP64) || (B->precond == FFP_PRECOND_COMBO);
    const PairArgs *T = B->dpairs + g.p0;
    const dim3 gv(g.nb_max, g.np), gf(1, g.np);
    const cudaError_t e = group_precond(B, g, s);
    if (e != cudaSuccess) return e;
    b_dot_rz<<<gv, kThreads, 0, s>>>(T);
    b_finalize<<<gf, 32, 0, s>>>(T, CTL_ITER, FIN_RZ, flexible);
    b_update_p<<<gv, kThreads, 0, s>>>(T);
    b_spmv_dot<<<gv, kThreads, 0, s>>>(T);
    b_finalize<<<gf, 32, 0, s>>>(T, CTL_ITER, FIN_PQ, flexible);
    b_update_xr<<<gv, kThreads, 0, s>>>(T);
    b_finalize<<<gf, 32, 0, s>>>(T, CTL_ITER, FIN_RR, flexible);
    return cudaGetLastError();
}

// All groups, as parallel branches off stream gs or one after another on it.
template <class Fn>
cudaError_t all_groups(ffp_batch *B, Fn fn) {
    cudaError_t e = cudaSuccess;
    const int ng = (int)B->groups.size();
    if (!B->cfg.branches || ng == 1) {
        for (int k = 0; k < ng && e == cudaSuccess; ++k) e = fn(B->groups[k], B->gs);
        return e;
    }
    e = cudaEventRecord(B->fork, B->gs);
    for (int k = 0; k < ng && e == cudaSuccess; ++k) {
        e = cudaStreamWaitEvent(B->side[k], B->fork, 0);
        if (e == cudaSuccess) e = fn(B->groups[k], B->side[k]);
        if (e == cudaSuccess) e = cudaEventRecord(B->join[k], B->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B->gs, B->join[k], 0);
    }
    return e;
}

template <class Fn>
cudaError_t capture(cudaStream_t st, cudaGraphExec_t *out, Fn fn) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t e2 = fn();
    e = cudaStreamEndCapture(st, &g);
    if (e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e2;
    }
    if (e != cudaSuccess) return e;
    // kernel nodes keep the priority of the stream they were captured from
    e = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    return e;
}

void drop_graphs(ffp_batch *B) {
    if (B->g_iter) cudaGraphExecDestroy(B->g_iter);
    if (B->g_resid) cudaGraphExecDestroy(B->g_resid);
    B->g_iter = nullptr;
    B->g_resid = nullptr;
}

cudaError_t build_graphs(ffp_batch *B) {
    const int np = B->npairs;
    cudaError_t e = capture(B->gs, &B->g_iter, [&]() {
        cudaError_t x = cudaMemcpyAsync(B->dctl, B->hctl, 4 * (size_t)np, cudaMemcpyHostToDevice, B->gs);
        if (x == cudaSuccess)
            x = all_groups(B, [&](const Group &g, cudaStream_t s) { return group_iteration(B, g, s); });
        if (x == cudaSuccess)
            x = cudaMemcpyAsync(B->hscal, B->dscal, kPairScal * np, cudaMemcpyDeviceToHost, B->gs);
        return x;
    });
    if (e != cudaSuccess) return e;
    B->iter_launches = kernel_count_of(B->groups, B->precond == FFP_PRECOND_COMBO, B->prec != FFP_FP64);
    e = capture(B->gs, &B->g_resid, [&]() {
        cudaError_t x = cudaMemcpyAsync(B->dctl, B->hctl, 4 * (size_t)np, cudaMemcpyHostToDevice, B->gs);
        if (x == cudaSuccess) {
            b_resid<<<dim3(B->nb_max, np), kThreads, 0, B->gs>>>(B->dpairs);
            b_finalize<<<dim3(1, np), 32, 0, B->gs>>>(B->dpairs, CTL_RESID, FIN_RESID, 0);
            x = cudaGetLastError();
        }
        if (x == cudaSuccess)
            x = cudaMemcpyAsync(B->hscal, B->dscal, kPairScal * np, cudaMemcpyDeviceToHost, B->gs);
        return x;
    });
    B->resid_launches = 2;
    return e;
}

const double *pscal(const ffp_batch *B, int k) {
    return reinterpret_cast<const double *>(B->hscal + kPairScal * k);
}
const int *pflags(const ffp_batch *B, int k) { return reinterpret_cast<const int *>(pscal(B, k) + kScal); }

std::string batch_key(const ffp_batch *B) {
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, B->device);
    unsigned long long h = 1469598103934665603ULL;  // FNV-1a over the instance grids
    for (const KernelCtx &c : B->inst)
        for (int v : {c.nx, c.ny, c.nz}) {
            h ^= (unsigned long long)v;
            h *= 1099511628211ULL;
        }
    char buf[320];
    std::snprintf(buf, sizeof(buf), "%s|sm%d%d|prec%d|pc%d|count%d|nrhs%d|grids%016llx", prop.name,
                  prop.major, prop.minor, B->prec, B->precond, B->count, B->nrhs, h);
    for (char *p = buf; *p; ++p)
        if (*p == ' ' || *p == '\t' || *p == '\n') *p = '_';
    return buf;
}

// cache lines: "<key> <ilu_warps> <branches> <ms> <ntd_ms> <rhs_per_cta>"
bool cache_lookup(const char *path, const std::string &key, ffp_batch_config *cfg) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char k[512];
    int w = 0, br = 0, nr = 0;
    double ms = 0.0, nms = 0.0;
    bool found = false;
    while (std::fscanf(f, "%511s %d %d %lf %lf %d", k, &w, &br, &ms, &nms, &nr) == 6)
        if (key == k && w >= 1 && w <= 8 && (br == 0 || br == 1) && (nr == 1 || nr == 2)) {
            cfg->ilu_warps = w; cfg->branches = br; cfg->ms = ms; cfg->ntd_ms = nms;
            cfg->rhs_per_cta = nr;
            found = true;  // the last matching line wins
        }
    std::fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const ffp_batch_config &cfg) {
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %.6f %.6f %d\n", key.c_str(), cfg.ilu_warps, cfg.branches, cfg.ms, cfg.ntd_ms,
                 cfg.rhs_per_cta);
    std::fclose(f);
}

}  // namespace

extern "C" {

size_t ffp_batch_workspace_bytes(int count, const ffp_grid *grids, int nrhs, int precision) {
    if (count < 1 || nrhs < 1 || !grids || prec_bytes(precision) == 0) return 0;
    if ((long long)count * nrhs > FFP_BATCH_MAX_PAIRS) return 0;
    for (int i = 0; i < count; ++i)
        if (!grid_ok(grids[i])) return 0;
    return batch_layout(count, grids, nrhs, precision, nullptr, nullptr, nullptr);
}

int ffp_batch_setup(int count, const ffp_grid *grids, const double *const *kappa,
                    const ffp_bc *bcs, const double *const *t, int nrhs, int precision,
                    int precond, void *workspace, size_t ws_bytes, void *stream, ffp_batch **out) {
    if (out) *out = nullptr;
    if (count < 1 || nrhs < 1 || !grids || !kappa || !bcs || !workspace || !out) return FFP_ERR_ARG;
    if (prec_bytes(precision) == 0) return FFP_ERR_ARG;
    const int schur = (precond & FFP_SCHUR_BETA) ? 1 : 0;
    precond &= ~FFP_SCHUR_BETA;
    if (precond != FFP_PRECOND_NTD && precond != FFP_PRECOND_COMBO) return FFP_ERR_ARG;
    if (((uintptr_t)workspace & 255) != 0) return FFP_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        if (!grid_ok(grids[i]) || !kappa[i]) return FFP_ERR_ARG;
        for (int f = 0; f < 6; ++f)
            if (bcs[i].face[f] != FFP_DIRICHLET && bcs[i].face[f] != FFP_NEUMANN) return FFP_ERR_ARG;
    }
    const size_t need = ffp_batch_workspace_bytes(count, grids, nrhs, precision);
    if (need == 0 || ws_bytes < need) return FFP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ffp_batch *B = new (std::nothrow) ffp_batch;
    if (!B) return FFP_ERR_ARG;
    B->count = count; B->nrhs = nrhs; B->npairs = count * nrhs; B->prec = precision;
    B->precond = precond;
    B->nb_max = 1;
    B->hctl = nullptr; B->hscal = nullptr; B->gs = nullptr; B->fork = nullptr;
    B->tev[0] = B->tev[1] = nullptr;
    B->g_iter = nullptr; B->g_resid = nullptr;
    B->iter_launches = 0; B->resid_launches = 0; B->setup_launches = 0;
    B->cfg.ilu_warps = 4; B->cfg.branches = 1; B->cfg.ms = 0.0; B->cfg.ntd_ms = 0.0;
    B->cfg.from_cache = 0; B->cfg.rhs_per_cta = 1;
    B->inst.resize(count);
    B->pairs.assign(B->npairs, PairArgs());
    std::memset(B->pairs.data(), 0, sizeof(PairArgs) * B->npairs);
    auto fail = [&](int status) {
        ffp_batch_destroy(B);
        return status;
    };
    if (cudaGetDevice(&B->device) != cudaSuccess) return fail(FFP_ERR_CUDA);
    std::vector<void *> ascr(B->npairs, nullptr);
    batch_layout(count, grids, nrhs, precision, (char *)workspace, B, &ascr);
    for (int i = 0; i < count; ++i) {
        KernelCtx &c = B->inst[i];
        c.nx = grids[i].nx; c.ny = grids[i].ny; c.nz = grids[i].nz;
        c.n = (long long)c.nx * c.ny * c.nz;
        c.lx = grids[i].lx > 0 ? grids[i].lx : 1.0;
        c.ly = grids[i].ly > 0 ? grids[i].ly : 1.0;
        c.lz = grids[i].lz > 0 ? grids[i].lz : 1.0;
        c.prec = precision; c.precond = precond; c.schur = schur; c.slots = slots_for(c.nx);
        c.dbg_stall = 0; c.dbg_tries = 0;
    }
    if (cudaMallocHost((void **)&B->hctl, 4 * (size_t)B->npairs) != cudaSuccess ||
        cudaMallocHost((void **)&B->hscal, kPairScal * (size_t)B->npairs) != cudaSuccess)
        return fail(FFP_ERR_CUDA);
    cudaError_t e = cudaMemsetAsync(B->dscal, 0, kPairScal * B->npairs, st);
    // ---- operators (per instance) and the checks of kappa and of user filters
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        const KernelCtx &c = B->inst[i];
        const size_t recb = prec_bytes(precision) * (size_t)c.ny * c.nz * (size_t)rec_len(c.slots);
        e = cudaMemsetAsync(c.ws.scal, 0, 8 * (size_t)kScal + 4 * 16, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c.ws.rec, 0, recb, st);  // record pads read as 0
        if (e == cudaSuccess) e = launch_assemble(c, kappa[i], bcs[i].face, st);
        if (e == cudaSuccess && t && t[i]) e = launch_check_filter(c, t[i], st);
        if (e == cudaSuccess) e = launch_convert_bands(c, st);
        B->setup_launches += 1 + ((t && t[i]) ? 1 : 0) + (precond == FFP_PRECOND_COMBO ? 4 : 2);
    }
    if (e != cudaSuccess) return fail(FFP_ERR_CUDA);
    std::vector<int> fl(16 * (size_t)count, 0);
    auto read_flags = [&]() -> int {
        for (int i = 0; i < count; ++i)
            if (cudaMemcpyAsync(&fl[16 * (size_t)i], B->inst[i].ws.flags, 4 * 16, cudaMemcpyDeviceToHost,
                                st) != cudaSuccess)
                return FFP_ERR_CUDA;
        return cuda_status(cudaStreamSynchronize(st));
    };
    {
        const int s = read_flags();
        if (s != FFP_OK) return fail(s);
        for (int i = 0; i < count; ++i)
            if (fl[16 * i + FL_ARG]) return fail(FFP_ERR_ARG);
    }
    // ---- setup: one launch per phase for all instances of one slot count
    {
        std::vector<int> ord(count);
        for (int i = 0; i < count; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return B->inst[a].slots < B->inst[b].slots; });
        std::vector<SetupArgs> sa(count);
        for (int k = 0; k < count; ++k) fill_setup_args(B->inst[ord[k]], t ? t[ord[k]] : nullptr, &sa[k]);
        e = cudaMemcpyAsync(B->dsetup, sa.data(), sizeof(SetupArgs) * count, cudaMemcpyHostToDevice, st);
        for (int k0 = 0; k0 < count && e == cudaSuccess;) {
            int k1 = k0, nxm = 1;
            while (k1 < count && B->inst[ord[k1]].slots == B->inst[ord[k0]].slots)
                nxm = std::max(nxm, B->inst[ord[k1++]].nx);
            e = launch_setup_table(B->inst[ord[k0]].slots, B->dsetup + k0, k1 - k0, nxm, st);
            B->setup_launches += 2;
            k0 = k1;
        }
        std::vector<IluPivArgs> pa(count);
        if (e == cudaSuccess && precond == FFP_PRECOND_COMBO) {
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
                return ilu_slots(B->inst[a].nx) < ilu_slots(B->inst[b].nx);
            });
            for (int k = 0; k < count; ++k) {
                const KernelCtx &c = B->inst[ord[k]];
                IluPivArgs &a = pa[k];
                a.nx = c.nx; a.ny = c.ny; a.nz = c.nz; a.prec = c.prec;
                a.d = c.ws.d; a.cx = c.ws.cx; a.cy = c.ws.cy; a.cz = c.ws.cz;
                a.D64 = c.ws.p;  // the CG vector p is free until a solve
                a.dinv = c.ws.dinv; a.flags = c.ws.flags;
            }
            e = cudaMemcpyAsync(B->dpiv, pa.data(), sizeof(IluPivArgs) * count, cudaMemcpyHostToDevice, st);
            for (int k0 = 0; k0 < count && e == cudaSuccess;) {
                const int Si = ilu_slots(B->inst[ord[k0]].nx);
                int k1 = k0, nd = 1, ml = 1;
                while (k1 < count && ilu_slots(B->inst[ord[k1]].nx) == Si) {
                    const KernelCtx &c = B->inst[ord[k1++]];
                    nd = std::max(nd, c.ny + c.nz - 1);
                    ml = std::max(ml, std::min(c.ny, c.nz));
                }
                e = launch_ilu_setup_table(Si, B->dpiv + k0, k1 - k0, nd, ml, st);
                B->setup_launches += nd;
                k0 = k1;
            }
        }
        // the host tables must outlive the copies above
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return fail(FFP_ERR_CUDA);
    {
        const int s = read_flags();
        if (s != FFP_OK) return fail(s);
        for (int i = 0; i < count; ++i)
            if (fl[16 * i + FL_BREAKDOWN]) return fail(FFP_ERR_BREAKDOWN);
    }
    // ---- pair tables in device order: groups of equal (S, ILU S), longest chain first
    auto key = [&](int up) {
        const KernelCtx &c = B->inst[up / nrhs];
        return std::make_pair(c.slots, ilu_slots(c.nx));
    };
    std::vector<int> ord(B->npairs);
    for (int k = 0; k < B->npairs; ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        if (key(a) != key(b)) return key(a) < key(b);
        const KernelCtx &ca = B->inst[a / nrhs], &cb = B->inst[b / nrhs];
        return (long long)ca.ny * ca.nz > (long long)cb.ny * cb.nz;
    });
    B->order = ord;
    std::vector<PairArgs> pt(B->npairs);
    std::vector<ApplyArgs> at(B->npairs);
    std::vector<IluArgs> it(B->npairs);
    for (int k = 0; k < B->npairs; ++k) {
        const int up = ord[k], i = up / nrhs;
        const KernelCtx &c = B->inst[i];
        PairArgs P = B->pairs[up];
        P.nx = c.nx; P.ny = c.ny; P.nz = c.nz; P.nxy = c.nx * c.ny; P.n = c.n;
        P.nb = grid_for(c.n);
        P.S = c.slots;
        P.d = c.ws.d; P.cx = c.ws.cx; P.cy = c.ws.cy; P.cz = c.ws.cz;
        P.b = nullptr; P.x = nullptr;
        P.scal = reinterpret_cast<double *>(B->dscal + kPairScal * k);
        P.flags = reinterpret_cast<int *>(P.scal + kScal);
        P.ctl = B->dctl + k;
        if (precond != FFP_PRECOND_COMBO || precision == FFP_FP64) {
            P.r32 = nullptr;
            P.tw = nullptr;
        }
        pt[k] = P;
        ApplyArgs &A = at[k];
        A.nx = c.nx; A.ny = c.ny; A.nz = c.nz;
        A.rec = c.ws.rec; A.l3n = c.ws.l3;
        A.r = P.ra;
        A.z = P.za;
        A.scr = ascr[up];
        A.flags = P.flags;
        A.ctl = P.ctl;
        A.r1 = nullptr; A.z1 = nullptr; A.scr1 = nullptr; A.flags1 = nullptr; A.ctl1 = nullptr;
        A.wait_tries = kWaitTries;
        A.stall = 0;
        IluArgs &L = it[k];
        std::memset(&L, 0, sizeof(L));
        L.nx = c.nx; L.ny = c.ny; L.nz = c.nz;
        L.dinv = c.ws.dinv; L.lx = c.ws.lx; L.ly = c.ws.ly; L.lz = c.ws.l3;
        if (P.r32) {  // FP32 sweeps on tagged words; the backward sweep also stores c1 in FP64
            L.r = P.r32; L.t = nullptr; L.tw = P.tw; L.out64 = P.c1;
        } else {
            L.r = P.r; L.t = P.c1;
        }
        L.ctl = P.ctl;
        L.err = P.flags;
        B->nb_max = std::max(B->nb_max, P.nb);
    }
    B->pairs = pt;
    // groups; each gets its ILU(0) sync region: counters, then its pairs' ready flags
    int *sync = B->dsync;
    std::vector<ApplyArgs> at2;
    for (int k0 = 0; k0 < B->npairs;) {
        Group g;
        g.p0 = k0;
        g.S = key(ord[k0]).first;
        g.Si = key(ord[k0]).second;
        g.nx_max = 1; g.nb_max = 1; g.nitems = 0; g.chain = 0;
        g.sync = sync;
        int *ready = sync + kSyncHead;
        int k1 = k0;
        while (k1 < B->npairs && key(ord[k1]) == key(ord[k0])) {
            IluArgs &L = it[k1];
            const PairArgs &P = pt[k1++];
            g.nx_max = std::max(g.nx_max, P.nx);
            g.nb_max = std::max(g.nb_max, P.nb);
            g.chain = std::max(g.chain, (long long)(P.ny + 1) * (P.nz + 1));
            L.item0 = g.nitems;
            L.ready = ready;
            L.sync = sync;
            g.nitems += P.nz;
            ready += (size_t)P.ny * P.nz;
        }
        g.np = k1 - k0;
        g.q0 = (int)at2.size();
        g.nq = 0;
        // two-RHS entries: consecutive pairs (i, 2j), (i, 2j + 1) of one instance, if every
        // pair of the group has its partner and the two-RHS kernels exist for its slot count
        bool pairs_up = (g.np % 2 == 0) && apply_two_rhs_ok(precision, g.S);
        for (int k = k0; k < k1 && pairs_up; k += 2)
            pairs_up = (ord[k] % 2 == 0) && (ord[k + 1] == ord[k] + 1) && (ord[k] / nrhs == ord[k + 1] / nrhs);
        if (pairs_up) {
            for (int k = k0; k < k1; k += 2) {
                ApplyArgs E = at[k];
                const ApplyArgs &P2 = at[k + 1];
                E.r1 = P2.r; E.z1 = P2.z; E.scr1 = P2.scr; E.flags1 = P2.flags; E.ctl1 = P2.ctl;
                at2.push_back(E);
            }
            g.nq = g.np / 2;
        }
        g.sync_bytes = 4 * (size_t)(ready - sync);
        sync = ready;
        B->groups.push_back(g);
        k0 = k1;
    }
    e = cudaMemcpyAsync(B->dpairs, pt.data(), sizeof(PairArgs) * B->npairs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->dapply, at.data(), sizeof(ApplyArgs) * B->npairs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->dilu, it.data(), sizeof(IluArgs) * B->npairs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !at2.empty())
        e = cudaMemcpyAsync(B->dapply2, at2.data(), sizeof(ApplyArgs) * at2.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->dctl, 0, 4 * (size_t)B->npairs, st);
    // padding positions of the apply input blocks must read 0; b_prec_in writes only cells;
    // ILU(0) epochs start at 0 and the tagged words untagged
    for (int k = 0; k < B->npairs && e == cudaSuccess; ++k) {
        const PairArgs &P = pt[k];
        e = cudaMemsetAsync(P.ra, 0, (precision == FFP_FP64 ? 8 : 4) * (size_t)P.ny * P.nz * lb_len(P.S), st);
        if (e == cudaSuccess && P.tw) e = cudaMemsetAsync(P.tw, 0, 8 * (size_t)P.n, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(B->dsync, 0, 4 * (size_t)(sync - B->dsync), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // ---- streams and events of the graphs
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->gs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreate(&B->tev[k]);
    B->side.assign(B->groups.size(), nullptr);
    B->join.assign(B->groups.size(), nullptr);
    // branch priorities: the group with the longest level-3 chain highest, so its
    // kernels (the batch's critical path) get SM slots first
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    std::vector<int> rank(B->groups.size());
    for (size_t k = 0; k < B->groups.size(); ++k) {
        int r = 0;
        for (size_t j = 0; j < B->groups.size(); ++j)
            if (B->groups[j].chain > B->groups[k].chain || (B->groups[j].chain == B->groups[k].chain && j < k)) ++r;
        rank[k] = r;
    }
    for (size_t k = 0; k < B->groups.size() && e == cudaSuccess; ++k) {
        const int prio = std::min(least, greatest + rank[k]);  // greatest is the numerically smallest
        e = cudaStreamCreateWithPriority(&B->side[k], cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return fail(FFP_ERR_CUDA);
    *out = B;
    return FFP_OK;
}

void ffp_batch_destroy(ffp_batch *B) {
    if (!B) return;
    drop_graphs(B);
    for (cudaStream_t s : B->side)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t ev : B->join)
        if (ev) cudaEventDestroy(ev);
    if (B->fork) cudaEventDestroy(B->fork);
    for (int k = 0; k < 2; ++k)
        if (B->tev[k]) cudaEventDestroy(B->tev[k]);
    if (B->gs) cudaStreamDestroy(B->gs);
    if (B->hctl) cudaFreeHost(B->hctl);
    if (B->hscal) cudaFreeHost(B->hscal);
    delete B;
}

int ffp_batch_info(const ffp_batch *B, int *ngroups, int *npairs, long long *launches_per_iter,
                   long long *setup_launches) {
    if (!B) return FFP_ERR_ARG;
    if (setup_launches) *setup_launches = B->setup_launches;
    if (ngroups) *ngroups = (int)B->groups.size();
    if (npairs) *npairs = B->npairs;
    if (launches_per_iter)
        *launches_per_iter = kernel_count_of(B->groups, B->precond == FFP_PRECOND_COMBO, B->prec != FFP_FP64);
    return FFP_OK;
}

int ffp_batch_get_config(const ffp_batch *B, ffp_batch_config *cfg) {
    if (!B || !cfg) return FFP_ERR_ARG;
    *cfg = B->cfg;
    return FFP_OK;
}

int ffp_batch_set_config(ffp_batch *B, const ffp_batch_config *cfg) {
    if (!B || !cfg) return FFP_ERR_ARG;
    if (cfg->ilu_warps < 1 || cfg->ilu_warps > 8 || (cfg->branches != 0 && cfg->branches != 1) ||
        (cfg->rhs_per_cta != 1 && cfg->rhs_per_cta != 2))
        return FFP_ERR_ARG;
    if (cfg->ilu_warps != B->cfg.ilu_warps || cfg->branches != B->cfg.branches ||
        cfg->rhs_per_cta != B->cfg.rhs_per_cta)
        drop_graphs(B);
    B->cfg = *cfg;
    return FFP_OK;
}

int ffp_batch_tune(ffp_batch *B, const char *cache_path, ffp_batch_config *out, void *stream) {
    if (!B) return FFP_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFP_ERR_CUDA;
    if (dev != B->device) return FFP_ERR_ARG;
    const std::string key = batch_key(B);
    ffp_batch_config best = B->cfg;
    if (cache_path && cache_lookup(cache_path, key, &best)) {
        best.from_cache = 1;
        const int s = ffp_batch_set_config(B, &best);
        if (out) *out = B->cfg;
        return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return FFP_ERR_CUDA;
    cudaError_t e = cudaEventRecord(ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->gs, ev, 0);
    // every pair takes part; the preconditioner reads r, set to zero here
    for (int k = 0; k < B->npairs; ++k) B->hctl[k] = CTL_ITER;
    for (int k = 0; k < B->npairs && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(B->pairs[k].r, 0, 8 * (size_t)B->pairs[k].n, B->gs);
        if (e == cudaSuccess && B->pairs[k].r32)
            e = cudaMemsetAsync(B->pairs[k].r32, 0, 4 * (size_t)B->pairs[k].n, B->gs);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->dctl, B->hctl, 4 * (size_t)B->npairs, cudaMemcpyHostToDevice, B->gs);
    const bool combo = B->precond == FFP_PRECOND_COMBO;
    bool any_two = false;
    for (const Group &g : B->groups) any_two = any_two || g.nq > 0;
    std::vector<ffp_batch_config> cand;
    for (int nr = 1; nr <= (any_two ? 2 : 1); ++nr)
        for (int br = 0; br <= 1; ++br)
            for (int w : {1, 2, 4, 8}) {
                if (!combo && w != 4) continue;
                ffp_batch_config c;
                c.ilu_warps = w; c.branches = br; c.ms = 0.0; c.ntd_ms = 0.0; c.from_cache = 0;
                c.rhs_per_cta = nr;
                cand.push_back(c);
            }
    // mean time of 3 replays (after one warm-up replay) of the graph of fn over all groups
    auto time_graph = [&](auto fn, double *ms_out) -> cudaError_t {
        cudaGraphExec_t g = nullptr;
        cudaError_t x = capture(B->gs, &g, [&]() { return all_groups(B, fn); });
        if (x != cudaSuccess) return x;
        double sum = 0.0;
        for (int rep = 0; rep < 4 && x == cudaSuccess; ++rep) {
            x = cudaEventRecord(B->tev[0], B->gs);
            if (x == cudaSuccess) x = cudaGraphLaunch(g, B->gs);
            if (x == cudaSuccess) x = cudaEventRecord(B->tev[1], B->gs);
            if (x == cudaSuccess) x = cudaEventSynchronize(B->tev[1]);
            float ms = 0.f;
            if (x == cudaSuccess) x = cudaEventElapsedTime(&ms, B->tev[0], B->tev[1]);
            if (rep > 0) sum += ms;
        }
        cudaGraphExecDestroy(g);
        *ms_out = sum / 3.0;
        return x;
    };
    auto precond_fn = [&](const Group &gr, cudaStream_t s) { return group_precond(B, gr, s); };
    auto ntd_fn = [&](const Group &gr, cudaStream_t s) {
        return (B->cfg.rhs_per_cta == 2 && gr.nq > 0)
                   ? launch_apply_table(B->prec, gr.S, B->dapply2 + gr.q0, gr.nq, gr.nx_max, 2, s)
                   : launch_apply_table(B->prec, gr.S, B->dapply + gr.p0, gr.np, gr.nx_max, 1, s);
    };
    double best_ms = 1e300;
    const ffp_batch_config keep = B->cfg;
    for (size_t q = 0; q < cand.size() && e == cudaSuccess; ++q) {
        B->cfg.ilu_warps = cand[q].ilu_warps;
        B->cfg.branches = cand[q].branches;
        B->cfg.rhs_per_cta = cand[q].rhs_per_cta;
        e = time_graph(precond_fn, &cand[q].ms);
        if (e == cudaSuccess && cand[q].ms < best_ms) {
            best_ms = cand[q].ms;
            best = cand[q];
        }
    }
    if (e == cudaSuccess) {
        B->cfg.ilu_warps = best.ilu_warps;
        B->cfg.branches = best.branches;
        B->cfg.rhs_per_cta = best.rhs_per_cta;
        e = time_graph(ntd_fn, &best.ntd_ms);
    }
    B->cfg = keep;
    int status = cuda_status(e);
    if (status == FFP_OK) {
        status = ffp_batch_set_config(B, &best);
        if (status == FFP_OK && cache_path) cache_store(cache_path, key, best);
    }
    if (cudaEventRecord(ev, B->gs) == cudaSuccess) cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
    if (out) *out = B->cfg;
    return status;
}

int ffp_batch_solve(ffp_batch *B, const double *const *b, double *const *x, double rtol, int maxit,
                    ffp_stats *stats, void *stream) {
    if (!B || !b || !x || !(rtol > 0.0) || maxit < 0) return FFP_ERR_ARG;
    const int np = B->npairs;
    for (int p = 0; p < np; ++p)
        if (!b[p] || !x[p]) return FFP_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFP_ERR_CUDA;
    if (dev != B->device) return FFP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t gs = B->gs;
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return FFP_ERR_CUDA;
    cudaError_t e = cudaEventRecord(ev, st);  // the caller's work on b and x comes first
    if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, ev, 0);
    for (int k = 0; k < np; ++k) {
        B->pairs[k].b = b[B->order[k]];
        B->pairs[k].x = x[B->order[k]];
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->dpairs, B->pairs.data(), sizeof(PairArgs) * np, cudaMemcpyHostToDevice, gs);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->dscal, 0, kPairScal * np, gs);
    // the host pair table is read by the copy above before it can change again
    if (e == cudaSuccess) e = cudaStreamSynchronize(gs);
    if (e == cudaSuccess && !B->g_iter) e = build_graphs(B);
    int status = cuda_status(e);
    long long launches = 0;
    std::vector<double> bb(np, 0.0), rr(np, 0.0);
    std::vector<int> it(np, 0), fresh(np, 1), done(np, 0), st_p(np, FFP_OK), it_rec(np, -1);
    std::vector<int> stalls(np, 0);           // as in the single-instance driver
    std::vector<double> best_true(np, -1.0);
    auto run = [&](cudaGraphExec_t g, long long nk) {
        launches += nk;
        return cudaGraphLaunch(g, gs) == cudaSuccess && cudaStreamSynchronize(gs) == cudaSuccess;
    };
    if (status == FFP_OK) {
        for (int k = 0; k < np; ++k) B->hctl[k] = CTL_RESID;
        if (!run(B->g_resid, B->resid_launches)) status = FFP_ERR_CUDA;
    }
    if (status == FFP_OK) {
        for (int k = 0; k < np; ++k) {
            bb[k] = pscal(B, k)[SC_BB];
            rr[k] = pscal(B, k)[SC_RR];
            if (bb[k] == 0.0) {
                if (cudaMemsetAsync(B->pairs[k].x, 0, 8 * (size_t)B->pairs[k].n, gs) != cudaSuccess)
                    status = FFP_ERR_CUDA;
                done[k] = 1;
            }
        }
    }
    while (status == FFP_OK) {
        // converged on the recursive residual: confirm with the true one, else restart from it
        bool check = false;
        for (int k = 0; k < np; ++k) {
            B->hctl[k] = 0;
            if (!done[k] && std::sqrt(rr[k] / bb[k]) < rtol) {
                if (it_rec[k] < 0) it_rec[k] = it[k];
                B->hctl[k] = CTL_RESID;
                check = true;
            }
        }
        if (check) {
            if (!run(B->g_resid, B->resid_launches)) { status = FFP_ERR_CUDA; break; }
            for (int k = 0; k < np; ++k)
                if (B->hctl[k] & CTL_RESID) {
                    rr[k] = pscal(B, k)[SC_RR];
                    if (std::sqrt(rr[k] / bb[k]) < rtol) {
                        done[k] = 1;
                        continue;
                    }
                    stalls[k] = (best_true[k] >= 0.0 && rr[k] > 0.25 * best_true[k]) ? stalls[k] + 1 : 0;
                    if (best_true[k] < 0.0 || rr[k] < best_true[k]) best_true[k] = rr[k];
                    if (stalls[k] >= kStallConfirms) {
                        st_p[k] = FFP_ERR_NOT_CONVERGED;
                        done[k] = 1;
                    } else {
                        fresh[k] = 1;
                    }
                }
        }
        bool any = false;
        for (int k = 0; k < np; ++k) {
            B->hctl[k] = 0;
            if (done[k]) continue;
            if (it[k] >= maxit) {
                st_p[k] = FFP_ERR_NOT_CONVERGED;
                done[k] = 1;
                continue;
            }
            B->hctl[k] = CTL_ITER | (fresh[k] ? CTL_FRESH : 0);
            any = true;
        }
        if (!any) break;
        if (!run(B->g_iter, B->iter_launches)) { status = FFP_ERR_CUDA; break; }
        for (int k = 0; k < np; ++k) {
            if (!(B->hctl[k] & CTL_ITER)) continue;
            fresh[k] = 0;
            ++it[k];
            rr[k] = pscal(B, k)[SC_RR];
            if (pflags(B, k)[FL_TIMEOUT]) { st_p[k] = FFP_ERR_TIMEOUT; done[k] = 1; }
            else if (pflags(B, k)[FL_PQ] || !std::isfinite(rr[k])) { st_p[k] = FFP_ERR_BREAKDOWN; done[k] = 1; }
        }
    }
    // true residuals of the final iterates
    if (status == FFP_OK) {
        for (int k = 0; k < np; ++k) B->hctl[k] = (bb[k] > 0.0) ? CTL_RESID : 0;
        if (!run(B->g_resid, B->resid_launches)) status = FFP_ERR_CUDA;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int worst = status;
    for (int k = 0; k < np; ++k) {
        if (worst == FFP_OK && st_p[k] != FFP_OK) worst = st_p[k];
        if (!stats) continue;
        ffp_stats &s = stats[B->order[k]];
        std::memset(&s, 0, sizeof(s));
        s.iters = it[k];
        s.status = (status != FFP_OK) ? status : st_p[k];
        s.rel_res = (bb[k] > 0.0) ? std::sqrt(rr[k] / bb[k]) : 0.0;
        s.rel_res_true = (status != FFP_OK) ? -1.0
                                            : (bb[k] > 0.0 ? std::sqrt(pscal(B, k)[SC_TRR] / bb[k]) : 0.0);
        s.solve_s = secs;
        s.napply = it[k];
        s.launches = launches;
        s.iters_rec = (bb[k] == 0.0) ? 0 : it_rec[k];
    }
    if (cudaEventRecord(ev, gs) == cudaSuccess) cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
    return worst;
}

}  // extern "C"
