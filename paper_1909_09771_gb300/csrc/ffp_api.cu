// ffp_api.cu -- the C ABI declared in include/ffp.h.
//
// The caller owns every device buffer, including the workspace, which this
// file carves into the operator bands, the stored factors, the CG vectors and
// small scratch; the handle is a host struct that only points into it.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ffp_kernels.h"

using namespace ffp;

struct ffp_handle {
    KernelCtx c;
    int device;
    double *host_scal;  // pinned copy of the scalar block + flags
    cudaEvent_t ev[6];  // preconditioner timing: start, B_NTD sweeps start and end, end;
                        // then the start and end of the SpMV + (p, Ap) launch
};

const KernelCtx *ffp::handle_ctx(const ffp_handle *h) { return h ? &h->c : nullptr; }
int ffp::handle_device(const ffp_handle *h) { return h ? h->device : -1; }

size_t ffp::prec_bytes(int prec) {
    switch (prec) {
        case FFP_FP64: return 8;
        case FFP_FP32: return 4;
        case FFP_BF16: return 2;
        default: return 0;
    }
}

namespace {
size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

bool grid_ok(const ffp_grid *g) {
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1 || g->nx > FFP_MAX_NX) return false;
    const long long n = (long long)g->nx * g->ny * g->nz;
    return n <= 2000000000LL;
}

}  // namespace

// Carve the workspace (base may be 0 to compute the size) for line slot count
// S (0: the one the grid needs).  Returns the total size.
size_t ffp::carve_workspace(const ffp_grid *g, int prec, int S_force, char *base, Ws *ws) {
    const size_t n = (size_t)g->nx * g->ny * g->nz;
    const size_t nxy = (size_t)g->nx * g->ny;
    const size_t fb = prec_bytes(prec);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += align_up(bytes);
        return p;
    };
    Ws w;
    std::memset(&w, 0, sizeof(w));
    w.d = (double *)take(8 * n); w.cx = (double *)take(8 * n);
    w.cy = (double *)take(8 * n); w.cz = (double *)take(8 * n);
    const int S = S_force > 0 ? S_force : slots_for(g->nx);
    const size_t nlines = (size_t)g->ny * g->nz;
    w.rec = take(fb * nlines * (size_t)rec_len(S > 0 ? S : 1));
    w.l3 = take(fb * n);
    w.l1 = take(fb * n);
    w.dinv = take(fb * n); w.lx = take(fb * n); w.ly = take(fb * n);
    w.r = (double *)take(8 * n); w.z = (double *)take(8 * n);
    w.p = (double *)take(8 * n); w.q = (double *)take(8 * n);
    w.c1 = (double *)take(8 * n); w.c2 = (double *)take(8 * n);
    {
        // the apply's vectors in the line-block layout, in its arithmetic type
        const size_t ab = (prec == FFP_FP64) ? 8 : 4;
        const size_t lb = (size_t)lb_len(S > 0 ? S : 1);
        w.ra = take(ab * nlines * lb);
        w.za = take(ab * nlines * lb);
        w.ascr = take(ab * 2 * (size_t)g->ny * lb);
    }
    for (int h = 0; h < 2; ++h) {
        for (int pp = 0; pp < 2; ++pp)
            for (int b = 0; b < 3; ++b) w.sP[h][pp][b] = (double *)take(8 * nxy);
        for (int b = 0; b < 2; ++b) w.sF[h][b] = (double *)take(8 * nxy);
        for (int b = 0; b < 2; ++b) w.sW[h][b] = (double *)take(8 * nxy);
        for (int b = 0; b < 3; ++b) w.sC[h][b] = (double *)take(8 * nxy);
    }
    w.ilu_ready = (int *)take(4 * (size_t)g->ny * g->nz);
    w.ilu_sync = (int *)take(4 * 32);
    w.ilu_v = (prec != FFP_FP64) ? take(4 * n) : nullptr;
    w.ilu_tw = (prec != FFP_FP64) ? (unsigned long long *)take(8 * n) : nullptr;
    w.red = (double *)take(8 * (size_t)kRedSlots);
    // scalar block and flags are contiguous so one copy brings both back
    w.scal = (double *)take(8 * (size_t)kScal + 4 * 16);
    w.flags = base ? (int *)(w.scal + kScal) : nullptr;
    if (ws) *ws = w;
    return off;
}

namespace {
size_t carve(const ffp_grid *g, int prec, char *base, Ws *ws) { return carve_workspace(g, prec, 0, base, ws); }

constexpr size_t kScalBytes = 8 * (size_t)kScal + 4 * 16;

int cuda_status(cudaError_t e) { return e == cudaSuccess ? FFP_OK : FFP_ERR_CUDA; }

// kernels launched by one B_NTD apply (conversions to and from the line-block
// layout around the sweeps) / one ILU(0) solve
long long ntd_launches(const KernelCtx &c) {
    const int mz = (c.nz - 1) / 2;
    return ((mz > 0 || c.nz - 1 - mz > 0) ? 3 : 1) + 2;
}
long long ilu_launches(const KernelCtx &c) { return ilu_solve_launches(c); }

// Extreme eigenvalues of the Lanczos tridiagonal that k CG steps define (the
// Lanczos-CG relation: with p_j = z_j + b_j p_{j-1}, b_0 = 0, the tridiagonal of
// B^{-1}A in the basis of the preconditioned residuals has diagonal
// 1/a_j + b_j/a_{j-1} and off-diagonal sqrt(b_j)/a_{j-1}).  Bisection on the
// Sturm count (the number of negative pivots of T - s I), from the Gershgorin
// interval, to the last bit.
void lanczos_extremes(const std::vector<double> &a, const std::vector<double> &b, double *lmin,
                      double *lmax) {
    const size_t k = a.size();
    *lmin = *lmax = 0.0;
    if (k == 0) return;
    std::vector<double> d(k), e2(k, 0.0);
    double lo = 0.0, hi = 0.0;
    for (size_t j = 0; j < k; ++j) {
        if (!(a[j] > 0.0) || !(j == 0 || b[j] >= 0.0)) return;  // not a Lanczos sequence
        d[j] = 1.0 / a[j] + (j > 0 ? b[j] / a[j - 1] : 0.0);
        if (j > 0) e2[j] = b[j] / (a[j - 1] * a[j - 1]);
    }
    for (size_t j = 0; j < k; ++j) {
        const double r = (j > 0 ? std::sqrt(e2[j]) : 0.0) + (j + 1 < k ? std::sqrt(e2[j + 1]) : 0.0);
        if (j == 0 || d[j] - r < lo) lo = d[j] - r;
        if (j == 0 || d[j] + r > hi) hi = d[j] + r;
    }
    auto below = [&](double s) {  // eigenvalues < s
        int cnt = 0;
        double q = 1.0;
        for (size_t j = 0; j < k; ++j) {
            q = d[j] - s - (j > 0 ? e2[j] / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++cnt;
        }
        return cnt;
    };
    auto kth = [&](int want) {  // the eigenvalue with `want` eigenvalues below it
        double l = lo, h = hi;
        for (int it = 0; it < 200 && h - l > 0.0; ++it) {
            const double m = 0.5 * (l + h);
            if (m <= l || m >= h) break;
            if (below(m) > want) h = m; else l = m;
        }
        return 0.5 * (l + h);
    };
    *lmin = kth(0);
    *lmax = kth((int)k - 1);
}

// z = B^{-1} r for the handle's preconditioner (r and z distinct from c1, c2).
// ev (optional): events recorded at the start, just before and just after the
// three B_NTD sweep launches, and at the end.
cudaError_t precond_apply(const KernelCtx &c, const double *r, double *z, cudaStream_t st,
                          long long *launches, cudaEvent_t *ev = nullptr) {
    cudaError_t e = cudaSuccess;
    if (ev) e = cudaEventRecord(ev[0], st);
    if (c.precond != FFP_PRECOND_COMBO) {
        if (e == cudaSuccess) e = launch_apply(c, r, z, st, ev ? ev + 1 : nullptr);
        *launches += ntd_launches(c);
    } else {
        // B_c^{-1} r = y + B_NTD^{-1} (r - A y), y = B_ILU0^{-1} r
        if (e == cudaSuccess) e = launch_ilu_solve(c, r, c.ws.c1, st);
        if (e == cudaSuccess) e = launch_resid_vec(c, r, c.ws.c1, c.ws.c2, st);
        if (e == cudaSuccess) e = launch_apply(c, c.ws.c2, z, st, ev ? ev + 1 : nullptr, c.ws.c1);
        *launches += ilu_launches(c) + 1 + ntd_launches(c);
    }
    if (ev && e == cudaSuccess) e = cudaEventRecord(ev[3], st);
    return e;
}

int read_scalars(ffp_handle *h, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(h->host_scal, h->c.ws.scal, kScalBytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return FFP_ERR_CUDA;
    e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

const int *host_flags(const ffp_handle *h) { return (const int *)(h->host_scal + kScal); }

}  // namespace

extern "C" {

size_t ffp_workspace_bytes(const ffp_grid *grid, int precision) {
    if (!grid_ok(grid) || prec_bytes(precision) == 0) return 0;
    return carve(grid, precision, nullptr, nullptr);
}

int ffp_setup(const ffp_grid *grid, const double *kappa, const ffp_bc *bc, int filter,
              const double *t, int precision, int precond, void *workspace, size_t ws_bytes,
              void *stream, ffp_handle **out) {
    if (out) *out = nullptr;
    if (!grid_ok(grid) || !kappa || !bc || !workspace || !out) return FFP_ERR_ARG;
    if (prec_bytes(precision) == 0) return FFP_ERR_ARG;
    if (filter != FFP_FILTER_ROWSUM && filter != FFP_FILTER_USER) return FFP_ERR_ARG;
    const int schur = (precond & FFP_SCHUR_BETA) ? 1 : 0;
    precond &= ~FFP_SCHUR_BETA;
    if (precond != FFP_PRECOND_NTD && precond != FFP_PRECOND_COMBO) return FFP_ERR_ARG;
    if (filter == FFP_FILTER_USER && !t) return FFP_ERR_ARG;
    if (((uintptr_t)workspace & 255) != 0) return FFP_ERR_ARG;
    for (int f = 0; f < 6; ++f)
        if (bc->face[f] != FFP_DIRICHLET && bc->face[f] != FFP_NEUMANN) return FFP_ERR_ARG;
    const size_t need = carve(grid, precision, nullptr, nullptr);
    if (ws_bytes < need) return FFP_ERR_ARG;
    const int slots = slots_for(grid->nx);
    if (slots < 0) return FFP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;

    ffp_handle *h = new (std::nothrow) ffp_handle;
    if (!h) return FFP_ERR_ARG;
    std::memset(h, 0, sizeof(*h));
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return FFP_ERR_CUDA; }
    if (cudaMallocHost((void **)&h->host_scal, kScalBytes) != cudaSuccess) { delete h; return FFP_ERR_CUDA; }
    for (int k = 0; k < 6; ++k)
        if (cudaEventCreate(&h->ev[k]) != cudaSuccess) { ffp_destroy(h); return FFP_ERR_CUDA; }
    KernelCtx &c = h->c;
    c.nx = grid->nx; c.ny = grid->ny; c.nz = grid->nz;
    c.n = (long long)c.nx * c.ny * c.nz;
    c.lx = grid->lx > 0 ? grid->lx : 1.0;
    c.ly = grid->ly > 0 ? grid->ly : 1.0;
    c.lz = grid->lz > 0 ? grid->lz : 1.0;
    c.prec = precision;
    c.precond = precond;
    c.schur = schur;
    c.slots = slots;
    carve(grid, precision, (char *)workspace, &c.ws);

    cudaError_t e = cudaMemsetAsync(c.ws.scal, 0, kScalBytes, st);
    // ILU(0) sweep epoch 0 and untagged result words (no tag of a solve is 0)
    if (e == cudaSuccess) e = cudaMemsetAsync(c.ws.ilu_sync, 0, 4 * 32, st);
    if (e == cudaSuccess && c.ws.ilu_tw) e = cudaMemsetAsync(c.ws.ilu_tw, 0, 8 * (size_t)c.n, st);
    if (e == cudaSuccess)   // record pads must read as 0
        e = cudaMemsetAsync(c.ws.rec, 0,
                            prec_bytes(precision) * (size_t)c.ny * c.nz * (size_t)rec_len(slots), st);
    if (e == cudaSuccess) e = launch_assemble(c, kappa, bc->face, st);
    if (e == cudaSuccess && filter == FFP_FILTER_USER) e = launch_check_filter(c, t, st);
    int status = cuda_status(e);
    if (status == FFP_OK) status = read_scalars(h, st);
    if (status == FFP_OK && host_flags(h)[FL_ARG]) status = FFP_ERR_ARG;
    if (status == FFP_OK) {
        e = launch_convert_bands(c, st);
        if (e == cudaSuccess) e = launch_setup(c, filter == FFP_FILTER_USER ? t : nullptr, st);
        // ILU(0) pivots in FP64 use the CG vector p as scratch (free until a solve)
        if (e == cudaSuccess && precond == FFP_PRECOND_COMBO) e = launch_ilu_setup(c, c.ws.p, st);
        status = cuda_status(e);
    }
    if (status == FFP_OK) status = read_scalars(h, st);
    if (status == FFP_OK && host_flags(h)[FL_BREAKDOWN]) status = FFP_ERR_BREAKDOWN;
    if (status != FFP_OK) {
        ffp_destroy(h);
        return status;
    }
    *out = h;
    return FFP_OK;
}

int ffp_spmv(ffp_handle *h, const double *x, double *y, void *stream) {
    if (!h || !x || !y) return FFP_ERR_ARG;
    return cuda_status(launch_spmv(h->c, x, y, (cudaStream_t)stream));
}

int ffp_apply(ffp_handle *h, const double *r, double *z, void *stream) {
    if (!h || !r || !z || r == z) return FFP_ERR_ARG;
    long long n = 0;
    return cuda_status(precond_apply(h->c, r, z, (cudaStream_t)stream, &n));
}

int ffp_export(ffp_handle *h, double *d, double *cx, double *cy, double *cz, double *l3,
               double *l2, double *l1, double *minv, double *dinv, void *stream) {
    if (!h) return FFP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = 8 * (size_t)h->c.n;
    cudaError_t e = cudaSuccess;
    if (d && e == cudaSuccess) e = cudaMemcpyAsync(d, h->c.ws.d, nb, cudaMemcpyDeviceToDevice, st);
    if (cx && e == cudaSuccess) e = cudaMemcpyAsync(cx, h->c.ws.cx, nb, cudaMemcpyDeviceToDevice, st);
    if (cy && e == cudaSuccess) e = cudaMemcpyAsync(cy, h->c.ws.cy, nb, cudaMemcpyDeviceToDevice, st);
    if (cz && e == cudaSuccess) e = cudaMemcpyAsync(cz, h->c.ws.cz, nb, cudaMemcpyDeviceToDevice, st);
    if (l3 && e == cudaSuccess) e = launch_export_rec(h->c, 3, l3, st);
    if (l2 && e == cudaSuccess) e = launch_export_rec(h->c, 2, l2, st);
    if (l1 && e == cudaSuccess) e = launch_export_rec(h->c, 0, l1, st);
    if (minv && e == cudaSuccess) e = launch_export_rec(h->c, 1, minv, st);
    if (dinv && e == cudaSuccess && h->c.precond == FFP_PRECOND_COMBO)
        e = launch_export(h->c, h->c.ws.dinv, dinv, st);
    return cuda_status(e);
}

int ffp_pcg_solve(ffp_handle *h, const double *b, double *x, double rtol, int maxit,
                  ffp_stats *stats, void *stream) {
    if (!h || !b || !x || !(rtol > 0.0) || maxit < 0) return FFP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const KernelCtx &c = h->c;
    const int flexible = (c.prec != FFP_FP64) || (c.precond == FFP_PRECOND_COMBO);
    auto t0 = std::chrono::steady_clock::now();
    int it = 0, fresh = 1, status = FFP_OK, it_rec = -1;
    // true residuals at confirmations: the best so far and the confirmations in a row
    // that did not halve it (the true residual has reached its FP64 floor)
    double best_true = -1.0;
    int stalls = 0;
    double bb = 0.0, rr = 0.0;
    double pre_ms = 0.0, ntd_ms = 0.0, spmv_ms = 0.0;
    long long nl = 0;
    // CG coefficients since the start, up to the first restart (Lanczos estimate)
    std::vector<double> lz_a, lz_b;
    bool lz_open = true;
#define FFP_TRY(expr)                                                 \
    do {                                                              \
        cudaError_t _e = (expr);                                      \
        if (_e != cudaSuccess) { status = FFP_ERR_CUDA; goto done; } \
    } while (0)
    FFP_TRY(cudaMemsetAsync(c.ws.flags, 0, 4 * 16, st));
    FFP_TRY(launch_resid(c, b, x, st));
    FFP_TRY(launch_finalize(c, FIN_RESID, 0, flexible, st));
    nl += 2;
    if ((status = read_scalars(h, st)) != FFP_OK) goto done;
    bb = h->host_scal[SC_BB];
    rr = h->host_scal[SC_RR];
    if (bb == 0.0) {
        FFP_TRY(cudaMemsetAsync(x, 0, 8 * (size_t)c.n, st));
        if (stats) {
            std::memset(stats, 0, sizeof(*stats));
            stats->launches = nl;
        }
        cudaStreamSynchronize(st);
        return FFP_OK;
    }
    for (;;) {
        if (std::sqrt(rr / bb) < rtol) {
            if (it_rec < 0) it_rec = it;
            // confirm with the true residual; continue from it if it is not converged
            FFP_TRY(launch_resid(c, b, x, st));
            FFP_TRY(launch_finalize(c, FIN_RESID, 0, flexible, st));
            nl += 2;
            if ((status = read_scalars(h, st)) != FFP_OK) goto done;
            rr = h->host_scal[SC_RR];
            if (std::sqrt(rr / bb) < rtol) break;
            stalls = (best_true >= 0.0 && rr > 0.25 * best_true) ? stalls + 1 : 0;
            if (best_true < 0.0 || rr < best_true) best_true = rr;
            if (stalls >= kStallConfirms) { status = FFP_ERR_NOT_CONVERGED; break; }
            fresh = 1;
            lz_open = false;
        }
        if (it >= maxit) { status = FFP_ERR_NOT_CONVERGED; break; }
        FFP_TRY(precond_apply(c, c.ws.r, c.ws.z, st, &nl, h->ev));
        FFP_TRY(launch_dot_rz(c, st));
        FFP_TRY(launch_finalize(c, FIN_RZ, fresh, flexible, st));
        FFP_TRY(launch_update_p(c, fresh, st));
        fresh = 0;
        FFP_TRY(cudaEventRecord(h->ev[4], st));
        FFP_TRY(launch_spmv_dot(c, st));
        FFP_TRY(cudaEventRecord(h->ev[5], st));
        FFP_TRY(launch_finalize(c, FIN_PQ, 0, flexible, st));
        FFP_TRY(launch_update_xr(c, x, st));
        FFP_TRY(launch_finalize(c, FIN_RR, 0, flexible, st));
        nl += 8;
        ++it;
        if ((status = read_scalars(h, st)) != FFP_OK) goto done;
        if (lz_open) {
            lz_a.push_back(h->host_scal[SC_ALPHA]);
            lz_b.push_back(lz_a.size() == 1 ? 0.0 : h->host_scal[SC_BETA]);
        }
        {
            float a = 0.f, b2 = 0.f;
            if (cudaEventElapsedTime(&a, h->ev[0], h->ev[3]) == cudaSuccess) pre_ms += a;
            if (cudaEventElapsedTime(&b2, h->ev[1], h->ev[2]) == cudaSuccess) ntd_ms += b2;
            float c2 = 0.f;
            if (cudaEventElapsedTime(&c2, h->ev[4], h->ev[5]) == cudaSuccess) spmv_ms += c2;
        }
        if (host_flags(h)[FL_TIMEOUT]) { status = FFP_ERR_TIMEOUT; break; }
        if (host_flags(h)[FL_PQ]) { status = FFP_ERR_BREAKDOWN; break; }
        rr = h->host_scal[SC_RR];
        if (!std::isfinite(rr)) { status = FFP_ERR_BREAKDOWN; break; }
    }
done:
#undef FFP_TRY
    if (stats) {
        stats->iters = it;
        stats->status = status;
        stats->precond_ms = pre_ms;
        stats->ntd_ms = ntd_ms;
        stats->spmv_ms = spmv_ms;
        stats->napply = it;
        stats->rel_res = (bb > 0.0) ? std::sqrt(rr / bb) : 0.0;
        stats->rel_res_true = -1.0;
        if (status != FFP_ERR_CUDA) {
            if (launch_resid(c, b, x, st) == cudaSuccess &&
                launch_finalize(c, FIN_RESID, 0, flexible, st) == cudaSuccess &&
                read_scalars(h, st) == FFP_OK)
                stats->rel_res_true = std::sqrt(h->host_scal[SC_TRR] / bb);
            nl += 2;
        }
        stats->launches = nl;
        stats->iters_rec = it_rec;
        lanczos_extremes(lz_a, lz_b, &stats->lanczos_min, &stats->lanczos_max);
        stats->solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

int ffp_debug_stall(ffp_handle *h, int mode, unsigned wait_tries) {
    if (!h || mode < 0 || mode > 1) return FFP_ERR_ARG;
    h->c.dbg_stall = mode;
    h->c.dbg_tries = wait_tries;
    return FFP_OK;
}

void ffp_destroy(ffp_handle *h) {
    if (!h) return;
    for (int k = 0; k < 6; ++k)
        if (h->ev[k]) cudaEventDestroy(h->ev[k]);
    if (h->host_scal) cudaFreeHost(h->host_scal);
    delete h;
}

const char *ffp_strerror(int status) {
    switch (status) {
        case FFP_OK: return "ok";
        case FFP_ERR_ARG: return "invalid argument";
        case FFP_ERR_CUDA: return "CUDA runtime error";
        case FFP_ERR_BREAKDOWN: return "breakdown: non-positive pivot or (p, Ap) <= 0";
        case FFP_ERR_NOT_CONVERGED: return "not converged within maxit";
        case FFP_ERR_TIMEOUT: return "a bounded wait in a kernel timed out";
        case FFP_ERR_UNSUPPORTED: return "unsupported option";
        default: return "unknown status";
    }
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free apply
// Scratch for ffp_apply_noalloc: the two upper-sweep planes of the B_NTD apply.
// In host code `g_noalloc_scratch` is only a host-side stand-in for the symbol;
// its device address is looked up once per device and cached.
static __device__ __align__(256) double g_noalloc_scratch[2 * FFP_NOALLOC_MAX_PLANE];

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on first use).
int noalloc_scratch(int device, double **out) {
    if (device < 0 || device >= kMaxDevices) return FFP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FFP_ERR_CUDA;
        g_noalloc_ptr[device] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[device];
    return FFP_OK;
}
}  // namespace

extern "C" int ffp_apply_noalloc(ffp_handle *h, const double *r, double *z, void *stream) {
    if (!h || !r || !z || r == z) return FFP_ERR_ARG;
    // one scratch plane (line-block layout, the apply's arithmetic type) must fit
    // FFP_NOALLOC_MAX_PLANE FP64 values
    const long long plane_bytes = (long long)h->c.ny * lb_len(h->c.slots) *
                                  (h->c.prec == FFP_FP64 ? 8 : 4);
    if ((long long)h->c.nx * h->c.ny > FFP_NOALLOC_MAX_PLANE ||
        plane_bytes > 8LL * FFP_NOALLOC_MAX_PLANE)
        return FFP_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFP_ERR_CUDA;
    if (dev != h->device) return FFP_ERR_ARG;
    double *scr = nullptr;
    const int st = noalloc_scratch(dev, &scr);
    if (st != FFP_OK) return st;
    KernelCtx c = h->c;
    c.ws.ascr = static_cast<void *>(scr);
    return cuda_status(launch_apply(c, r, z, (cudaStream_t)stream));
}
