// ffp_ops.cu -- operator assembly, SpMV and the FP64 CG vector kernels.
//
// Assembly (Sec. I Eq. (2), finite-volume reading): face coefficient
// kappa_f * area / distance with kappa_f = 2 ka kb / (ka + kb); a Dirichlet
// face at half a cell contributes 2 kappa * area / h to the diagonal; faces
// are summed in the order x-, x+, y-, y+, z-, z+.
// SpMV (Sec. II band storage): y_a = d_a x_a + sum of the six couplings.
// Reductions are deterministic: a fixed grid, a fixed per-block tree and a
// fixed-order final sum in finalize_kernel.
#include "ffp_vecops.cuh"

namespace ffp {

__device__ __forceinline__ double harmonic(double ka, double kb) { return 2.0 * ka * kb / (ka + kb); }

__global__ void __launch_bounds__(kThreads) assemble_kernel(Geo g, double ax, double ay, double az,
                                                           const double *__restrict__ kappa,
                                                           uchar4 bc03, uchar2 bc45, double *d,
                                                           double *cx, double *cy, double *cz,
                                                           int *flags) {
    const unsigned char bc[6] = {bc03.x, bc03.y, bc03.z, bc03.w, bc45.x, bc45.y};
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.n;
         a += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(a % g.nx);
        const int y = (int)((a / g.nx) % g.ny);
        const int z = (int)(a / g.nxy);
        const double ka = kappa[a];
        if (!(ka > 0.0) || !isfinite(ka)) atomicOr(flags + FL_ARG, 1);
        double diag = 0.0;
        if (x > 0) diag += harmonic(ka, kappa[a - 1]) * ax;
        else if (bc[0] == FFP_DIRICHLET) diag += 2.0 * ka * ax;
        if (x + 1 < g.nx) { const double c = harmonic(ka, kappa[a + 1]) * ax; cx[a] = -c; diag += c; }
        else { cx[a] = 0.0; if (bc[1] == FFP_DIRICHLET) diag += 2.0 * ka * ax; }
        if (y > 0) diag += harmonic(ka, kappa[a - g.nx]) * ay;
        else if (bc[2] == FFP_DIRICHLET) diag += 2.0 * ka * ay;
        if (y + 1 < g.ny) { const double c = harmonic(ka, kappa[a + g.nx]) * ay; cy[a] = -c; diag += c; }
        else { cy[a] = 0.0; if (bc[3] == FFP_DIRICHLET) diag += 2.0 * ka * ay; }
        if (z > 0) diag += harmonic(ka, kappa[a - g.nxy]) * az;
        else if (bc[4] == FFP_DIRICHLET) diag += 2.0 * ka * az;
        if (z + 1 < g.nz) { const double c = harmonic(ka, kappa[a + g.nxy]) * az; cz[a] = -c; diag += c; }
        else { cz[a] = 0.0; if (bc[5] == FFP_DIRICHLET) diag += 2.0 * ka * az; }
        d[a] = diag;
    }
}

__global__ void check_filter_kernel(long long n, const double *__restrict__ t, int *flags) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const double v = t[a];
        if (!(v > 0.0) || !isfinite(v)) atomicOr(flags + FL_ARG, 1);
    }
}

template <typename F>
__global__ void convert_kernel(long long n, const double *__restrict__ s, F *o) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        o[a] = from_d<F>(s[a]);
}

template <typename F>
__global__ void export_kernel(long long n, const F *__restrict__ s, double *o) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        o[a] = (double)to_r(s[a], typename Compute<F>::type());
}

// l3 (z-band) into the factor line records
template <typename F>
__global__ void l3_records_kernel(Geo g, int S, const double *__restrict__ cz, F *rec) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.n;
         a += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(a % g.nx);
        const long long line = a / g.nx;
        rec[line * rec_len(S) + rec_cell(g.nx, S, REC_L3, MID_L3, x)] = from_d<F>(cz[a]);
    }
}

// natural-order 1/M, l2 or l3 from the records (what: 1..3)
template <typename F>
__global__ void export_rec_kernel(Geo g, int S, const F *__restrict__ rec, int what, double *o) {
    using R = typename Compute<F>::type;
    const int f = (what == 1) ? REC_MINV : ((what == 2) ? REC_L2 : REC_L3);
    const int mf = (what == 1) ? MID_MINV : ((what == 2) ? MID_L2 : MID_L3);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.n;
         a += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(a % g.nx);
        const F *rb = rec + (a / g.nx) * rec_len(S);
        o[a] = (double)to_r(rb[rec_cell(g.nx, S, f, mf, x)], R());
    }
}

__global__ void __launch_bounds__(kThreads) spmv_kernel(Geo g, const double *__restrict__ d,
                                                       const double *__restrict__ cx,
                                                       const double *__restrict__ cy,
                                                       const double *__restrict__ cz,
                                                       const double *__restrict__ x, double *y) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.n;
         a += (long long)gridDim.x * blockDim.x)
        y[a] = stencil(g, a, d, cx, cy, cz, x);
}

// w = r - A y
__global__ void __launch_bounds__(kThreads) resid_vec_kernel(Geo g, const double *__restrict__ d,
                                                            const double *__restrict__ cx,
                                                            const double *__restrict__ cy,
                                                            const double *__restrict__ cz,
                                                            const double *__restrict__ r,
                                                            const double *__restrict__ y,
                                                            double *w) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.n;
         a += (long long)gridDim.x * blockDim.x)
        w[a] = r[a] - stencil(g, a, d, cx, cy, cz, y);
}

__global__ void __launch_bounds__(kThreads) add_kernel(long long n, double *z,
                                                      const double *__restrict__ y) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        z[a] += y[a];
}

// natural FP64 -> line-block layout of type R (one thread per block position;
// padding positions are written as 0)
template <typename R>
__global__ void __launch_bounds__(kThreads) to_lb_kernel(long long nlines, int nx, int S,
                                                        const double *__restrict__ x, R *y) {
    const long long L = lb_len(S);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nlines * L;
         e += (long long)gridDim.x * blockDim.x) {
        const long long line = e / L;
        const int a = lb_cell(nx, S, (int)(e - line * L));
        y[e] = (a >= 0) ? (R)x[line * nx + a] : R(0);
    }
}

// line-block layout of type R -> natural FP64 (+ add)
template <typename R>
__global__ void __launch_bounds__(kThreads) from_lb_kernel(long long n, int nx, int S,
                                                          const R *__restrict__ xb, double *y,
                                                          const double *__restrict__ add) {
    const long long L = lb_len(S);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const long long line = a / nx;
        const double v = (double)xb[line * L + lb_pos(nx, S, (int)(a - line * nx))];
        y[a] = add ? v + add[a] : v;
    }
}

// r = b - A x ; partials (r.r, b.b)
__global__ void __launch_bounds__(kThreads) resid_kernel(Geo g, const double *__restrict__ d,
                                                        const double *__restrict__ cx,
                                                        const double *__restrict__ cy,
                                                        const double *__restrict__ cz,
                                                        const double *__restrict__ b,
                                                        const double *__restrict__ x, double *r,
                                                        double *red) {
    double acc[2] = {0.0, 0.0};
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.n;
         a += (long long)gridDim.x * blockDim.x) {
        const double ba = b[a];
        const double ra = ba - stencil(g, a, d, cx, cy, cz, x);
        r[a] = ra;
        acc[0] += ra * ra;
        acc[1] += ba * ba;
    }
    block_sum<2>(acc, red);
}

// q = A p ; partial (p.q)
__global__ void __launch_bounds__(kThreads) spmv_dot_kernel(Geo g, const double *__restrict__ d,
                                                           const double *__restrict__ cx,
                                                           const double *__restrict__ cy,
                                                           const double *__restrict__ cz,
                                                           const double *__restrict__ p, double *q,
                                                           double *red) {
    double acc[1] = {0.0};
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < g.n;
         a += (long long)gridDim.x * blockDim.x) {
        const double qa = stencil(g, a, d, cx, cy, cz, p);
        q[a] = qa;
        acc[0] += p[a] * qa;
    }
    block_sum<1>(acc, red);
}

// x += alpha p ; r -= alpha q ; partial (r.r)
__global__ void __launch_bounds__(kThreads) update_xr_kernel(long long n,
                                                            const double *__restrict__ scal,
                                                            const double *__restrict__ p,
                                                            const double *__restrict__ q, double *x,
                                                            double *r, double *red) {
    const double alpha = scal[SC_ALPHA];
    double acc[1] = {0.0};
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        x[a] += alpha * p[a];
        const double ra = r[a] - alpha * q[a];
        r[a] = ra;
        acc[0] += ra * ra;
    }
    block_sum<1>(acc, red);
}

// partials (r.z, z.q)
__global__ void __launch_bounds__(kThreads) dot_rz_kernel(long long n, const double *__restrict__ r,
                                                         const double *__restrict__ z,
                                                         const double *__restrict__ q,
                                                         double *red) {
    double acc[2] = {0.0, 0.0};
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const double za = z[a];
        acc[0] += r[a] * za;
        acc[1] += za * q[a];
    }
    block_sum<2>(acc, red);
}

// p = z + beta p  (p = z when the direction is (re)started)
__global__ void __launch_bounds__(kThreads) update_p_kernel(long long n,
                                                           const double *__restrict__ scal,
                                                           const double *__restrict__ z, double *p,
                                                           int fresh) {
    const double beta = scal[SC_BETA];
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        p[a] = fresh ? z[a] : z[a] + beta * p[a];
}

// Fold the partial sums and update the CG scalars (one warp).
__global__ void finalize_kernel(int mode, int nblk, int fresh, int flexible,
                                const double *__restrict__ red, double *scal, int *flags) {
    finalize_scalars(mode, nblk, fresh, flexible, red, scal, flags);
}

// ---------------------------------------------------------------- launchers
static Geo geo(const KernelCtx &c) {
    Geo g;
    g.nx = c.nx; g.ny = c.ny; g.nz = c.nz; g.n = c.n; g.nxy = c.nx * c.ny;
    return g;
}


cudaError_t launch_assemble(const KernelCtx &c, const double *kappa, const unsigned char bc[6],
                            cudaStream_t st) {
    const double hx = c.lx / c.nx, hy = c.ly / c.ny, hz = c.lz / c.nz;
    const double ax = hy * hz / hx, ay = hx * hz / hy, az = hx * hy / hz;
    uchar4 b03 = make_uchar4(bc[0], bc[1], bc[2], bc[3]);
    uchar2 b45 = make_uchar2(bc[4], bc[5]);
    assemble_kernel<<<grid_for(c.n), kThreads, 0, st>>>(geo(c), ax, ay, az, kappa, b03, b45,
                                                        c.ws.d, c.ws.cx, c.ws.cy, c.ws.cz,
                                                        c.ws.flags);
    return cudaGetLastError();
}

cudaError_t launch_check_filter(const KernelCtx &c, const double *t, cudaStream_t st) {
    check_filter_kernel<<<grid_for(c.n), kThreads, 0, st>>>(c.n, t, c.ws.flags);
    return cudaGetLastError();
}

static Geo geo(const KernelCtx &c);

template <typename F>
static void convert_all(const KernelCtx &c, cudaStream_t st) {
    convert_kernel<F><<<grid_for(c.n), kThreads, 0, st>>>(c.n, c.ws.cz, (F *)c.ws.l3);
    l3_records_kernel<F><<<grid_for(c.n), kThreads, 0, st>>>(geo(c), c.slots, c.ws.cz, (F *)c.ws.rec);
    if (c.precond == FFP_PRECOND_COMBO) {
        convert_kernel<F><<<grid_for(c.n), kThreads, 0, st>>>(c.n, c.ws.cx, (F *)c.ws.lx);
        convert_kernel<F><<<grid_for(c.n), kThreads, 0, st>>>(c.n, c.ws.cy, (F *)c.ws.ly);
    }
}

cudaError_t launch_convert_bands(const KernelCtx &c, cudaStream_t st) {
    switch (c.prec) {
        case FFP_FP64: convert_all<double>(c, st); break;
        case FFP_FP32: convert_all<float>(c, st); break;
        default: convert_all<__nv_bfloat16>(c, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_export_rec(const KernelCtx &c, int what, double *dst, cudaStream_t st) {
    if (what == 0) return launch_export(c, c.ws.l1, dst, st);
    switch (c.prec) {
        case FFP_FP64:
            export_rec_kernel<double><<<grid_for(c.n), kThreads, 0, st>>>(geo(c), c.slots, (const double *)c.ws.rec, what, dst);
            break;
        case FFP_FP32:
            export_rec_kernel<float><<<grid_for(c.n), kThreads, 0, st>>>(geo(c), c.slots, (const float *)c.ws.rec, what, dst);
            break;
        default:
            export_rec_kernel<__nv_bfloat16><<<grid_for(c.n), kThreads, 0, st>>>(geo(c), c.slots, (const __nv_bfloat16 *)c.ws.rec, what, dst);
    }
    return cudaGetLastError();
}

cudaError_t launch_export(const KernelCtx &c, const void *src, double *dst, cudaStream_t st) {
    switch (c.prec) {
        case FFP_FP64:
            export_kernel<double><<<grid_for(c.n), kThreads, 0, st>>>(c.n, (const double *)src, dst);
            break;
        case FFP_FP32:
            export_kernel<float><<<grid_for(c.n), kThreads, 0, st>>>(c.n, (const float *)src, dst);
            break;
        default:
            export_kernel<__nv_bfloat16><<<grid_for(c.n), kThreads, 0, st>>>(
                c.n, (const __nv_bfloat16 *)src, dst);
    }
    return cudaGetLastError();
}

cudaError_t launch_spmv(const KernelCtx &c, const double *x, double *y, cudaStream_t st) {
    spmv_kernel<<<grid_for(c.n), kThreads, 0, st>>>(geo(c), c.ws.d, c.ws.cx, c.ws.cy, c.ws.cz, x, y);
    return cudaGetLastError();
}

cudaError_t launch_resid_vec(const KernelCtx &c, const double *r, const double *y, double *w,
                             cudaStream_t st) {
    resid_vec_kernel<<<grid_for(c.n), kThreads, 0, st>>>(geo(c), c.ws.d, c.ws.cx, c.ws.cy, c.ws.cz,
                                                         r, y, w);
    return cudaGetLastError();
}

cudaError_t launch_add(const KernelCtx &c, double *z, const double *y, cudaStream_t st) {
    add_kernel<<<grid_for(c.n), kThreads, 0, st>>>(c.n, z, y);
    return cudaGetLastError();
}

cudaError_t launch_to_lb(const KernelCtx &c, const double *x, void *xb, cudaStream_t st) {
    const long long nlines = (long long)c.ny * c.nz;
    const long long tot = nlines * lb_len(c.slots);
    if (c.prec == FFP_FP64)
        to_lb_kernel<double><<<grid_for(tot), kThreads, 0, st>>>(nlines, c.nx, c.slots, x, (double *)xb);
    else
        to_lb_kernel<float><<<grid_for(tot), kThreads, 0, st>>>(nlines, c.nx, c.slots, x, (float *)xb);
    return cudaGetLastError();
}

cudaError_t launch_from_lb(const KernelCtx &c, const void *xb, double *y, const double *add,
                           cudaStream_t st) {
    if (c.prec == FFP_FP64)
        from_lb_kernel<double><<<grid_for(c.n), kThreads, 0, st>>>(c.n, c.nx, c.slots, (const double *)xb, y, add);
    else
        from_lb_kernel<float><<<grid_for(c.n), kThreads, 0, st>>>(c.n, c.nx, c.slots, (const float *)xb, y, add);
    return cudaGetLastError();
}

cudaError_t launch_resid(const KernelCtx &c, const double *b, const double *x, cudaStream_t st) {
    resid_kernel<<<grid_for(c.n), kThreads, 0, st>>>(geo(c), c.ws.d, c.ws.cx, c.ws.cy, c.ws.cz, b, x,
                                                     c.ws.r, c.ws.red);
    return cudaGetLastError();
}

cudaError_t launch_spmv_dot(const KernelCtx &c, cudaStream_t st) {
    spmv_dot_kernel<<<grid_for(c.n), kThreads, 0, st>>>(geo(c), c.ws.d, c.ws.cx, c.ws.cy, c.ws.cz,
                                                        c.ws.p, c.ws.q, c.ws.red);
    return cudaGetLastError();
}

cudaError_t launch_update_xr(const KernelCtx &c, double *x, cudaStream_t st) {
    update_xr_kernel<<<grid_for(c.n), kThreads, 0, st>>>(c.n, c.ws.scal, c.ws.p, c.ws.q, x, c.ws.r,
                                                         c.ws.red);
    return cudaGetLastError();
}

cudaError_t launch_dot_rz(const KernelCtx &c, cudaStream_t st) {
    dot_rz_kernel<<<grid_for(c.n), kThreads, 0, st>>>(c.n, c.ws.r, c.ws.z, c.ws.q, c.ws.red);
    return cudaGetLastError();
}

cudaError_t launch_update_p(const KernelCtx &c, int fresh, cudaStream_t st) {
    update_p_kernel<<<grid_for(c.n), kThreads, 0, st>>>(c.n, c.ws.scal, c.ws.z, c.ws.p, fresh);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const KernelCtx &c, int mode, int fresh, int flexible, cudaStream_t st) {
    finalize_kernel<<<1, 32, 0, st>>>(mode, grid_for(c.n), fresh, flexible, c.ws.red, c.ws.scal,
                                      c.ws.flags);
    return cudaGetLastError();
}

}  // namespace ffp
