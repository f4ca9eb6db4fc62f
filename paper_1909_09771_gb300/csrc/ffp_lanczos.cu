// ffp_lanczos.cu -- Ritz pairs of B_NTD^{-1} A (Lanczos) and the filter
// training target built from them.
//
// Sec. I: the error components hardest to damp are those along the
// eigenvectors of the smallest eigenvalues of B^{-1}A, and a filter vector
// approximating them helps PCG.  B^{-1}A is self-adjoint in the A-inner
// product <u, v>_A = u^T A v (A and B symmetric positive definite), so the
// Lanczos process runs in that product:
//   q_0 = v0 / ||v0||_A;  w = B^{-1} A q_j;  alpha_j = <w, q_j>_A;
//   w -= sum_i <w, q_i>_A q_i over every earlier q_i, twice (full
//   re-orthogonalisation; this also removes the alpha_j and beta_{j-1} terms);
//   A w recomputed after it; beta_j = ||w||_A; q_{j+1} = w / beta_j,
// keeping A q_j beside q_j so every A-product is a plain dot product.  The
// tridiagonal's eigenpairs (Jacobi rotations on the host, m <= 64) give the
// Ritz values theta and vectors Y = Q S.
//
// Target: t* = sqrt(sum_k (theta_0 / theta_k) (y_k / max|y_k|)^2) over the
// nvec smallest Ritz pairs, scaled to max 1 and floored; s* = log t* minus its
// mean (the filter acts through ratios only, so its scale is free).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ffp_vecops.cuh"

namespace ffp {
namespace {

constexpr int kLzBlocks = 608;  // 4 x 152 SMs
constexpr int kMaxM = 64;

// red[i * nblk + blockIdx.x] = partial of x . Y_i, i = blockIdx.y
__global__ void __launch_bounds__(256) ldot_kernel(long long n, const double *__restrict__ x,
                                                   const double *__restrict__ Y, long long ld,
                                                   double *red) {
    const double *y = Y + (long long)blockIdx.y * ld;
    double acc[1] = {0.0};
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        acc[0] += x[a] * y[a];
    block_sum<1>(acc, red + (long long)blockIdx.y * gridDim.x);
}

// coef[i] = sum of red[i * nblk ...] (fixed order), one warp per i
__global__ void lfold_kernel(const double *__restrict__ red, int nblk, double *coef) {
    const double s = warp_fold(red + (long long)blockIdx.x * nblk, nblk, 1, 0);
    if (threadIdx.x == 0) coef[blockIdx.x] = s;
}

// w -= sum_{i<k} coef[i] Q_i
__global__ void __launch_bounds__(256) lupdate_kernel(long long n, double *w,
                                                      const double *__restrict__ Q, long long ld,
                                                      int k, const double *__restrict__ coef) {
    __shared__ double c[kMaxM + 1];
    for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = coef[i];
    __syncthreads();
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        double s = w[a];
        for (int i = 0; i < k; ++i) s -= c[i] * Q[i * ld + a];
        w[a] = s;
    }
}

// q = x / nrm, aq = ax / nrm
__global__ void lscale_kernel(long long n, const double *__restrict__ x,
                              const double *__restrict__ ax, double *q, double *aq, double inv) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        q[a] = x[a] * inv;
        aq[a] = ax[a] * inv;
    }
}

// Y_v = sum_{j<k} S[j][v] Q_j for v < nvec (S row-major k x k, eigenvectors in columns)
__global__ void __launch_bounds__(256) ritz_kernel(long long n, const double *__restrict__ Q,
                                                   long long ld, int k, int nvec,
                                                   const double *__restrict__ S, double *Y) {
    __shared__ double s[kMaxM * 8];
    for (int i = threadIdx.x; i < k * nvec; i += blockDim.x) s[i] = S[(i / nvec) * k + i % nvec];
    __syncthreads();
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        double y[8];
        for (int v = 0; v < nvec; ++v) y[v] = 0.0;
        for (int j = 0; j < k; ++j) {
            const double q = Q[j * ld + a];
            for (int v = 0; v < nvec; ++v) y[v] += s[j * nvec + v] * q;
        }
        for (int v = 0; v < nvec; ++v) Y[v * n + a] = y[v];
    }
}

// block maxima of |x_v| (v = blockIdx.y) -> red[v * nblk + blockIdx.x]
__global__ void __launch_bounds__(256) lmax_kernel(long long n, const double *__restrict__ X,
                                                   double *red) {
    __shared__ double sh[8];
    const double *x = X + (long long)blockIdx.y * n;
    double m = 0.0;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(x[a]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t = fmax(t, sh[w]);
        red[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void lmax_fold(const double *__restrict__ red, int nblk, double *out) {
    const double *r = red + (long long)blockIdx.x * nblk;
    double m = 0.0;
    for (int i = threadIdx.x; i < nblk; i += 32) m = fmax(m, r[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) out[blockIdx.x] = m;
}

// t = sqrt(sum_v wt[v] (Y_v / ymax_v)^2)
__global__ void envelope_kernel(long long n, int nvec, const double *__restrict__ Y,
                                const double *__restrict__ ymax, const double *__restrict__ wt,
                                double *t) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int v = 0; v < nvec; ++v) {
            const double y = Y[v * n + a] / ymax[v];
            acc += wt[v] * y * y;
        }
        t[a] = sqrt(acc);
    }
}

// t = max(t / tmax, floor); s = log t; partial sums of s
__global__ void __launch_bounds__(256) floor_log_kernel(long long n, double *t,
                                                        const double *__restrict__ tmax,
                                                        double floor_, double *s, double *red) {
    const double inv = 1.0 / *tmax;
    double acc[1] = {0.0};
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const double v = fmax(t[a] * inv, floor_);
        t[a] = v;
        const double l = log(v);
        s[a] = l;
        acc[0] += l;
    }
    block_sum<1>(acc, red);
}

__global__ void center_kernel(long long n, const double *__restrict__ s, const double *__restrict__ sum,
                              float *s32) {
    const double mean = *sum / (double)n;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        s32[a] = (float)(s[a] - mean);
}

// Eigenpairs of a symmetric k x k matrix (row-major) by cyclic Jacobi rotations;
// eigenvalues ascending in ev, eigenvectors in the columns of V.
void jacobi_eig(int k, std::vector<double> T, std::vector<double> &ev, std::vector<double> &V) {
    V.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) V[i * k + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                tot += T[i * k + j] * T[i * k + j];
                if (i != j) off += T[i * k + j] * T[i * k + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = T[p * k + q];
                if (apq == 0.0) continue;
                const double app = T[p * k + p], aqq = T[q * k + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {  // columns p, q
                    const double trp = T[r * k + p], trq = T[r * k + q];
                    T[r * k + p] = c * trp - s * trq;
                    T[r * k + q] = s * trp + c * trq;
                }
                for (int r = 0; r < k; ++r) {  // rows p, q
                    const double tpr = T[p * k + r], tqr = T[q * k + r];
                    T[p * k + r] = c * tpr - s * tqr;
                    T[q * k + r] = s * tpr + c * tqr;
                }
                for (int r = 0; r < k; ++r) {
                    const double vrp = V[r * k + p], vrq = V[r * k + q];
                    V[r * k + p] = c * vrp - s * vrq;
                    V[r * k + q] = s * vrp + c * vrq;
                }
            }
    }
    std::vector<int> ord(k);
    for (int i = 0; i < k; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return T[a * k + a] < T[b * k + b]; });
    ev.resize(k);
    std::vector<double> W((size_t)k * k);
    for (int c = 0; c < k; ++c) {
        ev[c] = T[ord[c] * k + ord[c]];
        for (int r = 0; r < k; ++r) W[r * k + c] = V[r * k + ord[c]];
    }
    V.swap(W);
}

struct LzWs {
    double *Q, *AQ, *w, *Aw, *red, *coef, *S, *small;
};

size_t al256l(size_t v) { return (v + 255) & ~(size_t)255; }

size_t lz_layout(long long n, int m, char *base, LzWs *L) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += al256l(bytes);
        return p;
    };
    LzWs q;
    q.Q = (double *)take(8 * (size_t)n * (m + 1));
    q.AQ = (double *)take(8 * (size_t)n * (m + 1));
    q.w = (double *)take(8 * (size_t)n);
    q.Aw = (double *)take(8 * (size_t)n);
    q.red = (double *)take(8 * (size_t)kLzBlocks * (kMaxM + 1));
    q.coef = (double *)take(8 * (kMaxM + 1));
    q.S = (double *)take(8 * (size_t)kMaxM * kMaxM);
    q.small = (double *)take(8 * 64);
    if (L) *L = q;
    return off;
}

int nblk_for(long long n) { return (int)std::max<long long>(1, std::min<long long>(kLzBlocks, (n + 255) / 256)); }

// dots x . Y_i for i < k into host[0..k)
cudaError_t dots(long long n, const double *x, const double *Y, long long ld, int k, const LzWs &L,
                 double *host, cudaStream_t st) {
    const int nb = nblk_for(n);
    ldot_kernel<<<dim3(nb, k), 256, 0, st>>>(n, x, Y, ld, L.red);
    lfold_kernel<<<k, 32, 0, st>>>(L.red, nb, L.coef);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && host) {
        e = cudaMemcpyAsync(host, L.coef, 8 * (size_t)k, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e;
}

}  // namespace
}  // namespace ffp

using namespace ffp;

extern "C" {

size_t ffp_lanczos_scratch_bytes(const ffp_grid *grid, int m) {
    if (!grid || grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || m < 1 || m > kMaxM) return 0;
    return lz_layout((long long)grid->nx * grid->ny * grid->nz, m, nullptr, nullptr);
}

int ffp_lanczos_ritz(ffp_handle *h, const double *v0, int m, int nvec, void *scratch,
                     size_t scratch_bytes, double *theta, double *Y, int *steps, void *stream) {
    const KernelCtx *cp = handle_ctx(h);
    if (!cp || !v0 || !scratch || !theta || m < 1 || m > kMaxM || nvec < 0 || nvec > 8 ||
        (nvec > 0 && !Y))
        return FFP_ERR_ARG;
    const KernelCtx &c = *cp;
    const long long n = c.n;
    if (scratch_bytes < lz_layout(n, m, nullptr, nullptr) || ((uintptr_t)scratch & 255) != 0)
        return FFP_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FFP_ERR_CUDA;
    if (dev != handle_device(h)) return FFP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    LzWs L;
    lz_layout(n, m, (char *)scratch, &L);
    const int vb = nblk_for(n);
    std::vector<double> alpha, beta;
    double hv[kMaxM + 1];
    cudaError_t e = launch_spmv(c, v0, L.AQ, st);
    if (e == cudaSuccess) e = dots(n, v0, L.AQ, n, 1, L, hv, st);
    if (e != cudaSuccess) return FFP_ERR_CUDA;
    if (!(hv[0] > 0.0) || !std::isfinite(hv[0])) return FFP_ERR_BREAKDOWN;
    lscale_kernel<<<vb, 256, 0, st>>>(n, v0, L.AQ, L.Q, L.AQ, 1.0 / std::sqrt(hv[0]));
    for (int j = 0; j < m && e == cudaSuccess; ++j) {
        double *aqj = L.AQ + (size_t)j * n;
        e = launch_apply(c, aqj, L.w, st);  // w = B_NTD^{-1} A q_j
        if (e == cudaSuccess) e = dots(n, L.w, aqj, n, 1, L, hv, st);
        if (e != cudaSuccess) break;
        alpha.push_back(hv[0]);
        for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
            e = dots(n, L.w, L.AQ, n, j + 1, L, nullptr, st);
            if (e == cudaSuccess) {
                lupdate_kernel<<<vb, 256, 0, st>>>(n, L.w, L.Q, n, j + 1, L.coef);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess) e = launch_spmv(c, L.w, L.Aw, st);
        if (e == cudaSuccess) e = dots(n, L.w, L.Aw, n, 1, L, hv, st);
        if (e != cudaSuccess) break;
        const double b2 = std::max(hv[0], 0.0);
        const double bj = std::sqrt(b2);
        if (j == m - 1 || !(bj > 1e-14 * std::fabs(alpha[0]))) break;
        beta.push_back(bj);
        lscale_kernel<<<vb, 256, 0, st>>>(n, L.w, L.Aw, L.Q + (size_t)(j + 1) * n,
                                          L.AQ + (size_t)(j + 1) * n, 1.0 / bj);
    }
    if (e != cudaSuccess) return FFP_ERR_CUDA;
    const int k = (int)alpha.size();
    std::vector<double> T((size_t)k * k, 0.0), ev, V;
    for (int i = 0; i < k; ++i) {
        T[i * k + i] = alpha[i];
        if (i + 1 < k) T[i * k + i + 1] = T[(i + 1) * k + i] = beta[i];
    }
    jacobi_eig(k, T, ev, V);
    for (int i = 0; i < k; ++i) theta[i] = ev[i];
    if (steps) *steps = k;
    const int nv = std::min(nvec, k);
    if (nv > 0) {
        std::vector<double> Sv((size_t)k * k);
        for (int r = 0; r < k; ++r)
            for (int cc = 0; cc < k; ++cc) Sv[r * k + cc] = V[r * k + cc];
        e = cudaMemcpyAsync(L.S, Sv.data(), 8 * (size_t)k * k, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            // ritz_kernel takes S as k x k row-major and the first nv columns
            ritz_kernel<<<vb, 256, 0, st>>>(n, L.Q, n, k, nv, L.S, Y);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // Sv is read by the copy
    }
    return e == cudaSuccess ? FFP_OK : FFP_ERR_CUDA;
}

int ffp_filter_target(const ffp_grid *grid, int nvec, const double *theta, const double *Y,
                      double floor_, double *t, float *s, void *scratch, size_t scratch_bytes,
                      void *stream) {
    if (!grid || nvec < 1 || nvec > 8 || !theta || !Y || !t || !s || !scratch ||
        !(floor_ > 0.0) || !(floor_ <= 1.0))
        return FFP_ERR_ARG;
    const long long n = (long long)grid->nx * grid->ny * grid->nz;
    if (n < 1 || scratch_bytes < ffp_lanczos_scratch_bytes(grid, 1) || ((uintptr_t)scratch & 255) != 0)
        return FFP_ERR_ARG;
    for (int v = 0; v < nvec; ++v)
        if (!(theta[v] > 0.0)) return FFP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    LzWs L;
    lz_layout(n, 1, (char *)scratch, &L);
    const int vb = nblk_for(n);
    double wt[8];
    for (int v = 0; v < nvec; ++v) wt[v] = theta[0] / theta[v];
    // small: [0..8) ymax, [8..16) weights, [16] tmax, [17] sum of log t
    cudaError_t e = cudaMemcpyAsync(L.small + 8, wt, 8 * (size_t)nvec, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        lmax_kernel<<<dim3(vb, nvec), 256, 0, st>>>(n, Y, L.red);
        lmax_fold<<<nvec, 32, 0, st>>>(L.red, vb, L.small);
        envelope_kernel<<<vb, 256, 0, st>>>(n, nvec, Y, L.small, L.small + 8, t);
        lmax_kernel<<<dim3(vb, 1), 256, 0, st>>>(n, t, L.red);
        lmax_fold<<<1, 32, 0, st>>>(L.red, vb, L.small + 16);
        floor_log_kernel<<<vb, 256, 0, st>>>(n, t, L.small + 16, floor_, L.w, L.red);
        lfold_kernel<<<1, 32, 0, st>>>(L.red, vb, L.small + 17);
        center_kernel<<<vb, 256, 0, st>>>(n, L.w, L.small + 17, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // wt is read by the copy
    return e == cudaSuccess ? FFP_OK : FFP_ERR_CUDA;
}

}  // extern "C"
