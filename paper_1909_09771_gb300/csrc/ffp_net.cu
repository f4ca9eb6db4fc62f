// ffp_net.cu -- the learned filter: a 3-D convolutional network that maps
// log10(kappa) to the filter vector t > 0 of the filtering property B t = A t
// (Sec. I Eq. (3)), its training kernels (gradient, Adam), and the Lanczos
// Ritz vectors of B^{-1}A that its training targets come from (Sec. I: the
// error components hardest to damp lie along the eigenvectors of the
// smallest eigenvalues of B^{-1}A, so t should approximate them).
//
// Network: four 3x3x3 convolutions with zero padding, channels 1 -> 16 -> 16
// -> 16 -> 1, ReLU after the first three; input x0 = log10(kappa) / 3; output
// s = log t.  Weights are stored in BF16 (master copy and Adam moments in
// FP32), all arithmetic is FP32.  Activations are [batch][channel][cell] FP32
// with the cell index a = x + nx (y + ny z).
//
// Convolution kernels work on tiles of 32 x 4 x 2 cells (x, y, z), one thread
// per output cell computing every output channel from a shared-memory copy of
// the input tile with its one-cell halo (zeros outside the grid) and of the
// layer's weights as FP32 [in][tap][out], so the weights are broadcast reads.
// The data gradient of a layer is the same kernel with the taps mirrored and
// the channel roles exchanged, the ReLU derivative applied on load.  The
// weight gradient is a persistent kernel: each thread owns one (out, in)
// channel pair (or a share of the rows of a tile for the thin layers), slides
// a three-cell window along x, and keeps its 27 tap sums in registers over
// all the tiles it visits; the per-block sums are folded in a fixed order.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "ffp_kernels.h"

namespace ffp {
namespace net {

constexpr int TX = 32, TY = 4, TZ = 2, TT = TX * TY * TZ;   // output tile, 256 cells
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int kCS = HX * HY * HZ + 1;  // channel stride of a halo tile (odd: no bank conflicts)
constexpr int kThreadsN = 256;
constexpr int kWgradBlocks = 1216;     // 8 x 152 SMs

struct LayerOff {
    int w, b, cin, cout;
};
__host__ __device__ constexpr LayerOff layer(int l) {
    return l == 0 ? LayerOff{0, 432, 1, 16}
         : l == 1 ? LayerOff{448, 7360, 16, 16}
         : l == 2 ? LayerOff{7376, 14288, 16, 16}
                  : LayerOff{14304, 14736, 16, 1};
}
static_assert(layer(3).b + 1 == FFP_NET_PARAMS, "parameter layout");

struct NetGeo {
    int nx, ny, nz;
    long long n;
    int tx, ty, tz;  // tiles per axis
    int ntile;
};

inline NetGeo make_geo(const ffp_grid &g) {
    NetGeo q;
    q.nx = g.nx; q.ny = g.ny; q.nz = g.nz;
    q.n = (long long)g.nx * g.ny * g.nz;
    q.tx = (g.nx + TX - 1) / TX; q.ty = (g.ny + TY - 1) / TY; q.tz = (g.nz + TZ - 1) / TZ;
    q.ntile = q.tx * q.ty * q.tz;
    return q;
}

__device__ __forceinline__ void tile_origin(const NetGeo &g, int t, int &x0, int &y0, int &z0) {
    x0 = (t % g.tx) * TX;
    t /= g.tx;
    y0 = (t % g.ty) * TY;
    z0 = (t / g.ty) * TZ;
}

// Halo tile of CIN channels of `in` (batch b) into smem; MASK: value kept where mask > 0.
template <int CIN, bool MASK>
__device__ __forceinline__ void load_halo(const NetGeo &g, const float *__restrict__ in,
                                          const float *__restrict__ mask, int x0, int y0, int z0,
                                          float *tile) {
    for (int i = threadIdx.x; i < CIN * (HX * HY * HZ); i += blockDim.x) {
        const int c = i / (HX * HY * HZ);
        int r = i - c * (HX * HY * HZ);
        const int hx = r % HX;
        r /= HX;
        const int hy = r % HY, hz = r / HY;
        const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
        float v = 0.f;
        if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
            const long long a = x + (long long)g.nx * (y + (long long)g.ny * z) + c * g.n;
            v = in[a];
            if (MASK && !(mask[a] > 0.f)) v = 0.f;
        }
        tile[c * kCS + (hz * HY + hy) * HX + hx] = v;
    }
}

// out = conv(in) (+ bias) (ReLU); FLIP: data gradient of a layer with CIN / COUT
// exchanged (W is then the layer's [COUT][CIN][27] weights read as [CIN][COUT],
// taps mirrored); MASK: the input is masked by mask > 0 (ReLU derivative).
template <int CIN, int COUT, bool FLIP, bool RELU, bool MASK>
__global__ void __launch_bounds__(kThreadsN) conv_kernel(NetGeo g, const float *__restrict__ in,
                                                         const float *__restrict__ mask,
                                                         const __nv_bfloat16 *__restrict__ W,
                                                         const float *__restrict__ bias,
                                                         float *__restrict__ out) {
    extern __shared__ __align__(16) float sm[];
    float *ws = sm;                       // [CIN][27][COUT]
    float *tile = sm + CIN * 27 * COUT;   // [CIN][kCS]
    for (int i = threadIdx.x; i < CIN * 27 * COUT; i += blockDim.x) {
        const int o = i % COUT, r = i / COUT, tap = r % 27, c = r / 27;
        const int src = FLIP ? (c * COUT + o) * 27 + (26 - tap) : (o * CIN + c) * 27 + tap;
        ws[i] = __bfloat162float(W[src]);
    }
    int x0, y0, z0;
    tile_origin(g, blockIdx.x, x0, y0, z0);
    const long long boff = (long long)blockIdx.y * g.n;
    load_halo<CIN, MASK>(g, in + boff * CIN, MASK ? mask + boff * CIN : nullptr, x0, y0, z0, tile);
    __syncthreads();
    const int lx = threadIdx.x % TX, ly = (threadIdx.x / TX) % TY, lz = threadIdx.x / (TX * TY);
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = bias ? bias[o] : 0.f;
    for (int c = 0; c < CIN; ++c) {
        const float *tc = tile + c * kCS + (lz * HY + ly) * HX + lx;
        const float *wc = ws + c * 27 * COUT;
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const float v = tc[(dz * HY + dy) * HX + dx];
                    const float *w = wc + ((dz * 3 + dy) * 3 + dx) * COUT;
#pragma unroll
                    for (int o = 0; o < COUT; ++o) acc[o] = fmaf(w[o], v, acc[o]);
                }
    }
    const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
    if (x < g.nx && y < g.ny && z < g.nz) {
        const long long a = x + (long long)g.nx * (y + (long long)g.ny * z);
        float *ob = out + boff * COUT + a;
#pragma unroll
        for (int o = 0; o < COUT; ++o) ob[o * g.n] = RELU ? fmaxf(acc[o], 0.f) : acc[o];
    }
}

// Weight and bias gradient partial sums of one layer over the tiles this block
// visits: gw[o][c][tap] = sum_cells gy[o] * x[c](cell + tap - 1), gb[o] = sum gy[o],
// with gy = gY masked by M > 0 when MASK.  Output partial[blockIdx.x][E],
// E = COUT*CIN*27 weights then COUT biases.
template <int CIN, int COUT, bool MASK>
__global__ void __launch_bounds__(kThreadsN) wgrad_kernel(NetGeo g, int batch,
                                                          const float *__restrict__ X,
                                                          const float *__restrict__ gY,
                                                          const float *__restrict__ M,
                                                          float *__restrict__ partial) {
    constexpr int NP = CIN * COUT;          // channel pairs
    constexpr int NG = kThreadsN / NP;      // thread groups sharing the tile rows
    constexpr int NROW = TY * TZ;           // 8 rows of 32 cells per tile
    static_assert(NG >= 1 && kThreadsN % NP == 0, "pairs per block");
    extern __shared__ __align__(16) float sm[];
    float *xt = sm;                         // [CIN][kCS]
    float *gt = sm + CIN * kCS;             // [COUT][TT]
    const int p = threadIdx.x % NP, grp = threadIdx.x / NP;
    const int o = p / CIN, c = p % CIN;
    // rows and (dz, dy) combinations of this thread's group
    const int rows_per = (NROW + NG - 1) / NG;  // NG <= 8: whole rows; NG = 16: rows shared
    const int row_lo = (NG <= NROW) ? grp * rows_per : grp % NROW;
    const int row_hi = (NG <= NROW) ? min(NROW, row_lo + rows_per) : row_lo + 1;
    const int cmb_lo = (NG <= NROW) ? 0 : (grp / NROW) * 5;
    const int cmb_hi = (NG <= NROW) ? 9 : min(9, cmb_lo + 5);
    float acc[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) acc[k] = 0.f;
    float accb = 0.f;
    const int total = g.ntile * batch;
    for (int tid = blockIdx.x; tid < total; tid += gridDim.x) {
        const int b = tid / g.ntile, t = tid % g.ntile;
        int x0, y0, z0;
        tile_origin(g, t, x0, y0, z0);
        const long long boff = (long long)b * g.n;
        __syncthreads();  // the previous tile is no longer read
        load_halo<CIN, false>(g, X + boff * CIN, nullptr, x0, y0, z0, xt);
        for (int i = threadIdx.x; i < COUT * TT; i += blockDim.x) {
            const int oo = i / TT, r = i % TT;
            const int x = x0 + r % TX, y = y0 + (r / TX) % TY, z = z0 + r / (TX * TY);
            float v = 0.f;  // cells past the grid contribute nothing
            if (x < g.nx && y < g.ny && z < g.nz) {
                const long long a = x + (long long)g.nx * (y + (long long)g.ny * z) + oo * g.n + boff * COUT;
                v = gY[a];
                if (MASK && !(M[a] > 0.f)) v = 0.f;
            }
            gt[i] = v;
        }
        __syncthreads();
        for (int row = row_lo; row < row_hi; ++row) {
            const int ly = row % TY, lz = row / TY;
            const float *gr = gt + o * TT + row * TX;
            if (cmb_lo == 0 && c == 0)
                for (int x = 0; x < TX; ++x) accb += gr[x];
            for (int cmb = cmb_lo; cmb < cmb_hi; ++cmb) {
                const int dz = cmb / 3, dy = cmb % 3;
                const float *xr = xt + c * kCS + ((lz + dz) * HY + (ly + dy)) * HX;
                float w0 = xr[0], w1 = xr[1];
                float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll 8
                for (int x = 0; x < TX; ++x) {
                    const float w2 = xr[x + 2];
                    const float gv = gr[x];
                    s0 = fmaf(gv, w0, s0);
                    s1 = fmaf(gv, w1, s1);
                    s2 = fmaf(gv, w2, s2);
                    w0 = w1;
                    w1 = w2;
                }
                // acc index = tap = (dz*3 + dy)*3 + dx; cmb is compile-time unknown, so
                // accumulate through a small switch-free write
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    if (k == cmb) { acc[3 * k] += s0; acc[3 * k + 1] += s1; acc[3 * k + 2] += s2; }
            }
        }
    }
    // fold the groups (fixed order) and write this block's partial sums
    constexpr int E = COUT * CIN * 27 + COUT;
    float *out = partial + (size_t)blockIdx.x * E;
    if (NG == 1) {
#pragma unroll
        for (int k = 0; k < 27; ++k) out[p * 27 + k] = acc[k];
        if (c == 0) out[COUT * CIN * 27 + o] = accb;
    } else {
        __syncthreads();
        float *red = sm;  // [NG][NP][28]
        for (int k = 0; k < 27; ++k) red[(grp * NP + p) * 28 + k] = acc[k];
        red[(grp * NP + p) * 28 + 27] = accb;
        __syncthreads();
        for (int i = threadIdx.x; i < NP * 28; i += blockDim.x) {
            const int pp = i / 28, k = i % 28;
            float s = 0.f;
            for (int q = 0; q < NG; ++q) s += red[(q * NP + pp) * 28 + k];
            const int oo = pp / CIN, cc = pp % CIN;
            if (k < 27) out[pp * 27 + k] = s;
            else if (cc == 0) out[COUT * CIN * 27 + oo] = s;
        }
    }
}

// grad[off_w + e] (e < Ew) and grad[off_b + o] = fixed-order sums of the block partials
__global__ void wgrad_fold(const float *__restrict__ partial, int nblk, int E, int Ew, int off_w,
                           int off_b, float *grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += (double)partial[(size_t)k * E + e];
    if (e < Ew) grad[off_w + e] = (float)s;
    else grad[off_b + (e - Ew)] = (float)s;
}

__global__ void features_kernel(long long n, const double *__restrict__ kappa, float *x0) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        x0[a] = (float)(log10(kappa[a]) / 3.0);
}

__global__ void head_kernel(long long n, const float *__restrict__ s, double *t) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        t[a] = exp(fmin(fmax((double)s[a], -30.0), 30.0));
}

// gs = 2 (s - s*) / n, partial sums of (s - s*)^2 per block
__global__ void __launch_bounds__(256) loss_kernel(long long n, const float *__restrict__ s,
                                                   const float *__restrict__ st, float *gs,
                                                   double *red) {
    __shared__ double sh[8];
    double acc = 0.0;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x) {
        const float d = s[a] - st[a];
        gs[a] = 2.f * d / (float)n;
        acc += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        red[blockIdx.x] = t;
    }
}

__global__ void loss_fold(const double *__restrict__ red, int nblk, long long n, double *loss) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += red[k];
    *loss = s / (double)n;
}

__global__ void adam_kernel(int np, float *p, __nv_bfloat16 *wb, float *m, float *v,
                            const float *__restrict__ g, float lr, float b1, float b2, float eps,
                            float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    wb[i] = __float2bfloat16_rn(pi);
}

__global__ void cast_kernel(int np, const float *__restrict__ p, __nv_bfloat16 *wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) wb[i] = __float2bfloat16_rn(p[i]);
}

// ---------------------------------------------------------------- host side
template <int CIN, int COUT>
constexpr size_t conv_smem() {
    return sizeof(float) * ((size_t)CIN * 27 * COUT + (size_t)CIN * kCS);
}
template <int CIN, int COUT>
constexpr size_t wgrad_smem() {
    const size_t a = sizeof(float) * ((size_t)CIN * kCS + (size_t)COUT * TT);
    const size_t r = sizeof(float) * (size_t)kThreadsN * 28;
    return a > r ? a : r;
}

template <int CIN, int COUT, bool FLIP, bool RELU, bool MASK>
cudaError_t conv(const NetGeo &g, int batch, const float *in, const float *mask,
                 const __nv_bfloat16 *W, const float *bias, float *out, cudaStream_t st) {
    const size_t smem = conv_smem<CIN, COUT>();
    auto k = conv_kernel<CIN, COUT, FLIP, RELU, MASK>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(g.ntile, batch), kThreadsN, smem, st>>>(g, in, mask, W, bias, out);
    return cudaGetLastError();
}

template <int CIN, int COUT, bool MASK>
cudaError_t wgrad(const NetGeo &g, int batch, const float *X, const float *gY, const float *M,
                  float *partial, float *grad, int l, cudaStream_t st) {
    const size_t smem = wgrad_smem<CIN, COUT>();
    auto k = wgrad_kernel<CIN, COUT, MASK>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nblk = std::min(kWgradBlocks, g.ntile * batch);
    k<<<nblk, kThreadsN, smem, st>>>(g, batch, X, gY, M, partial);
    const int E = COUT * CIN * 27 + COUT;
    wgrad_fold<<<(E + 255) / 256, 256, 0, st>>>(partial, nblk, E, COUT * CIN * 27, layer(l).w,
                                                layer(l).b, grad);
    return cudaGetLastError();
}

// workspace: x0 [B][1][N], a1..a3 [B][16][N], s [B][1][N] (training keeps every
// activation; inference ping-pongs two 16-channel buffers), gradient buffers,
// partial sums
struct NetWs {
    float *x0, *a[3], *s, *g16[2], *gs, *partial;
    double *red, *loss;
};

size_t al256n(size_t v) { return (v + 255) & ~(size_t)255; }

size_t net_layout(const ffp_grid &grid, int batch, int train, char *base, NetWs *w) {
    const size_t n = (size_t)grid.nx * grid.ny * grid.nz * (size_t)batch;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += al256n(bytes);
        return p;
    };
    NetWs q;
    std::memset(&q, 0, sizeof(q));
    q.x0 = (float *)take(4 * n);
    q.a[0] = (float *)take(4 * 16 * n);
    q.a[1] = (float *)take(4 * 16 * n);
    q.a[2] = train ? (float *)take(4 * 16 * n) : q.a[0];
    q.s = (float *)take(4 * n);
    if (train) {
        q.g16[0] = (float *)take(4 * 16 * n);
        q.g16[1] = (float *)take(4 * 16 * n);
        q.gs = (float *)take(4 * n);
        q.partial = (float *)take(4 * (size_t)kWgradBlocks * (16 * 16 * 27 + 16));
        q.red = (double *)take(8 * 1216);
        q.loss = (double *)take(8);
    }
    if (w) *w = q;
    return off;
}

int grid_ok_net(const ffp_grid *g, int batch) {
    return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && batch >= 1 &&
           (long long)g->nx * g->ny * g->nz * batch <= 2000000000LL / 16;
}

cudaError_t forward(const NetGeo &g, int batch, const double *kappa, const float *P,
                    const __nv_bfloat16 *Wb, const NetWs &w, cudaStream_t st) {
    const long long nb = g.n * batch;
    const int vb = (int)std::min<long long>((nb + 255) / 256, 1216 * 4);
    features_kernel<<<vb, 256, 0, st>>>(nb, kappa, w.x0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = conv<1, 16, false, true, false>(g, batch, w.x0, nullptr, Wb + layer(0).w, P + layer(0).b, w.a[0], st);
    if (e == cudaSuccess) e = conv<16, 16, false, true, false>(g, batch, w.a[0], nullptr, Wb + layer(1).w, P + layer(1).b, w.a[1], st);
    if (e == cudaSuccess) e = conv<16, 16, false, true, false>(g, batch, w.a[1], nullptr, Wb + layer(2).w, P + layer(2).b, w.a[2], st);
    if (e == cudaSuccess) e = conv<16, 1, false, false, false>(g, batch, w.a[2], nullptr, Wb + layer(3).w, P + layer(3).b, w.s, st);
    return e;
}

}  // namespace net
}  // namespace ffp

using namespace ffp::net;

extern "C" {

size_t ffp_net_workspace_bytes(const ffp_grid *grid, int batch, int train) {
    if (!grid_ok_net(grid, batch)) return 0;
    return net_layout(*grid, batch, train ? 1 : 0, nullptr, nullptr);
}

int ffp_net_init(unsigned long long seed, float *params, unsigned short *wbf16, void *stream) {
    if (!params || !wbf16) return FFP_ERR_ARG;
    std::vector<float> h(FFP_NET_PARAMS, 0.f);
    std::mt19937_64 gen(seed);
    for (int l = 0; l < 4; ++l) {
        const LayerOff L = layer(l);
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (27.0 * L.cin)));
        for (int i = 0; i < L.cout * L.cin * 27; ++i) h[L.w + i] = (float)nd(gen);
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(params, h.data(), sizeof(float) * FFP_NET_PARAMS,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        cast_kernel<<<(FFP_NET_PARAMS + 255) / 256, 256, 0, st>>>(FFP_NET_PARAMS, params,
                                                                  (__nv_bfloat16 *)wbf16);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // h is read by the copy
    return e == cudaSuccess ? FFP_OK : FFP_ERR_CUDA;
}

int ffp_net_cast(const float *params, unsigned short *wbf16, void *stream) {
    if (!params || !wbf16) return FFP_ERR_ARG;
    cast_kernel<<<(FFP_NET_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        FFP_NET_PARAMS, params, (__nv_bfloat16 *)wbf16);
    return cudaGetLastError() == cudaSuccess ? FFP_OK : FFP_ERR_CUDA;
}

int ffp_net_forward(const ffp_grid *grid, int batch, const double *kappa, const float *params,
                    const unsigned short *wbf16, void *workspace, size_t ws_bytes, double *t,
                    void *stream) {
    if (!grid_ok_net(grid, batch) || !kappa || !params || !wbf16 || !workspace || !t)
        return FFP_ERR_ARG;
    if (((uintptr_t)workspace & 255) != 0 || ws_bytes < ffp_net_workspace_bytes(grid, batch, 0))
        return FFP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    NetWs w;
    net_layout(*grid, batch, 0, (char *)workspace, &w);
    const NetGeo g = make_geo(*grid);
    cudaError_t e = forward(g, batch, kappa, params, (const __nv_bfloat16 *)wbf16, w, st);
    if (e == cudaSuccess) {
        const long long nb = g.n * batch;
        head_kernel<<<(int)std::min<long long>((nb + 255) / 256, 4864), 256, 0, st>>>(nb, w.s, t);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? FFP_OK : FFP_ERR_CUDA;
}

int ffp_net_grad(const ffp_grid *grid, int batch, const double *kappa, const float *s_target,
                 const float *params, const unsigned short *wbf16, void *workspace,
                 size_t ws_bytes, float *grad, double *loss, void *stream) {
    if (!grid_ok_net(grid, batch) || !kappa || !s_target || !params || !wbf16 || !workspace ||
        !grad)
        return FFP_ERR_ARG;
    if (((uintptr_t)workspace & 255) != 0 || ws_bytes < ffp_net_workspace_bytes(grid, batch, 1))
        return FFP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    NetWs w;
    net_layout(*grid, batch, 1, (char *)workspace, &w);
    const NetGeo g = make_geo(*grid);
    const __nv_bfloat16 *Wb = (const __nv_bfloat16 *)wbf16;
    cudaError_t e = forward(g, batch, kappa, params, Wb, w, st);
    const long long nb = g.n * batch;
    const int lb = (int)std::min<long long>((nb + 255) / 256, 1216);
    if (e == cudaSuccess) {
        loss_kernel<<<lb, 256, 0, st>>>(nb, w.s, s_target, w.gs, w.red);
        loss_fold<<<1, 32, 0, st>>>(w.red, lb, nb, w.loss);
        e = cudaGetLastError();
    }
    // layer 3 (16 -> 1, linear): weights from (a3, gs); data gradient g16[0] = conv^T(gs)
    if (e == cudaSuccess) e = wgrad<16, 1, false>(g, batch, w.a[2], w.gs, nullptr, w.partial, grad, 3, st);
    if (e == cudaSuccess) e = conv<1, 16, true, false, false>(g, batch, w.gs, nullptr, Wb + layer(3).w, nullptr, w.g16[0], st);
    // layer 2 (16 -> 16, ReLU output a3)
    if (e == cudaSuccess) e = wgrad<16, 16, true>(g, batch, w.a[1], w.g16[0], w.a[2], w.partial, grad, 2, st);
    if (e == cudaSuccess) e = conv<16, 16, true, false, true>(g, batch, w.g16[0], w.a[2], Wb + layer(2).w, nullptr, w.g16[1], st);
    // layer 1 (16 -> 16, ReLU output a2)
    if (e == cudaSuccess) e = wgrad<16, 16, true>(g, batch, w.a[0], w.g16[1], w.a[1], w.partial, grad, 1, st);
    if (e == cudaSuccess) e = conv<16, 16, true, false, true>(g, batch, w.g16[1], w.a[1], Wb + layer(1).w, nullptr, w.g16[0], st);
    // layer 0 (1 -> 16, ReLU output a1); no gradient w.r.t. the features
    if (e == cudaSuccess) e = wgrad<1, 16, true>(g, batch, w.x0, w.g16[0], w.a[0], w.partial, grad, 0, st);
    if (e == cudaSuccess && loss) {
        e = cudaMemcpyAsync(loss, w.loss, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e == cudaSuccess ? FFP_OK : FFP_ERR_CUDA;
}

int ffp_net_adam(float *params, unsigned short *wbf16, float *m, float *v, const float *grad,
                 int step, double lr, void *stream) {
    if (!params || !wbf16 || !m || !v || !grad || step < 1 || !(lr > 0.0)) return FFP_ERR_ARG;
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    const double bc1 = 1.0 - std::pow(b1, step), bc2 = 1.0 - std::pow(b2, step);
    adam_kernel<<<(FFP_NET_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        FFP_NET_PARAMS, params, (__nv_bfloat16 *)wbf16, m, v, grad, (float)lr, (float)b1,
        (float)b2, (float)eps, (float)bc1, (float)bc2);
    return cudaGetLastError() == cudaSuccess ? FFP_OK : FFP_ERR_CUDA;
}

}  // extern "C"
