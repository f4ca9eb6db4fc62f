// ffp_net.cu -- the learned filter: a 3-D convolutional network that maps
// log10(kappa) to the filter vector t > 0 of the filtering property B t = A t
// (Sec. I Eq. (3)), and its training kernels (gradient, Adam).  Sec. I: the
// error components hardest to damp lie along the eigenvectors of the smallest
// eigenvalues of B^{-1}A, so t should approximate them; the Ritz vectors the
// targets come from are in ffp_lanczos.cu.
//
// Network: four 3x3x3 convolutions with zero padding, channels 1 -> 16 -> 16
// -> 16 -> 1, ReLU after the first three; input x0 = log10(kappa) / 3; output
// s = log t.  Weights in BF16 (master copy and Adam moments in FP32).
//
// Tensor-core form.  Activations live in a padded, channel-split BF16 layout
// (PCS): every instance of the batch is padded by one zero cell on each side
// (X = nx+2, Y = ny+2, Z = nz+2), the padded volumes are concatenated into one
// flat index q, and the 16 channels are split into two planes of 8 (16 bytes
// per cell and plane).  In the flat padded index a 3x3x3 convolution is a 1-D
// correlation with the 27 offsets dz*X*Y + dy*X + dx, so for 128 consecutive
// outputs every tap reads 128 consecutive cells: one M=128, N=16, K=16 BF16
// MMA (tcgen05, FP32 accumulator in tensor memory) whose A descriptor is the
// staged tile shifted by the tap's offset (a shift of 16 bytes per cell).
// Outputs that fall on the padding are computed and discarded (written as 0,
// which keeps the padding zero for the next layer).  Thin layers use the same
// kernels: the 1-channel input x0 and loss gradient are 16-channel tensors
// with 15 zero channels, and the 1-output layer a 16-output one with 15 zero
// weight rows.
//
//  tconv_kernel   forward (bias + ReLU, or the FP32 head s) and data gradient
//                 (mirrored taps, transposed weights, ReLU mask of the
//                 layer's input applied in the epilogue).  One CTA per SM,
//                 persistent over tiles of 128 NT outputs: warp 0 stages three
//                 slabs (dz = -1, 0, 1) of the input per tile with bulk copies
//                 into a ring, warp 1 issues the 27 NT MMAs, warps 2-5 drain
//                 the two tensor-memory accumulators (one per tile in flight).
//  twgrad_kernel  weight gradient: dW_tap[o][c] = sum_q gz[q][o] in[q+off][c],
//                 M = 128 (rows 0-15 are o; the others are not read), N = 16
//                 (c), K = 16 cells per MMA, both operands MN-major; one MMA
//                 per tap and 16 cells, and one more against a ones operand
//                 for the bias gradient sum_q gz[q][o].  The 28 accumulators
//                 stay in tensor memory over all of the CTA's tiles.
// Every mbarrier wait is bounded; a wait that runs out sets a flag the host
// turns into FFP_ERR_TIMEOUT, and the kernel drains its copies and MMAs in
// flight (again with bounded waits) before it frees its tensor memory.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "ffp_kernels.h"
#include "ffp_umma.cuh"

namespace ffp {
namespace net {

constexpr int kWgradBlocks = 1216;   // upper bound of CTAs of one weight-gradient launch
constexpr int kWimg = 27 * 512;      // bytes of one B-operand image (27 taps x 16 x 16 BF16)
constexpr int kMaxStages = 4;
constexpr int kTK = 256;             // cells per weight-gradient tile
constexpr int kSmemCap = 232448;     // dynamic shared memory of one CTA (227 KB)
constexpr int kSmemOneCta = 120832;  // at least this much: one CTA per SM (tensor memory)
constexpr int kBarBytes = 128;       // barriers, the tensor-memory slot, the abort word

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

// Padded channel-split layout of one batch: plane 0 (channels 0-7) at the
// buffer's start, plane 1 (8-15) `pitch` bytes later; cell q (flat padded
// index, -G <= q < L - G) at byte 16 (G + q) of its plane.
struct Pcs {
    int nx, ny, nz, batch;
    int X, Y, XY;     // padded row and plane
    int V;            // padded cells per instance
    long long n;      // cells per instance
    int Q;            // padded cells of the batch
    int G;            // guard cells before q = 0 (the largest tap offset)
    long long L;      // cells per plane: guards, batch and the tail of the last tile
    long long pitch;  // 16 L
};

Pcs make_pcs(const ffp_grid &g, int batch) {
    Pcs p;
    p.nx = g.nx; p.ny = g.ny; p.nz = g.nz; p.batch = batch;
    p.X = g.nx + 2; p.Y = g.ny + 2; p.XY = p.X * p.Y;
    p.V = p.XY * (g.nz + 2);
    p.n = (long long)g.nx * g.ny * g.nz;
    p.Q = p.V * batch;
    p.G = p.XY + p.X + 1;
    p.L = ((long long)2 * p.G + p.Q + 512 + 7) / 8 * 8;
    p.pitch = 16 * p.L;
    return p;
}

// Flat padded index -> instance-major cell index a (false on the padding).
__device__ __forceinline__ bool interior(const Pcs &p, int q, long long &a) {
    const int b = q / p.V;
    int r = q - b * p.V;
    const int z = r / p.XY;
    r -= z * p.XY;
    const int y = r / p.X, x = r - y * p.X;
    if (x < 1 || x > p.nx || y < 1 || y > p.ny || z < 1 || z > p.nz) return false;
    a = (long long)b * p.n + (x - 1) + (long long)p.nx * ((y - 1) + (long long)p.ny * (z - 1));
    return true;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// ---------------------------------------------------------------- elementwise kernels
// Zero the guard cells (before q = 0 and after q = Q) of up to 8 buffers.
struct GuardArgs {
    char *buf[8];
    int nbuf;
};
__global__ void guard_zero_kernel(Pcs p, GuardArgs g) {
    const long long head = p.G, tail = p.L - p.G - p.Q, per = 2 * (head + tail);  // cells per buffer
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per * g.nbuf;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / per);
        long long r = i - b * per;
        const int plane = (int)(r / (head + tail));
        r -= plane * (head + tail);
        const long long cell = r < head ? r : p.G + p.Q + (r - head);
        *(uint4 *)(g.buf[b] + plane * p.pitch + 16 * cell) = make_uint4(0, 0, 0, 0);
    }
}

// x0 = log10(kappa) / 3 in channel 0 of a PCS buffer (channels 1-15 and the padding 0).
__global__ void features_kernel(Pcs p, const double *__restrict__ kappa, char *x0) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.Q; q += gridDim.x * blockDim.x) {
        long long a;
        float v = 0.f;
        if (interior(p, q, a)) v = (float)(log10(kappa[a]) / 3.0);
        *(uint4 *)(x0 + 16 * ((long long)p.G + q)) = make_uint4(pack2(v, 0.f), 0, 0, 0);
        *(uint4 *)(x0 + p.pitch + 16 * ((long long)p.G + q)) = make_uint4(0, 0, 0, 0);
    }
}

// B-operand images [tap][k/8][n][k%8] (BF16) of every layer: images 0-3 the
// forward convolutions (n = output, k = input channel), images 4-6 the data
// gradients of layers 1-3 (n = input, k = output channel, taps mirrored).
__global__ void wimg_kernel(const __nv_bfloat16 *__restrict__ W, __nv_bfloat16 *img) {
    const int im = blockIdx.y;
    const int l = im < 4 ? im : im - 3;
    const bool flip = im >= 4;
    const LayerOff L = layer(l);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 27 * 256; i += gridDim.x * blockDim.x) {
        const int tap = i / 256, r = i % 256;
        const int k = (r / 128) * 8 + r % 8, n = (r / 8) % 16;
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (!flip) {
            if (n < L.cout && k < L.cin) v = W[L.w + (n * L.cin + k) * 27 + tap];
        } else {
            if (k < L.cout && n < L.cin) v = W[L.w + (k * L.cin + n) * 27 + (26 - tap)];
        }
        img[(size_t)im * 27 * 256 + i] = v;
    }
}

__global__ void head_kernel(long long n, const float *__restrict__ s, double *t) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        t[a] = exp(fmin(fmax((double)s[a], -30.0), 30.0));
}

// gs = 2 (s - s*) / n_b into channel 0 of a PCS buffer (BF16), block partial
// sums of (s - s*)^2.
__global__ void __launch_bounds__(256) loss_kernel(Pcs p, const float *__restrict__ s,
                                                   const float *__restrict__ st, char *gs,
                                                   double *red) {
    __shared__ double sh[8];
    const float inv = 2.f / (float)(p.n * p.batch);
    double acc = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.Q; q += gridDim.x * blockDim.x) {
        long long a;
        float g = 0.f;
        if (interior(p, q, a)) {
            const float d = s[a] - st[a];
            g = d * inv;
            acc += (double)d * d;
        }
        *(uint4 *)(gs + 16 * ((long long)p.G + q)) = make_uint4(pack2(g, 0.f), 0, 0, 0);
        *(uint4 *)(gs + p.pitch + 16 * ((long long)p.G + q)) = make_uint4(0, 0, 0, 0);
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

// ---------------------------------------------------------------- tensor-core convolution
enum { CM_ACT = 0, CM_HEAD = 1, CM_DGRAD = 2 };

struct ConvArgs {
    Pcs p;
    const char *in;            // input PCS buffer
    char *out;                 // CM_ACT, CM_DGRAD: output PCS buffer
    const char *mask;          // CM_DGRAD: the layer input's forward activation (ReLU mask)
    float *s;                  // CM_HEAD: FP32 [batch][n]
    const __nv_bfloat16 *wimg; // the layer's B-operand image
    const float *bias;         // CM_ACT, CM_HEAD: `cout` biases
    int *flags;                // [0]: a bounded wait ran out
    int mode, cout, ntiles, stages, R;
    unsigned tries;
};

__host__ __device__ inline size_t conv_stage_bytes(int R) { return (size_t)6 * R * 16; }

template <int NT>
__device__ __forceinline__ void conv_store(const ConvArgs &A, int q, const float (&v)[16],
                                           const float (&bias)[16]) {
    long long a;
    const bool in = interior(A.p, q, a);
    const long long off = 16 * ((long long)A.p.G + q);
    if (A.mode == CM_HEAD) {
        if (in) A.s[a] = v[0] + bias[0];
        return;
    }
    uint32_t w[8];
    if (!in) {
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = 0;
    } else if (A.mode == CM_ACT) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            w[i] = pack2(fmaxf(v[2 * i] + bias[2 * i], 0.f), fmaxf(v[2 * i + 1] + bias[2 * i + 1], 0.f));
    } else {
        const uint4 m0 = *(const uint4 *)(A.mask + off), m1 = *(const uint4 *)(A.mask + A.p.pitch + off);
        const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
            w[i] = pack2(bf_lo(mw[i]) > 0.f ? v[2 * i] : 0.f, bf_hi(mw[i]) > 0.f ? v[2 * i + 1] : 0.f);
    }
    *(uint4 *)(A.out + off) = make_uint4(w[0], w[1], w[2], w[3]);
    *(uint4 *)(A.out + A.p.pitch + off) = make_uint4(w[4], w[5], w[6], w[7]);
}

template <int NT>
__global__ void __launch_bounds__(192, 1) tconv_kernel(const __grid_constant__ ConvArgs A) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int TM = 128 * NT;
    constexpr uint32_t kCols = 2 * NT * 16;  // two accumulators of NT x 16 columns
    const int S = A.stages, R = A.R;
    const size_t stage_b = conv_stage_bytes(R);
    unsigned long long *bars = (unsigned long long *)(sm + kWimg + (size_t)S * stage_b);
    unsigned long long *full = bars, *empty = bars + kMaxStages, *tfull = bars + 2 * kMaxStages,
                       *tempty = tfull + 2, *drain = tfull + 4;
    uint32_t *tslot = (uint32_t *)(drain + 1);
    volatile int *abort_s = (volatile int *)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    {  // the weight image, read by the tensor cores from shared memory
        const uint4 *src = (const uint4 *)A.wimg;
        uint4 *dst = (uint4 *)sm;
        for (int i = threadIdx.x; i < kWimg / 16; i += blockDim.x) dst[i] = src[i];
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(tfull + k, 1);
            mbar_init(tempty + k, 128);
        }
        mbar_init(drain, 1);
        *abort_s = 0;
        umma::fence_barrier_init();
    }
    umma::fence_proxy_async();
    if (warp == 0) umma::tmem_alloc(tslot, kCols);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // producer: three slabs (dz = -1, 0, 1) x two planes of R cells per tile
        int it = 0;
        for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x, ++it) {
            const int s = it % S;
            if (it >= S) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait(empty + s, ((it / S) & 1) ^ 1, A.tries);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) { atomicExch(A.flags, 1); *abort_s = 1; }
                    break;
                }
            }
            if (*abort_s) break;
            unsigned char *st = sm + kWimg + (size_t)s * stage_b;
            if (lane == 0) umma::mbar_arrive_expect_tx(full + s, (uint32_t)stage_b);
            __syncwarp();
            if (lane < 6) {
                const int dz = lane / 2 - 1, cg = lane & 1;
                const long long q = (long long)tile * TM + (long long)dz * A.p.XY - A.p.X - 1;
                umma::bulk_g2s(st + (size_t)lane * R * 16, A.in + cg * A.p.pitch + 16 * (A.p.G + q),
                               (uint32_t)R * 16, full + s);
            }
            __syncwarp();
        }
        // every copy issued has landed before the CTA moves on (bounded)
        if (lane == 0)
            for (int k = max(0, it - S); k < it; ++k)
                if (!mbar_wait(full + k % S, (k / S) & 1, A.tries)) atomicExch(A.flags, 1);
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = umma::idesc_bf16(128, 16, 0, 0);
            const uint32_t wbase = smem_u32(sm);
            int it = 0;
            bool any = false;
            for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x, ++it) {
                const int s = it % S, acc = it & 1;
                if (*abort_s) break;
                if (!mbar_wait(full + s, (it / S) & 1, A.tries)) {
                    atomicExch(A.flags, 1);
                    *abort_s = 1;
                    break;
                }
                if (it >= 2 && !mbar_wait(tempty + acc, ((it >> 1) & 1) ^ 1, A.tries)) {
                    atomicExch(A.flags, 1);
                    *abort_s = 1;
                    break;
                }
                umma::fence_after_sync();
                const uint32_t sbase = smem_u32(sm + kWimg + (size_t)s * stage_b);
#pragma unroll 1
                for (int j = 0; j < NT; ++j) {
                    const uint32_t d = tbase + (uint32_t)(acc * NT * 16 + j * 16);
#pragma unroll
                    for (int tap = 0; tap < 27; ++tap) {
                        const int dz = tap / 9, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                        // output cell j*128 + i reads slab cell j*128 + i + X + 1 + dy X + dx
                        const uint32_t a_addr = sbase + (uint32_t)(dz * 2) * R * 16 +
                                                (uint32_t)(j * 128 + A.p.X + 1 + dy * A.p.X + dx) * 16;
                        umma::mma_bf16(d, umma::sdesc(a_addr, (uint32_t)R * 16, 128),
                                       umma::sdesc(wbase + tap * 512, 256, 128), idesc, tap > 0);
                    }
                }
                umma::mma_commit(empty + s);
                umma::mma_commit(tfull + acc);
                any = true;
            }
            if (any) {  // every MMA issued has completed (bounded)
                umma::mma_commit(drain);
                if (!mbar_wait(drain, 0, A.tries)) atomicExch(A.flags, 1);
            }
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. +31
        const int quarter = warp & 3, row = quarter * 32 + lane;
        float bias[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) bias[c] = (A.bias && c < A.cout) ? A.bias[c] : 0.f;
        int it = 0;
        for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x, ++it) {
            const int acc = it & 1;
            if (*abort_s) break;
            const int ok = __all_sync(0xffffffffu, mbar_wait(tfull + acc, (it >> 1) & 1, A.tries));
            if (!ok) {
                if (lane == 0) { atomicExch(A.flags, 1); *abort_s = 1; }
                break;
            }
            umma::fence_after_sync();
#pragma unroll 1
            for (int j = 0; j < NT; ++j) {
                float v[16];
                umma::tmem_ld16(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * NT * 16 + j * 16), v);
                const int q = tile * TM + j * 128 + row;
                if (q < A.p.Q) conv_store<NT>(A, q, v, bias);
            }
            umma::fence_before_sync();
            mbar_arrive(tempty + acc);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(tbase, kCols);
}

// ---------------------------------------------------------------- tensor-core weight gradient
struct WgradArgs {
    Pcs p;
    const char *in;   // the layer's input (B operand, shifted per tap)
    const char *gz;   // the gradient at the layer's pre-activation output (A operand)
    float *partial;   // [gridDim.x][E], E = cout cin 27 + cout
    int *flags;
    int cin, cout, ntiles, stages, R;
    unsigned tries;
};

__host__ __device__ inline size_t wgrad_stage_bytes(int R) { return (size_t)kTK * 32 + (size_t)6 * R * 16; }

__global__ void __launch_bounds__(64, 1) twgrad_kernel(const __grid_constant__ WgradArgs A) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int S = A.stages, R = A.R;
    const size_t stage_b = wgrad_stage_bytes(R);
    unsigned char *stages = sm + 1024;  // sm[0, 512): the ones operand
    unsigned long long *bars = (unsigned long long *)(stages + (size_t)S * stage_b);
    unsigned long long *full = bars, *empty = bars + kMaxStages, *done = bars + 2 * kMaxStages;
    uint32_t *tslot = (uint32_t *)(done + 1);
    volatile int *abort_s = (volatile int *)(tslot + 1);
    volatile int *issued = abort_s + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        ((uint32_t *)sm)[i] = 0x3F803F80u;  // BF16 1.0 pairs
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        *abort_s = 0;
        *issued = 0;
        umma::fence_barrier_init();
    }
    umma::fence_proxy_async();
    if (warp == 0) umma::tmem_alloc(tslot, 512);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        int it = 0;
        for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x, ++it) {
            const int s = it % S;
            if (it >= S) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait(empty + s, ((it / S) & 1) ^ 1, A.tries);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) { atomicExch(A.flags, 1); *abort_s = 1; }
                    break;
                }
            }
            if (*abort_s) break;
            unsigned char *st = stages + (size_t)s * stage_b;
            if (lane == 0) umma::mbar_arrive_expect_tx(full + s, (uint32_t)stage_b);
            __syncwarp();
            const long long k0 = (long long)tile * kTK;
            // gz tile as [k-group of 8 cells][plane][8 cells x 16 bytes]
            for (int k = lane; k < kTK / 8 * 2; k += 32) {
                const int kg = k >> 1, cg = k & 1;
                umma::bulk_g2s(st + kg * 256 + cg * 128, A.gz + cg * A.p.pitch + 16 * (A.p.G + k0 + kg * 8), 128,
                               full + s);
            }
            if (lane < 6) {
                const int dz = lane / 2 - 1, cg = lane & 1;
                const long long q = k0 + (long long)dz * A.p.XY - A.p.X - 1;
                umma::bulk_g2s(st + kTK * 32 + (size_t)lane * R * 16, A.in + cg * A.p.pitch + 16 * (A.p.G + q),
                               (uint32_t)R * 16, full + s);
            }
            __syncwarp();
        }
        if (lane == 0)
            for (int k = max(0, it - S); k < it; ++k)
                if (!mbar_wait(full + k % S, (k / S) & 1, A.tries)) atomicExch(A.flags, 1);
        __syncwarp();
    } else if (lane == 0) {
        const uint32_t idesc = umma::idesc_bf16(128, 16, 1, 1);
        const uint64_t ones = umma::sdesc(smem_u32(sm), 128, 256);
        int it = 0;
        uint32_t acc = 0;
        for (int tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x, ++it) {
            const int s = it % S;
            if (*abort_s) break;
            if (!mbar_wait(full + s, (it / S) & 1, A.tries)) {
                atomicExch(A.flags, 1);
                *abort_s = 1;
                break;
            }
            umma::fence_after_sync();
            const uint32_t sbase = smem_u32(stages + (size_t)s * stage_b);
#pragma unroll 1
            for (int kk = 0; kk < kTK / 16; ++kk) {
                // A: gz, rows o (M-groups 128 bytes apart), 16 cells (K-groups 256 bytes apart)
                const uint64_t ad = umma::sdesc(sbase + kk * 512, 256, 128);
#pragma unroll
                for (int tap = 0; tap < 27; ++tap) {
                    const int dz = tap / 9, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                    // B: the input shifted by the tap, channels c (N-groups R*16 apart), cells (K-groups 128 apart)
                    const uint32_t b_addr = sbase + kTK * 32 + (uint32_t)(dz * 2) * R * 16 +
                                            (uint32_t)(kk * 16 + A.p.X + 1 + dy * A.p.X + dx) * 16;
                    umma::mma_bf16(tbase + tap * 16, ad, umma::sdesc(b_addr, 128, (uint32_t)R * 16), idesc, acc);
                }
                umma::mma_bf16(tbase + 27 * 16, ad, ones, idesc, acc);
                acc = 1;
            }
            umma::mma_commit(empty + s);
        }
        if (acc) {
            umma::mma_commit(done);
            *issued = 1;
        }
    }
    __syncthreads();
    if (warp == 0) {
        int ok = 0;
        if (lane == 0 && *issued) {
            ok = mbar_wait(done, 0, A.tries);
            if (!ok) atomicExch(A.flags, 1);
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) {
            umma::fence_after_sync();
            const int E = A.cout * A.cin * 27 + A.cout;
            float *out = A.partial + (size_t)blockIdx.x * E;
#pragma unroll 1
            for (int t = 0; t < 28; ++t) {
                float v[16];
                umma::tmem_ld16(tbase + t * 16, v);  // lanes 0-31 = rows o
                if (lane < A.cout) {
                    if (t < 27) {
                        for (int c = 0; c < A.cin; ++c) out[(lane * A.cin + c) * 27 + t] = v[c];
                    } else {
                        out[A.cout * A.cin * 27 + lane] = v[0];
                    }
                }
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------- host side
int sm_count() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
        return 1;
    return v;
}

// Tile shape of the convolution for a padded row X: NT = 4 with at least two
// stages, else NT = 2; 0 if not even one stage fits.
int conv_shape(int X, int *R, int *stages) {
    for (int nt : {4, 2}) {
        const int r = 128 * nt + 2 * X + 2;
        const long long avail = (long long)kSmemCap - kWimg - kBarBytes;
        const int s = (int)std::min<long long>(kMaxStages, avail / (long long)conv_stage_bytes(r));
        if ((nt == 4 && s >= 2) || (nt == 2 && s >= 1)) {
            *R = r;
            *stages = s;
            return nt;
        }
    }
    return 0;
}

int wgrad_shape(int X, int *R, int *stages) {
    const int r = kTK + 2 * X + 2;
    const long long avail = (long long)kSmemCap - 1024 - kBarBytes;
    const int s = (int)std::min<long long>(kMaxStages, avail / (long long)wgrad_stage_bytes(r));
    *R = r;
    *stages = s;
    return s >= 1;
}

template <int NT>
cudaError_t launch_tconv(const ConvArgs &a, cudaStream_t st) {
    const size_t smem = std::max<size_t>(kSmemOneCta, kWimg + (size_t)a.stages * conv_stage_bytes(a.R) + kBarBytes);
    auto k = tconv_kernel<NT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<std::min(a.ntiles, sm_count()), 192, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t tconv(const Pcs &p, const char *in, char *out, const char *mask, float *s,
                  const __nv_bfloat16 *wimg, const float *bias, int mode, int cout, int *flags,
                  cudaStream_t st) {
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.p = p; a.in = in; a.out = out; a.mask = mask; a.s = s; a.wimg = wimg; a.bias = bias;
    a.flags = flags; a.mode = mode; a.cout = cout; a.tries = kWaitTries;
    const int nt = conv_shape(p.X, &a.R, &a.stages);
    if (nt == 0) return cudaErrorInvalidValue;
    a.ntiles = (p.Q + 128 * nt - 1) / (128 * nt);
    return nt == 4 ? launch_tconv<4>(a, st) : launch_tconv<2>(a, st);
}

cudaError_t twgrad(const Pcs &p, const char *in, const char *gz, int cin, int cout, float *partial,
                   float *grad, int l, int *flags, cudaStream_t st) {
    WgradArgs a;
    std::memset(&a, 0, sizeof(a));
    a.p = p; a.in = in; a.gz = gz; a.partial = partial; a.flags = flags;
    a.cin = cin; a.cout = cout; a.tries = kWaitTries;
    if (!wgrad_shape(p.X, &a.R, &a.stages)) return cudaErrorInvalidValue;
    a.ntiles = (p.Q + kTK - 1) / kTK;
    const int nblk = std::min({a.ntiles, sm_count(), kWgradBlocks});
    const size_t smem = std::max<size_t>(kSmemOneCta, 1024 + (size_t)a.stages * wgrad_stage_bytes(a.R) + kBarBytes);
    cudaError_t e = cudaFuncSetAttribute(twgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    twgrad_kernel<<<nblk, 64, smem, st>>>(a);
    const int E = cout * cin * 27 + cout;
    wgrad_fold<<<(E + 255) / 256, 256, 0, st>>>(partial, nblk, E, cout * cin * 27, layer(l).w, layer(l).b, grad);
    return cudaGetLastError();
}

// workspace: PCS buffers (inference: two, ping-pong; training: x0, the three
// hidden activations, the loss gradient and two gradient buffers), s, the
// seven weight images, partial sums, flags
struct NetWs {
    char *x0, *a[3], *gs, *g[2];
    float *s;
    __nv_bfloat16 *wimg;
    float *partial;
    double *red, *loss;
    int *flags;
    char *pcs[8];
    int npcs;
};

size_t al256n(size_t v) { return (v + 255) & ~(size_t)255; }

size_t net_layout(const ffp_grid &grid, int batch, int train, char *base, NetWs *w) {
    const Pcs p = make_pcs(grid, batch);
    const size_t n = (size_t)p.n * (size_t)batch;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *q = base ? base + off : nullptr;
        off += al256n(bytes);
        return q;
    };
    NetWs q;
    std::memset(&q, 0, sizeof(q));
    const size_t pcs = 2 * (size_t)p.pitch;
    q.x0 = take(pcs);
    q.a[0] = take(pcs);
    if (train) {
        q.a[1] = take(pcs);
        q.a[2] = take(pcs);
        q.gs = take(pcs);
        q.g[0] = take(pcs);
        q.g[1] = take(pcs);
    } else {
        q.a[1] = q.x0;   // layer 1 writes over x0, layer 2 over a[0]
        q.a[2] = q.a[0];
    }
    q.npcs = train ? 7 : 2;
    char *list[7] = {q.x0, q.a[0], q.a[1], q.a[2], q.gs, q.g[0], q.g[1]};
    for (int i = 0; i < q.npcs; ++i) q.pcs[i] = list[i];
    q.s = (float *)take(4 * n);
    q.wimg = (__nv_bfloat16 *)take((size_t)7 * kWimg);
    q.flags = (int *)take(64);
    if (train) {
        q.partial = (float *)take(4 * (size_t)kWgradBlocks * (16 * 16 * 27 + 16));
        q.red = (double *)take(8 * 1216);
        q.loss = (double *)take(8);
    }
    if (w) *w = q;
    return off;
}

int grid_ok_net(const ffp_grid *g, int batch) {
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1 || batch < 1 || g->nx > FFP_NET_MAX_NX) return 0;
    const long long V = (long long)(g->nx + 2) * (g->ny + 2) * (g->nz + 2);
    return V * batch + 4 * V + 1024 < (1LL << 31);
}

cudaError_t forward(const Pcs &p, const double *kappa, const float *P, const __nv_bfloat16 *Wb,
                    const NetWs &w, int train, cudaStream_t st) {
    GuardArgs ga;
    std::memset(&ga, 0, sizeof(ga));
    for (int i = 0; i < w.npcs; ++i) ga.buf[i] = w.pcs[i];
    ga.nbuf = w.npcs;
    cudaError_t e = cudaMemsetAsync(w.flags, 0, 64, st);
    if (e != cudaSuccess) return e;
    guard_zero_kernel<<<152 * 2, 256, 0, st>>>(p, ga);
    wimg_kernel<<<dim3(8, train ? 7 : 4), 256, 0, st>>>(Wb, w.wimg);
    features_kernel<<<152 * 8, 256, 0, st>>>(p, kappa, w.x0);
    e = cudaGetLastError();
    const __nv_bfloat16 *im = w.wimg;
    constexpr size_t IM = kWimg / 2;  // BF16 elements per image
    if (e == cudaSuccess) e = tconv(p, w.x0, w.a[0], nullptr, nullptr, im + 0 * IM, P + layer(0).b, CM_ACT, 16, w.flags, st);
    if (e == cudaSuccess) e = tconv(p, w.a[0], w.a[1], nullptr, nullptr, im + 1 * IM, P + layer(1).b, CM_ACT, 16, w.flags, st);
    if (e == cudaSuccess) e = tconv(p, w.a[1], w.a[2], nullptr, nullptr, im + 2 * IM, P + layer(2).b, CM_ACT, 16, w.flags, st);
    if (e == cudaSuccess) e = tconv(p, w.a[2], nullptr, nullptr, w.s, im + 3 * IM, P + layer(3).b, CM_HEAD, 1, w.flags, st);
    return e;
}

// FFP_OK, FFP_ERR_TIMEOUT (a bounded wait ran out) or FFP_ERR_CUDA
int finish(const NetWs &w, cudaStream_t st) {
    int h = 0;
    if (cudaMemcpyAsync(&h, w.flags, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FFP_ERR_CUDA;
    return h ? FFP_ERR_TIMEOUT : FFP_OK;
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
    const Pcs p = make_pcs(*grid, batch);
    cudaError_t e = forward(p, kappa, params, (const __nv_bfloat16 *)wbf16, w, 0, st);
    if (e == cudaSuccess) {
        const long long nb = p.n * batch;
        head_kernel<<<(int)std::min<long long>((nb + 255) / 256, 4864), 256, 0, st>>>(nb, w.s, t);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return FFP_ERR_CUDA;
    return finish(w, st);
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
    const Pcs p = make_pcs(*grid, batch);
    const __nv_bfloat16 *im = w.wimg;
    constexpr size_t IM = kWimg / 2;
    cudaError_t e = forward(p, kappa, params, (const __nv_bfloat16 *)wbf16, w, 1, st);
    const int lb = 1216;
    if (e == cudaSuccess) {
        loss_kernel<<<lb, 256, 0, st>>>(p, w.s, s_target, w.gs, w.red);
        loss_fold<<<1, 32, 0, st>>>(w.red, lb, p.n * batch, w.loss);
        e = cudaGetLastError();
    }
    // layer 3 (16 -> 1, linear): weights from (a3, gs); g[0] = conv^T(gs) masked by a3 > 0
    if (e == cudaSuccess) e = twgrad(p, w.a[2], w.gs, 16, 1, w.partial, grad, 3, w.flags, st);
    if (e == cudaSuccess) e = tconv(p, w.gs, w.g[0], w.a[2], nullptr, im + 6 * IM, nullptr, CM_DGRAD, 16, w.flags, st);
    // layer 2 (16 -> 16): weights from (a2, g[0]); g[1] = conv^T(g[0]) masked by a2 > 0
    if (e == cudaSuccess) e = twgrad(p, w.a[1], w.g[0], 16, 16, w.partial, grad, 2, w.flags, st);
    if (e == cudaSuccess) e = tconv(p, w.g[0], w.g[1], w.a[1], nullptr, im + 5 * IM, nullptr, CM_DGRAD, 16, w.flags, st);
    // layer 1 (16 -> 16): weights from (a1, g[1]); g[0] = conv^T(g[1]) masked by a1 > 0
    if (e == cudaSuccess) e = twgrad(p, w.a[0], w.g[1], 16, 16, w.partial, grad, 1, w.flags, st);
    if (e == cudaSuccess) e = tconv(p, w.g[1], w.g[0], w.a[0], nullptr, im + 4 * IM, nullptr, CM_DGRAD, 16, w.flags, st);
    // layer 0 (1 -> 16): weights from (x0, g[0]); no gradient w.r.t. the features
    if (e == cudaSuccess) e = twgrad(p, w.x0, w.g[0], 1, 16, w.partial, grad, 0, w.flags, st);
    if (e != cudaSuccess) return FFP_ERR_CUDA;
    if (loss && cudaMemcpyAsync(loss, w.loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FFP_ERR_CUDA;
    return finish(w, st);
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
