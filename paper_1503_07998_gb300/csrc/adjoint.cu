// PSF calibration: loss and gradient with respect to the PSFs through
// unrolled MV-RL iterations (Supp. Note 1 update equation, simultaneous
// order), computed by a hand-written reverse sweep with checkpoints.
//
// Forward:  psi_0 = per-plane mean;  psi_{t+1} = psi_t * prod_v c_v with
//           b_v = P_v * psi_t,  r_v = phi_v / max(b_v, eps),  c_v = P_v (*) r_v.
// Loss:     L = sum_planes sum_v sum_x [ y_v - phi_v log max(y_v, eps) ],
//           y_v = P_v * psi_T.
// Reverse (given psibar = dL/dpsi_{t+1}), per iteration:
//   psibar_t   = psibar * prod_v c_v
//   cbar_v     = psibar * psi_t * prod_{w != v} c_w
//   rbar_v     = P_v * cbar_v                      (adjoint of the correlation)
//   Pbar_v[k] += sum_x cbar_v(x) r_v(x + d_k)
//   bbar_v     = -rbar_v phi_v / b_v^2  where b_v > eps, else 0
//   psibar_t  += P_v (*) bbar_v                    (adjoint of the convolution)
//   Pbar_v[k] += sum_x bbar_v(x) psi_t(x - d_k)
// with d_k = (i-R, j-R) for tap k = (i, j).  Only psi at every
// `checkpoint_every`-th iteration is kept; each segment is recomputed from
// its checkpoint before it is swept backwards.
//
// The PSFs here are free kernels (full rank in general), so the
// convolutions are direct K x K stencils over shared-memory tiles; the K^2
// lag sums reduce tiles in FP32 and combine across tiles in FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "mvd_internal.h"

namespace mvd {
namespace adj {

namespace {

constexpr int kT = 32;          // output tile side
constexpr int kThreads = 256;   // 8 x 32: each thread 4 rows of one column

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Input tile of side kT + 2R around output tile (y0, x0) of plane `src`.
__device__ __forceinline__ void load_halo(float *tile, const float *__restrict__ src, int y0, int x0, int R, int H,
                                          int W, int circular) {
    const int S = kT + 2 * R;
    for (int i = threadIdx.x; i < S * S; i += kThreads) {
        const int r = i / S, c = i - r * S;
        int y = y0 - R + r, x = x0 - R + c;
        float v = 0.0f;
        if (circular) {
            v = src[static_cast<long long>(wrap(y, H)) * W + wrap(x, W)];
        } else if (y >= 0 && y < H && x >= 0 && x < W) {
            v = src[static_cast<long long>(y) * W + x];
        }
        tile[i] = v;
    }
}

// out (=|+=) conv or corr of `in` with one K x K PSF, for every plane.
//   conv: out(y,x) = sum_ij P[i][j] in(y-i+R, x-j+R)
//   corr: out(y,x) = sum_ij P[i][j] in(y+i-R, x+j-R)
__global__ void __launch_bounds__(kThreads)
stencil_kernel(const float *__restrict__ in, float *__restrict__ out, const float *__restrict__ psf, int K, int H,
               int W, int circular, int correlate, int accumulate) {
    extern __shared__ float sm[];
    const int R = (K - 1) / 2;
    const int S = kT + 2 * R;
    float *tile = sm;
    float *p = sm + S * S;
    const long long plane = static_cast<long long>(H) * W;
    const float *src = in + blockIdx.z * plane;
    float *dst = out + blockIdx.z * plane;
    const int y0 = blockIdx.y * kT, x0 = blockIdx.x * kT;
    for (int i = threadIdx.x; i < K * K; i += kThreads) p[i] = psf[i];
    load_halo(tile, src, y0, x0, R, H, W, circular);
    __syncthreads();
    const int tx = threadIdx.x & 31, ty0 = threadIdx.x >> 5;   // rows ty0, ty0+8, ty0+16, ty0+24
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j < K; ++j) {
            // tile coordinate of the input tap for output row ty: conv -> ty+2R-i, corr -> ty+i
            const float w = correlate ? p[i * K + j] : p[(K - 1 - i) * K + (K - 1 - j)];
            const float *col = tile + i * S + j + tx;
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = fmaf(w, col[(ty0 + 8 * k) * S], acc[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int y = y0 + ty0 + 8 * k, x = x0 + tx;
        if (y < H && x < W) {
            const long long o = static_cast<long long>(y) * W + x;
            dst[o] = accumulate ? dst[o] + acc[k] : acc[k];
        }
    }
}

// G[i][j] += sum_planes sum_x g(x) img(x + s*d_ij), s = +1 (corr form) or -1
// (conv form), img zero or wrapped outside the plane.  One CTA per (tile,
// plane); every thread owns taps k = tid, tid + 256, ...; FP32 per tile,
// FP64 across tiles.
__global__ void __launch_bounds__(kThreads)
lag_sum_kernel(const float *__restrict__ g, const float *__restrict__ img, double *__restrict__ G, int K, int H, int W,
               int circular, int sign) {
    extern __shared__ float sm[];
    const int R = (K - 1) / 2;
    const int S = kT + 2 * R;
    float *tile = sm;               // img with halo
    float *gt = sm + S * S;         // g over the tile (zero outside the plane)
    const long long plane = static_cast<long long>(H) * W;
    const int y0 = blockIdx.y * kT, x0 = blockIdx.x * kT;
    load_halo(tile, img + blockIdx.z * plane, y0, x0, R, H, W, circular);
    for (int i = threadIdx.x; i < kT * kT; i += kThreads) {
        const int r = i / kT, c = i - r * kT;
        const int y = y0 + r, x = x0 + c;
        gt[i] = (y < H && x < W) ? g[blockIdx.z * plane + static_cast<long long>(y) * W + x] : 0.0f;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K * K; k += kThreads) {
        const int i = k / K, j = k - i * K;
        const int dy = sign * (i - R), dx = sign * (j - R);
        const float *base = tile + (R + dy) * S + (R + dx);
        float acc = 0.0f;
        for (int r = 0; r < kT; ++r) {
            const float *gr = gt + r * kT;
            const float *ir = base + r * S;
#pragma unroll 8
            for (int c = 0; c < kT; ++c) acc = fmaf(gr[c], ir[c], acc);
        }
        atomicAdd(G + k, static_cast<double>(acc));
    }
}

__global__ void fill_means_kernel(float *psi, const float *means, long long plane, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) psi[i] = means[i / plane];
}

__device__ __forceinline__ float data_at(const void *phi, int u16, long long i) {
    return u16 ? static_cast<float>(static_cast<const uint16_t *>(phi)[i]) : static_cast<const float *>(phi)[i];
}

// r = phi / max(b, eps)
__global__ void ratio_kernel(const void *phi, int u16, const float *b, float *r, long long n, float eps) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) r[i] = data_at(phi, u16, i) / fmaxf(b[i], eps);
}

// psi_next = psi * prod_v c_v     (c: [V][n])
__global__ void update_kernel(const float *psi, const float *c, float *psi_next, int V, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float prod = 1.0f;
    for (int v = 0; v < V; ++v) prod *= c[v * n + i];
    psi_next[i] = psi[i] * prod;
}

// terminal data fit: loss += y - phi log max(y, eps); ybar = 1 - phi/y (y > eps) else 1
__global__ void terminal_kernel(const void *phi, int u16, const float *y, float *ybar, double *loss, long long n,
                                float eps) {
    __shared__ double red[kThreads / 32];
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    double part = 0.0;
    if (i < n) {
        const float d = data_at(phi, u16, i), yy = y[i];
        part = static_cast<double>(yy) - static_cast<double>(d) * log(static_cast<double>(fmaxf(yy, eps)));
        ybar[i] = yy > eps ? 1.0f - d / yy : 1.0f;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        atomicAdd(loss, s);
    }
}

// psibar_new = psibar * prod_all c;  cbar_v = psibar * psi_t * prod_{w != v} c_w
__global__ void cbar_kernel(const float *psibar, const float *psi_t, const float *c, float *psibar_new, float *cbar,
                            int V, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float pb = psibar[i], ps = psi_t[i];
    float all = 1.0f;
    for (int v = 0; v < V; ++v) all *= c[v * n + i];
    psibar_new[i] = pb * all;
    for (int v = 0; v < V; ++v) {
        float others = 1.0f;
        for (int w = 0; w < V; ++w)
            if (w != v) others *= c[w * n + i];
        cbar[v * n + i] = pb * ps * others;
    }
}

// bbar = -rbar * phi / b^2 where b > eps, else 0
__global__ void bbar_kernel(const void *phi, int u16, const float *rbar, const float *b, float *bbar, long long n,
                            float eps) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float bb = b[i];
    bbar[i] = bb > eps ? -rbar[i] * data_at(phi, u16, i) / (bb * bb) : 0.0f;
}

__global__ void to_float_kernel(const double *G, float *out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = static_cast<float>(G[i]);
}

inline unsigned blocks(long long n) { return static_cast<unsigned>((n + kThreads - 1) / kThreads); }

}  // namespace

int stencil_smem_bytes(int K) {
    const int S = kT + 2 * ((K - 1) / 2);
    return (S * S + K * K) * 4;
}

int lag_smem_bytes(int K) {
    const int S = kT + 2 * ((K - 1) / 2);
    return (S * S + kT * kT) * 4;
}

cudaError_t stencil(const float *in, float *out, const float *psf, int K, int H, int W, int P, int circular,
                    int correlate, int accumulate, cudaStream_t s) {
    const int smem = stencil_smem_bytes(K);
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT, P);
    stencil_kernel<<<grid, kThreads, smem, s>>>(in, out, psf, K, H, W, circular, correlate, accumulate);
    count_launch();
    return cudaGetLastError();
}

cudaError_t lag_sum(const float *g, const float *img, double *G, int K, int H, int W, int P, int circular, int sign,
                    cudaStream_t s) {
    const int smem = lag_smem_bytes(K);
    cudaError_t e = cudaFuncSetAttribute(lag_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT, P);
    lag_sum_kernel<<<grid, kThreads, smem, s>>>(g, img, G, K, H, W, circular, sign);
    count_launch();
    return cudaGetLastError();
}

cudaError_t fill_means(float *psi, const float *means, long long plane, long long n, cudaStream_t s) {
    fill_means_kernel<<<blocks(n), kThreads, 0, s>>>(psi, means, plane, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t ratio(const void *phi, int u16, const float *b, float *r, long long n, float eps, cudaStream_t s) {
    ratio_kernel<<<blocks(n), kThreads, 0, s>>>(phi, u16, b, r, n, eps);
    count_launch();
    return cudaGetLastError();
}

cudaError_t update(const float *psi, const float *c, float *psi_next, int V, long long n, cudaStream_t s) {
    update_kernel<<<blocks(n), kThreads, 0, s>>>(psi, c, psi_next, V, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t terminal(const void *phi, int u16, const float *y, float *ybar, double *loss, long long n, float eps,
                     cudaStream_t s) {
    terminal_kernel<<<blocks(n), kThreads, 0, s>>>(phi, u16, y, ybar, loss, n, eps);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cbar(const float *psibar, const float *psi_t, const float *c, float *psibar_new, float *cb, int V,
                 long long n, cudaStream_t s) {
    cbar_kernel<<<blocks(n), kThreads, 0, s>>>(psibar, psi_t, c, psibar_new, cb, V, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t bbar(const void *phi, int u16, const float *rbar, const float *b, float *bb, long long n, float eps,
                 cudaStream_t s) {
    bbar_kernel<<<blocks(n), kThreads, 0, s>>>(phi, u16, rbar, b, bb, n, eps);
    count_launch();
    return cudaGetLastError();
}

cudaError_t to_float(const double *G, float *out, int n, cudaStream_t s) {
    to_float_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(G, out, n);
    count_launch();
    return cudaGetLastError();
}

}  // namespace adj
}  // namespace mvd
