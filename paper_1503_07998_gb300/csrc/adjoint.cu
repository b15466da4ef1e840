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

#include <algorithm>
#include <cstdint>

#include "mvd_internal.h"

namespace mvd {
namespace adj {

namespace {

constexpr int kThreads = 256;   // elementwise kernels and the lag sums
// Register-blocked stencils and lag sums: output tiles of TY x kTX pixels
// (64 x 64, 256 threads); taps and lag rows in chunks of kNB, so every
// shared-memory value a thread loads feeds kNB FMAs whatever K is (the last
// chunk's taps past K are zero).
constexpr int kTX = 64;
constexpr int kNB = 16;
constexpr int kStencilTY = 64;
constexpr int kStencilThreads = kTX * (kStencilTY / kNB);   // one item per thread
constexpr int kLagTY = 64;

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

__host__ __device__ constexpr int n_chunks(int K) { return (K + kNB - 1) / kNB; }
// Halo tile rows: TY + K - 1 input rows, then zero rows up to the chunked
// reach TY + kNB * chunks - 1 (read only against zero taps or dropped lags).
__host__ __device__ constexpr int halo_rows(int TY, int K) { return TY + kNB * n_chunks(K) - 1; }
__host__ __device__ constexpr int halo_cols(int K) { return kTX + K - 1; }
// Floats of the halo tile, rounded up to whole 16-byte quads so that the
// region after it starts 16-byte aligned.
__host__ __device__ constexpr int halo_floats(int TY, int K) {
    return (halo_rows(TY, K) * halo_cols(K) + 3) / 4 * 4;
}

// Halo tile around output tile (y0, x0) of plane `src`: tile[r][c] =
// src(y0 - R + r, x0 - R + c), zero (ZERO boundary) or wrapped (CIRCULAR)
// outside the plane, zero in the rows past TY + K - 1.  NT threads.
template <int TY, int NT>
__device__ __forceinline__ void load_halo(float *tile, const float *__restrict__ src, int y0, int x0, int K, int H,
                                          int W, int circular) {
    const int R = (K - 1) / 2, NC = halo_cols(K), NR = halo_rows(TY, K), valid = TY + K - 1;
    for (int i = threadIdx.x; i < NR * NC; i += NT) {
        const int r = i / NC, c = i - r * NC;
        const int y = y0 - R + r, x = x0 - R + c;
        float v = 0.0f;
        if (r < valid) {
            if (circular) {
                v = src[static_cast<long long>(wrap(y, H)) * W + wrap(x, W)];
            } else if (y >= 0 && y < H && x >= 0 && x < W) {
                v = src[static_cast<long long>(y) * W + x];
            }
        }
        tile[i] = v;
    }
}

// out (=|+=) conv or corr of `in` with one K x K PSF, for every plane:
//   corr: out(y,x) = sum_ij P[i][j] in(y+i-R, x+j-R)
//   conv: out(y,x) = sum_ij P[i][j] in(y-i+R, x-j+R) = corr with P turned by 180 degrees.
// Thread: one column and kNB consecutive output rows.  For every tap column
// j and chunk of kNB tap rows it walks the 2 kNB - 1 input rows in reach,
// each loaded once and multiplied into every output row it touches.
__global__ void __launch_bounds__(kStencilThreads)
stencil_kernel(const float *__restrict__ in, float *__restrict__ out, const float *__restrict__ psf, int K, int H,
               int W, int circular, int correlate, int accumulate) {
    constexpr int TY = kStencilTY;
    extern __shared__ __align__(16) float sm[];
    const int nch = n_chunks(K), KP = kNB * nch, NC = halo_cols(K);
    float *tile = sm;
    float *taps = sm + halo_floats(TY, K);   // [j][KP]: w(i, j), zero for i >= K (16-byte aligned rows)
    const long long plane = static_cast<long long>(H) * W;
    const float *src = in + blockIdx.z * plane;
    float *dst = out + blockIdx.z * plane;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * kTX;
    for (int k = threadIdx.x; k < K * KP; k += kStencilThreads) {
        const int j = k / KP, i = k - j * KP;
        taps[k] = i < K ? (correlate ? psf[i * K + j] : psf[(K - 1 - i) * K + (K - 1 - j)]) : 0.0f;
    }
    load_halo<TY, kStencilThreads>(tile, src, y0, x0, K, H, W, circular);
    __syncthreads();
    const int c = threadIdx.x % kTX, r0 = kNB * (threadIdx.x / kTX);
    float acc[kNB];
#pragma unroll
    for (int r = 0; r < kNB; ++r) acc[r] = 0.0f;
    for (int j = 0; j < K; ++j) {
        for (int ch = 0; ch < nch; ++ch) {
            float t[kNB];
            const float4 *tq = reinterpret_cast<const float4 *>(taps + j * KP + kNB * ch);
#pragma unroll
            for (int q = 0; q < kNB / 4; ++q) {
                const float4 v = tq[q];
                t[4 * q] = v.x;
                t[4 * q + 1] = v.y;
                t[4 * q + 2] = v.z;
                t[4 * q + 3] = v.w;
            }
            const float *col = tile + (r0 + kNB * ch) * NC + c + j;
#pragma unroll
            for (int m = 0; m < 2 * kNB - 1; ++m) {
                const float x = col[m * NC];
#pragma unroll
                for (int r = 0; r < kNB; ++r) {
                    const int i = m - r;
                    if (i >= 0 && i < kNB) acc[r] = fmaf(t[i], x, acc[r]);
                }
            }
        }
    }
    const int x = x0 + c;
    if (x >= W) return;
#pragma unroll
    for (int r = 0; r < kNB; ++r) {
        const int y = y0 + r0 + r;
        if (y < H) {
            const long long o = static_cast<long long>(y) * W + x;
            dst[o] = accumulate ? dst[o] + acc[r] : acc[r];
        }
    }
}

// G[i][j] += sum_planes sum_x g(x) img(x + s*d_ij), d_ij = (i-R, j-R),
// s = +1 (corr form) or -1 (conv form), img zero or wrapped outside the
// plane.  One CTA per (tile, plane) computes the tile's lag sums
//   Hs[i][j] = sum_{y,x in tile} g(y,x) img(y+i-R, x+j-R)
// (s = -1 takes Hs[K-1-i][K-1-j]).  Work unit: one lag column j, a chunk of
// kNB lag rows and a group of the tile's pixel columns; walking a pixel
// column down, each img value feeds kNB lags against a sliding window of
// kNB g values held in registers.  FP32 within a unit, FP64 across units
// (partial sums in shared memory, over the halo tile once it is read) and
// tiles (atomics).
__global__ void __launch_bounds__(kThreads)
lag_sum_kernel(const float *__restrict__ g, const float *__restrict__ img, double *__restrict__ G, int K, int H, int W,
               int circular, int sign) {
    constexpr int TY = kLagTY;
    extern __shared__ __align__(16) float sm[];
    const int nch = n_chunks(K), KP = kNB * nch, NC = halo_cols(K);
    const int items = K * nch;
    const int groups = min(kTX, max(1, kThreads / items));
    const int cpg = (kTX + groups - 1) / groups;
    float *tile = sm;                              // img with halo
    float *gt = tile + halo_floats(TY, K);         // g over the tile [TY][kTX], zero outside the plane
    float *red = tile;                             // [groups][KP][K] partial sums, once the tile is read
    const long long plane = static_cast<long long>(H) * W;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * kTX;
    load_halo<TY, kThreads>(tile, img + blockIdx.z * plane, y0, x0, K, H, W, circular);
    for (int i = threadIdx.x; i < TY * kTX; i += kThreads) {
        const int r = i / kTX, c = i - r * kTX;
        const int y = y0 + r, x = x0 + c;
        gt[i] = (y < H && x < W) ? g[blockIdx.z * plane + static_cast<long long>(y) * W + x] : 0.0f;
    }
    __syncthreads();
    const int u = threadIdx.x;
    const int gq = u / items, item = u - gq * items;
    const int ch = item / K, j = item - ch * K;
    float acc[kNB];
#pragma unroll
    for (int r = 0; r < kNB; ++r) acc[r] = 0.0f;
    if (gq < groups) {
        const int xb = gq * cpg, xe = min(kTX, xb + cpg);
        for (int x = xb; x < xe; ++x) {
            const float *tc = tile + kNB * ch * NC + x + j;   // rows 16ch + m, column x + j
            const float *gc = gt + x;
            float gv[TY];
#pragma unroll
            for (int m = 0; m < TY + kNB - 1; ++m) {
                if (m < TY) gv[m] = gc[m * kTX];
                const float t = tc[m * NC];
#pragma unroll
                for (int r = 0; r < kNB; ++r) {
                    const int y = m - r;   // lag row 16ch + r pairs pixel row y with img row y + 16ch + r
                    if (y >= 0 && y < TY) acc[r] = fmaf(gv[y], t, acc[r]);
                }
            }
        }
    }
    __syncthreads();   // the halo tile is read: its space takes the partial sums
    if (gq < groups) {
#pragma unroll
        for (int r = 0; r < kNB; ++r) red[(gq * KP + kNB * ch + r) * K + j] = acc[r];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K * K; k += kThreads) {
        double s = 0.0;
        for (int q = 0; q < groups; ++q) s += static_cast<double>(red[q * KP * K + k]);
        const int i = k / K, jj = k - i * K;
        atomicAdd(G + (sign > 0 ? k : (K - 1 - i) * K + (K - 1 - jj)), s);
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

int stencil_smem_bytes(int K) { return (halo_floats(kStencilTY, K) + K * kNB * n_chunks(K)) * 4; }

// The partial sums ([groups][KP][K], at most kThreads * kNB floats) reuse the
// halo tile, which is never smaller.
int lag_smem_bytes(int K) { return (halo_floats(kLagTY, K) + kLagTY * kTX) * 4; }
static_assert(kThreads * kNB <= (kLagTY + kNB - 1) * kTX, "partial sums fit the halo tile");

cudaError_t stencil(const float *in, float *out, const float *psf, int K, int H, int W, int P, int circular,
                    int correlate, int accumulate, cudaStream_t s) {
    const int smem = stencil_smem_bytes(K);
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((W + kTX - 1) / kTX, (H + kStencilTY - 1) / kStencilTY, P);
    stencil_kernel<<<grid, kStencilThreads, smem, s>>>(in, out, psf, K, H, W, circular, correlate, accumulate);
    count_launch();
    return cudaGetLastError();
}

cudaError_t lag_sum(const float *g, const float *img, double *G, int K, int H, int W, int P, int circular, int sign,
                    cudaStream_t s) {
    const int smem = lag_smem_bytes(K);
    cudaError_t e = cudaFuncSetAttribute(lag_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((W + kTX - 1) / kTX, (H + kLagTY - 1) / kLagTY, P);
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
