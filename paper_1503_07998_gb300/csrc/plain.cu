// Plain per-plane MV-RL path: one plane at a time and one kernel per step of
// the update (Supp. Note 1): for each view a vertical and a horizontal 1D
// pass per SVD term (or one K x K direct convolution), the ratio, the same
// for the correlation, then the product over views and the update.  Every
// kernel reads its operands straight from global memory, one output pixel
// per thread.  This is the comparison baseline for the fused path; it is
// also the route that needs no factorisation (MVD_ALGO_DIRECT).
#include <cuda_runtime.h>
#include <cstdint>

#include "mvd_internal.h"

namespace mvd {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// out[y][x] (+)= sum_m t[m] * in[y - R + m][x]  (dir 0)  or  in[y][x - R + m]  (dir 1),
// for `planes` consecutive H x W planes
__global__ void __launch_bounds__(kThreads)
pass1d(const float *__restrict__ in, float *__restrict__ out, const float *__restrict__ t, int K, int H,
       int W, int circular, int dir, int accumulate, int planes) {
    const long long plane = static_cast<long long>(H) * W;
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= plane * planes) return;
    const long long pbase = (i / plane) * plane;
    const long long ip = i - pbase;
    in += pbase;
    const int y = static_cast<int>(ip / W);
    const int x = static_cast<int>(ip - static_cast<long long>(y) * W);
    const int R = (K - 1) / 2;
    float s = 0.0f;
    for (int m = 0; m < K; ++m) {
        int yy = y, xx = x;
        if (dir == 0) yy = y - R + m; else xx = x - R + m;
        if (circular) {
            yy = wrap(yy, H);
            xx = wrap(xx, W);
        } else if (yy < 0 || yy >= H || xx < 0 || xx >= W) {
            continue;
        }
        s = fmaf(__ldg(t + m), __ldg(in + static_cast<long long>(yy) * W + xx), s);
    }
    out[i] = accumulate ? out[i] + s : s;
}

// K x K direct: conv  out(y,x) = sum_ij P[i][j] in(y-i+R, x-j+R)
//               corr  out(y,x) = sum_ij P[i][j] in(y+i-R, x+j-R)
__global__ void __launch_bounds__(kThreads)
direct2d(const float *__restrict__ in, float *__restrict__ out, const float *__restrict__ P, int K, int H,
         int W, int circular, int correlate) {
    const long long n = static_cast<long long>(H) * W;
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int y = static_cast<int>(idx / W);
    const int x = static_cast<int>(idx - static_cast<long long>(y) * W);
    const int R = (K - 1) / 2;
    const int sgn = correlate ? 1 : -1;
    float s = 0.0f;
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j < K; ++j) {
            int yy = y + sgn * (i - R), xx = x + sgn * (j - R);
            if (circular) {
                yy = wrap(yy, H);
                xx = wrap(xx, W);
            } else if (yy < 0 || yy >= H || xx < 0 || xx >= W) {
                continue;
            }
            s = fmaf(__ldg(P + i * K + j), __ldg(in + static_cast<long long>(yy) * W + xx), s);
        }
    }
    out[idx] = s;
}

__global__ void __launch_bounds__(kThreads)
fill_kernel(float *__restrict__ dst, const float *__restrict__ means, int plane, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __ldg(means + plane);
}

__global__ void __launch_bounds__(kThreads)
ratio_kernel(const void *__restrict__ phi, int u16, const float *__restrict__ w, const float *__restrict__ blur,
             float *__restrict__ r, long long n, float eps) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d = u16 ? static_cast<float>(static_cast<const uint16_t *>(phi)[i]) : static_cast<const float *>(phi)[i];
    if (w) d *= w[i];
    r[i] = __fdiv_rn(d, fmaxf(blur[i], eps));
}

// c = c / n_v where the footprint reaches a weighted pixel, else 1 (m < 0)
__global__ void __launch_bounds__(kThreads)
apply_norm_kernel(float *__restrict__ c, const float *__restrict__ m, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mi = m[i];
    c[i] = mi >= 0.0f ? c[i] * mi : 1.0f;
}

// footprint n -> 1 / n, or -1 below the floor
__global__ void __launch_bounds__(kThreads)
invert_norm_kernel(float *__restrict__ m, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = m[i];
    m[i] = v >= kNormFloor ? 1.0f / v : -1.0f;
}

__global__ void __launch_bounds__(kThreads)
multiply_kernel(float *__restrict__ acc, const float *__restrict__ c, long long n, int first) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) acc[i] = first ? c[i] : acc[i] * c[i];
}

__global__ void __launch_bounds__(kThreads)
update_kernel(float *__restrict__ psi, const float *__restrict__ prod, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) psi[i] *= prod[i];
}

inline unsigned blocks(long long n) { return static_cast<unsigned>((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t plain_convolve(const PlainArgs &a, int v, int correlate, int direct, const float *in,
                           float *tmp, float *out, cudaStream_t s) {
    const long long n = static_cast<long long>(a.H) * a.W;
    const int K = a.ft.K;
    if (direct) {
        const float *P = (correlate ? a.psf_corr : a.psf_dev) + static_cast<long long>(v) * K * K;
        direct2d<<<blocks(n), kThreads, 0, s>>>(in, out, P, K, a.H, a.W, a.circular, correlate);
        count_launch();
        return cudaGetLastError();
    }
    const int rank = correlate ? a.ft.crank[v] : a.ft.rank[v];
    const int off = correlate ? a.ft.ctap_off[v] : a.ft.tap_off[v];
    for (int q = 0; q < rank; ++q) {
        const float *tq = a.taps + static_cast<long long>(off + q) * 4 * K + (correlate ? 2 * K : 0);
        pass1d<<<blocks(n), kThreads, 0, s>>>(in, tmp, tq, K, a.H, a.W, a.circular, 0, 0, 1);
        pass1d<<<blocks(n), kThreads, 0, s>>>(tmp, out, tq + K, K, a.H, a.W, a.circular, 1, q > 0, 1);
        count_launch(2);
    }
    return cudaGetLastError();
}

cudaError_t plain_fill(float *dst, const float *means, int plane, size_t n, cudaStream_t s) {
    fill_kernel<<<blocks(static_cast<long long>(n)), kThreads, 0, s>>>(dst, means, plane, static_cast<long long>(n));
    count_launch();
    return cudaGetLastError();
}

cudaError_t plain_ratio(const void *phi, int u16, const float *weights, const float *blur, float *ratio, size_t n,
                        float eps, cudaStream_t s) {
    ratio_kernel<<<blocks(static_cast<long long>(n)), kThreads, 0, s>>>(phi, u16, weights, blur, ratio,
                                                                        static_cast<long long>(n), eps);
    count_launch();
    return cudaGetLastError();
}

cudaError_t plain_apply_norm(float *c, const float *wnorm, size_t n, cudaStream_t s) {
    apply_norm_kernel<<<blocks(static_cast<long long>(n)), kThreads, 0, s>>>(c, wnorm, static_cast<long long>(n));
    count_launch();
    return cudaGetLastError();
}

cudaError_t weight_norms(const PlainArgs &a, const float *weights, int P, float *tmp, float *wnorm, cudaStream_t s) {
    const long long plane = static_cast<long long>(a.H) * a.W;
    const long long n = plane * P;
    const int K = a.ft.K;
    for (int v = 0; v < a.ft.views; ++v) {
        const float *w = weights + v * n;
        float *out = wnorm + v * n;
        for (int q = 0; q < a.ft.crank[v]; ++q) {
            const float *tq = a.taps + static_cast<long long>(a.ft.ctap_off[v] + q) * 4 * K + 2 * K;
            pass1d<<<blocks(n), kThreads, 0, s>>>(w, tmp, tq, K, a.H, a.W, a.circular, 0, 0, P);
            pass1d<<<blocks(n), kThreads, 0, s>>>(tmp, out, tq + K, K, a.H, a.W, a.circular, 1, q > 0, P);
            count_launch(2);
        }
        invert_norm_kernel<<<blocks(n), kThreads, 0, s>>>(out, n);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t plain_multiply(float *acc, const float *c, size_t n, int first, cudaStream_t s) {
    multiply_kernel<<<blocks(static_cast<long long>(n)), kThreads, 0, s>>>(acc, c, static_cast<long long>(n), first);
    count_launch();
    return cudaGetLastError();
}

cudaError_t plain_update(float *psi, const float *prod, size_t n, cudaStream_t s) {
    update_kernel<<<blocks(static_cast<long long>(n)), kThreads, 0, s>>>(psi, prod, static_cast<long long>(n));
    count_launch();
    return cudaGetLastError();
}

}  // namespace mvd
