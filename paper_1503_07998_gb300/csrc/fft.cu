// Fourier route of the MV-RL iteration (Supp. Note 2 sec. 4: the
// convolutions are products of spectra), with a hand-written batched
// mixed-radix (4, 2, 3, 5) Stockham FFT in shared memory and the pointwise
// steps fused into the transforms:
//
//   rows  F   real rows of psi (zero beyond the plane) -> half spectra S0
//   cols  FM  S0 -> column FFT -> Psi; per view: Psi . H_v -> inverse column FFT -> T_v
//   rows  R   per view: T_v -> inverse row FFT -> blur b_v -> r_v = phi_v / max(b_v, eps)
//             (zero beyond the plane) -> forward row FFT -> T_v
//   cols  C   per view: T_v -> column FFT -> . conj(H_v) -> inverse column FFT -> T_v
//   rows  U   per view: T_v -> inverse row FFT -> c_v; psi <- psi * prod_v c_v
//
// H_v is the spectrum of view v's PSF wrapped onto the padded grid with its
// centre at the origin, scaled by 1 / (Ly Lx) so that both inverse
// transforms come out normalised; the correlation uses its conjugate.  For
// the ZERO boundary the grid is padded to Ly >= H + R, Lx >= W + R (enough
// for the cyclic product to equal the linear convolution on the plane); for
// CIRCULAR it is the plane itself.  Two real rows travel as one complex row
// (a + i b) and are separated by Hermitian symmetry.  Only the H rows of the
// plane are stored between passes: the padding rows of every real-space
// input are zero, so the column kernels fill them in shared memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "mvd_internal.h"

namespace mvd {
namespace fftr {

namespace {

constexpr int kThreads = 256;
// Element loops issue kBatch global loads into registers before the batch's
// shared-memory stores, so that several loads are in flight per thread
// (stores through generic pointers would otherwise order every load after
// the previous store).
constexpr int kBatch = 4;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// w^e with w = exp(sign * 2 pi i / N), from the table tw[k] = exp(+2 pi i k / N).
template <bool INV>
__device__ __forceinline__ float2 twid(const float2 *tw, int e, int N) {
    const float2 t = tw[e % N];
    return INV ? t : make_float2(t.x, -t.y);
}

// -i*d (forward) or +i*d (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 d) {
    return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
}

// Size-R DFT in registers, exponent sign -1 (forward) or +1 (inverse).  The
// constants are cos/sin of 2 pi/3, 2 pi/5 and 4 pi/5.
template <int R, bool INV>
__device__ __forceinline__ void small_dft(float2 (&a)[R]) {
    if (R == 2) {
        const float2 s = cadd(a[0], a[1]), d = csub(a[0], a[1]);
        a[0] = s;
        a[1] = d;
    } else if (R == 4) {
        const float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
        const float2 s13 = cadd(a[1], a[3]), d13 = rot<INV>(csub(a[1], a[3]));
        a[0] = cadd(s02, s13);
        a[1] = cadd(d02, d13);
        a[2] = csub(s02, s13);
        a[3] = csub(d02, d13);
    } else if (R == 3) {
        constexpr float s3 = 0.8660254037844386f;       // sin(2 pi / 3)
        const float2 t1 = cadd(a[1], a[2]);
        const float2 t2 = rot<INV>(csub(a[1], a[2]));
        const float2 m = make_float2(a[0].x - 0.5f * t1.x, a[0].y - 0.5f * t1.y);
        a[0] = cadd(a[0], t1);
        a[1] = make_float2(m.x + s3 * t2.x, m.y + s3 * t2.y);
        a[2] = make_float2(m.x - s3 * t2.x, m.y - s3 * t2.y);
    } else if (R == 5) {
        constexpr float c1 = 0.30901699437494745f, c2 = -0.8090169943749475f;   // cos(2pi/5), cos(4pi/5)
        constexpr float s1 = 0.9510565162951535f, s2 = 0.5877852522924731f;     // sin(2pi/5), sin(4pi/5)
        const float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
        const float2 t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
        const float2 b1 = make_float2(a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y);
        const float2 b2 = make_float2(a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y);
        const float2 d1 = rot<INV>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
        const float2 d2 = rot<INV>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
        a[0] = cadd(a[0], cadd(t1, t2));
        a[1] = cadd(b1, d1);
        a[4] = csub(b1, d1);
        a[2] = cadd(b2, d2);
        a[3] = csub(b2, d2);
    }
}

// One radix-R stage of the Stockham autosort: p = product of the radices
// before it.  q*k*stride < N, so the twiddle index needs no reduction.
template <int R, bool INV>
__device__ __forceinline__ void fft_stage(const float2 *__restrict__ x, float2 *__restrict__ y, int N, int p,
                                          const float2 *tw, int lane, int nl) {
    const int M = N / R, stride = N / (p * R);
    for (int i = lane; i < M; i += nl) {
        const int k = i % p;
        float2 a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = x[i + q * M];
#pragma unroll
        for (int q = 1; q < R; ++q) {
            const float2 t = tw[q * k * stride];
            a[q] = cmul(a[q], INV ? t : make_float2(t.x, -t.y));
        }
        small_dft<R, INV>(a);
        const int j = (i - k) * R + k;
#pragma unroll
        for (int m = 0; m < R; ++m) y[j + m * p] = a[m];
    }
}

// One transform of length N over x (input) / y (scratch); threads `lane` ..
// step `nl` of a group share it.  Returns the buffer that holds the result.
// Every thread of the CTA must call it with the same N and radix list (the
// stages synchronise the CTA).
template <bool INV>
__device__ float2 *fft_group(float2 *x, float2 *y, int N, const int *rad, int nrad, const float2 *tw, int lane,
                             int nl) {
    int p = 1;
    for (int s = 0; s < nrad; ++s) {
        const int R = rad[s];
        switch (R) {
            case 4: fft_stage<4, INV>(x, y, N, p, tw, lane, nl); break;
            case 2: fft_stage<2, INV>(x, y, N, p, tw, lane, nl); break;
            case 3: fft_stage<3, INV>(x, y, N, p, tw, lane, nl); break;
            default: fft_stage<5, INV>(x, y, N, p, tw, lane, nl); break;
        }
        __syncthreads();
        float2 *t = x;
        x = y;
        y = t;
        p *= R;
    }
    return x;
}

__device__ __forceinline__ float data_at(const void *phi, int u16, long long i) {
    return u16 ? static_cast<float>(static_cast<const uint16_t *>(phi)[i]) : __ldg(static_cast<const float *>(phi) + i);
}

// Row kernels.  A CTA handles NP row pairs of one plane; each pair is one
// complex transform of length Lx done by kThreads/NP threads.
enum RowMode { ROW_PSI = 0, ROW_RATIO = 1, ROW_UPDATE = 2 };

template <int MODE>
__global__ void __launch_bounds__(kThreads) fft_rows_kernel(const FftArgs a, int NP) {
    extern __shared__ float2 sm[];
    const int Lx = a.Lx;
    float2 *tw = sm;
    float2 *bufs = sm + Lx;                       // NP x 2 x Lx
    float *prod = reinterpret_cast<float *>(bufs + 2 * NP * Lx);   // NP x 2 x W (ROW_UPDATE)
    for (int i = threadIdx.x; i < Lx; i += kThreads) tw[i] = a.tw_x[i];
    const int per = kThreads / NP;
    const int g = threadIdx.x / per, lane = threadIdx.x - g * per;
    const int p = blockIdx.y;
    const int y0 = 2 * (blockIdx.x * NP + g);
    const bool have0 = y0 < a.H, have1 = y0 + 1 < a.H;
    float2 *x = bufs + 2 * g * Lx, *y = x + Lx;
    const long long plane = static_cast<long long>(a.H) * a.W;
    const long long srow = static_cast<long long>(a.LcP);
    const long long splane = static_cast<long long>(a.H) * srow;
    __syncthreads();

    if constexpr (MODE == ROW_PSI) {
        const float m = a.psi_in ? 0.0f : __ldg(a.means + p);
        for (int i0 = lane; i0 < Lx; i0 += kBatch * per) {
            float r0[kBatch], r1[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int i = i0 + u * per;
                r0[u] = r1[u] = 0.0f;
                if (i < a.W) {
                    if (have0) r0[u] = a.psi_in ? __ldg(a.psi_in + p * plane + static_cast<long long>(y0) * a.W + i) : m;
                    if (have1)
                        r1[u] = a.psi_in ? __ldg(a.psi_in + p * plane + static_cast<long long>(y0 + 1) * a.W + i) : m;
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                if (i0 + u * per < Lx) x[i0 + u * per] = make_float2(r0[u], r1[u]);
        }
        __syncthreads();
        float2 *Z = fft_group<false>(x, y, Lx, a.rad_x, a.nrad_x, tw, lane, per);
        for (int k = lane; k < a.Lc; k += per) {
            const float2 z = Z[k], zc = Z[(Lx - k) % Lx];
            const float2 A = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
            const float2 B = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
            if (have0) a.S0[p * splane + y0 * srow + k] = A;
            if (have1) a.S0[p * splane + (y0 + 1) * srow + k] = B;
        }
    } else {
        for (int v = a.view_lo; v < a.view_hi; ++v) {
            float2 *T = a.T + (static_cast<long long>(v) * a.P + p) * splane;
            // Hermitian rebuild of the two rows' full spectra into Z = A + iB
            for (int k0 = lane; k0 < Lx; k0 += kBatch * per) {
                float2 A[kBatch], B[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int k = k0 + u * per;
                    A[u] = B[u] = make_float2(0.f, 0.f);
                    if (k < Lx) {
                        const int kk = k < a.Lc ? k : Lx - k;
                        if (have0) A[u] = T[y0 * srow + kk];
                        if (have1) B[u] = T[(y0 + 1) * srow + kk];
                    }
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int k = k0 + u * per;
                    if (k >= Lx) continue;
                    if (k >= a.Lc) {
                        A[u].y = -A[u].y;
                        B[u].y = -B[u].y;
                    }
                    x[k] = make_float2(A[u].x - B[u].y, A[u].y + B[u].x);
                }
            }
            __syncthreads();
            float2 *z = fft_group<true>(x, y, Lx, a.rad_x, a.nrad_x, tw, lane, per);
            float2 *zo = (z == x) ? y : x;
            if (MODE == ROW_RATIO) {
                const long long dbase = (static_cast<long long>(v) * a.P + p) * plane;
                for (int i0 = lane; i0 < Lx; i0 += kBatch * per) {
                    float d0[kBatch], d1[kBatch];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const int i = i0 + u * per;
                        d0[u] = d1[u] = 0.f;
                        if (i < a.W) {
                            if (have0) d0[u] = data_at(a.phi, a.u16, dbase + static_cast<long long>(y0) * a.W + i);
                            if (have1) d1[u] = data_at(a.phi, a.u16, dbase + static_cast<long long>(y0 + 1) * a.W + i);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const int i = i0 + u * per;
                        if (i >= Lx) continue;
                        float r0 = 0.f, r1 = 0.f;
                        if (i < a.W) {
                            const float2 b = z[i];
                            if (have0) r0 = d0[u] / fmaxf(b.x, a.eps);
                            if (have1) r1 = d1[u] / fmaxf(b.y, a.eps);
                        }
                        zo[i] = make_float2(r0, r1);
                    }
                }
                __syncthreads();
                float2 *Z = fft_group<false>(zo, z, Lx, a.rad_x, a.nrad_x, tw, lane, per);
                for (int k = lane; k < a.Lc; k += per) {
                    const float2 q = Z[k], qc = Z[(Lx - k) % Lx];
                    if (have0) T[y0 * srow + k] = make_float2(0.5f * (q.x + qc.x), 0.5f * (q.y - qc.y));
                    if (have1) T[(y0 + 1) * srow + k] = make_float2(0.5f * (q.y + qc.y), -0.5f * (q.x - qc.x));
                }
                __syncthreads();
            } else {   // ROW_UPDATE
                float *pr = prod + 2 * g * a.W;
                const bool first = v == a.view_lo;
                for (int i = lane; i < a.W; i += per) {
                    const float2 c = z[i];
                    pr[i] = first ? c.x : pr[i] * c.x;
                    pr[a.W + i] = first ? c.y : pr[a.W + i] * c.y;
                }
                __syncthreads();
            }
        }
        if (MODE == ROW_UPDATE) {
            const float *pr = prod + 2 * g * a.W;
            const float m = a.psi_in ? 0.0f : __ldg(a.means + p);
            const long long o0 = p * plane + static_cast<long long>(y0) * a.W;
            const long long o1 = o0 + a.W;
            for (int i0 = lane; i0 < a.W; i0 += kBatch * per) {
                float q0[kBatch], q1[kBatch];   // psi (may be psi_out itself: each element is read before written)
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int i = i0 + u * per;
                    q0[u] = q1[u] = m;
                    if (i < a.W && a.psi_in) {
                        if (have0) q0[u] = a.psi_in[o0 + i];
                        if (have1) q1[u] = a.psi_in[o1 + i];
                    }
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int i = i0 + u * per;
                    if (i >= a.W) continue;
                    if (have0) a.psi_out[o0 + i] = q0[u] * pr[i];
                    if (have1) a.psi_out[o1 + i] = q1[u] * pr[a.W + i];
                }
            }
        }
    }
}

// Column kernels.  A CTA handles CB adjacent spectrum columns of one plane.
enum ColMode { COL_FWD_MUL_INV = 0, COL_CORR = 1 };

template <int MODE>
__global__ void __launch_bounds__(kThreads) fft_cols_kernel(const FftArgs a, int CB) {
    extern __shared__ float2 sm[];
    const int Ly = a.Ly, LD = Ly + 1;
    float2 *tw = sm;
    float2 *b0 = sm + Ly, *b1 = b0 + CB * LD, *b2 = b1 + CB * LD;
    for (int i = threadIdx.x; i < Ly; i += kThreads) tw[i] = a.tw_y[i];
    const int per = kThreads / CB;
    const int cl = threadIdx.x / per, lane = threadIdx.x - cl * per;
    const int p = blockIdx.y;
    const int c0 = blockIdx.x * CB;
    const long long srow = a.LcP, splane = static_cast<long long>(a.H) * srow;
    const long long hplane = static_cast<long long>(Ly) * srow;

    auto load = [&](const float2 *src, float2 *dst) {   // rows < H, zero beyond
        for (int idx0 = threadIdx.x; idx0 < Ly * CB; idx0 += kBatch * kThreads) {
            float2 v[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int idx = idx0 + u * kThreads, r = idx / CB, c = idx - r * CB;
                v[u] = make_float2(0.f, 0.f);
                if (idx < Ly * CB && r < a.H && c0 + c < a.Lc) v[u] = src[r * srow + c0 + c];
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int idx = idx0 + u * kThreads, r = idx / CB, c = idx - r * CB;
                if (idx < Ly * CB) dst[c * LD + r] = v[u];
            }
        }
    };
    auto store = [&](const float2 *src, float2 *dst) {  // rows < H
        for (int idx = threadIdx.x; idx < a.H * CB; idx += kThreads) {
            const int r = idx / CB, c = idx - r * CB;
            if (c0 + c < a.Lc) dst[r * srow + c0 + c] = src[c * LD + r];
        }
    };

    if (MODE == COL_FWD_MUL_INV) {
        load(a.S0 + p * splane, b0);
        __syncthreads();
        float2 *col = b0 + cl * LD, *alt = b1 + cl * LD;
        float2 *Psi = fft_group<false>(col, alt, Ly, a.rad_y, a.nrad_y, tw, lane, per);
        // Psi lives in b0 or b1; the other two buffers do the inverse transforms
        float2 *w0 = (Psi == col) ? b1 : b0, *w1 = b2;
        const float2 *psi_base = Psi - cl * LD;
        for (int v = a.view_lo; v < a.view_hi; ++v) {
            const float2 *Hs = a.spec + static_cast<long long>(v) * hplane;
            // columns fastest: each row's CB spectrum values are one coalesced run
            for (int idx0 = threadIdx.x; idx0 < Ly * CB; idx0 += kBatch * kThreads) {
                float2 h[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int idx = idx0 + u * kThreads, r = idx / CB, c = idx - r * CB;
                    h[u] = make_float2(0.f, 0.f);
                    if (idx < Ly * CB && c0 + c < a.Lc) h[u] = __ldg(Hs + r * srow + c0 + c);
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int idx = idx0 + u * kThreads, r = idx / CB, c = idx - r * CB;
                    if (idx < Ly * CB) w0[c * LD + r] = cmul(psi_base[c * LD + r], h[u]);
                }
            }
            __syncthreads();
            float2 *res = fft_group<true>(w0 + cl * LD, w1 + cl * LD, Ly, a.rad_y, a.nrad_y, tw, lane, per);
            store(res - cl * LD, a.T + (static_cast<long long>(v) * a.P + p) * splane);
            __syncthreads();
        }
    } else {
        for (int v = a.view_lo; v < a.view_hi; ++v) {
            float2 *T = a.T + (static_cast<long long>(v) * a.P + p) * splane;
            const float2 *Hs = a.cspec + static_cast<long long>(v) * hplane;
            load(T, b0);
            __syncthreads();
            float2 *F = fft_group<false>(b0 + cl * LD, b1 + cl * LD, Ly, a.rad_y, a.nrad_y, tw, lane, per);
            float2 *Fb = F - cl * LD;
            for (int idx0 = threadIdx.x; idx0 < Ly * CB; idx0 += kBatch * kThreads) {
                float2 h[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int idx = idx0 + u * kThreads, r = idx / CB, c = idx - r * CB;
                    h[u] = make_float2(0.f, 0.f);
                    if (idx < Ly * CB && c0 + c < a.Lc) h[u] = __ldg(Hs + r * srow + c0 + c);
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int idx = idx0 + u * kThreads, r = idx / CB, c = idx - r * CB;
                    if (idx < Ly * CB) Fb[c * LD + r] = cmulc(Fb[c * LD + r], h[u]);
                }
            }
            __syncthreads();
            float2 *o = (Fb == b0) ? b1 : b0;
            float2 *res = fft_group<true>(Fb + cl * LD, o + cl * LD, Ly, a.rad_y, a.nrad_y, tw, lane, per);
            store(res - cl * LD, T);
            __syncthreads();
        }
    }
}

int row_pairs_per_cta(int Lx) { return Lx <= 1024 ? 4 : 2; }
// Four columns per CTA: at Ly = 540 that is 56 KB of shared memory and four
// resident CTAs per SM (eight columns: two), which hides the column loads
// better (89.5 against 92.8 ms for 10 iterations on 512 planes of 512^2).
int cols_per_cta(int) { return 4; }

}  // namespace

// ---- host: sizes, twiddles and PSF spectra ---------------------------------

bool smooth_size(int n, int *out) {
    int best = 0;
    for (long long a = 1; a <= 8192; a *= 2)
        for (long long b = a; b <= 8192; b *= 3)
            for (long long c = b; c <= 8192; c *= 5)
                if (c >= n && (best == 0 || c < best)) best = static_cast<int>(c);
    if (best == 0) return false;
    *out = best;
    return true;
}

bool radix_list(int n, int *rad, int *nrad) {
    int k = 0;
    while (n % 4 == 0) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0) { rad[k++] = 2; n /= 2; }
    while (n % 3 == 0) { rad[k++] = 3; n /= 3; }
    while (n % 5 == 0) { rad[k++] = 5; n /= 5; }
    *nrad = k;
    return n == 1 && k <= kMaxRadices;
}

namespace {

// FP64 host transform (same Stockham recursion), used once per context for
// the PSF spectra.
void host_fft(std::vector<double> &re, std::vector<double> &im, int N, int sign) {
    int rad[kMaxRadices], nrad = 0;
    radix_list(N, rad, &nrad);
    std::vector<double> yr(N), yi(N), c(N), sn(N);
    for (int k = 0; k < N; ++k) {
        c[k] = std::cos(2.0 * M_PI * k / N);
        sn[k] = sign * std::sin(2.0 * M_PI * k / N);
    }
    int p = 1;
    for (int s = 0; s < nrad; ++s) {
        const int R = rad[s], M = N / R, stride = N / (p * R);
        for (int i = 0; i < M; ++i) {
            const int k = i % p;
            double ar[5], ai[5];
            for (int q = 0; q < R; ++q) {
                const double xr = re[i + q * M], xi = im[i + q * M];
                const int e = static_cast<int>((static_cast<long long>(q) * k * stride) % N);
                ar[q] = xr * c[e] - xi * sn[e];
                ai[q] = xr * sn[e] + xi * c[e];
            }
            const int j = (i / p) * p * R + k;
            for (int m = 0; m < R; ++m) {
                double sr = 0, si = 0;
                for (int q = 0; q < R; ++q) {
                    const int e = (q * m * (N / R)) % N;
                    sr += ar[q] * c[e] - ai[q] * sn[e];
                    si += ar[q] * sn[e] + ai[q] * c[e];
                }
                yr[j + m * p] = sr;
                yi[j + m * p] = si;
            }
        }
        re.swap(yr);
        im.swap(yi);
        p *= R;
    }
}

}  // namespace

void twiddles(int N, std::vector<float2> &out) {
    out.resize(N);
    for (int k = 0; k < N; ++k) {
        const double th = 2.0 * M_PI * k / N;
        out[k] = make_float2(static_cast<float>(std::cos(th)), static_cast<float>(std::sin(th)));
    }
}

// Spectrum of a K x K PSF wrapped onto Ly x Lx with its centre at the origin,
// scaled by 1 / (Ly Lx): columns 0 .. Lc-1 of every row, row pitch LcP.
void psf_spectrum(const float *psf, int K, int Ly, int Lx, int Lc, int LcP, std::vector<float2> &out) {
    const int R = (K - 1) / 2;
    std::vector<double> re(static_cast<size_t>(Ly) * Lx, 0.0), im(static_cast<size_t>(Ly) * Lx, 0.0);
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            const int y = ((i - R) % Ly + Ly) % Ly, x = ((j - R) % Lx + Lx) % Lx;
            re[static_cast<size_t>(y) * Lx + x] += psf[i * K + j];
        }
    std::vector<double> r(Lx), m(Lx);
    for (int y = 0; y < Ly; ++y) {       // rows
        for (int x = 0; x < Lx; ++x) {
            r[x] = re[static_cast<size_t>(y) * Lx + x];
            m[x] = im[static_cast<size_t>(y) * Lx + x];
        }
        host_fft(r, m, Lx, -1);
        for (int x = 0; x < Lx; ++x) {
            re[static_cast<size_t>(y) * Lx + x] = r[x];
            im[static_cast<size_t>(y) * Lx + x] = m[x];
        }
    }
    std::vector<double> cr(Ly), ci(Ly);
    out.assign(static_cast<size_t>(Ly) * LcP, make_float2(0.f, 0.f));
    const double scale = 1.0 / (static_cast<double>(Ly) * Lx);
    for (int x = 0; x < Lc; ++x) {       // columns
        for (int y = 0; y < Ly; ++y) {
            cr[y] = re[static_cast<size_t>(y) * Lx + x];
            ci[y] = im[static_cast<size_t>(y) * Lx + x];
        }
        host_fft(cr, ci, Ly, -1);
        for (int y = 0; y < Ly; ++y)
            out[static_cast<size_t>(y) * LcP + x] =
                make_float2(static_cast<float>(cr[y] * scale), static_cast<float>(ci[y] * scale));
    }
}

size_t rows_smem(int Lx, int W) {
    const int NP = row_pairs_per_cta(Lx);
    return (static_cast<size_t>(Lx) + 2ull * NP * Lx) * sizeof(float2) + 2ull * NP * W * sizeof(float);
}

size_t cols_smem(int Ly) {
    const int CB = cols_per_cta(Ly);
    return (static_cast<size_t>(Ly) + 3ull * CB * (Ly + 1)) * sizeof(float2);
}

cudaError_t launch_iteration(const FftArgs &a, cudaStream_t s) {
    const int NP = row_pairs_per_cta(a.Lx), CB = cols_per_cta(a.Ly);
    const size_t rs = rows_smem(a.Lx, a.W), cs = cols_smem(a.Ly);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(fft_rows_kernel<ROW_PSI>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) ||
        (e = cudaFuncSetAttribute(fft_rows_kernel<ROW_RATIO>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) ||
        (e = cudaFuncSetAttribute(fft_rows_kernel<ROW_UPDATE>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)) ||
        (e = cudaFuncSetAttribute(fft_cols_kernel<COL_FWD_MUL_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) ||
        (e = cudaFuncSetAttribute(fft_cols_kernel<COL_CORR>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)))
        return e;
    const int pairs = (a.H + 1) / 2;
    const dim3 rg((pairs + NP - 1) / NP, a.P), cg((a.Lc + CB - 1) / CB, a.P);
    fft_rows_kernel<ROW_PSI><<<rg, kThreads, rs, s>>>(a, NP);
    fft_cols_kernel<COL_FWD_MUL_INV><<<cg, kThreads, cs, s>>>(a, CB);
    fft_rows_kernel<ROW_RATIO><<<rg, kThreads, rs, s>>>(a, NP);
    fft_cols_kernel<COL_CORR><<<cg, kThreads, cs, s>>>(a, CB);
    fft_rows_kernel<ROW_UPDATE><<<rg, kThreads, rs, s>>>(a, NP);
    count_launch(5);
    return cudaGetLastError();
}

}  // namespace fftr
}  // namespace mvd
