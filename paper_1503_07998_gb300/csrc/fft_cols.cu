// Column passes of the Fourier route (Supp. Note 2 sec. 4): FM (column FFT
// of the estimate's row spectra, product with each view's PSF spectrum,
// inverse column FFT) and C (column FFT of each view's ratio spectra,
// product with the conjugate spectrum, inverse column FFT).  A CTA holds a
// block of CB adjacent spectrum columns of one plane (rows at the plane's H,
// zero rows up to Ly filled in shared memory); each warp transforms one of
// them.  Block loads and stores are cooperative (runs of CB columns along
// the rows); the PSF spectra are stored column by column, so that each warp
// reads its own column contiguously.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fft_engine.cuh"
#include "mvd_internal.h"

namespace mvd {
namespace fftr {

namespace {

constexpr int kWarps = 8;                // columns per CTA at most
constexpr int kThreads = 32 * kWarps;
constexpr size_t kSmemCap = 227 * 1024;
constexpr int kBatch = 8;
constexpr int kPlanBytes = 128;
static_assert(sizeof(FftPlan1) <= kPlanBytes, "plan copy");

enum ColMode { COL_BLUR = 0, COL_CORR = 1 };

// Column pitch: Ly rounded up to 2 mod 16 (8-byte words), so that the
// cooperative accesses (CB columns x 2 rows per half-warp) hit distinct banks.
__host__ __device__ inline int col_pitch(int Ly) { return Ly + ((2 - Ly % 16) + 16) % 16; }

template <int MODE>
__global__ void __launch_bounds__(kThreads) fft_cols_kernel(const FftArgs a, int nblk) {
    extern __shared__ __align__(16) unsigned char smem[];
    FftPlan1 *pl = reinterpret_cast<FftPlan1 *>(smem);
    float2 *tw = reinterpret_cast<float2 *>(smem + kPlanBytes);
    const int twl = (a.py.tw_len + 1) & ~1;
    const int CB = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Ly = a.Ly, LD = col_pitch(Ly);
    float2 *b0 = tw + twl, *b1 = b0 + CB * LD, *b2 = b1 + CB * LD;
    if (threadIdx.x == 0) *pl = a.py;
    for (int i = threadIdx.x; i < a.py.tw_len; i += blockDim.x) tw[i] = a.tw_y[i];

    const long long srow = a.LcP, splane = static_cast<long long>(a.H) * srow;
    const long long items = static_cast<long long>(a.P) * nblk;
    const int nthr = blockDim.x;
    // idx / CB as a multiply-high by ceil(2^32 / CB): exact for CB <= 8 and
    // idx < 2^32 / 7 (a block holds at most Ly * CB elements)
    const unsigned cb_magic = CB > 1 ? static_cast<unsigned>((0x100000000ull + CB - 1) / CB) : 0u;
    auto row_of = [&](int idx) -> int { return CB > 1 ? static_cast<int>(__umulhi(static_cast<unsigned>(idx), cb_magic)) : idx; };

    // rows < H of the block's columns into dst (column c at dst + c LD), zero beyond
    auto load = [&](const float2 *src, float2 *dst, int c0) {
        for (int idx0 = threadIdx.x; idx0 < Ly * CB; idx0 += kBatch * nthr) {
            float2 v[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int idx = idx0 + u * nthr, r = row_of(idx), c = idx - r * CB;
                v[u] = make_float2(0.f, 0.f);
                if (idx < Ly * CB && r < a.H && c0 + c < a.Lc) v[u] = src[r * srow + c0 + c];
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int idx = idx0 + u * nthr, r = row_of(idx), c = idx - r * CB;
                if (idx < Ly * CB) dst[c * LD + r] = v[u];
            }
        }
    };
    auto store = [&](const float2 *src, float2 *dst, int c0) {   // rows < H
        for (int idx = threadIdx.x; idx < a.H * CB; idx += nthr) {
            const int r = row_of(idx), c = idx - r * CB;
            if (c0 + c < a.Lc) dst[r * srow + c0 + c] = src[c * LD + r];
        }
    };
    // w[r] = s[r] * h[r] (or * conj h[r]) down the warp's column
    auto mul = [&](const float2 *s, float2 *w, const float2 *h, bool conj) {
        for (int r0 = lane; r0 < Ly; r0 += 32 * kBatch) {
            float2 hv[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int r = r0 + 32 * u;
                hv[u] = r < Ly ? __ldg(h + r) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int r = r0 + 32 * u;
                if (r < Ly) w[r] = conj ? cmulc(s[r], hv[u]) : cmul(s[r], hv[u]);
            }
        }
    };

    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int p = static_cast<int>(it / nblk);
        const int c0 = static_cast<int>(it - static_cast<long long>(p) * nblk) * CB;
        const int col = c0 + warp;
        const bool live = col < a.Lc;
        const size_t hoff = static_cast<size_t>(live ? col : 0) * Ly;
        // A transform started in buffer X with scratch Y ends in X after an
        // even number of stages and in Y after an odd one: the same buffer
        // for every warp, which the cooperative stores rely on.
        const bool odd = a.py.nst & 1;
        if (MODE == COL_BLUR) {
            load(a.S0 + p * splane, b0, c0);
            __syncthreads();
            if (live) fft_warp<false>(b0 + warp * LD, b1 + warp * LD, *pl, tw, lane);
            float2 *Psi = odd ? b1 : b0;
            // several views: the other two buffers do the inverse transforms;
            // one view: Psi . H_v in place, the other buffer as scratch
            const bool three = a.view_hi - a.view_lo > 1;
            float2 *w0 = three ? (odd ? b0 : b1) : Psi, *w1 = three ? b2 : (odd ? b0 : b1);
            float2 *res = odd ? w1 : w0;
            for (int v = a.view_lo; v < a.view_hi; ++v) {
                if (live) {
                    mul(Psi + warp * LD, w0 + warp * LD, a.spec + static_cast<size_t>(v) * a.Lc * Ly + hoff, false);
                    __syncwarp();
                    fft_warp<true>(w0 + warp * LD, w1 + warp * LD, *pl, tw, lane);
                }
                __syncthreads();
                store(res, a.T + (static_cast<long long>(v) * a.P + p) * splane, c0);
                __syncthreads();
            }
        } else {
            float2 *F = odd ? b1 : b0, *G = odd ? b0 : b1;      // forward result and its scratch
            float2 *res = odd ? G : F;
            for (int v = a.view_lo; v < a.view_hi; ++v) {
                float2 *T = a.T + (static_cast<long long>(v) * a.P + p) * splane;
                load(T, b0, c0);
                __syncthreads();
                if (live) {
                    fft_warp<false>(b0 + warp * LD, b1 + warp * LD, *pl, tw, lane);
                    mul(F + warp * LD, F + warp * LD, a.cspec + static_cast<size_t>(v) * a.Lc * Ly + hoff, true);
                    __syncwarp();
                    fft_warp<true>(F + warp * LD, G + warp * LD, *pl, tw, lane);
                }
                __syncthreads();
                store(res, T, c0);
                __syncthreads();
            }
        }
    }
}

}  // namespace

cudaError_t launch_cols(int mode, const FftArgs &a, int sms, cudaStream_t s) {
    const int LD = col_pitch(a.Ly);
    // the blur keeps Psi for every view of the launch: a third buffer only
    // when there is more than one
    const int nbuf = mode == COL_BLUR && a.view_hi - a.view_lo > 1 ? 3 : 2;
    const size_t fixed = kPlanBytes + static_cast<size_t>((a.py.tw_len + 1) & ~1) * sizeof(float2);
    const size_t per_col = static_cast<size_t>(nbuf) * LD * sizeof(float2);
    const int max_cb = static_cast<int>(std::min<size_t>(kWarps, (kSmemCap - fixed) / per_col));
    if (max_cb < 1) return cudaErrorInvalidValue;
    const void *fn = mode == COL_BLUR ? reinterpret_cast<const void *>(fft_cols_kernel<COL_BLUR>)
                                      : reinterpret_cast<const void *>(fft_cols_kernel<COL_CORR>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(fixed + max_cb * per_col));
    if (e != cudaSuccess) return e;
    // columns (warps) per CTA: the count that keeps the most warps resident per SM
    int CB = 0, per_sm = 0;
    for (int w = max_cb; w >= 1; --w) {
        int b = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, 32 * w, fixed + w * per_col)) != cudaSuccess)
            return e;
        if (b * w > per_sm * CB) {
            CB = w;
            per_sm = b;
        }
    }
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = fixed + CB * per_col;
    const int nblk = (a.Lc + CB - 1) / CB;
    const long long items = static_cast<long long>(a.P) * nblk;
    const int grid = static_cast<int>(std::min<long long>(items, static_cast<long long>(per_sm) * std::max(sms, 1)));
    if (grid < 1) return cudaSuccess;
    if (mode == COL_BLUR)
        fft_cols_kernel<COL_BLUR><<<grid, 32 * CB, smem, s>>>(a, nblk);
    else
        fft_cols_kernel<COL_CORR><<<grid, 32 * CB, smem, s>>>(a, nblk);
    return cudaGetLastError();
}

}  // namespace fftr
}  // namespace mvd
