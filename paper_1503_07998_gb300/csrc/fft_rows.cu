// Row passes of the Fourier route (Supp. Note 2 sec. 4): F (estimate rows to
// half spectra), R (inverse rows, ratio, forward rows) and U (inverse rows,
// multiplicative update).  One warp transforms one pair of real rows packed
// as one complex row (a + i b); the two half spectra are separated (and
// rebuilt) through Hermitian symmetry.  Warps take (plane, row pair) items
// in a grid-stride loop; the only CTA barrier is the one after the plan and
// the twiddles are staged into shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fft_engine.cuh"
#include "mvd_internal.h"
#include "tma.cuh"

namespace mvd {
namespace fftr {

namespace {

constexpr int kWarps = 8;                // at most; fewer when the rows are long
constexpr int kThreads = 32 * kWarps;
constexpr size_t kSmemCap = 227 * 1024;
// Element loops issue kBatch global loads into registers before the batch's
// shared-memory stores, so that several loads are in flight per lane.
constexpr int kBatch = 8;
constexpr int kPlanBytes = 128;
static_assert(sizeof(FftPlan1) <= kPlanBytes, "plan copy");

enum RowMode { ROW_PSI = 0, ROW_RATIO = 1, ROW_UPDATE = 2 };

__device__ __forceinline__ float data_at(const void *phi, int u16, long long i) {
    return u16 ? static_cast<float>(__ldg(static_cast<const uint16_t *>(phi) + i))
               : __ldg(static_cast<const float *>(phi) + i);
}

__host__ __device__ inline int buf_len(int Lx) { return (Lx + 1) & ~1; }

// Rebuild the full spectrum of the packed row pair (y0, y0 + 1) from their
// stored half spectra: Z_k = A_k + i B_k with A_{L-k} = conj(A_k).
__device__ __forceinline__ void load_pair_spectrum(const FftArgs &a, const float2 *T, int y0, bool have1,
                                                   float2 *x, int lane) {
    const int Lx = a.Lx, Lc = a.Lc;
    const long long srow = a.LcP;
    const float2 *r0 = T + y0 * srow, *r1 = r0 + srow;
    for (int k0 = lane; k0 < Lx; k0 += 32 * kBatch) {
        float2 A[kBatch], B[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int k = k0 + 32 * u;
            A[u] = B[u] = make_float2(0.f, 0.f);
            if (k < Lx) {
                const int kk = k < Lc ? k : Lx - k;
                A[u] = r0[kk];
                if (have1) B[u] = r1[kk];
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int k = k0 + 32 * u;
            if (k >= Lx) continue;
            if (k >= Lc) {
                A[u].y = -A[u].y;
                B[u].y = -B[u].y;
            }
            x[k] = make_float2(A[u].x - B[u].y, A[u].y + B[u].x);
        }
    }
}

// Separate the packed transform Z of rows (y0, y0 + 1) into their half
// spectra and store them: A_k = (Z_k + conj Z_{L-k}) / 2, B_k = (Z_k - conj Z_{L-k}) / (2i).
__device__ __forceinline__ void store_pair_spectrum(const FftArgs &a, const float2 *Z, float2 *dst, int y0,
                                                    bool have1, int lane) {
    const int Lx = a.Lx;
    const long long srow = a.LcP;
    float2 *r0 = dst + y0 * srow, *r1 = r0 + srow;
    for (int k = lane; k < a.Lc; k += 32) {
        const float2 z = Z[k], zc = Z[k == 0 ? 0 : Lx - k];
        r0[k] = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
        if (have1) r1[k] = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) fft_rows_kernel(const FftArgs a, int pairs, int use_prod) {
    extern __shared__ __align__(16) unsigned char smem[];
    FftPlan1 *pl = reinterpret_cast<FftPlan1 *>(smem);
    float2 *tw = reinterpret_cast<float2 *>(smem + kPlanBytes);
    const int twl = (a.px.tw_len + 1) & ~1;
    const int BL = buf_len(a.Lx);
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *x = tw + twl + static_cast<size_t>(warp) * 2 * BL;
    float2 *y = x + BL;
    float *prod = reinterpret_cast<float *>(tw + twl + static_cast<size_t>(nw) * 2 * BL) + warp * 2 * a.W;
    if (threadIdx.x == 0) *pl = a.px;
    for (int i = threadIdx.x; i < a.px.tw_len; i += blockDim.x) tw[i] = a.tw_x[i];
    __syncthreads();

    const int Lx = a.Lx, W = a.W;
    const long long plane = static_cast<long long>(a.H) * W;
    const long long splane = static_cast<long long>(a.H) * a.LcP;
    const long long items = static_cast<long long>(a.P) * pairs;
    for (long long it = static_cast<long long>(blockIdx.x) * nw + warp; it < items;
         it += static_cast<long long>(gridDim.x) * nw) {
        const int p = static_cast<int>(it / pairs);
        const int y0 = 2 * static_cast<int>(it - static_cast<long long>(p) * pairs);
        const bool have1 = y0 + 1 < a.H;
        const long long o0 = p * plane + static_cast<long long>(y0) * W;
        const long long o1 = o0 + W;
        const float m = a.psi_in ? 0.0f : __ldg(a.means + p);

        if constexpr (MODE == ROW_PSI) {
            for (int i0 = lane; i0 < Lx; i0 += 32 * kBatch) {
                float r0[kBatch], r1[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int i = i0 + 32 * u;
                    r0[u] = r1[u] = 0.0f;
                    if (i < W) {
                        r0[u] = a.psi_in ? __ldg(a.psi_in + o0 + i) : m;
                        if (have1) r1[u] = a.psi_in ? __ldg(a.psi_in + o1 + i) : m;
                    }
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u)
                    if (i0 + 32 * u < Lx) x[i0 + 32 * u] = make_float2(r0[u], r1[u]);
            }
            __syncwarp();
            const float2 *Z = fft_warp<false>(x, y, *pl, tw, lane);
            store_pair_spectrum(a, Z, a.S0 + p * splane, y0, have1, lane);
        } else {
            for (int v = a.view_lo; v < a.view_hi; ++v) {
                float2 *T = a.T + (static_cast<long long>(v) * a.P + p) * splane;
                load_pair_spectrum(a, T, y0, have1, x, lane);
                __syncwarp();
                float2 *z = fft_warp<true>(x, y, *pl, tw, lane);
                float2 *zo = (z == x) ? y : x;
                if constexpr (MODE == ROW_RATIO) {
                    const long long d0 = (static_cast<long long>(v) * a.P + p) * plane + static_cast<long long>(y0) * W;
                    for (int i0 = lane; i0 < Lx; i0 += 32 * kBatch) {
                        float q0[kBatch], q1[kBatch];
#pragma unroll
                        for (int u = 0; u < kBatch; ++u) {
                            const int i = i0 + 32 * u;
                            q0[u] = q1[u] = 0.f;
                            if (i < W) {
                                q0[u] = data_at(a.phi, a.u16, d0 + i);
                                if (have1) q1[u] = data_at(a.phi, a.u16, d0 + W + i);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kBatch; ++u) {
                            const int i = i0 + 32 * u;
                            if (i >= Lx) continue;
                            float r0 = 0.f, r1 = 0.f;
                            if (i < W) {
                                const float2 b = z[i];
                                r0 = __fdiv_rn(q0[u], fmaxf(b.x, a.eps));
                                if (have1) r1 = __fdiv_rn(q1[u], fmaxf(b.y, a.eps));
                            }
                            zo[i] = make_float2(r0, r1);
                        }
                    }
                    __syncwarp();
                    const float2 *Z = fft_warp<false>(zo, z, *pl, tw, lane);
                    store_pair_spectrum(a, Z, T, y0, have1, lane);
                } else if (use_prod) {   // ROW_UPDATE, several views: product of their c_v
                    const bool first = v == a.view_lo;
                    for (int i = lane; i < W; i += 32) {
                        const float2 c = z[i];
                        prod[i] = first ? c.x : prod[i] * c.x;
                        prod[W + i] = first ? c.y : prod[W + i] * c.y;
                    }
                } else {                 // ROW_UPDATE, one view: psi <- psi * c_v
                    for (int i0 = lane; i0 < W; i0 += 32 * kBatch) {
                        float q0[kBatch], q1[kBatch];   // psi (may be psi_out itself: read before written)
#pragma unroll
                        for (int u = 0; u < kBatch; ++u) {
                            const int i = i0 + 32 * u;
                            q0[u] = q1[u] = m;
                            if (i < W && a.psi_in) {
                                q0[u] = a.psi_in[o0 + i];
                                if (have1) q1[u] = a.psi_in[o1 + i];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kBatch; ++u) {
                            const int i = i0 + 32 * u;
                            if (i >= W) continue;
                            const float2 c = z[i];
                            a.psi_out[o0 + i] = q0[u] * c.x;
                            if (have1) a.psi_out[o1 + i] = q1[u] * c.y;
                        }
                    }
                }
                __syncwarp();
            }
            if (MODE == ROW_UPDATE && use_prod) {
                for (int i0 = lane; i0 < W; i0 += 32 * kBatch) {
                    float q0[kBatch], q1[kBatch];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const int i = i0 + 32 * u;
                        q0[u] = q1[u] = m;
                        if (i < W && a.psi_in) {
                            q0[u] = a.psi_in[o0 + i];
                            if (have1) q1[u] = a.psi_in[o1 + i];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const int i = i0 + 32 * u;
                        if (i >= W) continue;
                        a.psi_out[o0 + i] = q0[u] * prod[i];
                        if (have1) a.psi_out[o1 + i] = q1[u] * prod[W + i];
                    }
                }
            }
        }
        __syncwarp();
    }
}

// Row passes with every job's inputs prefetched.  A job is (row pair,
// view) for the ratio pass and a row pair for the others; its inputs are the
// two stored half-spectrum rows (ratio, update) and two rows of the data
// (ratio) or of the estimate (update, estimate; none on the first
// iteration, which starts from the plane means).  Lane 0 of each warp copies
// the next job's rows into the warp's staging buffers with bulk async copies
// (one per row pair) as soon as the current job has consumed them, so they
// land while the warp transforms; each buffer has its own mbarrier.  Waits
// are bounded: an expired wait sets the status word, and the warp drains its
// copies in flight and stops.  Taken when those rows are whole 16-byte units
// and, for the update, when a launch has one view (no product buffer).
constexpr int kBarBytes = kWarps * 16;
constexpr long long kDrainBudget = 4000000000LL;

__host__ __device__ inline int rup16(int b) { return (b + 15) & ~15; }

template <int MODE>
__global__ void __launch_bounds__(kThreads) fft_rows_pf_kernel(const FftArgs a, int pairs, int es) {
    constexpr bool kUsesT = MODE != ROW_PSI;
    extern __shared__ __align__(16) unsigned char smem[];
    FftPlan1 *pl = reinterpret_cast<FftPlan1 *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kPlanBytes);
    float2 *tw = reinterpret_cast<float2 *>(smem + kPlanBytes + kBarBytes);
    const int twl = (a.px.tw_len + 1) & ~1;
    const int Lx = a.Lx, W = a.W, Lc = a.Lc;
    const int BL = buf_len(Lx), SL = kUsesT ? 2 * a.LcP : 0, PB = rup16(2 * W * es);
    const size_t per_warp = static_cast<size_t>(2 * BL + SL) * sizeof(float2) + PB;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wb = reinterpret_cast<unsigned char *>(tw + twl) + warp * per_warp;
    float2 *x = reinterpret_cast<float2 *>(wb);
    float2 *y = x + BL;
    float2 *st = y + BL;                                              // staged half spectra, 2 rows of LcP
    unsigned char *ph = reinterpret_cast<unsigned char *>(st + SL);   // staged data / estimate, 2 rows of W
    uint64_t *barT = bars + 2 * warp, *barP = barT + 1;
    if (threadIdx.x == 0) *pl = a.px;
    for (int i = threadIdx.x; i < a.px.tw_len; i += blockDim.x) tw[i] = a.tw_x[i];
    if (lane == 0) {
        tma::mbar_init(barT, 1);
        tma::mbar_init(barP, 1);
        tma::fence_barrier_init();
    }
    __syncthreads();

    const long long plane = static_cast<long long>(a.H) * W;
    const long long splane = static_cast<long long>(a.H) * a.LcP;
    const long long items = static_cast<long long>(a.P) * pairs;
    const long long stride = static_cast<long long>(gridDim.x) * nw;
    const long long first = static_cast<long long>(blockIdx.x) * nw + warp;
    const int v_hi = MODE == ROW_RATIO ? a.view_hi : a.view_lo + 1;   // one job per row pair otherwise
    const bool usesP = MODE == ROW_RATIO || a.psi_in != nullptr;
    // lane 0: copy job (it, v)'s half-spectrum rows and/or its other rows
    auto issue = [&](long long it, int v, bool rows_T, bool rows_P) {
        if (lane != 0) return;
        const int p = static_cast<int>(it / pairs);
        const int y0 = 2 * static_cast<int>(it - static_cast<long long>(p) * pairs);
        const int nr = y0 + 1 < a.H ? 2 : 1;
        const long long vp = static_cast<long long>(v) * a.P + p;
        if (rows_T) {
            const uint32_t bytes = static_cast<uint32_t>(nr * a.LcP * sizeof(float2));
            tma::fence_proxy_async_smem();
            tma::mbar_arrive_expect_tx(barT, bytes);
            tma::bulk_g2s(st, a.T + vp * splane + static_cast<long long>(y0) * a.LcP, bytes, barT);
        }
        if (rows_P) {
            const uint32_t bytes = static_cast<uint32_t>(nr * W * es);
            const unsigned char *src =
                MODE == ROW_RATIO
                    ? static_cast<const unsigned char *>(a.phi) + (vp * plane + static_cast<long long>(y0) * W) * es
                    : reinterpret_cast<const unsigned char *>(a.psi_in + p * plane + static_cast<long long>(y0) * W);
            tma::fence_proxy_async_smem();
            tma::mbar_arrive_expect_tx(barP, bytes);
            tma::bulk_g2s(ph, src, bytes, barP);
        }
    };
    const long long budget = a.wait_budget < 0 ? kDrainBudget : a.wait_budget;
    uint32_t phT = 0, phP = 0;
    bool pendT = false, pendP = false;
    // every lane waits; false after an expired (or injected) timeout, with the
    // warp's copies in flight drained
    auto wait = [&](uint64_t *bar, uint32_t &pha, bool &pend) -> bool {
        const bool ok = tma::mbar_wait_bounded(bar, pha, budget) && a.wait_budget >= 0;
        if (__all_sync(0xffffffffu, ok)) {
            pend = false;
            pha ^= 1u;
            return true;
        }
        if (lane == 0) atomicOr(a.err, kDevTimeout);
        if (pendT) tma::mbar_wait_bounded(barT, phT, kDrainBudget);
        if (pendP) tma::mbar_wait_bounded(barP, phP, kDrainBudget);
        return false;
    };
    auto staged = [&](int i) -> float {   // element i of the staged data / estimate rows
        return es == 2 ? static_cast<float>(reinterpret_cast<const uint16_t *>(ph)[i])
                       : reinterpret_cast<const float *>(ph)[i];
    };
    if (first < items) {
        issue(first, a.view_lo, kUsesT, usesP);
        pendT = kUsesT;
        pendP = usesP;
    }
    for (long long it = first; it < items; it += stride) {
        const int p = static_cast<int>(it / pairs);
        const int y0 = 2 * static_cast<int>(it - static_cast<long long>(p) * pairs);
        const bool have1 = y0 + 1 < a.H;
        const float m = a.psi_in ? 0.0f : __ldg(a.means + p);
        for (int v = a.view_lo; v < v_hi; ++v) {
            long long nit = it;
            int nv = v + 1;
            if (nv >= v_hi) {
                nit = it + stride;
                nv = a.view_lo;
            }
            const bool next = nit < items;
            if constexpr (MODE == ROW_PSI) {
                // the two estimate rows -> forward row FFT -> half spectra S0
                if (usesP && !wait(barP, phP, pendP)) return;
                for (int i = lane; i < Lx; i += 32) {
                    float r0 = 0.f, r1 = 0.f;
                    if (i < W) {
                        r0 = usesP ? staged(i) : m;
                        if (have1) r1 = usesP ? staged(W + i) : m;
                    }
                    x[i] = make_float2(r0, r1);
                }
                __syncwarp();
                if (next && usesP) {
                    issue(nit, nv, false, true);
                    pendP = true;
                }
                const float2 *Z = fft_warp<false>(x, y, *pl, tw, lane);
                store_pair_spectrum(a, Z, a.S0 + p * splane, y0, have1, lane);
            } else {
                float2 *T = a.T + (static_cast<long long>(v) * a.P + p) * splane;
                // half spectra -> full spectrum of the packed pair
                if (!wait(barT, phT, pendT)) return;
                for (int k = lane; k < Lx; k += 32) {
                    const int kk = k < Lc ? k : Lx - k;
                    float2 A = st[kk], B = have1 ? st[a.LcP + kk] : make_float2(0.f, 0.f);
                    if (k >= Lc) {
                        A.y = -A.y;
                        B.y = -B.y;
                    }
                    x[k] = make_float2(A.x - B.y, A.y + B.x);
                }
                __syncwarp();
                if (next) {
                    issue(nit, nv, true, false);
                    pendT = true;
                }
                float2 *z = fft_warp<true>(x, y, *pl, tw, lane);
                if (usesP && !wait(barP, phP, pendP)) return;   // the data (ratio) or estimate (update) rows
                if constexpr (MODE == ROW_RATIO) {
                    float2 *zo = (z == x) ? y : x;
                    for (int i = lane; i < Lx; i += 32) {
                        float r0 = 0.f, r1 = 0.f;
                        if (i < W) {
                            const float2 b = z[i];
                            r0 = __fdiv_rn(staged(i), fmaxf(b.x, a.eps));
                            if (have1) r1 = __fdiv_rn(staged(W + i), fmaxf(b.y, a.eps));
                        }
                        zo[i] = make_float2(r0, r1);
                    }
                    __syncwarp();
                    if (next) {
                        issue(nit, nv, false, true);
                        pendP = true;
                    }
                    const float2 *Z = fft_warp<false>(zo, z, *pl, tw, lane);
                    store_pair_spectrum(a, Z, T, y0, have1, lane);
                } else {   // ROW_UPDATE, one view: psi <- psi * c_v
                    const long long o0 = p * plane + static_cast<long long>(y0) * W;
                    for (int i = lane; i < W; i += 32) {
                        const float2 c = z[i];
                        a.psi_out[o0 + i] = (usesP ? staged(i) : m) * c.x;
                        if (have1) a.psi_out[o0 + W + i] = (usesP ? staged(W + i) : m) * c.y;
                    }
                    __syncwarp();
                    if (next && usesP) {   // the next row pair's estimate rows
                        issue(nit, nv, false, true);
                        pendP = true;
                    }
                }
            }
            __syncwarp();
        }
    }
}

}  // namespace

// The prefetching row passes (rows in whole 16-byte units).
cudaError_t launch_rows_pf(int mode, const FftArgs &a, int sms, cudaStream_t s) {
    const int pairs = (a.H + 1) / 2;
    const int es = mode == ROW_RATIO ? (a.u16 ? 2 : 4) : 4;
    const int SL = mode == ROW_PSI ? 0 : 2 * a.LcP;
    const size_t fixed = kPlanBytes + kBarBytes + static_cast<size_t>((a.px.tw_len + 1) & ~1) * sizeof(float2);
    const size_t per_warp = static_cast<size_t>(2 * buf_len(a.Lx) + SL) * sizeof(float2) + rup16(2 * a.W * es);
    const int max_nw = static_cast<int>(std::min<size_t>(kWarps, (kSmemCap - fixed) / per_warp));
    if (max_nw < 1) return cudaErrorInvalidValue;
    const void *fn = mode == ROW_PSI     ? reinterpret_cast<const void *>(fft_rows_pf_kernel<ROW_PSI>)
                     : mode == ROW_RATIO ? reinterpret_cast<const void *>(fft_rows_pf_kernel<ROW_RATIO>)
                                         : reinterpret_cast<const void *>(fft_rows_pf_kernel<ROW_UPDATE>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(fixed + max_nw * per_warp));
    if (e != cudaSuccess) return e;
    int nw = 0, per_sm = 0;
    for (int w = max_nw; w >= 1; --w) {
        int b = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, 32 * w, fixed + w * per_warp)) != cudaSuccess)
            return e;
        if (b * w > per_sm * nw) {
            nw = w;
            per_sm = b;
        }
    }
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long items = static_cast<long long>(a.P) * pairs;
    const long long need = (items + nw - 1) / nw;
    const int grid = static_cast<int>(std::min<long long>(need, static_cast<long long>(per_sm) * std::max(sms, 1)));
    if (grid < 1) return cudaSuccess;
    const size_t smem = fixed + nw * per_warp;
    switch (mode) {
        case ROW_PSI: fft_rows_pf_kernel<ROW_PSI><<<grid, 32 * nw, smem, s>>>(a, pairs, es); break;
        case ROW_RATIO: fft_rows_pf_kernel<ROW_RATIO><<<grid, 32 * nw, smem, s>>>(a, pairs, es); break;
        default: fft_rows_pf_kernel<ROW_UPDATE><<<grid, 32 * nw, smem, s>>>(a, pairs, es); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_rows(int mode, const FftArgs &a, int sms, cudaStream_t s) {
    const int pairs = (a.H + 1) / 2;
    // prefetching passes where every staged row is a whole number of 16-byte units
    const bool psi_ok = a.psi_in == nullptr || (a.W % 4 == 0 && reinterpret_cast<uintptr_t>(a.psi_in) % 16 == 0);
    const bool pf = a.err != nullptr &&
                    (mode == ROW_RATIO ? (static_cast<long long>(a.W) * (a.u16 ? 2 : 4)) % 16 == 0 &&
                                             reinterpret_cast<uintptr_t>(a.phi) % 16 == 0
                     : mode == ROW_UPDATE ? psi_ok && a.view_hi - a.view_lo == 1
                                          : psi_ok);
    if (pf) return launch_rows_pf(mode, a, sms, s);
    const int use_prod = mode == ROW_UPDATE && a.view_hi - a.view_lo > 1;
    const size_t fixed = kPlanBytes + static_cast<size_t>((a.px.tw_len + 1) & ~1) * sizeof(float2);
    const size_t per_warp = 2ull * buf_len(a.Lx) * sizeof(float2) + (use_prod ? 2ull * a.W * sizeof(float) : 0);
    const int max_nw = static_cast<int>(std::min<size_t>(kWarps, (kSmemCap - fixed) / per_warp));
    if (max_nw < 1) return cudaErrorInvalidValue;
    const void *fn = mode == ROW_PSI     ? reinterpret_cast<const void *>(fft_rows_kernel<ROW_PSI>)
                     : mode == ROW_RATIO ? reinterpret_cast<const void *>(fft_rows_kernel<ROW_RATIO>)
                                         : reinterpret_cast<const void *>(fft_rows_kernel<ROW_UPDATE>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(fixed + max_nw * per_warp));
    if (e != cudaSuccess) return e;
    // warps per CTA: the count that keeps the most warps resident per SM
    // (registers and shared memory both limit the CTAs per SM)
    int nw = 0, per_sm = 0;
    for (int w = max_nw; w >= 1; --w) {
        int b = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, 32 * w, fixed + w * per_warp)) != cudaSuccess)
            return e;
        if (b * w > per_sm * nw) {
            nw = w;
            per_sm = b;
        }
    }
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = fixed + nw * per_warp;
    const long long items = static_cast<long long>(a.P) * pairs;
    const long long need = (items + nw - 1) / nw;
    const int grid = static_cast<int>(std::min<long long>(need, static_cast<long long>(per_sm) * std::max(sms, 1)));
    if (grid < 1) return cudaSuccess;
    switch (mode) {
        case ROW_PSI: fft_rows_kernel<ROW_PSI><<<grid, 32 * nw, smem, s>>>(a, pairs, use_prod); break;
        case ROW_RATIO: fft_rows_kernel<ROW_RATIO><<<grid, 32 * nw, smem, s>>>(a, pairs, use_prod); break;
        default: fft_rows_kernel<ROW_UPDATE><<<grid, 32 * nw, smem, s>>>(a, pairs, use_prod); break;
    }
    return cudaGetLastError();
}

}  // namespace fftr
}  // namespace mvd
