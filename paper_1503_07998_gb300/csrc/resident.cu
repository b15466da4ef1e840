// Plane-resident MV-RL (Supp. Note 1 update; every plane independent,
// Results section): one thread-block cluster keeps a plane on chip for all
// iterations, so HBM sees each plane's estimate once on the way in and once
// on the way out, and the data phi_v once per iteration and view.
//
// The C CTAs of a cluster (C <= 16) each hold a strip of `strip` rows x W of
// the plane in shared memory: the estimate psi, the current view's ratio r
// and, in the simultaneous order, the running product of the views'
// corrections.  A 2D convolution is the sum over SVD terms of a vertical
// 1D pass (8 output rows at a time, into a staging tile padded with the
// zero columns of the boundary) and a horizontal 1D pass (16-column items
// in registers).  The vertical pass reads the rows above and below its
// strip straight from the neighbouring CTAs' shared memory (distributed
// shared memory; a table maps each plane row to the CTA and offset that hold
// it, or to zero outside the plane).  Cluster barriers separate the phases:
//   per view v:  r_v = phi_v / max(P_v * psi, eps)       (A, own strip)
//                barrier (every r_v complete)
//                c_v = r_v correlated with P_v; psi *= c_v (sequential)
//                or prod = prod * c_v (simultaneous)     (B, own strip)
//                barrier (halo reads of r_v done)
//   simultaneous: psi *= prod, barrier.
// Factors are padded with zero taps to the launch's size class (17, 31,
// 47), which leaves every sum unchanged; the narrow factors run with their
// short_tap_count central taps like the fused kernels.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fused_common.cuh"
#include "mvd_internal.h"

namespace cg = cooperative_groups;

namespace mvd {
namespace res {

namespace {

constexpr int kThreads = 256;
constexpr int kCR = 8;        // rows per vertical chunk
constexpr int kNC = 16;       // columns per horizontal item
constexpr int kMaxC = 16;     // CTAs per cluster (non-portable above 8)
constexpr size_t kSmemCap = 227 * 1024;

__host__ __device__ constexpr int rup(int a, int b) { return (a + b - 1) / b * b; }
// Staging row pitch: covers the 16 * ceil(W / 16) + KC - 1 columns the
// horizontal items read, rounded to the 16-byte loads they read them with, a
// multiple of 4 floats with an odd number of quads (the 8 rows of a
// quarter-warp's loads then start in distinct bank groups).
__host__ __device__ constexpr int stage_pitch(int W, int KC) {
    const int w = rup(rup(W, kNC) + KC + 3, 4);
    return (w / 4) % 2 == 1 ? w : w + 4;
}

// Row pitch of the strip buffers: W rounded to whole quads, an odd number of
// them, so that the 16-byte stores of the 8 rows of a quarter-warp's items
// hit distinct bank groups.
__host__ __device__ constexpr int strip_pitch(int W) {
    const int w = rup(W, 4);
    return (w / 4) % 2 == 1 ? w : w + 4;
}

struct Layout {
    size_t rows_psi, rows_ratio, taps, psi, prod, ratio, stage, total;
};
__host__ __device__ inline Layout layout(int W, int strip, int KC, int seq, int ntaps) {
    const int R = (KC - 1) / 2;
    Layout L;
    size_t o = 0;
    L.rows_psi = o;
    o += static_cast<size_t>(strip + 2 * R) * sizeof(void *);
    L.rows_ratio = o;
    o += static_cast<size_t>(strip + 2 * R) * sizeof(void *);
    L.taps = o = rup(static_cast<int>(o), 16);
    o += static_cast<size_t>(ntaps) * 4;
    const size_t plane = static_cast<size_t>(strip) * strip_pitch(W) * 4;
    L.psi = o = rup(static_cast<int>(o), 16);
    o += plane;
    L.prod = o;
    if (!seq) o += plane;
    L.ratio = o;
    o += plane;
    L.stage = o;
    o += static_cast<size_t>(kCR) * stage_pitch(W, KC) * 4;
    L.total = o;
    return L;
}

__device__ __forceinline__ float data_at(const void *phi, int u16, long long i) {
    return u16 ? static_cast<float>(__ldg(static_cast<const uint16_t *>(phi) + i))
               : __ldg(static_cast<const float *>(phi) + i);
}

// Columns c0 .. c0+15 of a strip row (16-byte aligned): whole quads inside
// the plane's W columns, single values for a partial last quad, zeros (load)
// or nothing (store) beyond.
__device__ __forceinline__ void store16(float *row, int c0, int W, const float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = c0 + 4 * q;
        if (c + 3 < W) {
            *reinterpret_cast<float4 *>(row + c) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (c + e < W) row[c + e] = v[4 * q + e];
        }
    }
}
__device__ __forceinline__ void load16(const float *row, int c0, int W, float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = c0 + 4 * q;
        if (c + 3 < W) {
            const float4 x = *reinterpret_cast<const float4 *>(row + c);
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[4 * q + e] = c + e < W ? row[c + e] : 0.0f;
        }
    }
}

// Vertical pass of chunk rows r0 .. r0+7 of the strip:
//   stage[i][R + c] = sum_m t[OFF + m] * row(r0 + i - R + OFF + m)[c]
// with rows[j + R] the row j of the strip (j in [-R, strip + R)), in this
// CTA's or a neighbour's shared memory, or nullptr (zero) outside the plane.
template <int KC, int KP>
__device__ __forceinline__ void vpass(const float *const *rows, const float *taps, float *stage, int pitch, int W,
                                      int r0) {
    constexpr int R = (KC - 1) / 2, OFF = (KC - KP) / 2;
    float t[KP];
#pragma unroll
    for (int m = 0; m < KP; ++m) t[m] = taps[OFF + m];
    for (int c = threadIdx.x; c < W; c += kThreads) {
        float acc[kCR];
#pragma unroll
        for (int i = 0; i < kCR; ++i) acc[i] = 0.0f;
#pragma unroll
        for (int m = 0; m < kCR + KP - 1; ++m) {
            const float *rp = rows[r0 + OFF + m];
            const float x = rp ? rp[c] : 0.0f;
#pragma unroll
            for (int i = 0; i < kCR; ++i) {
                const int j = m - i;
                if (j >= 0 && j < KP) acc[i] = fmaf(t[j], x, acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < kCR; ++i) stage[i * pitch + R + c] = acc[i];
    }
}

// Horizontal pass of item (row, g): acc[j] += sum_m t[OFF + m] * stage[row][16 g + OFF + j + m],
// on packed FP32 pairs with 16-byte loads (fused_common.cuh: same products
// and summation order as the scalar form).
template <int KC, int KP>
__device__ __forceinline__ void hpass(const float *stage, const float *taps, int pitch, int row, int g,
                                      float (&acc)[kNC]) {
    constexpr int OFF = (KC - KP) / 2, S = OFF & ~3, D = OFF - S, NIN = kNC + KP - 1 + D;
    float t[KP];
#pragma unroll
    for (int m = 0; m < KP; ++m) t[m] = taps[OFF + m];
    const float4 *src = reinterpret_cast<const float4 *>(stage + row * pitch + g * kNC + S);
    unsigned long long A[kNC / 2];
#pragma unroll
    for (int q = 0; q < kNC / 2; ++q) A[q] = fused::pk2(acc[2 * q], acc[2 * q + 1]);
    fused::hrow_x2<KP, D, NIN>(src, t, A);
#pragma unroll
    for (int q = 0; q < kNC / 2; ++q) fused::upk2(A[q], acc[2 * q], acc[2 * q + 1]);
}

}  // namespace

namespace {

template <int KC>
__global__ void __launch_bounds__(kThreads, 1) resident_kernel(const __grid_constant__ ResArgs a) {
    constexpr int R = (KC - 1) / 2;
    constexpr int KS = short_tap_count(KC);
    cg::cluster_group cl = cg::this_cluster();
    const int me = static_cast<int>(cl.block_rank());
    const int p = blockIdx.y;
    const int W = a.W, H = a.H, S = a.strip;
    const int pitch = stage_pitch(W, KC);
    const Layout L = layout(W, S, KC, a.seq, a.ntaps);
    extern __shared__ __align__(16) unsigned char smem[];
    const float **rows_psi = reinterpret_cast<const float **>(smem + L.rows_psi);
    const float **rows_ratio = reinterpret_cast<const float **>(smem + L.rows_ratio);
    float *taps = reinterpret_cast<float *>(smem + L.taps);
    float *psi = reinterpret_cast<float *>(smem + L.psi);
    float *prod = reinterpret_cast<float *>(smem + L.prod);
    float *ratio = reinterpret_cast<float *>(smem + L.ratio);
    float *stage = reinterpret_cast<float *>(smem + L.stage);
    const long long plane = static_cast<long long>(H) * W;
    const int WP = strip_pitch(W);
    const int g0 = me * S;                       // first plane row of this strip

    // row tables: strip row j (-R <= j < S + R) -> its CTA's buffer, or zero
    for (int j = threadIdx.x; j < S + 2 * R; j += kThreads) {
        const int gy = g0 + j - R;
        const float *rp = nullptr, *rr = nullptr;
        if (gy >= 0 && gy < H) {
            const unsigned owner = static_cast<unsigned>(gy / S);
            const int local = gy - static_cast<int>(owner) * S;
            rp = cl.map_shared_rank(psi, owner) + static_cast<long long>(local) * WP;
            rr = cl.map_shared_rank(ratio, owner) + static_cast<long long>(local) * WP;
        }
        rows_psi[j] = rp;
        rows_ratio[j] = rr;
    }
    for (int i = threadIdx.x; i < a.ntaps; i += kThreads) taps[i] = __ldg(a.taps + i);
    for (int i = threadIdx.x; i < kCR * pitch; i += kThreads) stage[i] = 0.0f;   // zero boundary columns
    // the strip's first estimate
    const float m0 = a.psi_in ? 0.0f : __ldg(a.means + p);
    for (int i = threadIdx.x; i < S * W; i += kThreads) {
        const int r = i / W, c = i - r * W;
        const int gy = g0 + r;
        float v = 0.0f;
        if (gy < H) v = a.psi_in ? __ldg(a.psi_in + p * plane + static_cast<long long>(gy) * W + c) : m0;
        psi[r * WP + c] = v;
    }
    cl.sync();

    const int G = (W + kNC - 1) / kNC;           // horizontal items per row
    const int step = a.seq ? 1 : a.V;
    for (int it = 0; it < a.iters; ++it) {
        for (int v0 = 0; v0 < a.V; v0 += step) {
            for (int v = v0; v < v0 + step; ++v) {
                // A: r_v = phi_v / max(P_v * psi, eps) on this strip
                const long long vplane = (static_cast<long long>(v) * a.P + p) * plane;
                for (int r0 = 0; r0 < S; r0 += kCR) {
                    float acc[kNC];
                    const int row = threadIdx.x % kCR, g = threadIdx.x / kCR;
                    const bool mine = g < G;    // one item per thread up to 256 / 8 = 32 groups
                    // items beyond one per thread: W > 512 is not planned
#pragma unroll
                    for (int j = 0; j < kNC; ++j) acc[j] = 0.0f;
                    for (int q = 0; q < a.rank[v]; ++q) {
                        const float *tq = taps + (a.tap_off[v] + q) * 4 * KC;
                        if (a.short_mask[v] & 1u) vpass<KC, KS>(rows_psi, tq, stage, pitch, W, r0);
                        else vpass<KC, KC>(rows_psi, tq, stage, pitch, W, r0);
                        __syncthreads();
                        if (mine) {
                            if (a.short_mask[v] & 2u) hpass<KC, KS>(stage, tq + KC, pitch, row, g, acc);
                            else hpass<KC, KC>(stage, tq + KC, pitch, row, g, acc);
                        }
                        __syncthreads();
                    }
                    const int lr = r0 + row, gy = g0 + lr;
                    if (mine && lr < S && gy < H) {
                        const long long off = vplane + static_cast<long long>(gy) * W;
                        float d[kNC];
#pragma unroll
                        for (int j = 0; j < kNC; ++j) {
                            const int c = g * kNC + j;
                            d[j] = c < W ? data_at(a.phi, a.u16, off + c) : 0.0f;
                        }
                        float r[kNC];
#pragma unroll
                        for (int j = 0; j < kNC; ++j) r[j] = __fdiv_rn(d[j], fmaxf(acc[j], a.eps));
                        store16(ratio + lr * WP, g * kNC, W, r);
                    }
                }
                cl.sync();   // every strip's ratio is complete (halos of B)
                // B: c_v = r_v correlated with P_v; psi *= c_v or prod *= c_v
                for (int r0 = 0; r0 < S; r0 += kCR) {
                    float acc[kNC];
                    const int row = threadIdx.x % kCR, g = threadIdx.x / kCR;
                    const bool mine = g < G;
#pragma unroll
                    for (int j = 0; j < kNC; ++j) acc[j] = 0.0f;
                    for (int q = 0; q < a.crank[v]; ++q) {
                        const float *tq = taps + (a.ctap_off[v] + q) * 4 * KC + 2 * KC;
                        if (a.short_mask[v] & 4u) vpass<KC, KS>(rows_ratio, tq, stage, pitch, W, r0);
                        else vpass<KC, KC>(rows_ratio, tq, stage, pitch, W, r0);
                        __syncthreads();
                        if (mine) {
                            if (a.short_mask[v] & 8u) hpass<KC, KS>(stage, tq + KC, pitch, row, g, acc);
                            else hpass<KC, KC>(stage, tq + KC, pitch, row, g, acc);
                        }
                        __syncthreads();
                    }
                    const int lr = r0 + row;
                    if (mine && lr < S && g0 + lr < H) {
                        float *row_buf = (a.seq ? psi : prod) + lr * WP;
                        if (a.seq || v != v0) {
                            float old[kNC];
                            load16(row_buf, g * kNC, W, old);
#pragma unroll
                            for (int j = 0; j < kNC; ++j) acc[j] *= old[j];
                        }
                        store16(row_buf, g * kNC, W, acc);
                    }
                }
                cl.sync();   // halo reads of r_v (and, sequential, of psi) are done
            }
            if (!a.seq) {    // simultaneous: psi *= prod_v c_v
                for (int i = threadIdx.x; i < S * WP; i += kThreads) psi[i] *= prod[i];
                cl.sync();
            }
        }
    }
    for (int i = threadIdx.x; i < S * W; i += kThreads) {
        const int r = i / W, c = i - r * W;
        const int gy = g0 + r;
        if (gy < H) a.psi_out[p * plane + static_cast<long long>(gy) * W + c] = psi[r * WP + c];
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

template <int KC>
cudaError_t launch_kc(const ResArgs &a, size_t smem, cudaStream_t s) {
    auto fn = resident_kernel<KC>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess && a.C > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.C, a.P, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg)) != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

}  // namespace

bool plan(int H, int W, int cls, int seq, int ntaps, int *C, int *strip, size_t *smem) {
    if (H < 1 || W < 1 || W > kNC * (kThreads / kCR) || cls < 0 || cls > 2) return false;
    const int KC = cls == 0 ? 17 : (cls == 1 ? 31 : 47);
    int S = std::min(32, rup(H, kCR));
    int c = (H + S - 1) / S;
    if (c > kMaxC) {
        S = rup((H + kMaxC - 1) / kMaxC, kCR);
        c = (H + S - 1) / S;
    }
    if (c > kMaxC) return false;
    const Layout L = layout(W, S, KC, seq, ntaps);
    if (L.total > kSmemCap) return false;
    *C = c;
    *strip = S;
    *smem = L.total;
    return true;
}

cudaError_t launch(const ResArgs &a, int cls, size_t smem, cudaStream_t s) {
    switch (cls) {
        case 0: return launch_kc<17>(a, smem, s);
        case 1: return launch_kc<31>(a, smem, s);
        default: return launch_kc<47>(a, smem, s);
    }
}

}  // namespace res
}  // namespace mvd
