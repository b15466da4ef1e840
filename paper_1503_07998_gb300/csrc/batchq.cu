// Persistent batched launch of the fused MV-RL iteration (Supp. Note 1
// update; planes and volumes are independent, Results section): one kernel
// walks a device-side queue of work items covering every iteration of every
// volume of a batch that runs on the separable fused path.
//
// Work item = (phase s of volume j, plane p, output tile k).  The phases of
// a volume are, per iteration, A (blur psi with a view's PSF, ratio
// phi_v / max(blur, eps)) and B (correlate the ratio with the flipped PSF,
// multiply into psi), one pair per view in the sequential order and one pair
// over all views in the simultaneous order.  Items are numbered phase-major
// over the whole batch (all volumes' phase 0, then phase 1, ...), and CTAs
// take them in that order from one atomic counter.  An item of phase s reads
// what phase s - 1 wrote anywhere on its plane (tile halos), so it first waits
// until the plane's counter of finished tiles reaches s * tiles.  Every item
// waited on was taken earlier by a CTA that is running it, so the waits
// always end; they are bounded all the same (the status word reports an
// expired wait and every CTA leaves).
//
// The tile arithmetic is the fused kernels' (fused_common.cuh: vertical and
// horizontal 1D passes per SVD term, 32 x 128 output tiles).  Data written
// inside the launch (the estimate and the ratios) are read through L2 only
// (ld.global.cg), never through the incoherent L1 or read-only paths.  One
// instance per PSF-size class (17, 31, 47): a volume's factors are padded
// with zero taps to its class, which leaves every sum unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "fused_common.cuh"
#include "mvd_internal.h"

namespace mvd {
namespace bq {

namespace {

using fused::Geo;
using fused::kNC;
using fused::kThreads;
constexpr int kTyQ = 32;                 // output tile rows
constexpr int kHeader = 128;             // item slot, flags
constexpr long long kDrainBudget = 4000000000LL;

__device__ __forceinline__ float load_data(const void *phi, int u16, long long i) {
    return u16 ? static_cast<float>(__ldg(static_cast<const uint16_t *>(phi) + i))
               : __ldg(static_cast<const float *>(phi) + i);
}

// Tile [BOX_H][BOX_W] of a plane written inside this launch (L2 reads);
// src == nullptr: the plane's constant first estimate `fill`.
template <int KC>
__device__ __forceinline__ void load_tile_l2(float *__restrict__ tile, const float *src, float fill, int y0, int x0,
                                             int H, int W, int circular) {
    using G = Geo<KC, kTyQ>;
    constexpr int N = G::BOX_H * G::BOX_W;
    for (int idx = threadIdx.x; idx < N; idx += kThreads) {
        const int r = idx / G::BOX_W;
        const int c = idx - r * G::BOX_W;
        int gy = y0 - G::R + r, gx = x0 - G::R4 + c;
        bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        if (circular) {
            gy %= H;
            if (gy < 0) gy += H;
            gx %= W;
            if (gx < 0) gx += W;
            in = true;
        }
        tile[idx] = in ? (src ? __ldcg(src + static_cast<long long>(gy) * W + gx) : fill) : 0.0f;
    }
}

// Phase s of a volume: iteration, views [v0, v1) and kind (0 = A, 1 = B).
struct PhaseInfo {
    int kind, v0, v1;
};
__device__ __forceinline__ PhaseInfo phase_info(const QVol &q, int s) {
    PhaseInfo f;
    f.kind = s & 1;
    if (q.seq) {
        f.v0 = (s >> 1) % q.V;
        f.v1 = f.v0 + 1;
    } else {
        f.v0 = 0;
        f.v1 = q.V;
    }
    return f;
}

// Bounded wait (thread 0) until `counter` reaches `need`; false when the
// budget ran out or another CTA has raised the abort flag.  A negative budget
// reports a timeout once the counter has been reached (fault injection).
__device__ bool wait_counter(const int *counter, int need, const QParams &qp) {
    const volatile int *c = counter;
    const volatile int *ab = qp.abort;
    if (*c >= need && qp.wait_budget >= 0) return true;
    const long long budget = qp.wait_budget < 0 ? kDrainBudget : qp.wait_budget;
    const long long t0 = clock64();
    while (*c < need) {
        if (*ab) return false;
        if (clock64() - t0 > budget) {
            atomicOr(qp.err, kDevTimeout);
            atomicExch(qp.abort, 1);
            return false;
        }
        __nanosleep(64);
    }
    if (qp.wait_budget < 0) {
        atomicOr(qp.err, kDevTimeout);
        atomicExch(qp.abort, 1);
        return false;
    }
    __threadfence();
    return true;
}

}  // namespace

namespace {

template <int KC>
__global__ void __launch_bounds__(kThreads, 2) queue_kernel(const __grid_constant__ QParams qp) {
    using G = Geo<KC, kTyQ>;
    static_assert(G::H_PER_THREAD == 1, "one horizontal item per thread");
    static_assert(kHeader == fused::kTileOffset, "tile placement");
    extern __shared__ __align__(128) unsigned char smem[];
    long long *slot = reinterpret_cast<long long *>(smem);
    int *slot_seg = reinterpret_cast<int *>(smem + 8);
    int *slot_ok = reinterpret_cast<int *>(smem + 12);
    float *tile = reinterpret_cast<float *>(smem + kHeader);
    float *stage = tile + G::BOX_H * G::BOX_W;
    constexpr int KS = fused::short_taps<KC>();

    for (;;) {
        if (threadIdx.x == 0) {
            const long long q = static_cast<long long>(atomicAdd(qp.head, 1ull));
            int ok = *reinterpret_cast<volatile int *>(qp.abort) == 0;
            int sg = 0;
            if (q < qp.total && ok) {
                int lo = 0, hi = qp.nseg - 1;   // last segment starting at or before q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (qp.segs[mid].start <= q) lo = mid;
                    else hi = mid - 1;
                }
                sg = lo;
                const QSeg &seg = qp.segs[sg];
                const QVol &v = qp.vols[seg.vol];
                const int p = static_cast<int>((q - seg.start) / v.tiles);
                ok = wait_counter(v.done + p, seg.phase * v.tiles, qp);
            }
            *slot = q;
            *slot_seg = sg;
            *slot_ok = ok;
        }
        __syncthreads();
        const long long q = *slot;
        if (q >= qp.total || !*slot_ok) break;
        const QSeg seg = qp.segs[*slot_seg];
        const QVol &v = qp.vols[seg.vol];
        const long long local = q - seg.start;
        const int p = static_cast<int>(local / v.tiles);
        const int k = static_cast<int>(local - static_cast<long long>(p) * v.tiles);
        const int ty = k / v.tiles_x;
        const int y0 = ty * G::TY, x0 = (k - ty * v.tiles_x) * G::TX;
        const int H = v.H, W = v.W, P = v.P;
        const long long plane = static_cast<long long>(H) * W;
        const PhaseInfo f = phase_info(v, seg.phase);
        int y, x;
        fused::item_origin<KC, kTyQ>(0, y0, x0, y, x);
        const int n = (y < H && x < W) ? min(kNC, W - x) : 0;

        if (f.kind == 0) {   // A: ratio_v = phi_v / max(P_v * psi, eps)
            const bool first = seg.phase == 0;
            load_tile_l2<KC>(tile, first ? nullptr : v.psi + p * plane, first ? __ldg(v.means + p) : 0.0f, y0,
                             x0, H, W, v.circular);
            __syncthreads();
            for (int vv = f.v0; vv < f.v1; ++vv) {
                float acc[1][kNC];
#pragma unroll
                for (int j = 0; j < kNC; ++j) acc[0][j] = 0.0f;
                const unsigned sm = v.short_mask[vv];
                for (int t = 0; t < v.rank[vv]; ++t) {
                    const float *tq = v.taps + static_cast<long long>(v.tap_off[vv] + t) * 4 * KC;
                    if (sm & 1u) fused::vertical_pass<KC, KS, kTyQ>(tile, stage, tq);
                    else fused::vertical_pass<KC, KC, kTyQ>(tile, stage, tq);
                    __syncthreads();
                    if (sm & 2u) fused::horizontal_pass<KC, KS, kTyQ>(stage, tq + KC, acc);
                    else fused::horizontal_pass<KC, KC, kTyQ>(stage, tq + KC, acc);
                    __syncthreads();
                }
                const long long off = (static_cast<long long>(vv) * P + p) * plane + static_cast<long long>(y) * W + x;
                float d[kNC];
#pragma unroll
                for (int e = 0; e < kNC; ++e) d[e] = e < n ? load_data(v.phi, v.u16, off + e) : 0.0f;
#pragma unroll
                for (int e = 0; e < kNC; ++e)
                    if (e < n) v.ratio[off + e] = __fdiv_rn(d[e], fmaxf(acc[0][e], v.eps));
            }
        } else {             // B: psi <- psi * prod_v (ratio_v correlated with P_v)
            float prod[1][kNC];
#pragma unroll
            for (int j = 0; j < kNC; ++j) prod[0][j] = 1.0f;
            for (int vv = f.v0; vv < f.v1; ++vv) {
                load_tile_l2<KC>(tile, v.ratio + (static_cast<long long>(vv) * P + p) * plane, 0.0f, y0, x0, H, W,
                                 v.circular);
                __syncthreads();
                const unsigned sm = v.short_mask[vv];
                if (v.crank[vv] == 1) {
                    const float *tq = v.taps + static_cast<long long>(v.ctap_off[vv]) * 4 * KC + 2 * KC;
                    if (sm & 4u) fused::vertical_pass<KC, KS, kTyQ>(tile, stage, tq);
                    else fused::vertical_pass<KC, KC, kTyQ>(tile, stage, tq);
                    __syncthreads();
                    if (sm & 8u) fused::horizontal_pass_mul<KC, KS, kTyQ>(stage, tq + KC, prod);
                    else fused::horizontal_pass_mul<KC, KC, kTyQ>(stage, tq + KC, prod);
                    __syncthreads();
                } else {
                    float c[1][kNC];
#pragma unroll
                    for (int j = 0; j < kNC; ++j) c[0][j] = 0.0f;
                    for (int t = 0; t < v.crank[vv]; ++t) {
                        const float *tq = v.taps + static_cast<long long>(v.ctap_off[vv] + t) * 4 * KC + 2 * KC;
                        if (sm & 4u) fused::vertical_pass<KC, KS, kTyQ>(tile, stage, tq);
                        else fused::vertical_pass<KC, KC, kTyQ>(tile, stage, tq);
                        __syncthreads();
                        if (sm & 8u) fused::horizontal_pass<KC, KS, kTyQ>(stage, tq + KC, c);
                        else fused::horizontal_pass<KC, KC, kTyQ>(stage, tq + KC, c);
                        __syncthreads();
                    }
#pragma unroll
                    for (int j = 0; j < kNC; ++j) prod[0][j] *= c[0][j];
                }
            }
            // the first update starts from the plane's mean
            const bool first = seg.phase == 1;
            const long long off = p * plane + static_cast<long long>(y) * W + x;
            const float m = first ? __ldg(v.means + p) : 0.0f;
            float b[kNC];
#pragma unroll
            for (int e = 0; e < kNC; ++e) b[e] = e < n ? (first ? m : __ldcg(v.psi + off + e)) : 0.0f;
#pragma unroll
            for (int e = 0; e < kNC; ++e)
                if (e < n) v.psi[off + e] = b[e] * prod[0][e];
        }
        // publish the tile: every thread's stores, then the plane's counter
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(v.done + p, 1);
    }
}

template <int KC>
cudaError_t launch_class(const QParams &qp, int sms, cudaStream_t s) {
    using G = Geo<KC, kTyQ>;
    const size_t smem = G::SMEM_BYTES;
    cudaError_t e = cudaFuncSetAttribute(queue_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, queue_kernel<KC>, kThreads, smem)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long want = std::min<long long>(qp.total, static_cast<long long>(per_sm) * std::max(sms, 1));
    if (want < 1) return cudaSuccess;
    queue_kernel<KC><<<static_cast<int>(want), kThreads, smem, s>>>(qp);
    return cudaGetLastError();
}

}  // namespace

int size_class(int K) { return K <= 17 ? 0 : (K <= 31 ? 1 : (K <= kFusedMaxK ? 2 : -1)); }
int class_k(int cls) { return cls == 0 ? 17 : (cls == 1 ? 31 : 47); }

cudaError_t launch_queue(int cls, const QParams &qp, int sms, cudaStream_t s) {
    switch (cls) {
        case 0: return launch_class<17>(qp, sms, s);
        case 1: return launch_class<31>(qp, sms, s);
        default: return launch_class<47>(qp, sms, s);
    }
}

}  // namespace bq
}  // namespace mvd
