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
#include "tma.cuh"

namespace mvd {
namespace bq {

namespace {

using fused::Geo;
using fused::kNC;
using fused::kThreads;
constexpr int kTyQ = 32;                 // output tile rows
constexpr int kHeader = 128;             // item slots, barrier, flags
// The current volume's descriptor and (up to kTapCache floats of) factor
// taps live in shared memory while the CTA works on its items.
constexpr int kQvBytes = (static_cast<int>(sizeof(QVol)) + 127) / 128 * 128;
constexpr int kTapCache = 4096;
constexpr int kTileAt = kHeader + kQvBytes + kTapCache * 4;
static_assert(kTileAt % 128 == 0, "TMA destination alignment");
static_assert(sizeof(QVol) % 16 == 0, "descriptor copied as 16-byte words");
constexpr long long kDrainBudget = 4000000000LL;

__device__ __forceinline__ float load_data(const void *phi, int u16, long long i) {
    return u16 ? static_cast<float>(__ldg(static_cast<const uint16_t *>(phi) + i))
               : __ldg(static_cast<const float *>(phi) + i);
}

// Tile [BOX_H][BOX_W] of a plane written inside this launch, for volumes
// without a TMA map (circular boundary, unaligned rows): L2 reads, eight in
// flight per thread before their shared-memory stores.
template <int KC>
__device__ __forceinline__ void load_tile_l2(float *__restrict__ tile, const float *src, int y0, int x0, int H, int W,
                                             int circular) {
    using G = Geo<KC, kTyQ>;
    constexpr int N = G::BOX_H * G::BOX_W;
    constexpr int B = 8;
    for (int i0 = threadIdx.x; i0 < N; i0 += B * kThreads) {
        float r[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int idx = i0 + u * kThreads;
            r[u] = 0.0f;
            if (idx < N) {
                const int row = idx / G::BOX_W;
                int gy = y0 - G::R + row, gx = x0 - G::R4 + (idx - row * G::BOX_W);
                bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
                if (circular) {
                    gy %= H;
                    if (gy < 0) gy += H;
                    gx %= W;
                    if (gx < 0) gx += W;
                    in = true;
                }
                if (in) r[u] = __ldcg(src + static_cast<long long>(gy) * W + gx);
            }
        }
#pragma unroll
        for (int u = 0; u < B; ++u)
            if (i0 + u * kThreads < N) tile[i0 + u * kThreads] = r[u];
    }
}

// The item's input tile into shared memory: the plane's constant first
// estimate, a TMA copy from the volume's map (plane z), or L2 loads.  Every
// thread waits on the copy's barrier; an expired wait flags the status word
// and the batch's abort flag, drains the copy and returns false (uniform).
template <int KC>
__device__ __forceinline__ bool stage_tile(float *tile, uint64_t *bar, uint32_t &phase, volatile int *cta_abort,
                                           const QVol &v, const QParams &qp, const CUtensorMap *map,
                                           const float *src, bool constant, float fill, int z, int y0, int x0) {
    using G = Geo<KC, kTyQ>;
    if (constant) {
        fused::fill_tile_const<KC, kTyQ>(tile, fill, y0, x0, v.H, v.W, v.circular);
    } else if (v.use_tma) {
        if (threadIdx.x == 0) {
            tma::fence_proxy_async_global();
            tma::fence_proxy_async_smem();
            tma::mbar_arrive_expect_tx(bar, G::TILE_BYTES);
            tma::load_3d(tile, map, bar, x0 - G::R4, y0 - G::R, z);
        }
        const long long budget = qp.wait_budget < 0 ? kDrainBudget : qp.wait_budget;
        if (!tma::mbar_wait_bounded(bar, phase, budget)) {
            atomicOr(qp.err, kDevTimeout);
            atomicExch(qp.abort, 1);
            tma::mbar_wait_bounded(bar, phase, kDrainBudget);
            *cta_abort = 1;
        }
        phase ^= 1u;
    } else {
        load_tile_l2<KC>(tile, src, y0, x0, v.H, v.W, v.circular);
    }
    __syncthreads();
    return *cta_abort == 0;
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

// Row-wise epilogue over the 32 x 128 results parked in the staging tile:
// warp w takes rows w, w + 8, ...; lane l columns l, l + 32, l + 64, l + 96,
// so every load and store of a warp is one contiguous 128-byte run.
//   RATIO:  out = phi / max(result, eps)      (out, phi: the view's plane)
//   UPDATE: psi = psi * result, or mean * result on the first update
// The tile's rows of one plane of `base` (es-byte elements) into L2, one
// 128-byte line per thread and step: the item's epilogue reads them after
// its passes.
template <int KC>
__device__ __forceinline__ void prefetch_rows(const void *base, int es, long long plane_off, int y0, int x0, int H,
                                              int W) {
    using G = Geo<KC, kTyQ>;
    const int lpr = (G::TX * es + 127) / 128;   // lines per tile row
    for (int i = threadIdx.x; i < G::TY * lpr; i += kThreads) {
        const int row = i / lpr, x = x0 + (i - row * lpr) * (128 / es), y = y0 + row;
        if (y < H && x < W)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const char *>(base) +
                                                          (plane_off + static_cast<long long>(y) * W + x) * es));
    }
}

template <int KC, bool RATIO>
__device__ __forceinline__ void row_out(const float *__restrict__ stage, const QVol &v, long long plane_off,
                                        int y0, int x0, bool first, float mean) {
    using G = Geo<KC, kTyQ>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < G::TY; r += kThreads / 32) {
        const int y = y0 + r;
        if (y >= v.H) break;
        const long long row = plane_off + static_cast<long long>(y) * v.W;
        float in[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int x = x0 + lane + 32 * e;
            in[e] = 0.0f;
            if (x < v.W) {
                if (RATIO) in[e] = load_data(v.phi, v.u16, row + x);
                else in[e] = first ? mean : __ldcg(v.psi + row + x);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int x = x0 + lane + 32 * e;
            if (x >= v.W) continue;
            const float s = stage[r * G::VB_LD + lane + 32 * e];
            if (RATIO) v.ratio[row + x] = __fdiv_rn(in[e], fmaxf(s, v.eps));
            else v.psi[row + x] = in[e] * s;
        }
    }
}

}  // namespace

namespace {

template <int KC>
__global__ void __launch_bounds__(kThreads, 2) queue_kernel(const __grid_constant__ QParams qp) {
    using G = Geo<KC, kTyQ>;
    static_assert(G::H_PER_THREAD == 1, "one horizontal item per thread");
    extern __shared__ __align__(128) unsigned char smem[];
    // header: the current item (q, segment, go), the tile barrier, the CTA's
    // abort flag, and the next item taken ahead (q, segment, its plane's
    // counter and the count it needs)
    long long *slot = reinterpret_cast<long long *>(smem);
    int *slot_seg = reinterpret_cast<int *>(smem + 8);
    int *slot_ok = reinterpret_cast<int *>(smem + 12);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 16);
    volatile int *cta_abort = reinterpret_cast<volatile int *>(smem + 24);
    long long *next_q = reinterpret_cast<long long *>(smem + 32);
    int *next_seg = reinterpret_cast<int *>(smem + 40);
    int *next_need = reinterpret_cast<int *>(smem + 44);
    const int **next_done = reinterpret_cast<const int **>(smem + 48);
    QVol *vs = reinterpret_cast<QVol *>(smem + kHeader);
    float *taps_s = reinterpret_cast<float *>(smem + kHeader + kQvBytes);
    float *tile = reinterpret_cast<float *>(smem + kTileAt);
    float *stage = tile + G::BOX_H * G::BOX_W;
    constexpr int KS = fused::short_taps<KC>();
    uint32_t phase = 0;
    // One thread of warp 1 takes the next item from the queue while the CTA
    // works on the current one: items come in increasing order, so its
    // segment search starts from the last segment found.
    constexpr int kTaker = 32;
    int sg_cache = 0;
    int cached_vol = -1;
    auto take_next = [&]() {
        const long long q = static_cast<long long>(atomicAdd(qp.head, 1ull));
        *next_q = q;
        if (q >= qp.total) return;
        if (sg_cache + 1 < qp.nseg && qp.segs[sg_cache + 1].start <= q) {
            int lo = sg_cache + 1, hi = qp.nseg - 1;   // last segment starting at or before q
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (qp.segs[mid].start <= q) lo = mid;
                else hi = mid - 1;
            }
            sg_cache = lo;
        }
        const QSeg &seg = qp.segs[sg_cache];
        const QVol &v = qp.vols[seg.vol];
        const int p = static_cast<int>((q - seg.start) / v.tiles);
        *next_seg = sg_cache;
        *next_need = seg.phase * v.tiles;
        *next_done = v.done + p;
    };
    if (threadIdx.x == 0) {
        *cta_abort = 0;
        tma::mbar_init(bar, 1);
        tma::fence_barrier_init();
    }
    if (threadIdx.x == kTaker) take_next();
    __syncthreads();

    for (;;) {
        if (threadIdx.x == 0) {
            const long long q = *next_q;
            int ok = *reinterpret_cast<volatile int *>(qp.abort) == 0;
            if (q < qp.total && ok) ok = wait_counter(*next_done, *next_need, qp);
            *slot = q;
            *slot_seg = *next_seg;
            *slot_ok = ok;
        }
        __syncthreads();
        const long long q = *slot;
        if (q >= qp.total || !*slot_ok) break;
        if (threadIdx.x == kTaker) take_next();
        const QSeg seg = qp.segs[*slot_seg];
        if (seg.vol != cached_vol) {   // uniform: the descriptor and taps of a new volume
            const QVol *g = qp.vols + seg.vol;
            for (int i = threadIdx.x; i < static_cast<int>(sizeof(QVol) / 16); i += kThreads)
                reinterpret_cast<int4 *>(vs)[i] = reinterpret_cast<const int4 *>(g)[i];
            const int nt = g->ntaps;
            if (nt <= kTapCache)
                for (int i = threadIdx.x; i < nt; i += kThreads) taps_s[i] = __ldg(g->taps + i);
            __syncthreads();
            cached_vol = seg.vol;
        }
        const QVol &v = *vs;
        const QVol *vg = qp.vols + seg.vol;
        const float *taps = v.ntaps <= kTapCache ? taps_s : v.taps;
        const long long local = q - seg.start;
        const int p = static_cast<int>(local / v.tiles);
        const int k = static_cast<int>(local - static_cast<long long>(p) * v.tiles);
        const int ty = k / v.tiles_x;
        const int y0 = ty * G::TY, x0 = (k - ty * v.tiles_x) * G::TX;
        const int P = v.P;
        const long long plane = static_cast<long long>(v.H) * v.W;
        const PhaseInfo f = phase_info(v, seg.phase);
        if (f.kind == 0) {
            for (int vv = f.v0; vv < f.v1; ++vv)
                prefetch_rows<KC>(v.phi, v.u16 ? 2 : 4, (static_cast<long long>(vv) * P + p) * plane, y0, x0, v.H, v.W);
        } else if (seg.phase != 1) {
            prefetch_rows<KC>(v.psi, 4, p * plane, y0, x0, v.H, v.W);
        }

        if (f.kind == 0) {   // A: ratio_v = phi_v / max(P_v * psi, eps)
            const bool first = seg.phase == 0;
            if (!stage_tile<KC>(tile, bar, phase, cta_abort, v, qp, &vg->psi_map, v.psi + p * plane, first,
                                first ? __ldg(v.means + p) : 0.0f, p, y0, x0))
                break;
            for (int vv = f.v0; vv < f.v1; ++vv) {
                float acc[1][kNC];
#pragma unroll
                for (int j = 0; j < kNC; ++j) acc[0][j] = 0.0f;
                const unsigned sm = v.short_mask[vv];
                for (int t = 0; t < v.rank[vv]; ++t) {
                    const float *tq = taps + static_cast<long long>(v.tap_off[vv] + t) * 4 * KC;
                    fused::vertical_pass_sel<KC, kTyQ>(sm & 1u, sm & 2u, tile, stage, tq);
                    __syncthreads();
                    if (sm & 2u) fused::horizontal_pass<KC, KS, kTyQ>(stage, tq + KC, acc);
                    else fused::horizontal_pass<KC, KC, kTyQ>(stage, tq + KC, acc);
                    __syncthreads();
                }
                fused::park_items<KC, kTyQ>(stage, acc);
                __syncthreads();
                row_out<KC, true>(stage, v, (static_cast<long long>(vv) * P + p) * plane, y0, x0, false, 0.0f);
                __syncthreads();   // the staging tile is rewritten by the next pass
            }
        } else {             // B: psi <- psi * prod_v (ratio_v correlated with P_v)
            float prod[1][kNC];
#pragma unroll
            for (int j = 0; j < kNC; ++j) prod[0][j] = 1.0f;
            bool dead = false;
            for (int vv = f.v0; vv < f.v1; ++vv) {
                if (!stage_tile<KC>(tile, bar, phase, cta_abort, v, qp, &vg->ratio_map,
                                    v.ratio + (static_cast<long long>(vv) * P + p) * plane, false, 0.0f, vv * P + p,
                                    y0, x0)) {
                    dead = true;
                    break;
                }
                const unsigned sm = v.short_mask[vv];
                if (v.crank[vv] == 1) {
                    const float *tq = taps + static_cast<long long>(v.ctap_off[vv]) * 4 * KC + 2 * KC;
                    fused::vertical_pass_sel<KC, kTyQ>(sm & 4u, sm & 8u, tile, stage, tq);
                    __syncthreads();
                    if (sm & 8u) fused::horizontal_pass_mul<KC, KS, kTyQ>(stage, tq + KC, prod);
                    else fused::horizontal_pass_mul<KC, KC, kTyQ>(stage, tq + KC, prod);
                    __syncthreads();
                } else {
                    float c[1][kNC];
#pragma unroll
                    for (int j = 0; j < kNC; ++j) c[0][j] = 0.0f;
                    for (int t = 0; t < v.crank[vv]; ++t) {
                        const float *tq = taps + static_cast<long long>(v.ctap_off[vv] + t) * 4 * KC + 2 * KC;
                        fused::vertical_pass_sel<KC, kTyQ>(sm & 4u, sm & 8u, tile, stage, tq);
                        __syncthreads();
                        if (sm & 8u) fused::horizontal_pass<KC, KS, kTyQ>(stage, tq + KC, c);
                        else fused::horizontal_pass<KC, KC, kTyQ>(stage, tq + KC, c);
                        __syncthreads();
                    }
#pragma unroll
                    for (int j = 0; j < kNC; ++j) prod[0][j] *= c[0][j];
                }
            }
            if (dead) break;
            // the first update starts from the plane's mean
            const bool first = seg.phase == 1;
            fused::park_items<KC, kTyQ>(stage, prod);
            __syncthreads();
            row_out<KC, false>(stage, v, p * plane, y0, x0, first, first ? __ldg(v.means + p) : 0.0f);
        }
        // publish the tile: every thread's stores (to plain loads and to the
        // TMA copies of later items), then the plane's counter
        tma::fence_proxy_async_global();
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(v.done + p, 1);
    }
}

template <int KC>
cudaError_t launch_class(const QParams &qp, int sms, cudaStream_t s) {
    using G = Geo<KC, kTyQ>;
    const size_t smem = kTileAt + (G::BOX_H * G::BOX_W + G::TY * G::VB_LD) * 4;
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

template <int KC>
void box_of(int *w, int *h) {
    *w = Geo<KC, kTyQ>::BOX_W;
    *h = Geo<KC, kTyQ>::BOX_H;
}

void tile_box(int cls, int *box_w, int *box_h) {
    if (cls == 0) box_of<17>(box_w, box_h);
    else if (cls == 1) box_of<31>(box_w, box_h);
    else box_of<47>(box_w, box_h);
}

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
