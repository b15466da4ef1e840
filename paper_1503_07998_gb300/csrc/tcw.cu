// Warp-specialised tensor-core kernels of the fused MV-RL iteration (Supp.
// Note 1 update equation), for launches whose views share one rank-1
// separable PSF factorisation (every launch of the sequential update order;
// for the blur, also views with identical PSFs in a simultaneous one):
//
//   tcw_blur_ratio        r_v = phi_v / max(psi * P, eps)
//   tcw_correlate_update  psi <- psi * (r_v (*) P_v^*)     (one view per launch)
//
// Each 2D convolution is two banded (Toeplitz) matrix products on the
// tcgen05 tensor cores in BF16x3: every FP32 operand x is split into
// hi = bf16(x) and lo = bf16(x - hi), and a product a*b is accumulated in
// FP32 in tensor memory as lo_a hi_b + hi_a lo_b + hi_a hi_b.  The ratio, the
// product over views and the update stay FP32 on the CUDA cores.
//
// Output tile: 128 x 128 pixels of one plane.  M = 128 = the tile's output
// columns x_out (the tensor-memory lane) in both passes:
//   pass 1 (along x): D1[x_out][n] = sum_k T1[x_out][k] B[k][n]
//       k = input column (KH of them), n = input row (KV); A = T1, the
//       horizontal taps' Toeplitz matrix (tensor memory, built once per CTA),
//       B = the input tile (shared memory, K-major, 16 columns per K-step).
//       N = KV <= 176.
//   pass 2 (along y): D2[x_out][y_out] = sum_n A2[x_out][n] T2[n][y_out]
//       A2 = D1 split into BF16 hi/lo in place in tensor memory, B = T2, the
//       vertical taps' Toeplitz matrix (shared memory, built once).  N = 128.
// Tensor memory: T1 (KH columns) + D1/A2 (KV) + D2 (128) <= 480 of 512.
//
// The input tile arrives in one of three ways (the launch's input mode):
//   split     the input was written already split, hi and lo BF16 planes in
//             a column-blocked layout (element (y, x) of a plane at
//             ((x / 8) * H + y) * 8 + x % 8, lo after hi), in which the 16
//             columns of a K-step are two contiguous runs: TMA copies them
//             (1.4 KB pieces) straight into the K-step's B slot (no
//             conversion).  The blur/ratio kernel writes its ratio this way
//             for the correlate/update kernel, which writes a split copy of
//             the estimate (beside the FP32 one) for the next blur.  The
//             split is exactly the one the BF16x3 products use, so nothing
//             changes in the arithmetic.
//   fp32      TMA copies FP32 column chunks (32 columns x KV rows) into a
//             ring, and converter warps split them into the B slots (the
//             first blur of a given initial estimate).
//   constant  the estimate is the plane's mean (the first iteration): the
//             converter warps write its split B slots directly.
//
// Warp roles (18 warps, 576 threads); every hand-off is an mbarrier whose
// waits are bounded (an expired wait sets the device status word, the CTA
// stops, drains its copies and MMAs and frees its tensor memory):
//   warp 16     TMA producer (one thread): B slots (split mode) or FP32
//               chunks (fp32 mode)
//   warps 0-3   converters (fp32 and constant modes)
//   warp 17     MMA issuer (one thread): pass 1 K-step by K-step (each
//               K-step's commit frees its B slot), then pass 2
//   warps 4-7   split D1 into A2 (tensor-memory lane quarter = warp % 4)
//   warps 8-15  epilogue: D2 rows of lane quarter warp % 4 (a block of
//               output rows per warp); ratio or update with coalesced
//               global loads and stores (consecutive lanes, consecutive x)
// One thread's MMAs complete in issue order, so the next tile's pass 1 can
// follow a pass 2 at once: it never overwrites D1 before pass 2 has read it.
//
// HBM traffic per pixel and view of a launch in split mode: the blur reads
// the split estimate (4 B) and phi_v (2 B uint16) and writes the split
// ratio (4 B); the correlation reads the split ratio (4 B) and the FP32
// estimate (4 B) and writes the FP32 and the split estimate (8 B).  Halo
// columns and rows of neighbouring tiles are re-read from L2.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "mvd_internal.h"
#include "tc5.cuh"
#include "tma.cuh"

namespace mvd {
namespace tcw {

namespace {

constexpr int kThreads = 576;
constexpr int kConvWarp0 = 0;    // 4 warps
constexpr int kSplitWarp0 = 4;   // 4 warps
constexpr int kEpiWarp0 = 8;     // 8 warps
constexpr int kTmaWarp = 16;
constexpr int kMmaWarp = 17;
constexpr int kNF = 4;           // FP32 chunk ring slots (fp32 mode)
constexpr int kMaxNB = 8;        // B slots: 8 in split mode, 4 otherwise
constexpr int kTX = 128, kTY = 128;
constexpr uint32_t kTmemCols = 512;
constexpr long long kDrainBudget = 4000000000LL;
constexpr int kMaxK = 47;

// Tile geometry and shared-memory layout (host-computed, in the parameters).
struct Geom {
    int K, R, R8, COL0;
    int KH;              // input columns = pass-1 K (multiple of 16)
    int KV;              // input rows = pass-1 N = pass-2 K (multiple of 16)
    int nb;              // B slots
    uint32_t c_t1lo, c_d1, c_d2;   // tensor-memory columns (T1 hi at 0)
    uint32_t f_bytes;    // FP32 chunk [KV][32]
    uint32_t b_lbo;      // k-group stride of a B slot
    uint32_t bh_bytes;   // hi (or lo) half of a B slot
    uint32_t t2_lbo;     // k-group stride of T2
    uint32_t t2h_bytes;  // hi (or lo) half of T2
    uint32_t off_t2, off_f, off_b, smem_bytes;
};

struct Params {
    CUtensorMap map;   // split: 8-byte {2H, G, 2 planes}, box {KV, 1, 1}; fp32: {W, H, planes}, box {32, KV, 1}
    FusedArgs a;
    TcwIo io;
    Geom g;
    int term;             // factor-table term whose taps this launch uses
    int kind_u, kind_w;   // vertical / horizontal tap kinds (0, 1 blur; 2, 3 correlation)
    int G;                // column blocks of the split layout (W rounded up to 8, / 8)
};

__host__ Geom make_geom(int K, int in_mode) {
    Geom g{};
    g.K = K;
    g.R = (K - 1) / 2;
    g.R8 = (g.R + 7) / 8 * 8;   // tile column origin x0 - R8 on a column block
    g.COL0 = g.R8 - g.R;
    g.KH = (g.COL0 + kTX + 2 * g.R + 15) / 16 * 16;
    g.KV = (kTY + 2 * g.R + 15) / 16 * 16;
    g.c_t1lo = g.KH / 2;
    g.c_d1 = g.KH;
    g.c_d2 = g.KH + g.KV;
    g.f_bytes = g.KV * 32 * 4;
    const bool split = in_mode == kInSplit;
    g.nb = split ? kMaxNB : 4;
    // TMA writes a split slot as it lands ([k-group][row][16 B]); the
    // converters' slots get a 64-byte offset between k-groups (bank spread)
    g.b_lbo = g.KV * 16 + (split ? 0 : 64);
    g.bh_bytes = (g.b_lbo + g.KV * 16 + 127) / 128 * 128;
    g.t2_lbo = kTY * 16;
    g.t2h_bytes = g.KV / 8 * g.t2_lbo;
    g.off_t2 = 1024;
    g.off_f = g.off_t2 + 2 * g.t2h_bytes;
    g.off_b = g.off_f + (split ? 0 : kNF * g.f_bytes);
    g.smem_bytes = g.off_b + g.nb * 2 * g.bh_bytes + 1024;   // + slack to align the base
    return g;
}

// Barriers and flags at the start of shared memory.
struct Bars {
    uint64_t full_f[kNF], empty_f[kNF], full_b[kMaxNB], empty_b[kMaxNB];
    uint64_t full_d1, ready_a2, full_d2, empty_d2, drain;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(Bars) <= 1024, "barrier block");

// BF16 hi and lo parts of two FP32 values, packed (first value in the low half).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
    hi = *reinterpret_cast<const uint32_t *>(&hb);
    const float h0 = __uint_as_float(hi << 16);
    const float h1 = __uint_as_float(hi & 0xFFFF0000u);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - h0, x1 - h1);
    lo = *reinterpret_cast<const uint32_t *>(&lb);
}

// The same split of one value: hi and lo BF16 bit patterns.
__device__ __forceinline__ void split1(float x, uint16_t &hi, uint16_t &lo) {
    const __nv_bfloat16 hb = __float2bfloat16_rn(x);
    hi = *reinterpret_cast<const uint16_t *>(&hb);
    const __nv_bfloat16 lb = __float2bfloat16_rn(x - __uint_as_float(static_cast<uint32_t>(hi) << 16));
    lo = *reinterpret_cast<const uint16_t *>(&lb);
}

struct Ctl {
    long long budget;
    int *err;
    volatile int *abort;
};

// Bounded wait for phase `parity` of `bar`.  False (and the CTA told to stop)
// on an expired budget or when another role has stopped already.  A negative
// budget reports a timeout once the phase has completed (fault injection).
__device__ __forceinline__ bool wait_or_stop(uint64_t *bar, uint32_t parity, const Ctl &c) {
    const bool inject = c.budget < 0;
    if (!inject && tma::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64(), budget = inject ? kDrainBudget : c.budget;
    bool done = false;
    while (!(done = tma::mbar_try_wait(bar, parity))) {
        if (*c.abort) return false;
        if (clock64() - t0 > budget) break;
    }
    if (done && !inject) return true;
    atomicOr(c.err, kDevTimeout);
    *c.abort = 1;
    return false;
}

// The same wait by every lane of a warp, with one outcome for the whole
// warp (each lane observes the phase itself; the warp continues only if
// every lane's wait succeeded), so that the warp-collective tensor-memory
// loads and stores that follow run converged.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, const Ctl &c) {
    const bool ok = wait_or_stop(bar, parity, c);
    return __all_sync(0xffffffffu, ok);
}

// Work item i of this CTA: tile t = blockIdx.x + (i / nv) * gridDim.x, view
// view_lo + i % nv (kernel B walks the launch's views per tile; kernel A has
// nv = 1).  False past the last tile.
struct Item {
    int p, y0, x0, v;
};
__device__ __forceinline__ bool item_of(int i, int nv, int tiles_x, int tiles_y, int n_tiles, int view_lo, Item &it) {
    const long long t = blockIdx.x + static_cast<long long>(i / nv) * gridDim.x;
    if (t >= n_tiles) return false;
    const int per_plane = tiles_x * tiles_y;
    const int tt = static_cast<int>(t);
    it.p = tt / per_plane;
    const int r = tt - it.p * per_plane;
    const int ty = r / tiles_x;
    it.y0 = ty * kTY;
    it.x0 = (r - ty * tiles_x) * kTX;
    it.v = view_lo + i % nv;
    return true;
}

// Toeplitz operands of the launch's term, built once per CTA.
//   T2 (shared memory, pass-2 B operand, K-major): element (y_out, k = input
//       row) = u[k - y_out], at (y_out % 8) * 16 + (y_out / 8) * 128 +
//       (k / 8) * t2_lbo + (k % 8) * 2; hi half then lo half.
//   T1 (tensor memory, pass-1 A operand): lane x_out, column c holds input
//       columns 2c, 2c+1: w[k - COL0 - x_out]; hi at c, lo at c_t1lo + c.
__device__ void build_t2(const Geom &g, const float *__restrict__ u, unsigned char *t2) {
    const int items = kTY * (g.KV / 8);
    for (int it = threadIdx.x; it < items; it += kThreads) {
        const int n = it % kTY, kg = it / kTY;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = 8 * kg + e - n;
            x[e] = (j >= 0 && j < g.K) ? __ldg(u + j) : 0.0f;
        }
        uint4 h, l;
        split2(x[0], x[1], h.x, l.x);
        split2(x[2], x[3], h.y, l.y);
        split2(x[4], x[5], h.z, l.z);
        split2(x[6], x[7], h.w, l.w);
        const uint32_t addr = (n & 7) * 16 + (n >> 3) * 128 + kg * g.t2_lbo;
        *reinterpret_cast<uint4 *>(t2 + addr) = h;
        *reinterpret_cast<uint4 *>(t2 + g.t2h_bytes + addr) = l;
    }
}

// Warps kSplitWarp0 .. +3 (lane quarter q = warp % 4).
__device__ void build_t1(const Geom &g, const float *__restrict__ w, uint32_t tmem) {
    const int q = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
    const int x_out = 32 * q + lane;
    const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
#pragma unroll 1
    for (int c0 = 0; c0 < g.KH / 2; c0 += 8) {
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int j0 = 2 * (c0 + c) - g.COL0 - x_out;
            const float a = (j0 >= 0 && j0 < g.K) ? __ldg(w + j0) : 0.0f;
            const float b = (j0 + 1 >= 0 && j0 + 1 < g.K) ? __ldg(w + j0 + 1) : 0.0f;
            split2(a, b, hi[c], lo[c]);
        }
        tc5::st8(tmem + lane_off + c0, hi);
        tc5::st8(tmem + lane_off + g.c_t1lo + c0, lo);
    }
    tc5::wait_st();
}

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~static_cast<uintptr_t>(1023));
}

// Common set-up: barriers, tensor memory, Toeplitz operands.
__device__ void setup(const Params &kp, unsigned char *smem, Bars *bars) {
    const Geom &g = kp.g;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNF; ++s) {
            tma::mbar_init(&bars->full_f[s], 1);
            tma::mbar_init(&bars->empty_f[s], 4);
        }
        for (int s = 0; s < g.nb; ++s) {
            // a B slot fills by TMA (one expect_tx arrival) or by the four converter warps
            tma::mbar_init(&bars->full_b[s], kp.io.in_mode == kInSplit ? 1 : 4);
            tma::mbar_init(&bars->empty_b[s], 1);
        }
        tma::mbar_init(&bars->full_d1, 1);
        tma::mbar_init(&bars->ready_a2, 4);
        tma::mbar_init(&bars->full_d2, 1);
        tma::mbar_init(&bars->empty_d2, 8);   // epilogue warps
        tma::mbar_init(&bars->drain, 1);
        bars->abort = 0;
        tma::fence_barrier_init();
    }
    if (warp == kMmaWarp) {
        __syncwarp();
        tc5::alloc(&bars->tmem_base, kTmemCols);
        tc5::relinquish();
    }
    const float *taps = kp.a.taps + static_cast<long long>(kp.term) * 4 * g.K;
    build_t2(g, taps + kp.kind_u * g.K, smem + g.off_t2);
    tma::fence_proxy_async_smem();   // T2 is read by the tensor core
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (warp >= kSplitWarp0 && warp < kSplitWarp0 + 4) {
        __syncwarp();
        build_t1(g, taps + kp.kind_w * g.K, bars->tmem_base);
    }
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
}

// ---- roles -----------------------------------------------------------------

// TMA producer (one thread).  Split mode: per K-step j the hi and lo blocks
// of its two column blocks, straight into B slot c % nb.  fp32 mode: FP32
// chunks of 32 columns into the F ring.  Copies in flight land before the
// CTA leaves.
__device__ void role_tma(const Params &kp, unsigned char *smem, Bars *bars, const Ctl &ctl, int nv, int tiles_x,
                         int tiles_y, int n_tiles, int kind) {
    const Geom &g = kp.g;
    const FusedArgs &a = kp.a;
    const int mode = kp.io.in_mode;
    int last_use[kMaxNB];
#pragma unroll
    for (int s = 0; s < kMaxNB; ++s) last_use[s] = -1;
    uint32_t c = 0;
    Item it;
    if (mode != kInConst) {
        for (int i = 0; item_of(i, nv, tiles_x, tiles_y, n_tiles, a.view_lo, it); ++i) {
            const int z = kind == 1 ? it.v * a.P + it.p : it.p;
            bool ok = true;
            if (mode == kInSplit) {
                const int blk0 = (it.x0 - g.R8) / 8;   // exact: x0 and R8 are multiples of 8
#pragma unroll 1
                for (int j = 0; j < g.KH / 16; ++j, ++c) {
                    const int s = c % g.nb, u = c / g.nb;
                    if (u > 0 && !wait_or_stop(&bars->empty_b[s], (u - 1) & 1, ctl)) {
                        ok = false;
                        break;
                    }
                    unsigned char *slot = smem + g.off_b + s * 2 * g.bh_bytes;
                    tma::mbar_arrive_expect_tx(&bars->full_b[s], 8 * g.KV * 8);
                    // hi / lo half, column block (k-group), upper / lower KV/2 rows
                    for (int hl = 0; hl < 2; ++hl)
                        for (int kg = 0; kg < 2; ++kg)
                            for (int rh = 0; rh < 2; ++rh)
                                tma::load_3d(slot + hl * g.bh_bytes + kg * g.b_lbo + rh * g.KV * 8, &kp.map,
                                             &bars->full_b[s], 2 * (it.y0 - g.R) + rh * g.KV, blk0 + 2 * j + kg,
                                             2 * z + hl);
                    last_use[s] = u;
                }
            } else {
#pragma unroll 1
                for (int j = 0; j < (g.KH + 31) / 32; ++j, ++c) {
                    const int s = c % kNF, u = c / kNF;
                    if (u > 0 && !wait_or_stop(&bars->empty_f[s], (u - 1) & 1, ctl)) {
                        ok = false;
                        break;
                    }
                    tma::mbar_arrive_expect_tx(&bars->full_f[s], g.f_bytes);
                    tma::load_3d(smem + g.off_f + s * g.f_bytes, &kp.map, &bars->full_f[s], it.x0 - g.R8 + 32 * j,
                                 it.y0 - g.R, z);
                    last_use[s] = u;
                }
            }
            if (!ok) break;
        }
    }
    const int nslots = mode == kInSplit ? g.nb : kNF;
    for (int s = 0; s < nslots; ++s)
        if (last_use[s] >= 0)
            tma::mbar_wait_bounded(mode == kInSplit ? &bars->full_b[s] : &bars->full_f[s], last_use[s] & 1,
                                   kDrainBudget);
}

// Converters (warps 0-3; fp32 and constant modes): FP32 chunk [KV rows][32
// columns] -> the B slots of its K-steps 2f and 2f+1: element (row n,
// column k of the K-step) at (k / 8) * b_lbo + n * 16 + (k % 8) * 2, in the
// hi and in the lo half.  Item = (row n, quad q8 of 4 columns): eight lanes
// read one row's 128 contiguous bytes; a thread's items are all loaded
// before they are split and stored.  A last chunk with one K-step converts
// its first 16 columns only.
constexpr int kConvItems = (176 * 8 + 127) / 128;   // items per thread and chunk at the largest KV

__device__ void role_convert(const Params &kp, unsigned char *smem, Bars *bars, const Ctl &ctl, int nv, int tiles_x,
                             int tiles_y, int n_tiles) {
    const Geom &g = kp.g;
    const FusedArgs &a = kp.a;
    const int mode = kp.io.in_mode;
    if (mode == kInSplit) return;
    const int ct = threadIdx.x - 32 * kConvWarp0;   // 0..127
    const int lane = threadIdx.x & 31;
    const int nks = g.KH / 16;                      // K-steps per item
    uint32_t cf = 0, c = 0;                         // chunk and K-step counters
    Item it;
    for (int i = 0; item_of(i, nv, tiles_x, tiles_y, n_tiles, a.view_lo, it); ++i) {
        const float mean = mode == kInConst ? __ldg(a.means + it.p) : 0.0f;
        bool ok = true;
#pragma unroll 1
        for (int j = 0; j < nks; j += 2, ++cf) {
            const int two = (j + 1 < nks) ? 2 : 1;   // K-steps in this chunk
            const int sf = cf % kNF, uf = cf / kNF;
            if (mode == kInF32 && !warp_wait(&bars->full_f[sf], uf & 1, ctl)) {
                ok = false;
                break;
            }
            for (int h = 0; h < two && ok; ++h) {
                const uint32_t ch = c + h;
                if (ch >= static_cast<uint32_t>(g.nb) &&
                    !warp_wait(&bars->empty_b[ch % g.nb], ((ch / g.nb) - 1) & 1, ctl))
                    ok = false;
            }
            if (!ok) break;
            const float *f = reinterpret_cast<const float *>(smem + g.off_f + sf * g.f_bytes);
            const int n_items = g.KV * 4 * two;
            const int sh = two == 2 ? 3 : 2;   // items per row: 8 (two K-steps) or 4
            float4 v[kConvItems];
#pragma unroll
            for (int k = 0; k < kConvItems; ++k) {
                const int e = ct + 128 * k;
                if (e >= n_items) break;
                const int n = e >> sh, q8 = e & ((1 << sh) - 1);
                if (mode == kInF32) {
                    v[k] = *reinterpret_cast<const float4 *>(f + n * 32 + 4 * q8);
                } else {   // the constant first estimate: the mean inside the plane, zero outside
                    const int gy = it.y0 - g.R + n, gx = it.x0 - g.R8 + 16 * j + 4 * q8;
                    const bool row_in = gy >= 0 && gy < a.H;
                    v[k].x = (row_in && gx >= 0 && gx < a.W) ? mean : 0.0f;
                    v[k].y = (row_in && gx + 1 >= 0 && gx + 1 < a.W) ? mean : 0.0f;
                    v[k].z = (row_in && gx + 2 >= 0 && gx + 2 < a.W) ? mean : 0.0f;
                    v[k].w = (row_in && gx + 3 >= 0 && gx + 3 < a.W) ? mean : 0.0f;
                }
            }
#pragma unroll
            for (int k = 0; k < kConvItems; ++k) {
                const int e = ct + 128 * k;
                if (e >= n_items) break;
                const int n = e >> sh, q8 = e & ((1 << sh) - 1), q = q8 & 3;
                uint2 hi, lo;
                split2(v[k].x, v[k].y, hi.x, lo.x);
                split2(v[k].z, v[k].w, hi.y, lo.y);
                unsigned char *b = smem + g.off_b + ((c + (q8 >> 2)) % g.nb) * 2 * g.bh_bytes;
                const uint32_t off = (q >> 1) * g.b_lbo + n * 16 + (q & 1) * 8;
                *reinterpret_cast<uint2 *>(b + off) = hi;
                *reinterpret_cast<uint2 *>(b + g.bh_bytes + off) = lo;
            }
            tma::fence_proxy_async_smem();   // the tensor core reads the slots
            __syncwarp();
            if (lane == 0) {
                if (mode == kInF32) tma::mbar_arrive(&bars->empty_f[sf]);
                for (int h = 0; h < two; ++h) tma::mbar_arrive(&bars->full_b[(c + h) % g.nb]);
            }
            c += two;
        }
        if (!ok) break;
    }
}

// MMA issuer (one thread).
__device__ void role_mma(const Params &kp, unsigned char *smem, Bars *bars, const Ctl &ctl, int nv, int tiles_x,
                         int tiles_y, int n_tiles) {
    const Geom &g = kp.g;
    const uint32_t tmem = bars->tmem_base;
    const uint32_t idesc1 = tc5::idesc_bf16(128, g.KV, false, false);
    const uint32_t idesc2 = tc5::idesc_bf16(128, kTY, false, false);
    const uint32_t b0 = tc5::smem_u32(smem + g.off_b), t2 = tc5::smem_u32(smem + g.off_t2);
    uint32_t c = 0;
    Item it;
    for (int i = 0; item_of(i, nv, tiles_x, tiles_y, n_tiles, kp.a.view_lo, it); ++i) {
        bool ok = true;
        // pass 1: D1 = T1 x B, one K-step per B slot
#pragma unroll 1
        for (int j = 0; j < g.KH / 16; ++j, ++c) {
            const int sb = c % g.nb, ub = c / g.nb;
            if (!wait_or_stop(&bars->full_b[sb], ub & 1, ctl)) {
                ok = false;
                break;
            }
            tc5::fence_after();
            const uint32_t bh = b0 + sb * 2 * g.bh_bytes, bl = bh + g.bh_bytes;
            const uint64_t dh = tc5::sdesc(bh, g.b_lbo, 128), dl = tc5::sdesc(bl, g.b_lbo, 128);
            const uint32_t ah = tmem + 8 * j, al = tmem + g.c_t1lo + 8 * j;
            tc5::mma_bf16_ta(tmem + g.c_d1, al, dh, idesc1, j > 0);
            tc5::mma_bf16_ta(tmem + g.c_d1, ah, dl, idesc1, 1);
            tc5::mma_bf16_ta(tmem + g.c_d1, ah, dh, idesc1, 1);
            tc5::commit(&bars->empty_b[sb]);   // the slot is free once these MMAs are done
        }
        if (!ok) break;
        tc5::commit(&bars->full_d1);
        // pass 2: D2 = A2 x T2 once A2 is split and the epilogue has read D2
        if (!wait_or_stop(&bars->ready_a2, i & 1, ctl)) break;
        if (i > 0 && !wait_or_stop(&bars->empty_d2, (i - 1) & 1, ctl)) break;
        tc5::fence_after();
#pragma unroll 1
        for (int s = 0; s < g.KV / 16; ++s) {
            const uint32_t bo = static_cast<uint32_t>(2 * s) * g.t2_lbo;
            const uint64_t dh = tc5::sdesc(t2 + bo, g.t2_lbo, 128), dl = tc5::sdesc(t2 + g.t2h_bytes + bo, g.t2_lbo, 128);
            const uint32_t ah = tmem + g.c_d1 + 16 * s, al = ah + 8;
            tc5::mma_bf16_ta(tmem + g.c_d2, al, dh, idesc2, s > 0);
            tc5::mma_bf16_ta(tmem + g.c_d2, ah, dl, idesc2, 1);
            tc5::mma_bf16_ta(tmem + g.c_d2, ah, dh, idesc2, 1);
        }
        tc5::commit(&bars->full_d2);
    }
    // every MMA has completed before the tensor memory is released
    tc5::commit(&bars->drain);
    tma::mbar_wait_bounded(&bars->drain, 0, kDrainBudget);
}

// Split warps (4-7): D1 (FP32, columns c_d1 + n) -> A2 in place: for each
// K-step s of 16 input rows, BF16 hi pairs in columns c_d1 + 16s .. +7 and
// lo pairs in c_d1 + 16s + 8 .. +15.
__device__ void role_split(const Params &kp, Bars *bars, const Ctl &ctl, int nv, int tiles_x, int tiles_y,
                           int n_tiles) {
    const Geom &g = kp.g;
    const int q = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
    const uint32_t base = bars->tmem_base + (static_cast<uint32_t>(32 * q) << 16) + g.c_d1;
    Item it;
    for (int i = 0; item_of(i, nv, tiles_x, tiles_y, n_tiles, kp.a.view_lo, it); ++i) {
        if (!warp_wait(&bars->full_d1, i & 1, ctl)) break;
        tc5::fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < g.KV; c0 += 32) {
            uint32_t r[32];
            const bool full = c0 + 32 <= g.KV;   // else 16 columns are left
            __syncwarp();
            if (full)
                tc5::ld32(base + c0, r);
            else
                tc5::ld16(base + c0, r);
            tc5::wait_ld();
            uint32_t w[16];
            // K-step s0 = c0 / 16: values r[0..15]; step s0 + 1: r[16..31]
#pragma unroll
            for (int st = 0; st < 2; ++st) {
                if (st == 1 && !full) break;
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    split2(__uint_as_float(r[16 * st + 2 * e]), __uint_as_float(r[16 * st + 2 * e + 1]), w[e],
                           w[8 + e]);
                tc5::st16(base + c0 + 16 * st, w);
            }
        }
        tc5::wait_st();
        tc5::fence_before();
        __syncwarp();
        if (lane == 0) tma::mbar_arrive(&bars->ready_a2);
    }
}

// Element (y, x) of a plane of the split layout (hi; lo at + G*H*8).
__device__ __forceinline__ long long split_index(int H, int y, int x) {
    return (static_cast<long long>(x >> 3) * H + y) * 8 + (x & 7);
}

// Epilogue warps 8-15.  Thread: output column x = x0 + 32 q + lane (q =
// warp % 4, its tensor-memory lane quarter) and nr consecutive output rows
// from r0: rows 0-63 (warps 8-11) and 64-127 (12-15).  (Giving the idle
// converter warps of the split mode a third of the rows was measured
// slower.)  D2 is read in loads of up to 32 columns (the last
// load frees it for the next pass 2), and rows are processed in groups of 16
// whose global loads are all issued before the first use (they hit L2: the
// warp prefetched them one item ahead).  KIND 0: ratio of every view of the
// launch, FP32 or split; KIND 1: the update (one view per launch), FP32 and,
// if asked, split.  A split output also holds zeros in its columns W .. 8G-1.
template <int KIND>
__device__ void role_epilogue(const Params &kp, Bars *bars, const Ctl &ctl, int nv, int tiles_x, int tiles_y,
                              int n_tiles, int r0, int nr) {
    const FusedArgs &a = kp.a;
    const Geom &g = kp.g;
    const int q = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
    const uint32_t base = bars->tmem_base + (static_cast<uint32_t>(32 * q) << 16) + g.c_d2 + r0;
    const long long plane_px = static_cast<long long>(a.H) * a.W;
    const long long split_plane = 2LL * kp.G * 8 * a.H;   // hi + lo of one plane
    const long long lo_off = static_cast<long long>(kp.G) * 8 * a.H;
    const bool split_out = KIND == 0 ? kp.io.ratio_split != 0 : kp.io.write_psi_split != 0;
    uint16_t *sout = KIND == 0 ? reinterpret_cast<uint16_t *>(a.ratio) : kp.io.psi_split;
    Item it;
    for (int i = 0; item_of(i, nv, tiles_x, tiles_y, n_tiles, a.view_lo, it); ++i) {
        if (!warp_wait(&bars->full_d2, i & 1, ctl)) break;
        tc5::fence_after();
        const int x = it.x0 + 32 * q + lane;
        {   // the next item's rows of this warp's 32 columns into L2: they lie in
            // one 128-byte line per row, so lane l fetches rows l and l + 32
            Item nx;
            if (item_of(i + 1, nv, tiles_x, tiles_y, n_tiles, a.view_lo, nx) && nx.x0 + 32 * q < a.W) {
                const int x1 = nx.x0 + 32 * q;
                const int y1 = nx.y0 + r0, n1 = min(nr, a.H - y1);
                for (int r = lane; r < n1; r += 32) {
                    if (KIND == 0) {
                        const int es = a.phi_u16 ? 2 : 4;
                        for (int v = a.view_lo; v < a.view_hi; ++v)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(
                                static_cast<const char *>(a.phi) +
                                ((static_cast<long long>(v) * a.P + nx.p) * plane_px + static_cast<long long>(y1 + r) * a.W +
                                 x1) * es));
                    } else if (a.psi_in) {
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psi_in + nx.p * plane_px +
                                                                      static_cast<long long>(y1 + r) * a.W + x1));
                    }
                }
            }
        }
#pragma unroll 1
        for (int c0 = 0; c0 < nr; c0 += 32) {
            uint32_t dr[32];
            const bool full = c0 + 32 <= nr;   // else 16 rows are left
            __syncwarp();
            if (full)
                tc5::ld32(base + c0, dr);
            else
                tc5::ld16(base + c0, dr);
            tc5::wait_ld();
            if (c0 + 32 >= nr) {   // D2 is free for the next pass 2
                tc5::fence_before();
                __syncwarp();
                if (lane == 0) tma::mbar_arrive(&bars->empty_d2);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && !full) break;
                // 16 rows y0 + r0 + c0 + 16 h + j; rows past the plane load
                // the last row (so that every load is issued unconditionally,
                // all before the first use) and are not stored
                const int yb = it.y0 + r0 + c0 + 16 * h;
                const int nrow = min(16, a.H - yb);
                if (x < a.W) {
                    if (KIND == 0) {
#pragma unroll 1
                        for (int v = a.view_lo; v < a.view_hi; ++v) {
                            const long long vp = static_cast<long long>(v) * a.P + it.p;
                            const long long vb = vp * plane_px + x;
                            float ph[16];
                            if (a.phi_u16) {
                                const uint16_t *src =
                                    static_cast<const uint16_t *>(a.phi) + vb + static_cast<long long>(yb) * a.W;
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    ph[j] = static_cast<float>(__ldg(src + static_cast<long long>(min(j, nrow - 1)) * a.W));
                            } else {
                                const float *src =
                                    static_cast<const float *>(a.phi) + vb + static_cast<long long>(yb) * a.W;
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    ph[j] = __ldg(src + static_cast<long long>(min(j, nrow - 1)) * a.W);
                            }
                            if (split_out) {
                                uint16_t *dst = sout + vp * split_plane + split_index(a.H, yb, x);
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    if (j < nrow) {
                                        uint16_t hi, lo;
                                        split1(__fdiv_rn(ph[j], fmaxf(__uint_as_float(dr[16 * h + j]), a.eps)), hi, lo);
                                        dst[8 * j] = hi;
                                        dst[8 * j + lo_off] = lo;
                                    }
                            } else {
                                float *dst = a.ratio + vb + static_cast<long long>(yb) * a.W;
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    if (j < nrow)
                                        dst[static_cast<long long>(j) * a.W] =
                                            __fdiv_rn(ph[j], fmaxf(__uint_as_float(dr[16 * h + j]), a.eps));
                            }
                        }
                    } else {
                        const long long pb = it.p * plane_px + x + static_cast<long long>(yb) * a.W;
                        float ps[16];
                        if (a.psi_in) {
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                ps[j] = __ldg(a.psi_in + pb + static_cast<long long>(min(j, nrow - 1)) * a.W);
                        } else {
                            const float mean = __ldg(a.means + it.p);
#pragma unroll
                            for (int j = 0; j < 16; ++j) ps[j] = mean;
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) ps[j] *= __uint_as_float(dr[16 * h + j]);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (j < nrow) a.psi_out[pb + static_cast<long long>(j) * a.W] = ps[j];
                        if (split_out) {
                            uint16_t *dst = sout + it.p * split_plane + split_index(a.H, yb, x);
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (j < nrow) {
                                    uint16_t hi, lo;
                                    split1(ps[j], hi, lo);
                                    dst[8 * j] = hi;
                                    dst[8 * j + lo_off] = lo;
                                }
                        }
                    }
                } else if (split_out && x < 8 * kp.G) {   // the split layout's columns past the plane hold zeros
                    const int np = KIND == 0 ? a.view_hi - a.view_lo : 1;
                    for (int w = 0; w < np; ++w) {
                        const long long pl = KIND == 0 ? static_cast<long long>(a.view_lo + w) * a.P + it.p : it.p;
                        uint16_t *dst = sout + pl * split_plane + split_index(a.H, yb, x);
                        for (int j = 0; j < nrow; ++j) {
                            dst[8 * j] = 0;
                            dst[8 * j + lo_off] = 0;
                        }
                    }
                }
            }
        }
    }
}

// KIND 0: blur/ratio (one input tile per tile), 1: correlate/update (one per
// view and tile).
template <int KIND>
__global__ void __launch_bounds__(kThreads, 1) tcw_kernel(const __grid_constant__ Params kp) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = align1024(smem_raw);
    Bars *bars = reinterpret_cast<Bars *>(smem);
    setup(kp, smem, bars);
    const FusedArgs &a = kp.a;
    const Ctl ctl{a.wait_budget, a.err, &bars->abort};
    const int tiles_x = (a.W + kTX - 1) / kTX, tiles_y = (a.H + kTY - 1) / kTY;
    const int n_tiles = tiles_x * tiles_y * a.P;
    const int nv = KIND == 0 ? 1 : a.view_hi - a.view_lo;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < kConvWarp0 + 4) {
        role_convert(kp, smem, bars, ctl, nv, tiles_x, tiles_y, n_tiles);
    } else if (warp < kSplitWarp0 + 4) {
        role_split(kp, bars, ctl, nv, tiles_x, tiles_y, n_tiles);
    } else if (warp < kEpiWarp0 + 8) {
        const int e = warp - kEpiWarp0;   // 0-3 rows from 0, 4-7 the next block
        role_epilogue<KIND>(kp, bars, ctl, nv, tiles_x, tiles_y, n_tiles, e < 4 ? 0 : 64, 64);
    } else if (warp == kTmaWarp) {
        if (lane == 0) role_tma(kp, smem, bars, ctl, nv, tiles_x, tiles_y, n_tiles, KIND);
    } else if (warp == kMmaWarp) {
        if (lane == 0) role_mma(kp, smem, bars, ctl, nv, tiles_x, tiles_y, n_tiles);
    }
    tc5::fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        __syncwarp();
        tc5::fence_after();
        tc5::dealloc(bars->tmem_base, kTmemCols);
    }
}

// ---- host side ------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// FP32 [D][H][W] planes, box 32 columns x KV rows x 1 plane, zero fill.
bool encode_f32(CUtensorMap *m, const void *base, int W, int H, long long D, int box_h) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H), static_cast<cuuint64_t>(D)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(W) * 4, static_cast<cuuint64_t>(W) * H * 4};
    cuuint32_t box[3] = {32, static_cast<cuuint32_t>(box_h), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Split layout of D planes, seen as 8-byte elements so that a column
// block's rows (16 bytes each, contiguous) form one long innermost run:
// {2 H (elements of one column block), G (column blocks), 2 D (hi, lo of
// each plane)}, box {KV, 1, 1} = KV/2 rows of one block, which land as
// consecutive 16-byte rows (two boxes per k-group of a K-step).  Rows
// outside the plane and blocks outside [0, G) read as zeros.
bool encode_split(CUtensorMap *m, const void *base, int H, int G, long long D, int box_h) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {2 * static_cast<cuuint64_t>(H), static_cast<cuuint64_t>(G), static_cast<cuuint64_t>(2 * D)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(H) * 16, static_cast<cuuint64_t>(G) * H * 16};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(box_h), 1, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline bool aligned16(const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

}  // namespace

// The launch's term when these kernels can take it, else -1: zero boundary,
// 16-byte aligned buffers and rows (TMA), no weights or blur-only mode, odd
// K <= 47, and a rank-1 factorisation shared by the launch's views (kernel
// A: one blur group; kernel B: one view per launch, as in the sequential
// update order).
int eligible_term(const FusedArgs &a, int which) {
    const int K = a.ft.K;
    if (a.circular || a.W % 4 != 0 || K < 1 || K > kMaxK || K % 2 == 0) return -1;
    if (a.weights || a.wnorm || a.store_blur || !a.taps || !a.taps_host) return -1;
    if (!aligned16(a.ratio) || !aligned16(a.psi_out) || (a.psi_in && !aligned16(a.psi_in))) return -1;
    if (a.view_hi <= a.view_lo) return -1;
    if (which == 0) {
        const int g = a.ft.group[a.view_lo];
        for (int v = a.view_lo; v < a.view_hi; ++v)
            if (a.ft.group[v] != g) return -1;
        const int lead = a.ft.group_leader[g];
        return a.ft.rank[lead] == 1 ? a.ft.tap_off[lead] : -1;
    }
    if (a.view_hi - a.view_lo != 1) return -1;   // one view per launch: the update needs no running product
    return a.ft.crank[a.view_lo] == 1 ? a.ft.ctap_off[a.view_lo] : -1;
}

}  // namespace tcw

bool tcw_eligible(const FusedArgs &a, int which) { return tcw::eligible_term(a, which) >= 0; }

size_t tcw_split_bytes(int W, int H, long long planes) {
    return static_cast<size_t>(planes) * H * ((W + 7) / 8 * 8) * 4;
}

cudaError_t launch_tcw(const FusedArgs &a, int which, const TcwIo &io, cudaStream_t st) {
    using namespace tcw;
    const int term = eligible_term(a, which);
    if (term < 0) return cudaErrorInvalidValue;
    if (io.in_mode < kInConst || io.in_mode > kInSplit || (which == 1 && io.in_mode == kInConst) ||
        (which == 0 && (io.in_mode == kInConst) != (a.psi_in == nullptr)))
        return cudaErrorInvalidValue;
    if ((which == 0 && io.in_mode == kInSplit) || (which == 1 && io.write_psi_split))
        if (!io.psi_split || !aligned16(io.psi_split)) return cudaErrorInvalidValue;
    Params kp;
    std::memset(&kp, 0, sizeof kp);
    kp.a = a;
    kp.io = io;
    kp.g = make_geom(a.ft.K, io.in_mode);
    kp.G = (a.W + 7) / 8;
    kp.term = term;
    kp.kind_u = which == 0 ? 0 : 2;
    kp.kind_w = which == 0 ? 1 : 3;
    const Geom &g = kp.g;
    int dev = 0;
    cudaGetDevice(&dev);
    static unsigned long long attr_set[2] = {0, 0};
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set[which] & bit)) {
        // the largest layout, so that one opt-in serves every K and mode
        uint32_t need = 0;
        for (int m = kInConst; m <= kInSplit; ++m) need = std::max(need, make_geom(kMaxK, m).smem_bytes);
        const cudaError_t e = cudaFuncSetAttribute(which == 0 ? tcw_kernel<0> : tcw_kernel<1>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        if (e != cudaSuccess) return e;
        attr_set[which] |= bit;
    }
    const long long planes = which == 0 ? a.P : static_cast<long long>(a.ft.views) * a.P;
    const void *src = which == 0 ? static_cast<const void *>(a.psi_in) : static_cast<const void *>(a.ratio);
    if (io.in_mode == kInSplit) {
        if (!encode_split(&kp.map, which == 0 ? static_cast<const void *>(io.psi_split) : src, a.H, kp.G, planes, g.KV))
            return cudaErrorInvalidValue;
    } else if (io.in_mode == kInF32) {
        if (!encode_f32(&kp.map, src, a.W, a.H, planes, g.KV)) return cudaErrorInvalidValue;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long n_tiles = static_cast<long long>((a.W + kTX - 1) / kTX) * ((a.H + kTY - 1) / kTY) * a.P;
    if (n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    long long ctas = sms > 0 ? sms : 1;   // one CTA per SM (shared and tensor memory)
    if (a.max_ctas > 0 && a.max_ctas < ctas) ctas = a.max_ctas;
    if (n_tiles < ctas) ctas = n_tiles;
    if (ctas < 1) return cudaSuccess;
    if (which == 0)
        tcw_kernel<0><<<dim3(static_cast<unsigned>(ctas)), kThreads, g.smem_bytes, st>>>(kp);
    else
        tcw_kernel<1><<<dim3(static_cast<unsigned>(ctas)), kThreads, g.smem_bytes, st>>>(kp);
    count_launch();
    return cudaGetLastError();
}

}  // namespace mvd
