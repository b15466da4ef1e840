// The two kernels of one fused MV-RL iteration (Supp. Note 1 update
// equation), for all planes of a batch in one launch each:
//
//   blur_ratio        r_v = phi_v / max(psi * P_v, eps)   for every view v
//   correlate_update  psi <- psi * prod_v (r_v (*) P_v^*)
//
// A CTA works on TY x 128 output tiles of the planes, one after another
// (persistent grid, one resident wave).  Kernel A stages the psi
// tile (halo R) once for all views; views whose PSFs are identical share
// one blur.  Kernel B stages each view's ratio tile with its halo, keeps the
// running product of the views' corrections in registers and updates psi in
// place: each CTA reads and writes only its own output pixels, and kernel A
// of the next iteration starts after kernel B ends in stream order.
//
// Tiles arrive by TMA (one thread issues a 3D box copy, hardware zero fill
// outside the plane = the ZERO boundary) whenever the plane rows are 16-byte
// multiples; the circular boundary, unaligned planes and the constant first
// estimate use a software load into the same layout.
//
// HBM traffic per voxel-iteration (uint16 data): kernel A reads psi (4 B) and
// phi_v (2V B) and writes r_v (4V B); kernel B reads r_v (4V B) and psi (4 B)
// and writes psi (4 B): 12 + 10V bytes.  Halo re-reads hit L2.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "fused_common.cuh"

namespace mvd {
namespace fused {

namespace {

constexpr long long kDrainBudget = 4000000000LL;

// Factor taps travel in the launch's parameter block (constant bank): the
// kernel's two kinds (blur or correlation) of every term, [vertical K]
// [horizontal K] per term.  Warp-uniform, they need no vector registers.
constexpr int kParamTaps = 4096;

struct KParams {
    CUtensorMap map;   // psi (kernel A) or the ratio planes (kernel B); valid if use_tma
    FusedArgs a;
    int use_tma;
    int vec_ok;    // rows are multiples of 4 elements and buffers 16-byte aligned
    int vec16;     // rows are multiples of 16 elements as well
    float taps[kParamTaps];
};

// Wait for the tile on `bar`; on an expired budget flag the device status,
// drain the copy (bounded again) and make the whole CTA leave.  A negative
// budget makes every wait report a timeout once its copy has landed (fault
// injection for testing the error path).
__device__ __forceinline__ bool wait_tile(uint64_t *bar, uint32_t parity, const FusedArgs &a,
                                          volatile int *abort_flag) {
    if (a.wait_budget < 0 || !tma::mbar_wait_bounded(bar, parity, a.wait_budget)) {
        atomicOr(a.err, kDevTimeout);
        tma::mbar_wait_bounded(bar, parity, kDrainBudget);
        *abort_flag = 1;
    }
    __syncthreads();
    return *abort_flag == 0;
}

// Four consecutive values of one row: uint16 or FP32 source.
__device__ __forceinline__ void load4(const void *src, int u16, long long off, bool vec, int n, float (&o)[4]) {
    if (u16) {
        const uint16_t *p = static_cast<const uint16_t *>(src) + off;
        if (vec) {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
            o[0] = static_cast<float>(w.x & 0xffffu);
            o[1] = static_cast<float>(w.x >> 16);
            o[2] = static_cast<float>(w.y & 0xffffu);
            o[3] = static_cast<float>(w.y >> 16);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = j < n ? static_cast<float>(p[j]) : 0.0f;
        }
    } else {
        const float *p = static_cast<const float *>(src) + off;
        if (vec) {
            const float4 w = __ldg(reinterpret_cast<const float4 *>(p));
            o[0] = w.x;
            o[1] = w.y;
            o[2] = w.z;
            o[3] = w.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = j < n ? __ldg(p + j) : 0.0f;
        }
    }
}

__device__ __forceinline__ void store4(float *dst, bool vec, int n, const float (&v)[4]) {
    if (vec) {
        *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < n) dst[j] = v[j];
    }
}

// Row-wise epilogue over the TY x TX output tile held in the staging tile.
// Warp w takes rows w, w+8, ...; lane l takes columns 4l .. 4l+3, so every
// warp reads and writes whole contiguous 512-byte row segments, and all of a
// warp's loads are issued before its stores.
//   MODE 0 (ratio):  ratio = phi / max(stage, eps)   (base: plane of view v)
//   MODE 1 (update): psi_out = psi_in * stage, or mean * stage on the first
//                    iteration                         (base: plane p)
template <int K, int MODE, int TYF = 0>
__device__ __forceinline__ void row_epilogue(const FusedArgs &a, int vec_ok, const float *__restrict__ stage,
                                             long long base, int y0, int x0, float mean) {
    using G = Geo<K, TYF>;
    constexpr int WARPS = kThreads / 32;
    constexpr int ROWS = G::TY / WARPS;
    static_assert(G::TX == 4 * 32, "one warp covers one tile row");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = x0 + 4 * lane;
    const int n = min(4, a.W - x);
    if (n <= 0) return;
    const bool vec = vec_ok && n == 4;
    float in[ROWS][4];
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
        const int y = y0 + warp + k * WARPS;
        if (y >= a.H) continue;
        const long long off = base + static_cast<long long>(y) * a.W + x;
        if (MODE == 0) {
            load4(a.phi, a.phi_u16, off, vec, n, in[k]);
        } else if (a.psi_in) {
            load4(a.psi_in, 0, off, vec, n, in[k]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) in[k][j] = mean;
        }
    }
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
        const int row = warp + k * WARPS;
        const int y = y0 + row;
        if (y >= a.H) continue;
        const float4 s4 = *reinterpret_cast<const float4 *>(stage + row * G::VB_LD + 4 * lane);
        const float s[4] = {s4.x, s4.y, s4.z, s4.w};
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = MODE == 0 ? __fdiv_rn(in[k][j], fmaxf(s[j], a.eps)) : in[k][j] * s[j];
        float *dst = (MODE == 0 ? a.ratio : a.psi_out) + base + static_cast<long long>(y) * a.W + x;
        store4(dst, vec, n, o);
    }
}

// Tile t of a launch: plane p, output origin (y0, x0); x fastest so that the
// CTAs working at the same time share halo rows in L2.
struct TileCoord {
    int p, y0, x0;
};

template <int K, int TYF = 0>
__device__ __forceinline__ TileCoord tile_coord(int t, int tiles_x, int tiles_y) {
    using G = Geo<K, TYF>;
    const int per_plane = tiles_x * tiles_y;
    const int p = t / per_plane;
    const int r = t - p * per_plane;
    const int ty = r / tiles_x;
    return {p, ty * G::TY, (r - ty * tiles_x) * G::TX};
}

// Tile heights: kernel A 0 (Geo's choice: 64 rows while two CTAs fit on an
// SM, else 32), kernel B 32 rows with three CTAs per SM where they fit.
constexpr int kTyA = 0;
constexpr int kTyB = 32;

// Persistent: each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// With TMA, the next tile's psi box is requested right after the last
// vertical pass of the current tile (the input tile is free from then on),
// so the copy overlaps the last horizontal pass and the epilogue.
template <int K>
__global__ void __launch_bounds__(kThreads, Geo<K, kTyA>::MIN_BLOCKS)
blur_ratio_kernel(const __grid_constant__ KParams kp) {
    using G = Geo<K, kTyA>;
    const FusedArgs &a = kp.a;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 8);
    float *tile = reinterpret_cast<float *>(smem + kTileOffset);
    float *stage = tile + G::BOX_H * G::BOX_W;

    const int tiles_x = (a.W + G::TX - 1) / G::TX;
    const int tiles_y = (a.H + G::TY - 1) / G::TY;
    const int n_tiles = tiles_x * tiles_y * a.P;
    const long long plane_px = static_cast<long long>(a.H) * a.W;
    const bool use_tma = kp.use_tma && a.psi_in != nullptr;

    // vertical passes per tile: one per SVD term of every blur group in use
    int passes = 0;
    for (int g = 0; g < a.ft.n_groups; ++g) {
        bool used = false;
        for (int v = a.view_lo; v < a.view_hi; ++v) used |= (a.ft.group[v] == g);
        if (used) passes += a.ft.rank[a.ft.group_leader[g]];
    }

    if (threadIdx.x == 0) {
        *abort_flag = 0;
        if (use_tma) {
            tma::mbar_init(bar, 1);
            tma::fence_barrier_init();
        }
    }
    __syncthreads();
    int t = blockIdx.x;
    if (use_tma && threadIdx.x == 0 && t < n_tiles) {
        const TileCoord c = tile_coord<K, kTyA>(t, tiles_x, tiles_y);
        tma::mbar_arrive_expect_tx(bar, G::TILE_BYTES);
        tma::load_3d(tile, &kp.map, bar, c.x0 - G::R4, c.y0 - G::R, c.p);
    }
    uint32_t phase = 0;
    for (; t < n_tiles; t += gridDim.x) {
        const TileCoord tc = tile_coord<K, kTyA>(t, tiles_x, tiles_y);
        const int p = tc.p, y0 = tc.y0, x0 = tc.x0;
        if (use_tma) {
            if (!wait_tile(bar, phase, a, abort_flag)) return;
            phase ^= 1u;
        } else {
            if (a.psi_in)
                load_tile_sw<K, kTyA>(tile, a.psi_in + p * plane_px, 0.0f, y0, x0, a.H, a.W, a.circular);
            else
                fill_tile_const<K, kTyA>(tile, __ldg(a.means + p), y0, x0, a.H, a.W, a.circular);
            __syncthreads();
        }
        const int t_next = t + gridDim.x;
        int left = passes;
        for (int g = 0; g < a.ft.n_groups; ++g) {
            bool used = false;
            for (int v = a.view_lo; v < a.view_hi; ++v) used |= (a.ft.group[v] == g);
            if (!used) continue;
            const int lead = a.ft.group_leader[g];
            float acc[G::H_PER_THREAD][kNC];
#pragma unroll
            for (int h = 0; h < G::H_PER_THREAD; ++h)
#pragma unroll
                for (int j = 0; j < kNC; ++j) acc[h][j] = 0.0f;
            // the first view of the group: its uint16 data for this thread's
            // items are requested before the last horizontal pass, so that the
            // loads land while the FMAs run
            int v_first = a.view_hi;
            for (int v = a.view_hi - 1; v >= a.view_lo; --v)
                if (a.ft.group[v] == g) v_first = v;
            const bool pre = kp.vec16 && a.phi_u16;
            // weighted runs have zero-weight regions whose only signal comes
            // through the factors' tails: full taps there
            const unsigned sm = a.weights ? 0u : a.ft.short_mask[lead];
            uint4 pf[G::H_PER_THREAD][2];
            for (int q = 0; q < a.ft.rank[lead]; ++q) {
                const float *tq = kp.taps + (a.ft.tap_off[lead] + q) * 2 * K;
                vertical_pass_sel<K, kTyA>(sm & 1u, sm & 2u, tile, stage, tq);
                __syncthreads();
                if (--left == 0 && use_tma && threadIdx.x == 0 && t_next < n_tiles) {
                    const TileCoord c = tile_coord<K, kTyA>(t_next, tiles_x, tiles_y);
                    tma::fence_proxy_async_smem();
                    tma::mbar_arrive_expect_tx(bar, G::TILE_BYTES);
                    tma::load_3d(tile, &kp.map, bar, c.x0 - G::R4, c.y0 - G::R, c.p);
                }
                if (pre && q == a.ft.rank[lead] - 1) {
                    const long long vplane = (static_cast<long long>(v_first) * a.P + p) * plane_px;
#pragma unroll
                    for (int h = 0; h < G::H_PER_THREAD; ++h) {
                        int y, x;
                        item_origin<K, kTyA>(h, y0, x0, y, x);
                        if (y < a.H && x < a.W) {
                            const uint4 *src = reinterpret_cast<const uint4 *>(
                                static_cast<const uint16_t *>(a.phi) + vplane + static_cast<long long>(y) * a.W + x);
                            pf[h][0] = __ldg(src);
                            pf[h][1] = __ldg(src + 1);
                        }
                    }
                }
                if (sm & 2u)
                    horizontal_pass<K, short_taps<K>(), kTyA>(stage, tq + K, acc);
                else
                    horizontal_pass<K, K, kTyA>(stage, tq + K, acc);
                __syncthreads();
            }
            // ratio epilogue per item (16 consecutive pixels of one row)
            for (int v = a.view_lo; v < a.view_hi; ++v) {
                if (a.ft.group[v] != g) continue;
                const long long vplane = (static_cast<long long>(v) * a.P + p) * plane_px;
#pragma unroll
                for (int h = 0; h < G::H_PER_THREAD; ++h) {
                    int y, x;
                    item_origin<K, kTyA>(h, y0, x0, y, x);
                    if (y >= a.H || x >= a.W) continue;
                    const int n = min(kNC, a.W - x);
                    const long long off = vplane + static_cast<long long>(y) * a.W + x;
                    float ph[kNC];
                    if (pre && v == v_first) {
                        const unsigned w[8] = {pf[h][0].x, pf[h][0].y, pf[h][0].z, pf[h][0].w,
                                               pf[h][1].x, pf[h][1].y, pf[h][1].z, pf[h][1].w};
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            ph[2 * k] = static_cast<float>(w[k] & 0xffffu);
                            ph[2 * k + 1] = static_cast<float>(w[k] >> 16);
                        }
                    } else {
#pragma unroll
                        for (int q4 = 0; q4 < kNC / 4; ++q4) {
                            float f[4];
                            load4(a.phi, a.phi_u16, off + 4 * q4, kp.vec_ok && n == kNC, max(0, min(4, n - 4 * q4)), f);
#pragma unroll
                            for (int e = 0; e < 4; ++e) ph[4 * q4 + e] = f[e];
                        }
                    }
                    if (a.weights) {   // weighted MV-RL: w_v phi_v / blur
                        const long long woff = (a.weights_bcast ? v * plane_px : vplane) +
                                               static_cast<long long>(y) * a.W + x;
#pragma unroll
                        for (int q4 = 0; q4 < kNC / 4; ++q4) {
                            float f[4];
                            load4(a.weights, 0, woff + 4 * q4, kp.vec_ok && n == kNC, max(0, min(4, n - 4 * q4)), f);
#pragma unroll
                            for (int e = 0; e < 4; ++e) ph[4 * q4 + e] *= f[e];
                        }
                    }
#pragma unroll
                    for (int q4 = 0; q4 < kNC / 4; ++q4) {
                        float r[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            r[e] = a.store_blur ? acc[h][4 * q4 + e]
                                                : __fdiv_rn(ph[4 * q4 + e], fmaxf(acc[h][4 * q4 + e], a.eps));
                        store4(a.ratio + off + 4 * q4, kp.vec_ok && n == kNC, max(0, min(4, n - 4 * q4)), r);
                    }
                }
            }
        }
    }
}

// Persistent like kernel A.  The ratio box of the next (tile, view) is
// requested right after the last vertical pass of the current view.
template <int K>
__global__ void __launch_bounds__(kThreads, Geo<K, kTyB>::MIN_BLOCKS)
correlate_update_kernel(const __grid_constant__ KParams kp) {
    using G = Geo<K, kTyB>;
    const FusedArgs &a = kp.a;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 8);
    float *tile = reinterpret_cast<float *>(smem + kTileOffset);
    float *stage = tile + G::BOX_H * G::BOX_W;

    const int tiles_x = (a.W + G::TX - 1) / G::TX;
    const int tiles_y = (a.H + G::TY - 1) / G::TY;
    const int n_tiles = tiles_x * tiles_y * a.P;
    const long long plane_px = static_cast<long long>(a.H) * a.W;
    const bool use_tma = kp.use_tma;
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        if (use_tma) {
            tma::mbar_init(bar, 1);
            tma::fence_barrier_init();
        }
    }
    __syncthreads();
    int t = blockIdx.x;
    if (use_tma && threadIdx.x == 0 && t < n_tiles) {
        const TileCoord c = tile_coord<K, kTyB>(t, tiles_x, tiles_y);
        tma::mbar_arrive_expect_tx(bar, G::TILE_BYTES);
        tma::load_3d(tile, &kp.map, bar, c.x0 - G::R4, c.y0 - G::R, a.view_lo * a.P + c.p);
    }
    uint32_t phase = 0;
    for (; t < n_tiles; t += gridDim.x) {
        const TileCoord tc = tile_coord<K, kTyB>(t, tiles_x, tiles_y);
        const int p = tc.p, y0 = tc.y0, x0 = tc.x0;
        const int t_next = t + gridDim.x;
        // the tile's estimate rows, read by the update epilogue after every
        // view's passes, are requested into L2 now: one 128-byte line per
        // thread (TY rows x TX columns = TY * 4 lines)
        if (a.psi_in && threadIdx.x < G::TY * (G::TX / 32)) {
            const int row = threadIdx.x / (G::TX / 32), seg = threadIdx.x % (G::TX / 32);
            const int y = y0 + row, x = x0 + 32 * seg;
            if (y < a.H && x < a.W)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psi_in + p * plane_px + static_cast<long long>(y) * a.W + x));
        }
        float prod[G::H_PER_THREAD][kNC];
#pragma unroll
        for (int h = 0; h < G::H_PER_THREAD; ++h)
#pragma unroll
            for (int j = 0; j < kNC; ++j) prod[h][j] = 1.0f;

        for (int v = a.view_lo; v < a.view_hi; ++v) {
            if (use_tma) {
                if (!wait_tile(bar, phase, a, abort_flag)) return;
                phase ^= 1u;
            } else {
                const float *rsrc = a.ratio + (static_cast<long long>(v) * a.P + p) * plane_px;
                load_tile_sw<K, kTyB>(tile, rsrc, 0.0f, y0, x0, a.H, a.W, a.circular);
                __syncthreads();
            }
            // the ratio box of the next (tile, view), requested once the tile is free
            auto prefetch_next = [&]() {
                if (!use_tma || threadIdx.x != 0) return;
                int nt = t, nv = v + 1;
                if (nv >= a.view_hi) {
                    nt = t_next;
                    nv = a.view_lo;
                }
                if (nt < n_tiles) {
                    const TileCoord c2 = tile_coord<K, kTyB>(nt, tiles_x, tiles_y);
                    tma::fence_proxy_async_smem();
                    tma::mbar_arrive_expect_tx(bar, G::TILE_BYTES);
                    tma::load_3d(tile, &kp.map, bar, c2.x0 - G::R4, c2.y0 - G::R, nv * a.P + c2.p);
                }
            };
            const unsigned sm = a.weights ? 0u : a.ft.short_mask[v];
            if (a.ft.crank[v] == 1 && !a.wnorm) {
                const float *tq = kp.taps + a.ft.ctap_off[v] * 2 * K;
                vertical_pass_sel<K, kTyB>(sm & 4u, sm & 8u, tile, stage, tq);
                __syncthreads();
                prefetch_next();
                if (sm & 8u)
                    horizontal_pass_mul<K, short_taps<K>(), kTyB>(stage, tq + K, prod);
                else
                    horizontal_pass_mul<K, K, kTyB>(stage, tq + K, prod);
                __syncthreads();
            } else {
                float c[G::H_PER_THREAD][kNC];
#pragma unroll
                for (int h = 0; h < G::H_PER_THREAD; ++h)
#pragma unroll
                    for (int j = 0; j < kNC; ++j) c[h][j] = 0.0f;
                for (int q = 0; q < a.ft.crank[v]; ++q) {
                    const float *tq = kp.taps + (a.ft.ctap_off[v] + q) * 2 * K;
                    vertical_pass_sel<K, kTyB>(sm & 4u, sm & 8u, tile, stage, tq);
                    __syncthreads();
                    if (q == a.ft.crank[v] - 1) prefetch_next();
                    if (sm & 8u)
                        horizontal_pass<K, short_taps<K>(), kTyB>(stage, tq + K, c);
                    else
                        horizontal_pass<K, K, kTyB>(stage, tq + K, c);
                    __syncthreads();
                }
                if (a.wnorm) {   // weighted MV-RL: c / n_v, or 1 where no weighted pixel is in reach
                    const long long vplane =
                        a.weights_bcast ? v * plane_px : (static_cast<long long>(v) * a.P + p) * plane_px;
#pragma unroll
                    for (int h = 0; h < G::H_PER_THREAD; ++h) {
                        int y, x;
                        item_origin<K, kTyB>(h, y0, x0, y, x);
                        if (y >= a.H || x >= a.W) continue;
                        const int n = min(kNC, a.W - x);
                        const long long off = vplane + static_cast<long long>(y) * a.W + x;
#pragma unroll
                        for (int q4 = 0; q4 < kNC / 4; ++q4) {
                            float m[4];
                            load4(a.wnorm, 0, off + 4 * q4, kp.vec_ok && n == kNC, max(0, min(4, n - 4 * q4)), m);
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                c[h][4 * q4 + e] = m[e] >= 0.0f ? c[h][4 * q4 + e] * m[e] : 1.0f;
                        }
                    }
                }
#pragma unroll
                for (int h = 0; h < G::H_PER_THREAD; ++h)
#pragma unroll
                    for (int j = 0; j < kNC; ++j) prod[h][j] *= c[h][j];
            }
        }

        // update epilogue, row by row: psi' = psi * prod with whole row segments
        park_items<K, kTyB>(stage, prod);
        __syncthreads();
        row_epilogue<K, 1, kTyB>(a, kp.vec_ok, stage, p * plane_px, y0, x0,
                          a.psi_in ? 0.0f : __ldg(a.means + p));
        __syncthreads();   // the staging tile is rewritten by the next pass
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

// 3D FP32 tensor [D][H][W] with a (box_w x box_h x 1) box; zero fill outside.
bool encode_3d(CUtensorMap *m, const void *base, int W, int H, long long D, int box_w, int box_h) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H), static_cast<cuuint64_t>(D)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(W) * 4, static_cast<cuuint64_t>(W) * H * 4};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline bool aligned16(const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

template <int K, int TYF>
cudaError_t launch_one(const FusedArgs &a, int which, cudaStream_t s) {
    using G = Geo<K, TYF>;
    // the shared-memory opt-in is per function (kernel A or B) and device
    static unsigned long long attr_set[2] = {0, 0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set[which] & bit)) {
        const cudaError_t e =
            which == 0 ? cudaFuncSetAttribute(blur_ratio_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              G::SMEM_BYTES)
                       : cudaFuncSetAttribute(correlate_update_kernel<K>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set[which] |= bit;
    }
    // persistent grid: as many CTAs as fit on the device at once, at most one per tile
    static int resident[64][2] = {};
    if (!resident[dev & 63][which]) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (which == 0)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, blur_ratio_kernel<K>, kThreads, G::SMEM_BYTES);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, correlate_update_kernel<K>, kThreads,
                                                          G::SMEM_BYTES);
        resident[dev & 63][which] = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    }
    const long long n_tiles = static_cast<long long>((a.W + G::TX - 1) / G::TX) * ((a.H + G::TY - 1) / G::TY) * a.P;
    if (n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    long long ctas = resident[dev & 63][which];
    if (a.max_ctas > 0 && a.max_ctas < ctas) ctas = a.max_ctas;
    const dim3 grid(static_cast<unsigned>(n_tiles < ctas ? n_tiles : ctas));
    KParams kp;   // about 18 KB with the taps; the launch copies it
    std::memset(&kp, 0, sizeof kp);
    kp.a = a;
    if (a.ft.total_terms * 2 * K > kParamTaps || !a.taps_host) return cudaErrorInvalidValue;
    for (int tt = 0; tt < a.ft.total_terms; ++tt)
        std::memcpy(kp.taps + tt * 2 * K, a.taps_host + (static_cast<size_t>(tt) * 4 + (which == 0 ? 0 : 2)) * K,
                    2 * K * sizeof(float));
    const bool aligned = aligned16(a.phi) && aligned16(a.ratio) && aligned16(a.psi_out) &&
                         (a.weights == nullptr || aligned16(a.weights)) && (a.wnorm == nullptr || aligned16(a.wnorm)) &&
                         (a.psi_in == nullptr || aligned16(a.psi_in));
    kp.vec_ok = aligned && (a.W % 4 == 0);
    kp.vec16 = aligned && (a.W % 16 == 0);
    const bool tma_ok = !a.circular && (a.W % 4 == 0);
    if (which == 0) {
        if (tma_ok && a.psi_in && aligned16(a.psi_in))
            kp.use_tma = encode_3d(&kp.map, a.psi_in, a.W, a.H, a.P, G::BOX_W, G::BOX_H);
        blur_ratio_kernel<K><<<grid, kThreads, G::SMEM_BYTES, s>>>(kp);
    } else {
        if (tma_ok && aligned16(a.ratio))
            kp.use_tma = encode_3d(&kp.map, a.ratio, a.W, a.H, static_cast<long long>(a.ft.views) * a.P,
                                   G::BOX_W, G::BOX_H);
        correlate_update_kernel<K><<<grid, kThreads, G::SMEM_BYTES, s>>>(kp);
    }
    count_launch();
    return cudaGetLastError();
}

#define MVD_FUSED_CASES(X) \
    X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(27) X(29) X(31) \
    X(33) X(35) X(37) X(39) X(41) X(43) X(45) X(47)

cudaError_t dispatch(const FusedArgs &a, int which, cudaStream_t s) {
    switch (a.ft.K) {
#define MVD_CASE(k) \
    case k:         \
        return which == 0 ? launch_one<k, kTyA>(a, 0, s) : launch_one<k, kTyB>(a, 1, s);
        MVD_FUSED_CASES(MVD_CASE)
#undef MVD_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace

// Tile map of an FP32 [D][H][W] tensor for other translation units (the
// batch queue): false if the encoder is missing or rejects the layout.
bool encode_plane_map(CUtensorMap *m, const void *base, int W, int H, long long D, int box_w, int box_h) {
    if (!aligned16(base) || (static_cast<long long>(W) * 4) % 16 != 0) return false;
    return encode_3d(m, base, W, H, D, box_w, box_h);
}

}  // namespace fused

bool fused_supported(int K) { return K >= 1 && K <= kFusedMaxK && (K % 2) == 1; }

bool fused_taps_fit(const FactorTable &ft) { return ft.total_terms * 2 * ft.K <= fused::kParamTaps; }

void fused_tile_shape(int K, int *tile_h, int *tile_w) {
    switch (K) {
#define MVD_CASE(k)                       \
    case k:                               \
        *tile_h = fused::Geo<k>::TY;      \
        *tile_w = fused::Geo<k>::TX;      \
        return;
        MVD_FUSED_CASES(MVD_CASE)
#undef MVD_CASE
        default:
            *tile_h = *tile_w = 0;
    }
}

cudaError_t launch_fused_blur_ratio(const FusedArgs &a, cudaStream_t s) { return fused::dispatch(a, 0, s); }

cudaError_t launch_fused_correlate_update(const FusedArgs &a, cudaStream_t s) {
    return fused::dispatch(a, 1, s);
}

}  // namespace mvd
