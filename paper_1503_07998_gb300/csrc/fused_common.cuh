// Tile machinery shared by the two kernels of one fused MV-RL iteration
// (Supp. Note 1 update equation):
//   kernel A  blur psi with every view's PSF, ratio phi_v / max(blur, eps)
//   kernel B  correlate every ratio with its flipped PSF, multiply the views'
//             corrections and update psi.
// Each 2D convolution is a sum over SVD terms of a vertical 1D pass (from the
// halo'd input tile in shared memory into a staging tile) followed by a
// horizontal 1D pass (from the staging tile into registers).
//
// Both passes are written in correlation form out[i] = sum_m t[m] in[i+m]
// (the host reverses the factors for the blur).  Every thread keeps a
// register block of 16 outputs so that each shared-memory value it loads
// feeds up to K FMAs:
//   vertical:   item = (column, block of 16 rows); lanes run along columns, so
//               the 4-byte loads of a warp hit 32 distinct banks;
//   horizontal: item = (row, group of 16 columns); lanes run along rows and
//               the staging tile's row pitch is an odd multiple of 4 floats,
//               so every 8-lane phase of a 16-byte load hits 8 distinct
//               4-bank groups.
//
// The input tile is the TMA box [BOX_H][BOX_W]: rows y0-R .. y0+TY+R-1 and
// columns x0-R4 .. x0+TX+R4-1, where R4 = R rounded up to a multiple of 4 so
// that the box starts on a 16-byte boundary; the vertical pass reads its
// TX+2R columns from column COL0 = R4-R on.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "mvd_internal.h"
#include "tma.cuh"

namespace mvd {
namespace fused {

constexpr int kThreads = 256;
template <int K>
__host__ __device__ constexpr int short_taps() { return short_tap_count(K); }
constexpr int kNR = 16;      // rows per vertical item
constexpr int kNC = 16;      // columns per horizontal item
constexpr int kTX = 128;     // output tile width
constexpr int kHeaderBytes = 128;   // mbarrier + abort flag
constexpr int kTileOffset = kHeaderBytes;   // a multiple of 128 for the TMA destination
// Two / three CTAs per SM: 228 KB per SM minus 1 KB reserved per CTA.
constexpr int kTwoCtaSmem = 113 * 1024;
constexpr int kThreeCtaSmem = 75 * 1024;

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Row pitch >= w with pitch/4 odd (see the bank argument above).
__host__ __device__ constexpr int odd_quad_pitch(int w) {
    return ((round_up(w, 4) / 4) % 2 == 1) ? round_up(w, 4) : round_up(w, 4) + 4;
}

// TYF = 0: the tile height of kernel A (64 rows while two CTAs fit on an
// SM, else 32); TYF > 0: that height, with three CTAs per SM where their
// shared memory fits (kernel B's choice: more resident warps hide its
// ratio-tile and estimate loads better than taller tiles save).
template <int K, int TYF = 0>
struct Geo {
    static constexpr int R = (K - 1) / 2;
    static constexpr int R4 = round_up(R, 4);
    static constexpr int TX = kTX;
    static constexpr int IN_W = TX + 2 * R;                  // columns the vertical pass computes
    static constexpr int BOX_W = TX + 2 * R4;                // tile pitch = TMA box width
    static constexpr int COL0 = R4 - R;
    static constexpr int HL = round_up(kNC + 2 * R, 4);       // horizontal load width
    static constexpr int VB_LD = odd_quad_pitch((TX / kNC - 1) * kNC + HL);
    static constexpr int smem_bytes(int ty) {
        return kTileOffset + ((ty + 2 * R) * BOX_W + ty * VB_LD) * 4;
    }
    // 64-row tiles while two CTAs still fit on an SM, else 32.
    static constexpr int TY = TYF ? TYF : ((smem_bytes(64) <= kTwoCtaSmem) ? 64 : 32);
    static constexpr int BOX_H = TY + 2 * R;
    static constexpr int SMEM_BYTES = smem_bytes(TY);
    static constexpr int TILE_BYTES = BOX_H * BOX_W * 4;
    static constexpr int V_ITEMS = IN_W * (TY / kNR);
    static constexpr int H_ITEMS = TY * (TX / kNC);
    static constexpr int H_PER_THREAD = H_ITEMS / kThreads;
    static_assert(H_ITEMS % kThreads == 0, "horizontal items must tile the CTA");
    static_assert(BOX_W <= 256 && BOX_H <= 256, "TMA box dimensions are at most 256");
    static constexpr int MIN_BLOCKS =
        (TYF && SMEM_BYTES <= kThreeCtaSmem) ? 3 : ((SMEM_BYTES <= kTwoCtaSmem) ? 2 : 1);
};

// Software tile load (circular boundary, unaligned planes): same layout as
// the TMA box.  src == nullptr means a constant plane of value `fill`
// (iteration 0 from the per-plane mean).  ZERO: zero outside the plane;
// CIRCULAR: indices modulo the plane size.
template <int K, int TYF = 0>
__device__ __forceinline__ void load_tile_sw(float *__restrict__ tile, const float *__restrict__ src,
                                             float fill, int y0, int x0, int H, int W, int circular) {
    using G = Geo<K, TYF>;
    constexpr int N = G::BOX_H * G::BOX_W;
    for (int idx = threadIdx.x; idx < N; idx += kThreads) {
        const int r = idx / G::BOX_W;
        const int c = idx - r * G::BOX_W;
        int gy = y0 - G::R + r;
        int gx = x0 - G::R4 + c;
        float v = 0.0f;
        if (circular) {
            gy %= H; if (gy < 0) gy += H;
            gx %= W; if (gx < 0) gx += W;
            v = src ? __ldg(src + static_cast<long long>(gy) * W + gx) : fill;
        } else if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            v = src ? __ldg(src + static_cast<long long>(gy) * W + gx) : fill;
        }
        tile[idx] = v;
    }
}

// The first iteration's tile: psi is the plane's mean inside the plane
// (and, for CIRCULAR, everywhere), zero outside for ZERO.  Same values as
// load_tile_sw with a null source, written as whole 16-byte quads.
template <int K, int TYF = 0>
__device__ __forceinline__ void fill_tile_const(float *__restrict__ tile, float fill, int y0, int x0, int H, int W,
                                                int circular) {
    using G = Geo<K, TYF>;
    static_assert(G::BOX_W % 4 == 0, "box rows are whole quads");
    constexpr int QW = G::BOX_W / 4;
    for (int q = threadIdx.x; q < G::BOX_H * QW; q += kThreads) {
        const int r = q / QW, c = 4 * (q - r * QW);
        const int gy = y0 - G::R + r, gx = x0 - G::R4 + c;
        const bool row_in = circular || (gy >= 0 && gy < H);
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = (row_in && (circular || (gx + e >= 0 && gx + e < W))) ? fill : 0.0f;
        *reinterpret_cast<float4 *>(tile + r * G::BOX_W + c) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// One vertical item: NR consecutive output rows r0.. of column c, with the
// KP central taps of the K-tap factor (KP = K: all of them).
template <int K, int NR, int KP, int TYF>
__device__ __forceinline__ void vertical_item(const float *__restrict__ tile, float *__restrict__ stage,
                                              const float (&t)[KP], int c, int r0) {
    using G = Geo<K, TYF>;
    constexpr int OFF = (K - KP) / 2;
    const float *col = tile + (r0 + OFF) * G::BOX_W + G::COL0 + c;
    float acc[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) acc[i] = 0.0f;
#pragma unroll
    for (int m = 0; m < NR + KP - 1; ++m) {
        const float x = col[m * G::BOX_W];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int j = m - i;
            if (j >= 0 && j < KP) acc[i] = fmaf(t[j], x, acc[i]);
        }
    }
    float *dst = stage + r0 * G::VB_LD + c;
#pragma unroll
    for (int i = 0; i < NR; ++i) dst[i * G::VB_LD] = acc[i];
}

// Vertical pass: stage[i][c] = sum_m t[m] * tile[i + m][COL0 + c] for the TY
// output rows and the columns that a horizontal pass of KH central taps
// reads: c = OFFH .. OFFH + TX + KH - 2 with OFFH = (K - KH) / 2 (all IN_W
// columns when KH = K).  The TX columns from OFFH on run as 16-row items
// (TX*TY/16 = a whole number of rounds of the CTA), the KH - 1 halo columns
// after them as 8-row items (one more round at most), so that no warp idles
// for long at the barrier that follows.  Staging columns outside that range
// keep stale values; the horizontal pass loads some of them as parts of
// quads but multiplies none of them.
template <int K, int KP = K, int TYF = 0, int KH = K>
__device__ __forceinline__ void vertical_pass(const float *__restrict__ tile, float *__restrict__ stage,
                                              const float *__restrict__ taps_s) {
    using G = Geo<K, TYF>;
    static_assert((G::TX * (G::TY / kNR)) % kThreads == 0, "main vertical items must tile the CTA");
    static_assert(KH >= 1 && KH <= K && (K - KH) % 2 == 0, "horizontal taps are central");
    constexpr int OFF = (K - KP) / 2;
    constexpr int OFFH = (K - KH) / 2;
    float t[KP];
#pragma unroll
    for (int m = 0; m < KP; ++m) t[m] = taps_s[OFF + m];
    for (int it = threadIdx.x; it < G::TX * (G::TY / kNR); it += kThreads) {
        const int rb = it / G::TX;
        vertical_item<K, kNR, KP, TYF>(tile, stage, t, OFFH + it - rb * G::TX, rb * kNR);
    }
    if (KH > 1) {
        constexpr int HC = KH > 1 ? KH - 1 : 1;   // halo columns OFFH+TX .. OFFH+TX+KH-2
        for (int it = threadIdx.x; it < HC * (G::TY / 8); it += kThreads) {
            const int r8 = it / HC;
            vertical_item<K, 8, KP, TYF>(tile, stage, t, OFFH + G::TX + (it - r8 * HC), r8 * 8);
        }
    }
}

// The vertical pass for a factor pair whose vertical (vs) and horizontal
// (hs) factors run their short_taps<K>() central taps (true) or all K.
template <int K, int TYF = 0>
__device__ __forceinline__ void vertical_pass_sel(bool vs, bool hs, const float *__restrict__ tile,
                                                  float *__restrict__ stage, const float *__restrict__ taps_s) {
    constexpr int S = short_taps<K>();
    if (vs) {
        if (hs) vertical_pass<K, S, TYF, S>(tile, stage, taps_s);
        else vertical_pass<K, S, TYF, K>(tile, stage, taps_s);
    } else {
        if (hs) vertical_pass<K, K, TYF, S>(tile, stage, taps_s);
        else vertical_pass<K, K, TYF, K>(tile, stage, taps_s);
    }
}

// Packed FP32 pairs (lo, hi) in one 64-bit register pair: one fma.rn.f32x2
// does two independent FP32 FMAs with the rounding of two fmaf calls.
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// One horizontal item on packed pairs: out[j] = sum_m t[m] in[j + m + D]
// for j = 0..15, as 8 output pairs (2p, 2p+1).  Output pair p takes tap m
// times the input pair starting at 2p + m + D: the quads' aligned pairs for
// even starts, pairs straddling two lanes of the quad (rebuilt) for odd
// ones.  Same products and the same summation order per output as the
// scalar form.
template <int KP, int D, int NIN>
__device__ __forceinline__ void hrow_x2(const float4 *__restrict__ src, const float (&t)[KP],
                                        unsigned long long (&A)[kNC / 2]) {
    float prev = 0.0f;
#pragma unroll
    for (int q = 0; q < (NIN + 3) / 4; ++q) {
        const float4 v = src[q];
        // pairs starting at 4q-1, 4q, 4q+1, 4q+2
        const unsigned long long pr[4] = {pk2(prev, v.x), pk2(v.x, v.y), pk2(v.y, v.z), pk2(v.z, v.w)};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = 4 * q - 1 + e;     // pair start (input index from S)
            if (i < 0 || i + 1 >= NIN) continue;
#pragma unroll
            for (int p = 0; p < kNC / 2; ++p) {
                const int m = i - 2 * p - D;
                if (m >= 0 && m < KP) A[p] = ffma2(pk2(t[m], t[m]), pr[e], A[p]);
            }
        }
        prev = v.w;
    }
}

// Horizontal pass for this thread's items: acc[h][j] += sum_m t[m] * stage[row][16g + j + m].
// Inputs stream through registers four at a time (one 16-byte load), each
// feeding every output it reaches, so only the 16 accumulators, the taps
// and one quad are live.
// With KP < K only the KP central taps run: inputs start at the quad
// boundary S <= OFF below the first one used, D = OFF - S places them.
template <int K, int KP = K, int TYF = 0>
__device__ __forceinline__ void horizontal_pass(const float *__restrict__ stage,
                                                const float *__restrict__ taps_s,
                                                float (&acc)[Geo<K, TYF>::H_PER_THREAD][kNC]) {
    using G = Geo<K, TYF>;
    constexpr int OFF = (K - KP) / 2, S = OFF & ~3, D = OFF - S;
    constexpr int NIN = kNC + KP - 1 + D;      // inputs read from S on
    float t[KP];
#pragma unroll
    for (int m = 0; m < KP; ++m) t[m] = taps_s[OFF + m];
#pragma unroll
    for (int h = 0; h < G::H_PER_THREAD; ++h) {
        const int it = threadIdx.x + h * kThreads;
        const int row = it % G::TY;
        const int g = it / G::TY;
        const float4 *src = reinterpret_cast<const float4 *>(stage + row * G::VB_LD + g * kNC + S);
        unsigned long long A[kNC / 2];
#pragma unroll
        for (int p = 0; p < kNC / 2; ++p) A[p] = pk2(acc[h][2 * p], acc[h][2 * p + 1]);
        hrow_x2<KP, D, NIN>(src, t, A);
#pragma unroll
        for (int p = 0; p < kNC / 2; ++p) upk2(A[p], acc[h][2 * p], acc[h][2 * p + 1]);
    }
}

// Horizontal pass of a one-term factorisation whose result multiplies into
// `prod` item by item (the running product over views of kernel B), so no
// second set of accumulators stays live.
template <int K, int KP = K, int TYF = 0>
__device__ __forceinline__ void horizontal_pass_mul(const float *__restrict__ stage,
                                                    const float *__restrict__ taps_s,
                                                    float (&prod)[Geo<K, TYF>::H_PER_THREAD][kNC]) {
    using G = Geo<K, TYF>;
    constexpr int OFF = (K - KP) / 2, S = OFF & ~3, D = OFF - S;
    constexpr int NIN = kNC + KP - 1 + D;
    float t[KP];
#pragma unroll
    for (int m = 0; m < KP; ++m) t[m] = taps_s[OFF + m];
#pragma unroll
    for (int h = 0; h < G::H_PER_THREAD; ++h) {
        const int it = threadIdx.x + h * kThreads;
        const float4 *src =
            reinterpret_cast<const float4 *>(stage + (it % G::TY) * G::VB_LD + (it / G::TY) * kNC + S);
        unsigned long long A[kNC / 2];
#pragma unroll
        for (int p = 0; p < kNC / 2; ++p) A[p] = 0ull;
        hrow_x2<KP, D, NIN>(src, t, A);
#pragma unroll
        for (int p = 0; p < kNC / 2; ++p) {
            float lo, hi;
            upk2(A[p], lo, hi);
            prod[h][2 * p] *= lo;
            prod[h][2 * p + 1] *= hi;
        }
    }
}

// Park this thread's horizontal-pass results in the staging tile at their
// output positions (row, 16g + j).  Lanes run along rows and the pitch is an
// odd multiple of 4 floats, so the 16-byte stores are conflict-free.  The
// caller synchronises before the tile is read back row by row.
template <int K, int TYF = 0>
__device__ __forceinline__ void park_items(float *__restrict__ stage,
                                           const float (&acc)[Geo<K, TYF>::H_PER_THREAD][kNC]) {
    using G = Geo<K, TYF>;
#pragma unroll
    for (int h = 0; h < G::H_PER_THREAD; ++h) {
        const int it = threadIdx.x + h * kThreads;
        float4 *dst = reinterpret_cast<float4 *>(stage + (it % G::TY) * G::VB_LD + (it / G::TY) * kNC);
#pragma unroll
        for (int q = 0; q < kNC / 4; ++q)
            dst[q] = make_float4(acc[h][4 * q], acc[h][4 * q + 1], acc[h][4 * q + 2], acc[h][4 * q + 3]);
    }
}

// Output coordinates of horizontal item h of this thread.
template <int K, int TYF = 0>
__device__ __forceinline__ void item_origin(int h, int y0, int x0, int &y, int &x) {
    using G = Geo<K, TYF>;
    const int it = threadIdx.x + h * kThreads;
    y = y0 + it % G::TY;
    x = x0 + (it / G::TY) * kNC;
}

}  // namespace fused
}  // namespace mvd
