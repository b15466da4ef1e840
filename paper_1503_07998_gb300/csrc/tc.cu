// Tensor-core route of the fused MV-RL iteration (Supp. Note 1 update
// equation): the same two kernels as the FP32 route,
//
//   tc_blur_ratio        r_v = phi_v / max(psi * P_v, eps)
//   tc_correlate_update  psi <- psi * prod_v (r_v (*) P_v^*)
//
// with every separable 1D pass of every SVD term run as a banded (Toeplitz)
// matrix product on the tcgen05 tensor cores.  The ratio, the product over
// views and the update stay FP32 on the CUDA cores.
//
// Precision (BF16x3): each FP32 operand x is split into hi = bf16(x) and
// lo = bf16(x - hi); a product a*b is formed as a_hi b_hi + a_lo b_hi +
// a_hi b_lo by three MMAs into one FP32 accumulator.  The dropped a_lo b_lo
// and the rounding of the lo parts leave about 2^-16 relative error per
// product, against 2^-24 for FP32 arithmetic.
//
// Tile: TY x 128 outputs of one plane (TY = 96 for K <= 33, 64 above); the
// input tile is 128 rows (TY + 2R of them used) x KA columns.
//
//   pass 1 (along x):  D1[y_in][x_out] = sum_k A1[y_in][k] T1[k][x_out]
//       A1 = input tile (BF16 hi/lo, K-major), T1 = Toeplitz matrix of the
//       horizontal taps, one 32-column output chunk per MMA group with a
//       K window of 32 + 2R (+ alignment) input columns;  D1 in tensor memory
//       (lanes = input rows, 128 columns).
//   hand-over: each thread reads its lane (one input row) of D1, splits the
//       values and stores them as A2 = D1^T (MN-major, x_out contiguous).
//   pass 2 (along y):  D2[x_out][y_out] = sum_k A2[x_out][k] T2[k][y_out]
//       T2 = Toeplitz matrix of the vertical taps, 32-row output chunks;
//       every SVD term accumulates into the same D2 (lanes = output columns).
//   epilogue: each thread reads its lane of D2, i.e. one output column, and
//       walks its rows: coalesced loads of phi / psi and stores of r / psi.
//
// Shared memory: the FP32 staging tile (TMA destination, later reused for
// A2), A1 hi/lo, and two buffers of Toeplitz operands built per term from
// the factor taps.  One CTA per SM (about 195-217 KB), 512 threads.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "mvd_internal.h"
#include "tc5.cuh"
#include "tma.cuh"

namespace mvd {
namespace tcr {

namespace {

constexpr int kThreads = 512;
constexpr long long kDrainBudget = 4000000000LL;
constexpr int kTmemCols = 256;

template <int K>
struct Geo {
    static constexpr int R = (K - 1) / 2;
    static constexpr int R4 = (R + 3) / 4 * 4;    // TMA x origin stays 16-byte aligned
    static constexpr int COL0 = R4 - R;           // input column of x0 - R within the staging tile
    static constexpr int TX = 128;
    static constexpr int TY = R == 0 ? 128 : (2 * R <= 32 ? 96 : 64);
    static constexpr int ROWS = 128;              // input rows = MMA M of pass 1
    static constexpr int WIN1 = (32 + COL0 + 2 * R + 15) / 16 * 16;
    static constexpr int NKS1 = WIN1 / 16;
    static constexpr int KA = 96 + WIN1;          // input columns
    static constexpr int NKB = KA / 8;
    static constexpr int WIN2 = (32 + 2 * R + 15) / 16 * 16;
    static constexpr int NKS2 = WIN2 / 16;
    static constexpr int NC2 = TY / 32;
    static constexpr int NE = TY / 4;             // output rows per epilogue thread
    static constexpr int STAGE_BYTES = ROWS * KA * 4;
    static constexpr uint32_t A1_LBO = 128 * 16 + 16;   // k-group stride; +16 B spreads banks
    static constexpr int A1_BYTES = NKB * A1_LBO;
    static constexpr uint32_t A2_LBO = 128;              // k-group stride (8 rows x 16 B)
    static constexpr uint32_t A2_SBO = 128 * 16;         // m-group stride (128 k rows x 16 B)
    static constexpr int A2_BYTES = 16 * A2_SBO;
    static constexpr uint32_t T_LBO = 32 * 16;           // k-group stride of a 32-column operand
    static constexpr uint32_t T_SBO = 128;
    static constexpr int T1_BYTES = WIN1 / 8 * T_LBO;
    static constexpr int T2_BYTES = WIN2 / 8 * T_LBO;
    static constexpr int TBUF_BYTES = 2 * (T1_BYTES + T2_BYTES);
    static constexpr int OFF_STAGE = 1024;
    static constexpr int OFF_A1 = OFF_STAGE + STAGE_BYTES;
    static constexpr int OFF_T = OFF_A1 + 2 * A1_BYTES;
    static constexpr int SMEM_USED = OFF_T + 2 * TBUF_BYTES;
    static constexpr int SMEM_BYTES = SMEM_USED + 128;   // room to align the dynamic base
    static_assert(TY + 2 * R <= ROWS, "input rows fit the pass-1 M");
    static_assert((NC2 - 1) * 32 + WIN2 <= ROWS, "pass-2 windows stay inside the input rows");
    static_assert(96 + WIN1 == KA && KA % 16 == 0, "pass-1 windows");
    static_assert(2 * A2_BYTES <= STAGE_BYTES, "A2 fits in the staging tile");
    static_assert(128 + TY <= kTmemCols, "D1 + D2 columns");
    static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
};

struct TcParams {
    CUtensorMap map;   // psi (kernel A) or the ratio planes (kernel B); valid if use_tma
    FusedArgs a;
    int use_tma;
};

__device__ __forceinline__ unsigned char *align128(unsigned char *p) {
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 127) & ~static_cast<uintptr_t>(127));
}

// Split 8 FP32 values into BF16 hi and lo parts (8 each, element 0 in the low
// half of the first word).
__device__ __forceinline__ void split8(const float (&x)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
        h[i] = *reinterpret_cast<const uint32_t *>(&hb);
        const float h0 = __uint_as_float(h[i] << 16);
        const float h1 = __uint_as_float(h[i] & 0xFFFF0000u);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * i] - h0, x[2 * i + 1] - h1);
        l[i] = *reinterpret_cast<const uint32_t *>(&lb);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void sts128(unsigned char *p, const uint4 &v) { *reinterpret_cast<uint4 *>(p) = v; }

// Software fill of the staging tile: rows y0-R.., columns x0-R4..; zero
// outside the plane (ZERO) or wrapped (CIRCULAR); `src` null = constant fill.
template <int K>
__device__ void load_stage_sw(float *__restrict__ stage, const float *__restrict__ src, float fill, int y0, int x0,
                              int H, int W, int circular) {
    using G = Geo<K>;
    constexpr int N = G::ROWS * G::KA;
    for (int idx = threadIdx.x; idx < N; idx += kThreads) {
        const int r = idx / G::KA;
        const int c = idx - r * G::KA;
        int gy = y0 - G::R + r;
        int gx = x0 - G::R4 + c;
        float v = 0.0f;
        if (circular) {
            gy %= H;
            if (gy < 0) gy += H;
            gx %= W;
            if (gx < 0) gx += W;
            v = src ? __ldg(src + static_cast<long long>(gy) * W + gx) : fill;
        } else if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            v = src ? __ldg(src + static_cast<long long>(gy) * W + gx) : fill;
        }
        stage[idx] = v;
    }
}

// Staging tile (FP32, row-major) -> A1 hi/lo (K-major BF16).  Item = one
// row and 8 consecutive columns.
template <int K>
__device__ __forceinline__ void convert_a1(const float *__restrict__ stage, unsigned char *a1) {
    using G = Geo<K>;
    constexpr int ITEMS = G::ROWS * G::NKB;
    for (int it = threadIdx.x; it < ITEMS; it += kThreads) {
        const int m = it / G::NKB;
        const int kb = it - m * G::NKB;
        const float4 *src = reinterpret_cast<const float4 *>(stage + m * G::KA + 8 * kb);
        const float4 p = src[0], q = src[1];
        const float x[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
        uint4 hi, lo;
        split8(x, hi, lo);
        const uint32_t off = static_cast<uint32_t>(m) * 16 + static_cast<uint32_t>(kb) * G::A1_LBO;
        sts128(a1 + off, hi);
        sts128(a1 + G::A1_BYTES + off, lo);
    }
}

// Toeplitz operands of one term (correlation-form taps: out(i) = sum_j t[j]
// in(i + j - R)): T1[k][n] = w[k - n - COL0] (horizontal), T2[k][n] = u[k - n]
// (vertical), each K-major BF16 hi/lo.  Item = one column n and 8 rows k.
template <int K>
__device__ __forceinline__ void build_toeplitz(const float *__restrict__ u, const float *__restrict__ w,
                                               unsigned char *tb) {
    using G = Geo<K>;
    constexpr int I1 = 32 * (G::WIN1 / 8), I2 = 32 * (G::WIN2 / 8);
    for (int it = threadIdx.x; it < I1 + I2; it += kThreads) {
        const bool second = it >= I1;
        const int i2 = second ? it - I1 : it;
        const int n = i2 & 31, kg = i2 >> 5;
        const float *t = second ? u : w;
        const int off = second ? 0 : G::COL0;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = 8 * kg + e - n - off;
            x[e] = (j >= 0 && j < K) ? __ldg(t + j) : 0.0f;
        }
        uint4 hi, lo;
        split8(x, hi, lo);
        unsigned char *base = tb + (second ? 2 * G::T1_BYTES : 0);
        const int bytes = second ? G::T2_BYTES : G::T1_BYTES;
        const uint32_t addr = (n & 7) * 16 + (n >> 3) * G::T_SBO + kg * G::T_LBO;
        sts128(base + addr, hi);
        sts128(base + bytes + addr, lo);
    }
}

// Pass 1 MMAs (one thread): D1 columns [32c, 32c+32) for c = 0..3.
template <int K>
__device__ __forceinline__ void issue_pass1(uint32_t tmem, uint32_t a1, uint32_t tb) {
    using G = Geo<K>;
    constexpr uint32_t idesc = tc5::idesc_bf16(128, 32, false, false);
    const uint32_t a1lo = a1 + G::A1_BYTES, t1lo = tb + G::T1_BYTES;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
#pragma unroll 1
        for (int s = 0; s < G::NKS1; ++s) {
            const uint32_t ao = static_cast<uint32_t>(4 * c + 2 * s) * G::A1_LBO;
            const uint32_t bo = static_cast<uint32_t>(2 * s) * G::T_LBO;
            const uint64_t ah = tc5::sdesc(a1 + ao, G::A1_LBO, 128), al = tc5::sdesc(a1lo + ao, G::A1_LBO, 128);
            const uint64_t bh = tc5::sdesc(tb + bo, G::T_LBO, G::T_SBO), bl = tc5::sdesc(t1lo + bo, G::T_LBO, G::T_SBO);
            const uint32_t d = tmem + 32 * c;
            tc5::mma_bf16(d, al, bh, idesc, s > 0);
            tc5::mma_bf16(d, ah, bl, idesc, 1);
            tc5::mma_bf16(d, ah, bh, idesc, 1);
        }
    }
}

// Pass 2 MMAs (one thread): D2 columns [128 + 32c, +32) for c < NC2.
template <int K>
__device__ __forceinline__ void issue_pass2(uint32_t tmem, uint32_t a2, uint32_t tb, bool accumulate) {
    using G = Geo<K>;
    constexpr uint32_t idesc = tc5::idesc_bf16(128, 32, true, false);
    const uint32_t a2lo = a2 + G::A2_BYTES;
    const uint32_t t2 = tb + 2 * G::T1_BYTES, t2lo = t2 + G::T2_BYTES;
#pragma unroll 1
    for (int c = 0; c < G::NC2; ++c) {
#pragma unroll 1
        for (int s = 0; s < G::NKS2; ++s) {
            const uint32_t ao = static_cast<uint32_t>(4 * c + 2 * s) * G::A2_LBO;
            const uint32_t bo = static_cast<uint32_t>(2 * s) * G::T_LBO;
            const uint64_t ah = tc5::sdesc(a2 + ao, G::A2_LBO, G::A2_SBO), al = tc5::sdesc(a2lo + ao, G::A2_LBO, G::A2_SBO);
            const uint64_t bh = tc5::sdesc(t2 + bo, G::T_LBO, G::T_SBO), bl = tc5::sdesc(t2lo + bo, G::T_LBO, G::T_SBO);
            const uint32_t d = tmem + 128 + 32 * c;
            tc5::mma_bf16(d, al, bh, idesc, (accumulate || s > 0) ? 1u : 0u);
            tc5::mma_bf16(d, ah, bl, idesc, 1);
            tc5::mma_bf16(d, ah, bh, idesc, 1);
        }
    }
}

// D1 -> A2: warp w reads lanes 32*(w%4).. (input rows) x columns 32*(w/4)..
// (one output chunk) and stores them transposed, BF16 hi/lo, MN-major.
template <int K>
__device__ __forceinline__ void handover(uint32_t tmem, unsigned char *a2) {
    using G = Geo<K>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qd = warp & 3, c = warp >> 2;
    uint32_t r[32];
    tc5::ld32(tmem + (static_cast<uint32_t>(32 * qd) << 16) + 32 * c, r);
    tc5::wait_ld();
    const uint32_t row = 32 * qd + lane;   // k index of A2
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float x[8] = {__uint_as_float(r[8 * v]),     __uint_as_float(r[8 * v + 1]),
                            __uint_as_float(r[8 * v + 2]), __uint_as_float(r[8 * v + 3]),
                            __uint_as_float(r[8 * v + 4]), __uint_as_float(r[8 * v + 5]),
                            __uint_as_float(r[8 * v + 6]), __uint_as_float(r[8 * v + 7])};
        uint4 hi, lo;
        split8(x, hi, lo);
        const uint32_t off = static_cast<uint32_t>(4 * c + v) * G::A2_SBO + row * 16;
        sts128(a2 + off, hi);
        sts128(a2 + G::A2_BYTES + off, lo);
    }
}

// This thread's column of D2: NE consecutive output rows.
template <int K>
__device__ __forceinline__ void read_d2(uint32_t tmem, float (&d)[Geo<K>::NE]) {
    using G = Geo<K>;
    const int warp = threadIdx.x >> 5;
    const int qd = warp & 3, cg = warp >> 2;
    const uint32_t base = tmem + (static_cast<uint32_t>(32 * qd) << 16) + 128 + cg * G::NE;
#pragma unroll
    for (int j = 0; j < G::NE / 8; ++j) tc5::ld8(base + 8 * j, reinterpret_cast<uint32_t *>(d) + 8 * j);
    tc5::wait_ld();
}

// Bounded wait on `bar`: thread 0 polls while the others park at the CTA
// barrier (spinning warps would take issue slots from the MMA-issuing
// thread); on a timeout flag the status, drain once more and make the CTA
// leave.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, const FusedArgs &a,
                                         volatile int *abort_flag) {
    if (threadIdx.x == 0) {
        if (a.wait_budget < 0 || !tma::mbar_wait_bounded(bar, parity, a.wait_budget)) {
            atomicOr(a.err, kDevTimeout);
            tma::mbar_wait_bounded(bar, parity, kDrainBudget);
            *abort_flag = 1;
        }
    }
    __syncthreads();
    return *abort_flag == 0;
}

struct Tile {
    int p, y0, x0;
};

template <int K>
__device__ __forceinline__ Tile tile_of(int t, int tiles_x, int tiles_y) {
    using G = Geo<K>;
    const int per_plane = tiles_x * tiles_y;
    const int p = t / per_plane;
    const int r = t - p * per_plane;
    const int ty = r / tiles_x;
    return {p, ty * G::TY, (r - ty * tiles_x) * G::TX};
}

// Shared setup: barriers, tensor memory.
struct Smem {
    uint64_t *bar_tma, *bar_mma;
    volatile int *abort_flag;
    uint32_t *tmem_slot;
};

__device__ __forceinline__ Smem setup(unsigned char *smem) {
    Smem s;
    s.bar_tma = reinterpret_cast<uint64_t *>(smem);
    s.bar_mma = reinterpret_cast<uint64_t *>(smem + 8);
    s.abort_flag = reinterpret_cast<volatile int *>(smem + 16);
    s.tmem_slot = reinterpret_cast<uint32_t *>(smem + 20);
    if (threadIdx.x == 0) {
        tma::mbar_init(s.bar_tma, 1);
        tma::mbar_init(s.bar_mma, 1);
        *s.abort_flag = 0;
        tma::fence_barrier_init();
    }
    if (threadIdx.x < 32) {
        tc5::alloc(s.tmem_slot, kTmemCols);
        tc5::relinquish();
    }
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    return s;
}

__device__ __forceinline__ void teardown(uint32_t tmem) {
    tc5::fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tc5::dealloc(tmem, kTmemCols);
}

// The Toeplitz operands of every term a launch uses stay resident (built once
// per CTA) when there are at most this many; otherwise two buffers alternate
// and each term's operands are built before its MMAs.
constexpr int kResidentTerms = 2;

// One group of SVD terms (a PSF's blur, or a view's correlation) on the input
// tile in A1: D2 = sum over the terms.  Returns with every MMA issued and
// their completion committed to bar_mma (the caller waits).  With
// `a2_last_in_a1` the last term's A2 goes to the A1 region (A1 is not read
// again), so the staging tile is free early: thread 0 calls `stage_free()`
// as soon as nothing can read it any more.  resident_slot >= 0: the terms'
// operands are resident from that slot on.  False if a wait timed out.
template <int K, typename F>
__device__ bool run_terms(const FusedArgs &a, const Smem &s, uint32_t tmem, unsigned char *smem, int term0,
                          int n_terms, int kind_u, int kind_w, int resident_slot, bool a2_last_in_a1,
                          F &&stage_free, uint32_t &ph_mma, int &tbuf) {
    using G = Geo<K>;
    unsigned char *a1 = smem + G::OFF_A1;
    for (int q = 0; q < n_terms; ++q) {
        const bool last = q == n_terms - 1;
        unsigned char *tb;
        if (resident_slot >= 0) {
            tb = smem + G::OFF_T + (resident_slot + q) * G::TBUF_BYTES;
        } else {
            tb = smem + G::OFF_T + tbuf * G::TBUF_BYTES;
            tbuf ^= 1;
            const float *tq = a.taps + static_cast<long long>(term0 + q) * 4 * K;
            build_toeplitz<K>(tq + kind_u * K, tq + kind_w * K, tb);
            tma::fence_proxy_async_smem();
        }
        tc5::fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc5::fence_after();
            issue_pass1<K>(tmem, tc5::smem_u32(a1), tc5::smem_u32(tb));
            tc5::commit(s.bar_mma);
            // one term: the staging tile was last read by the conversion
            if (last && a2_last_in_a1 && n_terms == 1) stage_free();
        }
        // pass 1 done, and with it every earlier MMA (D1 and the previous A2 are free)
        if (!wait_bar(s.bar_mma, ph_mma, a, s.abort_flag)) return false;
        ph_mma ^= 1;
        tc5::fence_after();
        if (threadIdx.x == 0 && last && a2_last_in_a1 && n_terms > 1) stage_free();
        unsigned char *a2 = (last && a2_last_in_a1) ? a1 : smem + G::OFF_STAGE;
        handover<K>(tmem, a2);
        tma::fence_proxy_async_smem();
        tc5::fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc5::fence_after();
            issue_pass2<K>(tmem, tc5::smem_u32(a2), tc5::smem_u32(tb), q > 0);
        }
    }
    if (threadIdx.x == 0) tc5::commit(s.bar_mma);
    return true;
}

// Wait for the MMAs run_terms committed; D2 is then readable.
__device__ __forceinline__ bool finish_terms(const FusedArgs &a, const Smem &s, uint32_t &ph_mma) {
    if (!wait_bar(s.bar_mma, ph_mma, a, s.abort_flag)) return false;
    ph_mma ^= 1;
    tc5::fence_after();
    return true;
}

// Build the operands of up to kResidentTerms terms once (slots 0, 1, ...).
template <int K>
__device__ __forceinline__ void build_resident(const FusedArgs &a, const int *terms, int n, int kind_u, int kind_w,
                                               unsigned char *smem) {
    using G = Geo<K>;
    for (int i = 0; i < n; ++i) {
        const float *tq = a.taps + static_cast<long long>(terms[i]) * 4 * K;
        build_toeplitz<K>(tq + kind_u * K, tq + kind_w * K, smem + G::OFF_T + i * G::TBUF_BYTES);
    }
    tma::fence_proxy_async_smem();
}

// Raw data of view v at this thread's output column and rows (NE values,
// uint16 or FP32 bits).  Nothing here consumes a loaded value, so all NE
// loads are in flight together; store_ratio converts them.
template <int K>
__device__ __forceinline__ void load_phi(const FusedArgs &a, int v, int p, int y0, int x,
                                         uint32_t (&phi)[Geo<K>::NE]) {
    using G = Geo<K>;
    const long long base = (static_cast<long long>(v) * a.P + p) * a.H * a.W + x;
    const int n = min(G::NE, a.H - y0);
    if (a.phi_u16) {
        const uint16_t *src = static_cast<const uint16_t *>(a.phi) + base;
#pragma unroll
        for (int j = 0; j < G::NE; ++j)
            phi[j] = j < n ? static_cast<uint32_t>(__ldg(src + static_cast<long long>(y0 + j) * a.W)) : 0u;
    } else {
        const float *src = static_cast<const float *>(a.phi) + base;
#pragma unroll
        for (int j = 0; j < G::NE; ++j)
            phi[j] = j < n ? __float_as_uint(__ldg(src + static_cast<long long>(y0 + j) * a.W)) : 0u;
    }
}

template <int K>
__device__ __forceinline__ void store_ratio(const FusedArgs &a, int v, int p, int y0, int x,
                                            const uint32_t (&phi)[Geo<K>::NE], const float (&d)[Geo<K>::NE]) {
    using G = Geo<K>;
    const long long base = (static_cast<long long>(v) * a.P + p) * a.H * a.W + x;
#pragma unroll
    for (int j = 0; j < G::NE; ++j) {
        const int y = y0 + j;
        const float f = a.phi_u16 ? static_cast<float>(phi[j]) : __uint_as_float(phi[j]);
        if (y < a.H) a.ratio[base + static_cast<long long>(y) * a.W] = __fdividef(f, fmaxf(d[j], a.eps));
    }
}

// Persistent kernel A: blur of every PSF group in use, then the ratios.
template <int K>
__global__ void __launch_bounds__(kThreads, 1) tc_blur_ratio_kernel(const __grid_constant__ TcParams kp) {
    using G = Geo<K>;
    const FusedArgs &a = kp.a;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = align128(smem_raw);
    const Smem s = setup(smem);
    const uint32_t tmem = *s.tmem_slot;
    float *stage = reinterpret_cast<float *>(smem + G::OFF_STAGE);

    const int tiles_x = (a.W + G::TX - 1) / G::TX;
    const int tiles_y = (a.H + G::TY - 1) / G::TY;
    const int n_tiles = tiles_x * tiles_y * a.P;
    const long long plane_px = static_cast<long long>(a.H) * a.W;
    const bool use_tma = kp.use_tma && a.psi_in != nullptr;
    uint32_t ph_tma = 0, ph_mma = 0;
    int tbuf = 0;
    bool tma_pending = false;

    // groups in use, the last of them, and the terms they need
    int last_g = -1, n_terms = 0, terms[kResidentTerms] = {0, 0};
    for (int g = 0; g < a.ft.n_groups; ++g) {
        bool used = false;
        for (int v = a.view_lo; v < a.view_hi; ++v) used |= (a.ft.group[v] == g);
        if (!used) continue;
        last_g = g;
        const int lead = a.ft.group_leader[g];
        for (int q = 0; q < a.ft.rank[lead]; ++q, ++n_terms)
            if (n_terms < kResidentTerms) terms[n_terms] = a.ft.tap_off[lead] + q;
    }
    const bool resident = n_terms <= kResidentTerms;
    if (resident) build_resident<K>(a, terms, n_terms, 0, 1, smem);

    if (use_tma && threadIdx.x == 0 && static_cast<int>(blockIdx.x) < n_tiles) {
        const Tile c = tile_of<K>(blockIdx.x, tiles_x, tiles_y);
        tma::mbar_arrive_expect_tx(s.bar_tma, G::STAGE_BYTES);
        tma::load_3d(stage, &kp.map, s.bar_tma, c.x0 - G::R4, c.y0 - G::R, c.p);
    }
    tma_pending = use_tma && static_cast<int>(blockIdx.x) < n_tiles;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x_out = 32 * (warp & 3) + lane;
    const int row0 = (warp >> 2) * G::NE;
    bool ok = true;

    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const Tile c = tile_of<K>(t, tiles_x, tiles_y);
        if (use_tma) {
            if (!wait_bar(s.bar_tma, ph_tma, a, s.abort_flag)) {
                tma_pending = false;   // drained by the wait
                break;
            }
            ph_tma ^= 1;
            tma_pending = false;
        } else {
            const float mean = a.psi_in ? 0.0f : __ldg(a.means + c.p);
            load_stage_sw<K>(stage, a.psi_in ? a.psi_in + c.p * plane_px : nullptr, mean, c.y0, c.x0, a.H, a.W,
                             a.circular);
            __syncthreads();
        }
        convert_a1<K>(stage, smem + G::OFF_A1);
        auto stage_free = [&]() {
            const int nt = t + gridDim.x;
            if (use_tma && nt < n_tiles) {
                const Tile c2 = tile_of<K>(nt, tiles_x, tiles_y);
                tma::fence_proxy_async_smem();
                tma::mbar_arrive_expect_tx(s.bar_tma, G::STAGE_BYTES);
                tma::load_3d(stage, &kp.map, s.bar_tma, c2.x0 - G::R4, c2.y0 - G::R, c2.p);
                tma_pending = true;   // thread 0's copy of the flag is the one used
            }
        };
        const int x = c.x0 + x_out;
        int slot = 0;
        for (int g = 0; g <= last_g && ok; ++g) {
            int v0 = -1;
            for (int v = a.view_lo; v < a.view_hi; ++v)
                if (a.ft.group[v] == g && v0 < 0) v0 = v;
            if (v0 < 0) continue;
            const int lead = a.ft.group_leader[g];
            const int rank = a.ft.rank[lead];
            ok = run_terms<K>(a, s, tmem, smem, a.ft.tap_off[lead], rank, 0, 1, resident ? slot : -1, g == last_g,
                              stage_free, ph_mma, tbuf);
            slot += rank;
            if (!ok) break;
            // the first view's data load overlaps the MMAs
            uint32_t phi[G::NE];
            if (x < a.W) load_phi<K>(a, v0, c.p, c.y0 + row0, x, phi);
            ok = finish_terms(a, s, ph_mma);
            if (!ok) break;
            float d[G::NE];
            read_d2<K>(tmem, d);
            if (x < a.W) {
                store_ratio<K>(a, v0, c.p, c.y0 + row0, x, phi, d);
                for (int v = v0 + 1; v < a.view_hi; ++v) {
                    if (a.ft.group[v] != g) continue;
                    load_phi<K>(a, v, c.p, c.y0 + row0, x, phi);
                    store_ratio<K>(a, v, c.p, c.y0 + row0, x, phi, d);
                }
            }
            tc5::fence_before();
            __syncthreads();
        }
    }
    if (tma_pending && threadIdx.x == 0) tma::mbar_wait_bounded(s.bar_tma, ph_tma, kDrainBudget);
    teardown(tmem);
}

// Persistent kernel B: per view, the correlation of its ratio tile; the
// product of the views' corrections stays in registers; then the update.
template <int K>
__global__ void __launch_bounds__(kThreads, 1) tc_correlate_update_kernel(const __grid_constant__ TcParams kp) {
    using G = Geo<K>;
    const FusedArgs &a = kp.a;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = align128(smem_raw);
    const Smem s = setup(smem);
    const uint32_t tmem = *s.tmem_slot;
    float *stage = reinterpret_cast<float *>(smem + G::OFF_STAGE);

    const int tiles_x = (a.W + G::TX - 1) / G::TX;
    const int tiles_y = (a.H + G::TY - 1) / G::TY;
    const int n_tiles = tiles_x * tiles_y * a.P;
    const long long plane_px = static_cast<long long>(a.H) * a.W;
    const bool use_tma = kp.use_tma != 0;
    uint32_t ph_tma = 0, ph_mma = 0;
    int tbuf = 0;
    bool tma_pending = false;

    int n_terms = 0, terms[kResidentTerms] = {0, 0};
    for (int v = a.view_lo; v < a.view_hi; ++v)
        for (int q = 0; q < a.ft.crank[v]; ++q, ++n_terms)
            if (n_terms < kResidentTerms) terms[n_terms] = a.ft.ctap_off[v] + q;
    const bool resident = n_terms <= kResidentTerms;
    if (resident) build_resident<K>(a, terms, n_terms, 2, 3, smem);

    if (use_tma && threadIdx.x == 0 && static_cast<int>(blockIdx.x) < n_tiles) {
        const Tile c = tile_of<K>(blockIdx.x, tiles_x, tiles_y);
        tma::mbar_arrive_expect_tx(s.bar_tma, G::STAGE_BYTES);
        tma::load_3d(stage, &kp.map, s.bar_tma, c.x0 - G::R4, c.y0 - G::R, a.view_lo * a.P + c.p);
    }
    tma_pending = use_tma && static_cast<int>(blockIdx.x) < n_tiles;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x_out = 32 * (warp & 3) + lane;
    const int row0 = (warp >> 2) * G::NE;
    bool ok = true;

    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const Tile c = tile_of<K>(t, tiles_x, tiles_y);
        float prod[G::NE];
#pragma unroll
        for (int j = 0; j < G::NE; ++j) prod[j] = 1.0f;
        int slot = 0;
        for (int v = a.view_lo; v < a.view_hi; ++v) {
            if (use_tma) {
                if (!wait_bar(s.bar_tma, ph_tma, a, s.abort_flag)) {
                    tma_pending = false;
                    ok = false;
                    break;
                }
                ph_tma ^= 1;
                tma_pending = false;
            } else {
                load_stage_sw<K>(stage, a.ratio + (static_cast<long long>(v) * a.P + c.p) * plane_px, 0.0f, c.y0,
                                 c.x0, a.H, a.W, a.circular);
                __syncthreads();
            }
            convert_a1<K>(stage, smem + G::OFF_A1);
            // the staging tile is free early: request the next (view, tile)
            int nv = v + 1, nt = t;
            if (nv >= a.view_hi) {
                nv = a.view_lo;
                nt = t + gridDim.x;
            }
            auto stage_free = [&]() {
                if (use_tma && nt < n_tiles) {
                    const Tile c2 = tile_of<K>(nt, tiles_x, tiles_y);
                    tma::fence_proxy_async_smem();
                    tma::mbar_arrive_expect_tx(s.bar_tma, G::STAGE_BYTES);
                    tma::load_3d(stage, &kp.map, s.bar_tma, c2.x0 - G::R4, c2.y0 - G::R, nv * a.P + c2.p);
                    tma_pending = true;   // thread 0's copy of the flag is the one used
                }
            };
            ok = run_terms<K>(a, s, tmem, smem, a.ft.ctap_off[v], a.ft.crank[v], 2, 3, resident ? slot : -1, true,
                              stage_free, ph_mma, tbuf);
            slot += a.ft.crank[v];
            if (!ok) break;
            ok = finish_terms(a, s, ph_mma);
            if (!ok) break;
            float d[G::NE];
            read_d2<K>(tmem, d);
#pragma unroll
            for (int j = 0; j < G::NE; ++j) prod[j] *= d[j];
            tc5::fence_before();
            __syncthreads();
        }
        if (!ok) break;
        const int x = c.x0 + x_out;
        if (x < a.W) {
            const long long base = c.p * plane_px + x;
            const float mean = a.psi_in ? 0.0f : __ldg(a.means + c.p);
            float psi[G::NE];
#pragma unroll
            for (int j = 0; j < G::NE; ++j) {
                const int y = c.y0 + row0 + j;
                psi[j] = mean;
                if (a.psi_in && y < a.H) psi[j] = __ldg(a.psi_in + base + static_cast<long long>(y) * a.W);
            }
#pragma unroll
            for (int j = 0; j < G::NE; ++j) {
                const int y = c.y0 + row0 + j;
                if (y < a.H) a.psi_out[base + static_cast<long long>(y) * a.W] = psi[j] * prod[j];
            }
        }
    }
    if (tma_pending && threadIdx.x == 0) tma::mbar_wait_bounded(s.bar_tma, ph_tma, kDrainBudget);
    teardown(tmem);
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

bool encode(CUtensorMap *m, const void *base, int W, int H, long long D, int box_w, int box_h) {
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

template <int K>
cudaError_t launch(const FusedArgs &a, int which, cudaStream_t st) {
    using G = Geo<K>;
    static unsigned long long attr_set = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set & bit)) {
        cudaError_t e = cudaFuncSetAttribute(tc_blur_ratio_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(tc_correlate_update_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set |= bit;
    }
    static int sms[64] = {};
    if (!sms[dev & 63]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms[dev & 63] = n > 0 ? n : 1;
    }
    const long long n_tiles = static_cast<long long>((a.W + G::TX - 1) / G::TX) * ((a.H + G::TY - 1) / G::TY) * a.P;
    if (n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    long long ctas = sms[dev & 63];   // one CTA per SM (shared memory and tensor memory)
    if (a.max_ctas > 0 && a.max_ctas < ctas) ctas = a.max_ctas;
    const dim3 grid(static_cast<unsigned>(n_tiles < ctas ? n_tiles : ctas));
    TcParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.a = a;
    const bool tma_ok = !a.circular && (a.W % 4 == 0);
    if (which == 0) {
        if (tma_ok && a.psi_in && aligned16(a.psi_in)) kp.use_tma = encode(&kp.map, a.psi_in, a.W, a.H, a.P, G::KA, G::ROWS);
        tc_blur_ratio_kernel<K><<<grid, kThreads, G::SMEM_BYTES, st>>>(kp);
    } else {
        if (tma_ok && aligned16(a.ratio))
            kp.use_tma = encode(&kp.map, a.ratio, a.W, a.H, static_cast<long long>(a.ft.views) * a.P, G::KA, G::ROWS);
        tc_correlate_update_kernel<K><<<grid, kThreads, G::SMEM_BYTES, st>>>(kp);
    }
    count_launch();
    return cudaGetLastError();
}

#define MVD_TC_CASES(X) \
    X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(27) X(29) X(31) \
    X(33) X(35) X(37) X(39) X(41) X(43) X(45) X(47)

cudaError_t dispatch(const FusedArgs &a, int which, cudaStream_t st) {
    switch (a.ft.K) {
#define MVD_CASE(k) \
    case k:         \
        return launch<k>(a, which, st);
        MVD_TC_CASES(MVD_CASE)
#undef MVD_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace tcr

bool tc_supported(int K) { return K >= 1 && K <= 47 && (K % 2) == 1; }

void tc_tile_shape(int K, int *tile_h, int *tile_w) {
    switch (K) {
#define MVD_CASE(k)                      \
    case k:                              \
        *tile_h = tcr::Geo<k>::TY;       \
        *tile_w = tcr::Geo<k>::TX;       \
        return;
        MVD_TC_CASES(MVD_CASE)
#undef MVD_CASE
        default:
            *tile_h = *tile_w = 0;
    }
}

cudaError_t launch_tc_blur_ratio(const FusedArgs &a, cudaStream_t s) { return tcr::dispatch(a, 0, s); }

cudaError_t launch_tc_correlate_update(const FusedArgs &a, cudaStream_t s) { return tcr::dispatch(a, 1, s); }

}  // namespace mvd
