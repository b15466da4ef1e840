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
// input tile is 128 rows (TY + 2R of them used) x KA columns.  An MMA costs
// about the same issue time up to N = 128, so both passes use wide MMAs:
//
//   pass 1 (along x):  D1[x_out][y_in] = sum_k T1[x_out][k] B1[k][y_in]
//       T1 = Toeplitz matrix of the horizontal taps, built by the threads in
//       tensor memory (A operand, one row per lane); B1 = input tile (BF16
//       hi/lo, K-major in shared memory); N = 128 input rows, K = KA columns.
//   split:  each thread reads its lane of D1 (one output column) and writes
//       it back as BF16 hi/lo: A2 = D1, again an A operand in tensor memory.
//   pass 2 (along y):  D2[x_out][y_out] = sum_k A2[x_out][k] T2[k][y_out]
//       T2 = Toeplitz matrix of the vertical taps (shared memory), N = TY,
//       K = 128 input rows; every SVD term accumulates into the same D2.
//   epilogue: each thread reads its lane of D2, i.e. one output column, and
//       walks its rows: coalesced loads of phi / psi and stores of r / psi.
//
// The FP32 staging tile (TMA destination) is free once converted to B1, so
// the next tile's copy overlaps all of the current tile's MMAs.  One CTA per
// SM (about 194-215 KB of shared memory, all 512 tensor-memory columns),
// 512 threads.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "tc_common.cuh"

namespace mvd {
namespace tcr {

namespace {

using tcc::kDrainBudget;
using tcc::kThreads;
using tcc::kTmemCols;
using tcc::Smem;
using tcc::TcParams;
using tcc::Tile;
using tcc::align128;
using tcc::load_phi;
using tcc::setup;
using tcc::store_ratio;
using tcc::teardown;
using tcc::wait_bar;

template <int K>
struct Geo {
    static constexpr int R = (K - 1) / 2;
    static constexpr int R4 = (R + 3) / 4 * 4;    // TMA x origin stays 16-byte aligned
    static constexpr int COL0 = R4 - R;           // input column of x0 - R within the staging tile
    static constexpr int TX = 128;
    static constexpr int TY = R == 0 ? 128 : (2 * R <= 32 ? 96 : 64);
    static constexpr int ROWS = 128;              // input rows = pass-1 N = pass-2 K
    static constexpr int KA = (128 + COL0 + 2 * R + 15) / 16 * 16;   // input columns = pass-1 K
    static constexpr int NKS1 = KA / 16;
    static constexpr int NKB = KA / 8;
    static constexpr int NKS2 = ROWS / 16;
    static constexpr int NE = TY / 4;             // output rows per epilogue thread
    static constexpr int QA = KA / 4;             // T1 columns (values) built per thread
    // tensor-memory columns
    static constexpr uint32_t C_T1 = 0, C_T1LO = KA / 2, C_D1 = KA, C_A2 = KA + 128, C_A2LO = KA + 192,
                              C_D2 = KA + 256;
    // shared memory
    static constexpr int STAGE_BYTES = ROWS * KA * 4;
    static constexpr uint32_t B1_LBO = 128 * 16 + 16;   // k-group stride; +16 B spreads banks
    static constexpr int B1_BYTES = NKB * B1_LBO;
    static constexpr uint32_t T2_LBO = TY * 16;         // k-group stride (TY rows x 16 B)
    static constexpr int T2_BYTES = ROWS / 8 * T2_LBO;
    static constexpr int OFF_STAGE = 1024;
    static constexpr int OFF_B1 = OFF_STAGE + STAGE_BYTES;
    static constexpr int OFF_T2 = OFF_B1 + 2 * B1_BYTES;
    static constexpr int SMEM_USED = OFF_T2 + 2 * T2_BYTES;
    static constexpr int SMEM_BYTES = SMEM_USED + 128;   // room to align the dynamic base
    static_assert(TY + 2 * R <= ROWS, "input rows fit pass 1's N");
    static_assert(KA >= 128 + COL0 + 2 * R && KA % 16 == 0, "pass-1 K covers the halo");
    static_assert(QA % 2 == 0, "T1 columns pair up");
    static_assert(C_D2 + TY <= kTmemCols, "tensor-memory columns");
    static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
};

// BF16 hi and lo parts of two FP32 values, packed (first value in the low half).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
    hi = *reinterpret_cast<const uint32_t *>(&hb);
    const float h0 = __uint_as_float(hi << 16);
    const float h1 = __uint_as_float(hi & 0xFFFF0000u);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - h0, x1 - h1);
    lo = *reinterpret_cast<const uint32_t *>(&lb);
}

// Split 8 FP32 values into BF16 hi and lo parts (8 each, element 0 in the low
// half of the first word).
__device__ __forceinline__ void split8(const float (&x)[8], uint4 &hi, uint4 &lo) {
    split2(x[0], x[1], hi.x, lo.x);
    split2(x[2], x[3], hi.y, lo.y);
    split2(x[4], x[5], hi.z, lo.z);
    split2(x[6], x[7], hi.w, lo.w);
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

// Staging tile (FP32, row-major) -> B1 hi/lo (BF16, K-major: element
// (input row n, column k) at n*16 + (k/8)*B1_LBO + (k%8)*2).  Item = one row
// and 8 consecutive columns.
template <int K>
__device__ __forceinline__ void convert_b1(const float *__restrict__ stage, unsigned char *b1) {
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
        const uint32_t off = static_cast<uint32_t>(m) * 16 + static_cast<uint32_t>(kb) * G::B1_LBO;
        sts128(b1 + off, hi);
        sts128(b1 + G::B1_BYTES + off, lo);
    }
}

// The Toeplitz operands of one term (correlation-form taps: out(i) = sum_j
// t[j] in(i + j - R)):
//   T1[x_out][k] = w[k - x_out - COL0]   (tensor memory, lane x_out; warp w
//                                         writes columns QA*(w/4) .. of its lanes)
//   T2[k][y_out] = u[k - y_out]          (shared memory, K-major, item = one
//                                         output row and 8 consecutive k)
// Callers make the writes visible (tcgen05 wait, proxy fence, barrier).
template <int K>
__device__ __forceinline__ void build_toeplitz(const float *__restrict__ u, const float *__restrict__ w, uint32_t tmem,
                                               unsigned char *t2) {
    using G = Geo<K>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x_out = 32 * (warp & 3) + lane;
    const int k0 = (warp >> 2) * G::QA;
    uint32_t hi[G::QA / 2], lo[G::QA / 2];
#pragma unroll
    for (int c = 0; c < G::QA / 2; ++c) {
        const int j0 = k0 + 2 * c - x_out - G::COL0;
        const float a = (j0 >= 0 && j0 < K) ? __ldg(w + j0) : 0.0f;
        const float b = (j0 + 1 >= 0 && j0 + 1 < K) ? __ldg(w + j0 + 1) : 0.0f;
        split2(a, b, hi[c], lo[c]);
    }
    const uint32_t lane_off = static_cast<uint32_t>(32 * (warp & 3)) << 16;
    tc5::st_cols<G::QA / 2>(tmem + lane_off + G::C_T1 + k0 / 2, hi);
    tc5::st_cols<G::QA / 2>(tmem + lane_off + G::C_T1LO + k0 / 2, lo);
    constexpr int ITEMS = G::TY * (G::ROWS / 8);
    for (int it = threadIdx.x; it < ITEMS; it += kThreads) {
        const int n = it % G::TY, kg = it / G::TY;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = 8 * kg + e - n;
            x[e] = (j >= 0 && j < K) ? __ldg(u + j) : 0.0f;
        }
        uint4 h, l;
        split8(x, h, l);
        const uint32_t addr = (n & 7) * 16 + (n >> 3) * 128 + kg * G::T2_LBO;
        sts128(t2 + addr, h);
        sts128(t2 + G::T2_BYTES + addr, l);
    }
    tc5::wait_st();
}

// Pass 1 MMAs (one thread): D1 = T1 (tensor memory) x B1 (shared memory).
template <int K>
__device__ __forceinline__ void issue_pass1(uint32_t tmem, uint32_t b1) {
    using G = Geo<K>;
    constexpr uint32_t idesc = tc5::idesc_bf16(128, 128, false, false);
    const uint32_t b1lo = b1 + G::B1_BYTES;
#pragma unroll 1
    for (int s = 0; s < G::NKS1; ++s) {
        const uint32_t bo = static_cast<uint32_t>(2 * s) * G::B1_LBO;
        const uint64_t bh = tc5::sdesc(b1 + bo, G::B1_LBO, 128), bl = tc5::sdesc(b1lo + bo, G::B1_LBO, 128);
        const uint32_t ah = tmem + G::C_T1 + 8 * s, al = tmem + G::C_T1LO + 8 * s;
        tc5::mma_bf16_ta(tmem + G::C_D1, al, bh, idesc, s > 0);
        tc5::mma_bf16_ta(tmem + G::C_D1, ah, bl, idesc, 1);
        tc5::mma_bf16_ta(tmem + G::C_D1, ah, bh, idesc, 1);
    }
}

// Pass 2 MMAs (one thread): D2 (+)= A2 (tensor memory) x T2 (shared memory).
template <int K>
__device__ __forceinline__ void issue_pass2(uint32_t tmem, uint32_t t2, bool accumulate) {
    using G = Geo<K>;
    constexpr uint32_t idesc = tc5::idesc_bf16(128, G::TY, false, false);
    const uint32_t t2lo = t2 + G::T2_BYTES;
#pragma unroll 1
    for (int s = 0; s < G::NKS2; ++s) {
        const uint32_t bo = static_cast<uint32_t>(2 * s) * G::T2_LBO;
        const uint64_t bh = tc5::sdesc(t2 + bo, G::T2_LBO, 128), bl = tc5::sdesc(t2lo + bo, G::T2_LBO, 128);
        const uint32_t ah = tmem + G::C_A2 + 8 * s, al = tmem + G::C_A2LO + 8 * s;
        tc5::mma_bf16_ta(tmem + G::C_D2, al, bh, idesc, (accumulate || s > 0) ? 1u : 0u);
        tc5::mma_bf16_ta(tmem + G::C_D2, ah, bl, idesc, 1);
        tc5::mma_bf16_ta(tmem + G::C_D2, ah, bh, idesc, 1);
    }
}

// D1 -> A2 in place per lane: warp w reads input rows 32*(w/4).. of its
// lanes' D1 and writes them back as BF16 hi/lo pairs.
template <int K>
__device__ __forceinline__ void split_d1(uint32_t tmem) {
    using G = Geo<K>;
    const int warp = threadIdx.x >> 5;
    const uint32_t lane_off = static_cast<uint32_t>(32 * (warp & 3)) << 16;
    const int cg = warp >> 2;
    uint32_t r[32];
    tc5::ld32(tmem + lane_off + G::C_D1 + 32 * cg, r);
    tc5::wait_ld();
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) split2(__uint_as_float(r[2 * c]), __uint_as_float(r[2 * c + 1]), hi[c], lo[c]);
    tc5::st16(tmem + lane_off + G::C_A2 + 16 * cg, hi);
    tc5::st16(tmem + lane_off + G::C_A2LO + 16 * cg, lo);
    tc5::wait_st();
}

// This thread's column of D2: NE consecutive output rows.
template <int K>
__device__ __forceinline__ void read_d2(uint32_t tmem, float (&d)[Geo<K>::NE]) {
    using G = Geo<K>;
    const int warp = threadIdx.x >> 5;
    const int qd = warp & 3, cg = warp >> 2;
    const uint32_t base = tmem + (static_cast<uint32_t>(32 * qd) << 16) + G::C_D2 + cg * G::NE;
#pragma unroll
    for (int j = 0; j < G::NE / 8; ++j) tc5::ld8(base + 8 * j, reinterpret_cast<uint32_t *>(d) + 8 * j);
    tc5::wait_ld();
}

template <int K>
__device__ __forceinline__ Tile tile_of(int t, int tiles_x, int tiles_y) {
    return tcc::tile_of<Geo<K>::TX, Geo<K>::TY>(t, tiles_x, tiles_y);
}

// One group of SVD terms (a PSF's blur, or a view's correlation) on the input
// tile in B1: D2 = sum over the terms.  Enter with every earlier MMA complete;
// returns with the last MMAs issued and committed to bar_mma (the caller
// waits, then reads D2).  False if a wait timed out.
template <int K>
__device__ bool run_terms(const FusedArgs &a, const Smem &s, uint32_t tmem, unsigned char *smem, int term0,
                          int n_terms, int kind_u, int kind_w, uint32_t &ph_mma) {
    using G = Geo<K>;
    unsigned char *b1 = smem + G::OFF_B1;
    unsigned char *t2 = smem + G::OFF_T2;
    for (int q = 0; q < n_terms; ++q) {
        if (q > 0) {
            // the previous term's pass 2 still reads T2 and A2
            if (!wait_bar(s.bar1, ph_mma, a, s.abort_flag)) return false;
            ph_mma ^= 1;
            tc5::fence_after();
        }
        const float *tq = a.taps + static_cast<long long>(term0 + q) * 4 * K;
        build_toeplitz<K>(tq + kind_u * K, tq + kind_w * K, tmem, t2);
        tma::fence_proxy_async_smem();
        tc5::fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc5::fence_after();
            issue_pass1<K>(tmem, tc5::smem_u32(b1));
            tc5::commit(s.bar1);
        }
        if (!wait_bar(s.bar1, ph_mma, a, s.abort_flag)) return false;
        ph_mma ^= 1;
        tc5::fence_after();
        split_d1<K>(tmem);
        tc5::fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc5::fence_after();
            issue_pass2<K>(tmem, tc5::smem_u32(t2), q > 0);
            tc5::commit(s.bar1);
        }
    }
    return true;
}

// Wait for the MMAs run_terms committed; D2 is then readable.
__device__ __forceinline__ bool finish_terms(const FusedArgs &a, const Smem &s, uint32_t &ph_mma) {
    if (!wait_bar(s.bar1, ph_mma, a, s.abort_flag)) return false;
    ph_mma ^= 1;
    tc5::fence_after();
    return true;
}

// Input tile of (tile t, z) into B1, then the staging tile is released: thread
// 0 requests the next copy (plane index nz of tile nt) if there is one.
// Returns false if the tile's copy timed out.
template <int K>
__device__ __forceinline__ bool take_tile(const TcParams &kp, const Smem &s, unsigned char *smem, bool use_tma,
                                          const float *sw_src, float sw_fill, const Tile &c, bool next, const Tile &c2,
                                          int nz, uint32_t &ph_tma, bool &tma_pending) {
    using G = Geo<K>;
    const FusedArgs &a = kp.a;
    float *stage = reinterpret_cast<float *>(smem + G::OFF_STAGE);
    if (use_tma) {
        if (!wait_bar(s.bar_tma, ph_tma, a, s.abort_flag)) {
            tma_pending = false;   // drained by the wait
            return false;
        }
        ph_tma ^= 1;
        tma_pending = false;
    } else {
        load_stage_sw<K>(stage, sw_src, sw_fill, c.y0, c.x0, a.H, a.W, a.circular);
        __syncthreads();
    }
    convert_b1<K>(stage, smem + G::OFF_B1);
    tma::fence_proxy_async_smem();
    __syncthreads();
    if (use_tma && next && threadIdx.x == 0) {
        tma::mbar_arrive_expect_tx(s.bar_tma, G::STAGE_BYTES);
        tma::load_3d(stage, &kp.map, s.bar_tma, c2.x0 - G::R4, c2.y0 - G::R, nz);
        tma_pending = true;   // thread 0's copy of the flag is the one used
    }
    return true;
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
    bool tma_pending = false;

    int last_g = -1;
    for (int g = 0; g < a.ft.n_groups; ++g)
        for (int v = a.view_lo; v < a.view_hi; ++v)
            if (a.ft.group[v] == g) last_g = g;

    if (use_tma && threadIdx.x == 0 && static_cast<int>(blockIdx.x) < n_tiles) {
        const Tile c = tile_of<K>(blockIdx.x, tiles_x, tiles_y);
        tma::mbar_arrive_expect_tx(s.bar_tma, G::STAGE_BYTES);
        tma::load_3d(stage, &kp.map, s.bar_tma, c.x0 - G::R4, c.y0 - G::R, c.p);
        tma_pending = true;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x_out = 32 * (warp & 3) + lane;
    const int row0 = (warp >> 2) * G::NE;
    bool ok = true;

    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const Tile c = tile_of<K>(t, tiles_x, tiles_y);
        const int nt = t + gridDim.x;
        const Tile c2 = tile_of<K>(nt < n_tiles ? nt : t, tiles_x, tiles_y);
        const float mean = a.psi_in ? 0.0f : __ldg(a.means + c.p);
        ok = take_tile<K>(kp, s, smem, use_tma, a.psi_in ? a.psi_in + c.p * plane_px : nullptr, mean, c,
                          nt < n_tiles, c2, c2.p, ph_tma, tma_pending);
        const int x = c.x0 + x_out;
        for (int g = 0; g <= last_g && ok; ++g) {
            int v0 = -1;
            for (int v = a.view_lo; v < a.view_hi; ++v)
                if (a.ft.group[v] == g && v0 < 0) v0 = v;
            if (v0 < 0) continue;
            const int lead = a.ft.group_leader[g];
            ok = run_terms<K>(a, s, tmem, smem, a.ft.tap_off[lead], a.ft.rank[lead], 0, 1, ph_mma);
            if (!ok) break;
            // the first view's data load overlaps the MMAs
            uint32_t phi[G::NE];
            if (x < a.W) load_phi<G::NE>(a, v0, c.p, c.y0 + row0, x, phi);
            ok = finish_terms(a, s, ph_mma);
            if (!ok) break;
            float d[G::NE];
            read_d2<K>(tmem, d);
            if (x < a.W) {
                store_ratio<G::NE>(a, v0, c.p, c.y0 + row0, x, phi, d);
                for (int v = v0 + 1; v < a.view_hi; ++v) {
                    if (a.ft.group[v] != g) continue;
                    load_phi<G::NE>(a, v, c.p, c.y0 + row0, x, phi);
                    store_ratio<G::NE>(a, v, c.p, c.y0 + row0, x, phi, d);
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
    bool tma_pending = false;

    if (use_tma && threadIdx.x == 0 && static_cast<int>(blockIdx.x) < n_tiles) {
        const Tile c = tile_of<K>(blockIdx.x, tiles_x, tiles_y);
        tma::mbar_arrive_expect_tx(s.bar_tma, G::STAGE_BYTES);
        tma::load_3d(stage, &kp.map, s.bar_tma, c.x0 - G::R4, c.y0 - G::R, a.view_lo * a.P + c.p);
        tma_pending = true;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x_out = 32 * (warp & 3) + lane;
    const int row0 = (warp >> 2) * G::NE;
    bool ok = true;

    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const Tile c = tile_of<K>(t, tiles_x, tiles_y);
        float prod[G::NE];
#pragma unroll
        for (int j = 0; j < G::NE; ++j) prod[j] = 1.0f;
        for (int v = a.view_lo; v < a.view_hi && ok; ++v) {
            int nv = v + 1, nt = t;
            if (nv >= a.view_hi) {
                nv = a.view_lo;
                nt = t + gridDim.x;
            }
            const Tile c2 = tile_of<K>(nt < n_tiles ? nt : t, tiles_x, tiles_y);
            ok = take_tile<K>(kp, s, smem, use_tma, a.ratio + (static_cast<long long>(v) * a.P + c.p) * plane_px,
                              0.0f, c, nt < n_tiles, c2, nv * a.P + c2.p, ph_tma, tma_pending);
            if (!ok) break;
            ok = run_terms<K>(a, s, tmem, smem, a.ft.ctap_off[v], a.ft.crank[v], 2, 3, ph_mma);
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
    const long long n_tiles = static_cast<long long>((a.W + G::TX - 1) / G::TX) * ((a.H + G::TY - 1) / G::TY) * a.P;
    if (n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    long long ctas = tcc::sm_count(dev);   // one CTA per SM (shared memory and tensor memory)
    if (a.max_ctas > 0 && a.max_ctas < ctas) ctas = a.max_ctas;
    const dim3 grid(static_cast<unsigned>(n_tiles < ctas ? n_tiles : ctas));
    TcParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.a = a;
    const bool tma_ok = !a.circular && (a.W % 4 == 0);
    if (which == 0) {
        if (tma_ok && a.psi_in && tcc::aligned16(a.psi_in)) kp.use_tma = tcc::encode(&kp.map, a.psi_in, a.W, a.H, a.P, G::KA, G::ROWS);
        tc_blur_ratio_kernel<K><<<grid, kThreads, G::SMEM_BYTES, st>>>(kp);
    } else {
        if (tma_ok && tcc::aligned16(a.ratio))
            kp.use_tma = tcc::encode(&kp.map, a.ratio, a.W, a.H, static_cast<long long>(a.ft.views) * a.P, G::KA, G::ROWS);
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
