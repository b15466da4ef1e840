// TF32 tensor-core route of the fused MV-RL iteration (Supp. Note 1 update
// equation), the precision configuration's reduced-precision arm:
//
//   tf32_blur_ratio        r_v = phi_v / max(psi * P_v, eps)
//   tf32_correlate_update  psi <- psi * prod_v (r_v (*) P_v^*)
//
// Every separable 1D pass of every SVD term is a banded (Toeplitz) matrix
// product on the tcgen05 tensor cores, kind::tf32: one MMA per K step of 8
// (against three per K step of 16 for BF16x3).  Operands are rounded to TF32
// (10 explicit mantissa bits, round to nearest) on the way in: the input
// tile, the taps and the pass-1 result; products accumulate in FP32.  The
// ratio, the product over views and the update stay FP32.  Expected error:
// about 2^-11 relative per product, against 2^-24 for FP32 arithmetic.
//
// Tile: TY x 128 outputs of one plane (TY = 96 for K <= 33, 64 above, 128
// for K = 1); the input tile is 128 rows x KA columns (KA = 128 + 2R rounded
// up to a multiple of 8, plus the alignment offset of the TMA origin).
//
//   pass 1 (along x):  D1[x_out][y_in] = sum_k T1[x_out][k] B1[y_in][k]
//       T1: horizontal taps as a Toeplitz matrix in tensor memory (A
//       operand, one TF32 value per column); B1: the input tile, K-major in
//       shared memory; M = N = 128, K = KA.
//   pass 2 (along y):  D2[x_out][y_out] = sum_k D1[x_out][k] T2[y_out][k]
//       A = D1 itself (rounded to TF32 in place), T2: vertical taps as a
//       Toeplitz matrix in shared memory; N = TY, K = 128.  Every SVD term
//       of a factor set accumulates into D2.
//   epilogue: each thread reads its lane of D2 (one output column) and
//       walks its rows: coalesced loads of phi / psi, stores of r / psi.
//
// Software pipeline over steps (one step = one SVD term on one tile):
// while pass 2 of step s runs, the input tile of step s+1 is converted from
// the TMA staging tile and its T1 is written; while pass 1 of step s+1 runs,
// T2 of step s+1 is written and the epilogue of step s runs.  The staging
// tile's next TMA copy is requested as soon as it has been converted.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "tc_common.cuh"

namespace mvd {
namespace tcf {

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
    static constexpr int COL0 = R4 - R;           // input column of x0 - R within the tile
    static constexpr int TX = 128;
    static constexpr int TY = R == 0 ? 128 : (2 * R <= 32 ? 96 : 64);
    static constexpr int ROWS = 128;              // input rows = pass-1 N = pass-2 K
    static constexpr int KA = (128 + COL0 + 2 * R + 7) / 8 * 8;   // input columns = pass-1 K
    static constexpr int NKG = KA / 4;            // 16-byte column groups of a row
    static constexpr int NKS1 = KA / 8;           // pass-1 MMAs
    static constexpr int NKS2 = ROWS / 8;         // pass-2 MMAs
    static constexpr int NE = TY / 4;             // output rows per epilogue thread
    static constexpr int QA = KA / 4;             // T1 columns written per thread
    // tensor-memory columns
    static constexpr uint32_t C_T1 = 0, C_D1 = KA, C_D2 = KA + 128;
    // shared memory
    static constexpr int STAGE_BYTES = ROWS * KA * 4;       // FP32 row-major input tile (TMA box)
    static constexpr uint32_t B1_LBO = 128 * 16 + 16;       // column-group stride; +16 B spreads banks
    static constexpr int B1_BYTES = NKG * B1_LBO;
    static constexpr uint32_t T2_LBO = TY * 16;             // k-group stride (TY rows x 16 B)
    static constexpr int T2_BYTES = ROWS / 4 * T2_LBO;
    static constexpr int OFF_STAGE = 1024;
    static constexpr int OFF_B1 = OFF_STAGE + STAGE_BYTES;
    static constexpr int OFF_T2 = OFF_B1 + B1_BYTES;
    static constexpr int SMEM_USED = OFF_T2 + T2_BYTES;
    static constexpr int SMEM_BYTES = SMEM_USED + 128;     // room to align the dynamic base
    static_assert(TY + 2 * R <= ROWS, "input rows fit pass 1's N");
    static_assert(KA >= 128 + COL0 + 2 * R && KA % 8 == 0 && KA <= 256, "pass-1 K covers the halo");
    static_assert(QA % 2 == 0, "T1 columns pair up");
    static_assert(C_D2 + TY <= kTmemCols, "tensor-memory columns");
    static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
};

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

// Staging tile (FP32, row-major) -> B1 (TF32, K-major: element (input row n,
// column k) at n*16 + (k/4)*B1_LBO + (k%4)*4).  Item = one row and 4
// consecutive columns.
template <int K>
__device__ __forceinline__ void convert_b1(const float *__restrict__ stage, unsigned char *b1) {
    using G = Geo<K>;
    constexpr int ITEMS = G::ROWS * G::NKG;
    for (int it = threadIdx.x; it < ITEMS; it += kThreads) {
        const int m = it / G::NKG;
        const int kg = it - m * G::NKG;
        const float4 v = *reinterpret_cast<const float4 *>(stage + m * G::KA + 4 * kg);
        const uint4 t = {tc5::to_tf32(v.x), tc5::to_tf32(v.y), tc5::to_tf32(v.z), tc5::to_tf32(v.w)};
        *reinterpret_cast<uint4 *>(b1 + static_cast<uint32_t>(m) * 16 + static_cast<uint32_t>(kg) * G::B1_LBO) = t;
    }
}

// The Toeplitz operands of one term (correlation-form taps: out(i) = sum_j
// t[j] in(i + j - R)):
//   T1[x_out][k] = w[k - x_out - COL0]   (tensor memory, lane x_out; warp w
//                                         writes columns QA*(w/4) .. of its lanes)
//   T2[y_out][k] = u[k - y_out]          (shared memory, K-major, item = one
//                                         output row and 4 consecutive k)
// Callers make the writes visible (proxy fence, tcgen05 fence, barrier).
template <int K>
__device__ __forceinline__ void build_t1(const float *__restrict__ w, uint32_t tmem) {
    using G = Geo<K>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x_out = 32 * (warp & 3) + lane;
    const int k0 = (warp >> 2) * G::QA;
    uint32_t t[G::QA];
#pragma unroll
    for (int c = 0; c < G::QA; ++c) {
        const int j = k0 + c - x_out - G::COL0;
        t[c] = tc5::to_tf32((j >= 0 && j < K) ? __ldg(w + j) : 0.0f);
    }
    const uint32_t lane_off = static_cast<uint32_t>(32 * (warp & 3)) << 16;
    tc5::st_cols<G::QA>(tmem + lane_off + G::C_T1 + k0, t);
    tc5::wait_st();
}

template <int K>
__device__ __forceinline__ void build_t2(const float *__restrict__ u, unsigned char *t2) {
    using G = Geo<K>;
    constexpr int ITEMS = G::TY * (G::ROWS / 4);
    for (int it = threadIdx.x; it < ITEMS; it += kThreads) {
        const int n = it % G::TY, kg = it / G::TY;
        uint32_t x[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 4 * kg + e - n;
            x[e] = tc5::to_tf32((j >= 0 && j < K) ? __ldg(u + j) : 0.0f);
        }
        const uint32_t addr = (n & 7) * 16 + (n >> 3) * 128 + kg * G::T2_LBO;
        *reinterpret_cast<uint4 *>(t2 + addr) = make_uint4(x[0], x[1], x[2], x[3]);
    }
}

// Pass 1 MMAs (one thread): D1 = T1 (tensor memory) x B1 (shared memory).
template <int K>
__device__ __forceinline__ void issue_pass1(uint32_t tmem, uint32_t b1) {
    using G = Geo<K>;
    constexpr uint32_t idesc = tc5::idesc_tf32(128, 128);
#pragma unroll 1
    for (int s = 0; s < G::NKS1; ++s) {
        const uint64_t b = tc5::sdesc(b1 + static_cast<uint32_t>(2 * s) * G::B1_LBO, G::B1_LBO, 128);
        tc5::mma_tf32_ta(tmem + G::C_D1, tmem + G::C_T1 + 8 * s, b, idesc, s > 0);
    }
}

// Pass 2 MMAs (one thread): D2 (+)= D1 (tensor memory) x T2 (shared memory).
template <int K>
__device__ __forceinline__ void issue_pass2(uint32_t tmem, uint32_t t2, bool accumulate) {
    using G = Geo<K>;
    constexpr uint32_t idesc = tc5::idesc_tf32(128, G::TY);
#pragma unroll 1
    for (int s = 0; s < G::NKS2; ++s) {
        const uint64_t b = tc5::sdesc(t2 + static_cast<uint32_t>(2 * s) * G::T2_LBO, G::T2_LBO, 128);
        tc5::mma_tf32_ta(tmem + G::C_D2, tmem + G::C_D1 + 8 * s, b, idesc, (accumulate || s > 0) ? 1u : 0u);
    }
}

// D1 rounded to TF32 in place: warp w rounds input rows 32*(w/4).. of its lanes.
template <int K>
__device__ __forceinline__ void round_d1(uint32_t tmem) {
    using G = Geo<K>;
    const int warp = threadIdx.x >> 5;
    const uint32_t addr = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + G::C_D1 + 32 * (warp >> 2);
    uint32_t r[32];
    tc5::ld32(addr, r);
    tc5::wait_ld();
#pragma unroll
    for (int c = 0; c < 32; ++c) r[c] = tc5::to_tf32(__uint_as_float(r[c]));
    tc5::st16(addr, r);
    tc5::st16(addr + 16, r + 16);
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

// One step of the pipeline: SVD term q of the factor set u (a PSF group's
// blur in kernel A, a view's correlation in kernel B) on tile t.
struct Step {
    int t, u, q;
    bool valid;
};

// The steps of a CTA in order: tiles blockIdx.x, blockIdx.x + gridDim.x, ...;
// per tile the factor sets in use; per set its terms.  `terms(u)` is the
// set's term count, `used(u)` whether the launch needs it, u in [0, n_sets).
template <typename Terms, typename Used>
__device__ __forceinline__ Step next_step(Step c, int n_tiles, int n_sets, Terms &&terms, Used &&used) {
    if (c.q + 1 < terms(c.u)) return {c.t, c.u, c.q + 1, true};
    for (int u = c.u + 1; u < n_sets; ++u)
        if (used(u)) return {c.t, u, 0, true};
    const int t = c.t + gridDim.x;
    if (t >= n_tiles) return {t, 0, 0, false};
    for (int u = 0; u < n_sets; ++u)
        if (used(u)) return {t, u, 0, true};
    return {t, 0, 0, false};
}

template <typename Terms, typename Used>
__device__ __forceinline__ Step first_step(int n_tiles, int n_sets, Terms &&terms, Used &&used) {
    const int t = blockIdx.x;
    if (t >= n_tiles) return {t, 0, 0, false};
    for (int u = 0; u < n_sets; ++u)
        if (used(u)) return {t, u, 0, true};
    return {t, 0, 0, false};
}

// The two kernels share the pipeline; KIND 0 = blur/ratio (factor sets =
// PSF groups, a new input tile per tile), 1 = correlate/update (sets =
// views, a new input tile per view).  MMAs complete in issue order, so pass
// 1 of step s+1 complete implies pass 2 of step s complete.
template <int K, int KIND>
__device__ void pipeline(const TcParams &kp, unsigned char *smem, const Smem &s, uint32_t tmem) {
    using G = Geo<K>;
    const FusedArgs &a = kp.a;
    const int tiles_x = (a.W + G::TX - 1) / G::TX;
    const int tiles_y = (a.H + G::TY - 1) / G::TY;
    const int n_tiles = tiles_x * tiles_y * a.P;
    const long long plane_px = static_cast<long long>(a.H) * a.W;
    unsigned char *b1 = smem + G::OFF_B1;
    unsigned char *t2 = smem + G::OFF_T2;
    float *stage = reinterpret_cast<float *>(smem + G::OFF_STAGE);
    const int n_sets = KIND == 0 ? a.ft.n_groups : a.view_hi;
    auto used = [&](int u) {
        if constexpr (KIND == 1) {
            return u >= a.view_lo && u < a.view_hi;
        } else {
            for (int v = a.view_lo; v < a.view_hi; ++v)
                if (a.ft.group[v] == u) return true;
            return false;
        }
    };
    auto terms = [&](int u) { return KIND == 0 ? a.ft.rank[a.ft.group_leader[u]] : a.ft.crank[u]; };
    // taps of step c: horizontal (pass 1) and vertical (pass 2) factor
    auto taps_of = [&](const Step &c) {
        const int t0 = KIND == 0 ? a.ft.tap_off[a.ft.group_leader[c.u]] : a.ft.ctap_off[c.u];
        return a.taps + static_cast<long long>(t0 + c.q) * 4 * K;
    };
    constexpr int kW = KIND == 0 ? 1 : 3, kU = KIND == 0 ? 0 : 2;
    auto tile = [&](int t) { return tcc::tile_of<G::TX, G::TY>(t, tiles_x, tiles_y); };
    auto needs_input = [&](const Step &c, const Step &prev) { return c.q == 0 && (KIND == 1 || c.t != prev.t); };
    auto plane_z = [&](const Step &c) { return KIND == 0 ? tile(c.t).p : c.u * a.P + tile(c.t).p; };
    const bool use_tma = kp.use_tma && (KIND == 1 || a.psi_in != nullptr);
    uint32_t ph1 = 0, ph2 = 0, ph_tma = 0;
    bool tma_pending = false;
    bool p1_out = false, p2_out = false;   // committed MMAs not yet waited for
    auto request = [&](const Step &c) {   // thread 0: the TMA copy of c's input tile
        const Tile tc = tile(c.t);
        tma::fence_proxy_async_smem();
        tma::mbar_arrive_expect_tx(s.bar_tma, G::STAGE_BYTES);
        tma::load_3d(stage, &kp.map, s.bar_tma, tc.x0 - G::R4, tc.y0 - G::R, plane_z(c));
        tma_pending = true;
    };
    // c's input tile -> B1; then the staging tile takes the next input
    auto take_input = [&](const Step &c) -> bool {
        const Tile tc = tile(c.t);
        if (use_tma) {
            if (!wait_bar(s.bar_tma, ph_tma, a, s.abort_flag)) {
                tma_pending = false;   // drained by the wait
                return false;
            }
            ph_tma ^= 1;
            tma_pending = false;
        } else {
            const float *src;
            float fill = 0.0f;
            if (KIND == 0) {
                src = a.psi_in ? a.psi_in + tc.p * plane_px : nullptr;
                if (!a.psi_in) fill = __ldg(a.means + tc.p);
            } else {
                src = a.ratio + (static_cast<long long>(c.u) * a.P + tc.p) * plane_px;
            }
            load_stage_sw<K>(stage, src, fill, tc.y0, tc.x0, a.H, a.W, a.circular);
            __syncthreads();
        }
        convert_b1<K>(stage, b1);
        tma::fence_proxy_async_smem();   // B1 is read by the MMAs (async proxy)
        __syncthreads();
        if (use_tma && threadIdx.x == 0) {
            Step prev = c, n = next_step(c, n_tiles, n_sets, terms, used);
            while (n.valid && !needs_input(n, prev)) {
                prev = n;
                n = next_step(n, n_tiles, n_sets, terms, used);
            }
            if (n.valid) request(n);
        }
        return true;
    };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x_out = 32 * (warp & 3) + lane;
    const int row0 = (warp >> 2) * G::NE;
    float prod[G::NE];
#pragma unroll
    for (int j = 0; j < G::NE; ++j) prod[j] = 1.0f;

    Step cur = first_step(n_tiles, n_sets, terms, used);
    bool ok = cur.valid;
    if (ok) {
        if (use_tma && threadIdx.x == 0) request(cur);
        ok = take_input(cur);
    }
    if (ok) {
        const float *tq = taps_of(cur);
        build_t1<K>(tq + kW * K, tmem);
        build_t2<K>(tq + kU * K, t2);
        tma::fence_proxy_async_smem();
        tc5::fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc5::fence_after();
            issue_pass1<K>(tmem, tc5::smem_u32(b1));
            tc5::commit(s.bar1);
        }
        p1_out = true;
    }
    while (ok && cur.valid) {
        p1_out = false;   // waited for, or drained by a wait that timed out
        if (!(ok = wait_bar(s.bar1, ph1, a, s.abort_flag))) break;
        ph1 ^= 1;
        tc5::fence_after();
        round_d1<K>(tmem);
        tc5::fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc5::fence_after();
            issue_pass2<K>(tmem, tc5::smem_u32(t2), cur.q > 0);
            tc5::commit(s.bar2);
        }
        p2_out = true;
        const Step nxt = next_step(cur, n_tiles, n_sets, terms, used);
        if (nxt.valid) {
            // B1 and T1 are free (pass 1 of this step is complete)
            if (needs_input(nxt, cur) && !(ok = take_input(nxt))) break;
            build_t1<K>(taps_of(nxt) + kW * K, tmem);
        }
        const bool last = cur.q + 1 == terms(cur.u);
        const Tile c = tile(cur.t);
        const int x = c.x0 + x_out;
        int v0 = -1;
        uint32_t phi[G::NE];
        if (KIND == 0 && last) {
            // the set's first view: data loads in flight while pass 2 runs
            for (int v = a.view_lo; v < a.view_hi && v0 < 0; ++v)
                if (a.ft.group[v] == cur.u) v0 = v;
            if (x < a.W) load_phi<G::NE>(a, v0, c.p, c.y0 + row0, x, phi);
        }
        p2_out = false;
        if (!(ok = wait_bar(s.bar2, ph2, a, s.abort_flag))) break;
        ph2 ^= 1;
        tc5::fence_after();
        if (nxt.valid) {
            // T2 and D1 are free (pass 2 of this step is complete): the next
            // step's pass 1 runs while this step's epilogue does
            build_t2<K>(taps_of(nxt) + kU * K, t2);
            tma::fence_proxy_async_smem();
            tc5::fence_before();
            __syncthreads();
            if (threadIdx.x == 0) {
                tc5::fence_after();
                issue_pass1<K>(tmem, tc5::smem_u32(b1));
                tc5::commit(s.bar1);
            }
            p1_out = true;
        }
        if (last) {
            float d[G::NE];
            read_d2<K>(tmem, d);
            if (KIND == 0) {
                if (x < a.W) {
                    store_ratio<G::NE>(a, v0, c.p, c.y0 + row0, x, phi, d);
                    for (int v = v0 + 1; v < a.view_hi; ++v) {
                        if (a.ft.group[v] != cur.u) continue;
                        load_phi<G::NE>(a, v, c.p, c.y0 + row0, x, phi);
                        store_ratio<G::NE>(a, v, c.p, c.y0 + row0, x, phi, d);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < G::NE; ++j) prod[j] *= d[j];
                if (!nxt.valid || nxt.t != cur.t) {   // the tile's last view: the update
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
#pragma unroll
                    for (int j = 0; j < G::NE; ++j) prod[j] = 1.0f;
                }
            }
        }
        // D2 has been read before the next step's pass 2 is issued (after
        // the barrier in the next wait)
        tc5::fence_before();
        cur = nxt;
    }
    // leaving early (a wait timed out): the copies and MMAs still in flight
    // complete before tensor memory is released
    if (threadIdx.x == 0) {
        if (tma_pending) tma::mbar_wait_bounded(s.bar_tma, ph_tma, kDrainBudget);
        if (p1_out) tma::mbar_wait_bounded(s.bar1, ph1, kDrainBudget);
        if (p2_out) tma::mbar_wait_bounded(s.bar2, ph2, kDrainBudget);
    }
}

// Persistent kernel A: blur of every PSF group in use, then the ratios.
template <int K>
__global__ void __launch_bounds__(kThreads, 1) tf32_blur_ratio_kernel(const __grid_constant__ TcParams kp) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = align128(smem_raw);
    const Smem s = setup(smem);
    const uint32_t tmem = *s.tmem_slot;
    pipeline<K, 0>(kp, smem, s, tmem);
    teardown(tmem);
}

// Persistent kernel B: per view, the correlation of its ratio tile; the
// product of the views' corrections stays in registers; then the update.
template <int K>
__global__ void __launch_bounds__(kThreads, 1) tf32_correlate_update_kernel(const __grid_constant__ TcParams kp) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = align128(smem_raw);
    const Smem s = setup(smem);
    const uint32_t tmem = *s.tmem_slot;
    pipeline<K, 1>(kp, smem, s, tmem);
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
        cudaError_t e = cudaFuncSetAttribute(tf32_blur_ratio_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(tf32_correlate_update_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
        if (tma_ok && a.psi_in && tcc::aligned16(a.psi_in))
            kp.use_tma = tcc::encode(&kp.map, a.psi_in, a.W, a.H, a.P, G::KA, G::ROWS);
        tf32_blur_ratio_kernel<K><<<grid, kThreads, G::SMEM_BYTES, st>>>(kp);
    } else {
        if (tma_ok && tcc::aligned16(a.ratio))
            kp.use_tma =
                tcc::encode(&kp.map, a.ratio, a.W, a.H, static_cast<long long>(a.ft.views) * a.P, G::KA, G::ROWS);
        tf32_correlate_update_kernel<K><<<grid, kThreads, G::SMEM_BYTES, st>>>(kp);
    }
    count_launch();
    return cudaGetLastError();
}

#define MVD_TF32_CASES(X) \
    X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(27) X(29) X(31) \
    X(33) X(35) X(37) X(39) X(41) X(43) X(45) X(47)

cudaError_t dispatch(const FusedArgs &a, int which, cudaStream_t st) {
    switch (a.ft.K) {
#define MVD_CASE(k) \
    case k:         \
        return launch<k>(a, which, st);
        MVD_TF32_CASES(MVD_CASE)
#undef MVD_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace tcf

void tf32_tile_shape(int K, int *tile_h, int *tile_w) {
    switch (K) {
#define MVD_CASE(k)                      \
    case k:                              \
        *tile_h = tcf::Geo<k>::TY;       \
        *tile_w = tcf::Geo<k>::TX;       \
        return;
        MVD_TF32_CASES(MVD_CASE)
#undef MVD_CASE
        default:
            *tile_h = *tile_w = 0;
    }
}

cudaError_t launch_tf32_blur_ratio(const FusedArgs &a, cudaStream_t s) { return tcf::dispatch(a, 0, s); }

cudaError_t launch_tf32_correlate_update(const FusedArgs &a, cudaStream_t s) { return tcf::dispatch(a, 1, s); }

}  // namespace mvd
