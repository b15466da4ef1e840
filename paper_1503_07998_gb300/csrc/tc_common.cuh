// Pieces shared by the two tensor-core routes of the fused MV-RL iteration
// (BF16x3 in tc.cu, TF32 in tc32.cu): the CTA shape, bounded barrier waits,
// the persistent walk over tiles, the data loads and ratio stores of the
// blur/ratio epilogue, and the FP32 tensor map of a stack of planes.
//
// Both routes run one CTA of 512 threads per SM.  The 16 warps form four
// lane quarters (warp % 4) of tensor memory times four column groups
// (warp / 4); in the epilogue thread (quarter q, lane l) owns output column
// 32 q + l of the tile and the column group's TY / 4 consecutive rows.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mvd_internal.h"
#include "tc5.cuh"
#include "tma.cuh"

namespace mvd {
namespace tcc {

constexpr int kThreads = 512;
constexpr long long kDrainBudget = 4000000000LL;
constexpr int kTmemCols = 512;

struct TcParams {
    CUtensorMap map;   // psi (kernel A) or the ratio planes (kernel B); valid if use_tma
    FusedArgs a;
    int use_tma;
};

__device__ __forceinline__ unsigned char *align128(unsigned char *p) {
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 127) & ~static_cast<uintptr_t>(127));
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

// Tile t of a launch: planes outermost, then TY-row bands, then TX-column
// blocks.
template <int TX, int TY>
__device__ __forceinline__ Tile tile_of(int t, int tiles_x, int tiles_y) {
    const int per_plane = tiles_x * tiles_y;
    const int p = t / per_plane;
    const int r = t - p * per_plane;
    const int ty = r / tiles_x;
    return {p, ty * TY, (r - ty * tiles_x) * TX};
}

// Shared setup: three mbarriers (MMA completions bar1 / bar2, TMA tile
// arrival bar_tma), the abort flag, all tensor-memory columns.
struct Smem {
    uint64_t *bar1, *bar2, *bar_tma;
    volatile int *abort_flag;
    uint32_t *tmem_slot;
};

__device__ __forceinline__ Smem setup(unsigned char *smem) {
    Smem s;
    s.bar1 = reinterpret_cast<uint64_t *>(smem);
    s.bar2 = reinterpret_cast<uint64_t *>(smem + 8);
    s.bar_tma = reinterpret_cast<uint64_t *>(smem + 16);
    s.abort_flag = reinterpret_cast<volatile int *>(smem + 24);
    s.tmem_slot = reinterpret_cast<uint32_t *>(smem + 28);
    if (threadIdx.x == 0) {
        tma::mbar_init(s.bar1, 1);
        tma::mbar_init(s.bar2, 1);
        tma::mbar_init(s.bar_tma, 1);
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

// Raw data of view v at column x, rows y0 .. y0 + NE (uint16 or FP32 bits).
// Nothing here consumes a loaded value, so all NE loads are in flight
// together; store_ratio converts them.
template <int NE>
__device__ __forceinline__ void load_phi(const FusedArgs &a, int v, int p, int y0, int x, uint32_t (&phi)[NE]) {
    const long long base = (static_cast<long long>(v) * a.P + p) * a.H * a.W + x;
    const int n = min(NE, a.H - y0);
    if (a.phi_u16) {
        const uint16_t *src = static_cast<const uint16_t *>(a.phi) + base;
#pragma unroll
        for (int j = 0; j < NE; ++j)
            phi[j] = j < n ? static_cast<uint32_t>(__ldg(src + static_cast<long long>(y0 + j) * a.W)) : 0u;
    } else {
        const float *src = static_cast<const float *>(a.phi) + base;
#pragma unroll
        for (int j = 0; j < NE; ++j)
            phi[j] = j < n ? __float_as_uint(__ldg(src + static_cast<long long>(y0 + j) * a.W)) : 0u;
    }
}

// r_v = phi_v / max(blur, eps) at column x, rows y0 .. y0 + NE.
template <int NE>
__device__ __forceinline__ void store_ratio(const FusedArgs &a, int v, int p, int y0, int x, const uint32_t (&phi)[NE],
                                            const float (&d)[NE]) {
    const long long base = (static_cast<long long>(v) * a.P + p) * a.H * a.W + x;
#pragma unroll
    for (int j = 0; j < NE; ++j) {
        const int y = y0 + j;
        const float f = a.phi_u16 ? static_cast<float>(phi[j]) : __uint_as_float(phi[j]);
        if (y < a.H) a.ratio[base + static_cast<long long>(y) * a.W] = __fdiv_rn(f, fmaxf(d[j], a.eps));
    }
}

// ---- host side ------------------------------------------------------------

inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// FP32 tensor [D][H][W] (W innermost), box box_w x box_h x 1, zero fill.
inline bool encode(CUtensorMap *m, const void *base, int W, int H, long long D, int box_w, int box_h) {
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

// Number of SMs of the current device (cached per device).
inline int sm_count(int dev) {
    static int sms[64] = {};
    if (!sms[dev & 63]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms[dev & 63] = n > 0 ? n : 1;
    }
    return sms[dev & 63];
}

}  // namespace tcc
}  // namespace mvd
