// 3D MV-RL for views turned about the rotation axis: the PSF of view v is
// a_v(y) P_v(z, x), the plane-wise in-plane PSF times a profile along the
// axis (the plane index y).  The in-plane blur and correlation run in the
// fused kernels; these two kernels add the passes along the plane axis:
//
//   axial_ratio  r[y] = phi[y] / max(sum_i a[i] b[y - (i - R)], eps)
//   axial_corr   c[y] = sum_i a[i] r[y + (i - R)]
//
// over the P planes of a call (planes outside are zero, or wrapped for the
// circular boundary).  A block stages kRun + Ka - 1 planes of 128
// consecutive pixel positions in shared memory (coalesced row segments, each
// value read once) and each thread walks the kRun output planes of its
// position.
#include <cuda_runtime.h>
#include <cstdint>

#include "mvd_internal.h"

namespace mvd {

namespace {

constexpr int kCols = 128;   // pixel positions per block (one per thread)
constexpr int kRun = 32;     // output planes per block

// Stage planes [y0 - R, y0 + kRun + R) of columns [px0, px0 + kCols) in
// shared memory: every input value is read from global memory once.
__device__ __forceinline__ void stage_planes(const float *__restrict__ in, float *tile, int y0, int R, int P,
                                             long long plane, long long px0, int circular) {
    const int rows = kRun + 2 * R;
    const long long px = px0 + threadIdx.x;
    constexpr int kBatch = 8;   // loads in flight per thread
    for (int r0 = 0; r0 < rows; r0 += kBatch) {
        float v[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            int y = y0 - R + r0 + b;
            v[b] = 0.0f;
            if (r0 + b >= rows || px >= plane) continue;
            if (circular) {
                y %= P;
                if (y < 0) y += P;
                v[b] = __ldg(in + y * plane + px);
            } else if (y >= 0 && y < P) {
                v[b] = __ldg(in + y * plane + px);
            }
        }
#pragma unroll
        for (int b = 0; b < kBatch; ++b)
            if (r0 + b < rows) tile[(r0 + b) * kCols + threadIdx.x] = v[b];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kCols)
axial_ratio_kernel(const float *__restrict__ blur, const void *__restrict__ phi, int u16,
                   const float *__restrict__ a, int Ka, int P, long long plane, int circular, float eps,
                   float *__restrict__ r) {
    extern __shared__ float tile[];
    const int R = (Ka - 1) / 2;
    const long long px0 = static_cast<long long>(blockIdx.x) * kCols;
    const int y0 = blockIdx.y * kRun;
    stage_planes(blur, tile, y0, R, P, plane, px0, circular);
    const long long px = px0 + threadIdx.x;
    if (px >= plane) return;
    for (int j = 0; j < kRun && y0 + j < P; ++j) {
        // sum_k a[k] b[y - (k - R)]: tile row (j + R) - (k - R)
        float sacc = 0.0f;
        for (int k = 0; k < Ka; ++k) sacc = fmaf(__ldg(a + k), tile[(j + 2 * R - k) * kCols + threadIdx.x], sacc);
        const long long o = static_cast<long long>(y0 + j) * plane + px;
        const float d = u16 ? static_cast<float>(static_cast<const uint16_t *>(phi)[o])
                            : static_cast<const float *>(phi)[o];
        r[o] = __fdiv_rn(d, fmaxf(sacc, eps));
    }
}

__global__ void __launch_bounds__(kCols)
axial_corr_kernel(const float *__restrict__ r, const float *__restrict__ a, int Ka, int P, long long plane,
                  int circular, float *__restrict__ c) {
    extern __shared__ float tile[];
    const int R = (Ka - 1) / 2;
    const long long px0 = static_cast<long long>(blockIdx.x) * kCols;
    const int y0 = blockIdx.y * kRun;
    stage_planes(r, tile, y0, R, P, plane, px0, circular);
    const long long px = px0 + threadIdx.x;
    if (px >= plane) return;
    for (int j = 0; j < kRun && y0 + j < P; ++j) {
        // sum_k a[k] r[y + (k - R)]: tile row j + k
        float sacc = 0.0f;
        for (int k = 0; k < Ka; ++k) sacc = fmaf(__ldg(a + k), tile[(j + k) * kCols + threadIdx.x], sacc);
        c[static_cast<long long>(y0 + j) * plane + px] = sacc;
    }
}

dim3 grid_of(int P, long long plane) {
    return dim3(static_cast<unsigned>((plane + kCols - 1) / kCols), static_cast<unsigned>((P + kRun - 1) / kRun));
}

size_t smem_of(int Ka) { return static_cast<size_t>(kRun + Ka - 1) * kCols * sizeof(float); }

cudaError_t allow_smem(const void *fn, size_t bytes) {
    return bytes > 48 * 1024 ? cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    static_cast<int>(bytes))
                             : cudaSuccess;
}

}  // namespace

cudaError_t launch_axial_ratio(const float *blur, const void *phi, int u16, const float *a, int Ka, int P,
                               long long plane, int circular, float eps, float *r, cudaStream_t s) {
    if (P == 0 || plane == 0) return cudaSuccess;
    const size_t sm = smem_of(Ka);
    cudaError_t e = allow_smem(reinterpret_cast<const void *>(axial_ratio_kernel), sm);
    if (e != cudaSuccess) return e;
    axial_ratio_kernel<<<grid_of(P, plane), kCols, sm, s>>>(blur, phi, u16, a, Ka, P, plane, circular, eps, r);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_axial_corr(const float *r, const float *a, int Ka, int P, long long plane, int circular, float *c,
                              cudaStream_t s) {
    if (P == 0 || plane == 0) return cudaSuccess;
    const size_t sm = smem_of(Ka);
    cudaError_t e = allow_smem(reinterpret_cast<const void *>(axial_corr_kernel), sm);
    if (e != cudaSuccess) return e;
    axial_corr_kernel<<<grid_of(P, plane), kCols, sm, s>>>(r, a, Ka, P, plane, circular, c);
    count_launch();
    return cudaGetLastError();
}

}  // namespace mvd
