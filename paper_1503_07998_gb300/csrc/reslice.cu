// Reslicing (Abstract; Fig. 1a) and the per-plane mean that starts the
// iterations.
//
// Reslicing [V][Z][Y][X] -> [V][Y][Z][X] keeps X innermost on both sides, so
// it is a gather of contiguous rows: no shared-memory transpose is needed and
// every load and store is a coalesced 16-byte access when a row is a multiple
// of 16 bytes.  It is bound by HBM bandwidth: 2 * bytes(stack) per call.
//
// The mean of plane p over all views is summed in FP64 (exactly in integers
// for uint16 data) by one CTA per plane, so results do not depend on launch
// order.
#include <cuda_runtime.h>
#include <cstdint>

#include "mvd_internal.h"

namespace mvd {

namespace {

constexpr int kResliceThreads = 256;

// One 16-byte unit per thread iteration; rows of `row_units` units.
__global__ void __launch_bounds__(kResliceThreads)
reslice_rows_vec16(const uint4 *__restrict__ src, uint4 *__restrict__ dst, int views, int nz,
                   int ny, long long row_units, long long total_units) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long u = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; u < total_units;
         u += stride) {
        // destination order: ((v * ny + y) * nz + z) * row_units + c
        const long long c = u % row_units;
        long long row = u / row_units;
        const long long z = row % nz;
        row /= nz;
        const long long y = row % ny;
        const long long v = row / ny;
        const long long s_off = ((v * nz + z) * ny + y) * row_units + c;
        dst[u] = __ldg(src + s_off);
    }
}

template <typename T>
__global__ void __launch_bounds__(kResliceThreads)
reslice_rows_scalar(const T *__restrict__ src, T *__restrict__ dst, int views, int nz, int ny,
                    long long nx, long long total) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long u = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; u < total;
         u += stride) {
        const long long x = u % nx;
        long long row = u / nx;
        const long long z = row % nz;
        row /= nz;
        const long long y = row % ny;
        const long long v = row / ny;
        dst[u] = src[((v * nz + z) * ny + y) * nx + x];
    }
}

constexpr int kMeanThreads = 512;

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// uint16 data: exact integer sums (per thread < 2^32 per pass, combined in 64 bits).
__global__ void __launch_bounds__(kMeanThreads)
plane_means_u16(const uint16_t *__restrict__ data, int views, int planes, long long plane_px,
                float *__restrict__ means) {
    const int p = blockIdx.x;
    unsigned long long acc = 0;
    for (int v = 0; v < views; ++v) {
        const uint16_t *src = data + (static_cast<long long>(v) * planes + p) * plane_px;
        unsigned int part = 0;
        int n = 0;
        const bool vec = (reinterpret_cast<uintptr_t>(src) % 16 == 0);
        long long i0 = 0;
        if (vec) {
            const long long nvec = plane_px / 8;
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
            for (long long i = threadIdx.x; i < nvec; i += blockDim.x) {
                const uint4 q = __ldg(s4 + i);
                part += (q.x & 0xffffu) + (q.x >> 16) + (q.y & 0xffffu) + (q.y >> 16) +
                        (q.z & 0xffffu) + (q.z >> 16) + (q.w & 0xffffu) + (q.w >> 16);
                if (++n == 4096) { acc += part; part = 0; n = 0; }
            }
            i0 = nvec * 8;
        }
        acc += part;
        for (long long i = i0 + threadIdx.x; i < plane_px; i += blockDim.x) acc += src[i];
    }
    __shared__ unsigned long long red[kMeanThreads / 32];
    acc = warp_sum_u64(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
        t = warp_sum_u64(t);
        if (threadIdx.x == 0)
            means[p] = static_cast<float>(static_cast<double>(t) /
                                          (static_cast<double>(plane_px) * views));
    }
}

// FP32 data: FP64 accumulation of every element.
__global__ void __launch_bounds__(kMeanThreads)
plane_means_f32(const float *__restrict__ data, int views, int planes, long long plane_px,
                float *__restrict__ means) {
    const int p = blockIdx.x;
    double acc = 0;
    for (int v = 0; v < views; ++v) {
        const float *src = data + (static_cast<long long>(v) * planes + p) * plane_px;
        for (long long i = threadIdx.x; i < plane_px; i += blockDim.x)
            acc += static_cast<double>(__ldg(src + i));
    }
    __shared__ double red[kMeanThreads / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0)
            means[p] = static_cast<float>(t / (static_cast<double>(plane_px) * views));
    }
}

int grid_for(long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    const long long cap = 152LL * 16;   // 16 resident CTAs of 256 threads per SM
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return static_cast<int>(g);
}

}  // namespace

cudaError_t launch_reslice(const void *src, void *dst, int elem_bytes, int views, int nz, int ny,
                           int nx, cudaStream_t s) {
    const long long row_bytes = static_cast<long long>(nx) * elem_bytes;
    const long long rows = static_cast<long long>(views) * nz * ny;
    const bool vec = (row_bytes % 16 == 0) && (reinterpret_cast<uintptr_t>(src) % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(dst) % 16 == 0);
    if (vec) {
        const long long row_units = row_bytes / 16;
        const long long total = rows * row_units;
        reslice_rows_vec16<<<grid_for(total, kResliceThreads), kResliceThreads, 0, s>>>(
            static_cast<const uint4 *>(src), static_cast<uint4 *>(dst), views, nz, ny, row_units,
            total);
    } else if (elem_bytes == 2) {
        const long long total = rows * nx;
        reslice_rows_scalar<uint16_t><<<grid_for(total, kResliceThreads), kResliceThreads, 0, s>>>(
            static_cast<const uint16_t *>(src), static_cast<uint16_t *>(dst), views, nz, ny, nx, total);
    } else {
        const long long total = rows * nx;
        reslice_rows_scalar<float><<<grid_for(total, kResliceThreads), kResliceThreads, 0, s>>>(
            static_cast<const float *>(src), static_cast<float *>(dst), views, nz, ny, nx, total);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_plane_means(const void *data, int u16, int views, int planes, int H, int W,
                               float *means, cudaStream_t s) {
    const long long px = static_cast<long long>(H) * W;
    if (u16)
        plane_means_u16<<<planes, kMeanThreads, 0, s>>>(static_cast<const uint16_t *>(data), views,
                                                        planes, px, means);
    else
        plane_means_f32<<<planes, kMeanThreads, 0, s>>>(static_cast<const float *>(data), views,
                                                        planes, px, means);
    count_launch();
    return cudaGetLastError();
}

namespace {

// Padded-domain estimate: plane (v, p) of H x W -> centre of a (H+2pad) x
// (W+2pad) plane, zeros around; weights 1 on the data, 0 in the padding.
template <typename T>
__global__ void embed_padded_kernel(const T *__restrict__ src, T *__restrict__ dst, float *__restrict__ w, int H,
                                    int W, int pad, long long n_out) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_out) return;
    const int Hp = H + 2 * pad, Wp = W + 2 * pad;
    const long long plane = i / (static_cast<long long>(Hp) * Wp);
    const long long r = i - plane * Hp * Wp;
    const int y = static_cast<int>(r / Wp) - pad;
    const int x = static_cast<int>(r % Wp) - pad;
    const bool in = y >= 0 && y < H && x >= 0 && x < W;
    dst[i] = in ? src[plane * H * W + static_cast<long long>(y) * W + x] : T(0);
    if (w) w[i] = in ? 1.0f : 0.0f;
}

__global__ void crop_planes_kernel(const float *__restrict__ src, float *__restrict__ dst, int Hp, int Wp, int pad,
                                   long long n_out) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_out) return;
    const int H = Hp - 2 * pad, W = Wp - 2 * pad;
    const long long plane = i / (static_cast<long long>(H) * W);
    const long long r = i - plane * H * W;
    const int y = static_cast<int>(r / W), x = static_cast<int>(r % W);
    dst[i] = src[plane * Hp * Wp + static_cast<long long>(y + pad) * Wp + x + pad];
}

}  // namespace

cudaError_t launch_embed_padded(const void *src, int elem_bytes, long long planes, int H, int W, int pad, void *dst,
                                float *weights, cudaStream_t s) {
    const long long n = planes * (H + 2LL * pad) * (W + 2LL * pad);
    if (n == 0) return cudaSuccess;
    const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
    if (elem_bytes == 2)
        embed_padded_kernel<uint16_t><<<blocks, 256, 0, s>>>(static_cast<const uint16_t *>(src),
                                                             static_cast<uint16_t *>(dst), weights, H, W, pad, n);
    else
        embed_padded_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(src), static_cast<float *>(dst),
                                                          weights, H, W, pad, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_crop_planes(const float *src, long long planes, int Hp, int Wp, int pad, float *dst,
                               cudaStream_t s) {
    const long long n = planes * (Hp - 2LL * pad) * (Wp - 2LL * pad);
    if (n == 0) return cudaSuccess;
    crop_planes_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(src, dst, Hp, Wp, pad, n);
    count_launch();
    return cudaGetLastError();
}

}  // namespace mvd
