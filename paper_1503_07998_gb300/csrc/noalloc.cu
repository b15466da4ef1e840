// mvd_deconvolve_planes_static: the fused deconvolution for callers that
// must not allocate GPU memory.
//
// Camera acquisition programs that deconvolve while they record, and plugins
// hosted by an application that owns the GPU's memory pool, often may not
// call cudaMalloc: an allocation can block on the whole device, its latency
// is unbounded, and the host application may account for every byte itself.
// This entry point therefore needs no context and allocates nothing.  The
// fused kernels' scratch (the device status word, the per-plane means and the
// ratio planes) lives in one file-scope device array of kStaticScratchBytes
// that every GPU loading this library holds until the process exits.  The
// factor taps travel in the kernels' parameter blocks, so they need no
// device copy.
//
// The array's name is only a host-side stand-in in host code, so its device
// address is looked up with cudaGetSymbolAddress once per device (with that
// device current) on the first call made on the device, and that address is
// what the kernels receive.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mvd.h"
#include "mvd_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;   // 32 MiB
constexpr int kStaticMaxViews = 8;
constexpr size_t kAlign = 256;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[64] = {};                                  // per device, set once
float g_taps_host[kStaticMaxViews * mvd::kFusedMaxK * 4 * mvd::kFusedMaxK];   // guarded by g_mu
std::atomic<long long> g_wait_budget{mvd::kDefaultWaitBudget};

inline size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

// Device address of the static array on the current device (looked up once
// per device); nullptr with the last error set on failure.  Caller holds g_mu.
unsigned char *scratch_base() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        mvd::set_last_error("cudaGetDevice failed");
        return nullptr;
    }
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            mvd::set_last_error("cudaGetSymbolAddress of the static scratch failed");
            return nullptr;
        }
        g_scratch_ptr[dev] = p;
    }
    return static_cast<unsigned char *>(g_scratch_ptr[dev]);
}

}  // namespace

extern "C" mvd_status mvd_deconvolve_planes_static(int views, const float *psfs_host, int psf_size,
                                                   int plane_h, int plane_w, int iters,
                                                   mvd_boundary boundary, float eps,
                                                   const void *data_dev, mvd_dtype dt,
                                                   float *estimate_dev, int n_planes, int init_mean,
                                                   void *stream) {
    auto fail = [](mvd_status s, const char *m) {
        mvd::set_last_error(m);
        return s;
    };
    mvd::set_last_error("");
    if (views < 1 || views > kStaticMaxViews) return fail(MVD_ERR_ARG, "views must be in [1, 8]");
    if (!psfs_host || !data_dev || !estimate_dev) return fail(MVD_ERR_ARG, "NULL buffer");
    if (!mvd::fused_supported(psf_size)) return fail(MVD_ERR_ARG, "PSF size must be odd and <= 47");
    if (plane_h < 1 || plane_w < 1 || iters < 0 || n_planes < 0 || n_planes > 65535)
        return fail(MVD_ERR_ARG, "bad sizes");
    if (!(eps > 0.0f)) return fail(MVD_ERR_ARG, "eps must be positive");
    if (dt != MVD_U16 && dt != MVD_F32) return fail(MVD_ERR_ARG, "unknown dtype");
    if (boundary != MVD_BOUNDARY_ZERO && boundary != MVD_BOUNDARY_CIRCULAR) return fail(MVD_ERR_ARG, "unknown boundary");
    if (boundary == MVD_BOUNDARY_CIRCULAR && (psf_size > plane_h || psf_size > plane_w))
        return fail(MVD_ERR_ARG, "circular boundary needs K <= min(H, W)");
    const size_t KK = static_cast<size_t>(psf_size) * psf_size;
    for (size_t i = 0; i < KK * views; ++i)
        if (!std::isfinite(psfs_host[i]) || psfs_host[i] < 0.0f) return fail(MVD_ERR_ARG, "PSF entries must be finite and >= 0");
    for (int v = 0; v < views; ++v) {
        double sum = 0.0;
        for (size_t i = 0; i < KK; ++i) sum += psfs_host[KK * v + i];
        if (!(sum > 0.0)) return fail(MVD_ERR_ARG, "every PSF must have a positive sum");
    }
    if (n_planes == 0) return MVD_OK;
    {
        const char *d0 = static_cast<const char *>(data_dev), *e0 = reinterpret_cast<const char *>(estimate_dev);
        const size_t px = static_cast<size_t>(plane_h) * plane_w * n_planes;
        const size_t dbytes = px * views * (dt == MVD_U16 ? 2 : 4), ebytes = px * sizeof(float);
        if (d0 < e0 + ebytes && e0 < d0 + dbytes) return fail(MVD_ERR_ARG, "data and estimate overlap");
    }

    // scratch layout: status word | means | ratio planes
    const size_t plane_px = static_cast<size_t>(plane_h) * plane_w;
    const size_t off_means = kAlign;
    const size_t off_ratio = off_means + round_up(static_cast<size_t>(n_planes) * sizeof(float));
    const size_t need = off_ratio + static_cast<size_t>(views) * n_planes * plane_px * sizeof(float);
    if (need > kStaticScratchBytes) {
        char m[200];
        std::snprintf(m, sizeof m,
                      "these sizes need %zu bytes of scratch; the static scratch holds %zu bytes "
                      "(call again with fewer planes)", need, kStaticScratchBytes);
        return fail(MVD_ERR_ARG, m);
    }

    std::lock_guard<std::mutex> lock(g_mu);
    unsigned char *base = scratch_base();
    if (!base) return MVD_ERR_CUDA;

    mvd::FactorTable ft;
    char msg[200] = {0};
    if (!mvd::factorise_psfs(psfs_host, views, psf_size, mvd::kDefaultRankTol, ft, g_taps_host,
                             static_cast<int>(sizeof g_taps_host / sizeof(float)), msg, sizeof msg))
        return fail(MVD_ERR_ARG, "PSF factorisation failed");
    if (!mvd::fused_taps_fit(ft)) return fail(MVD_ERR_ARG, "the PSFs need too many separable terms for this call");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(base, 0, kAlign, s);   // status word starts at zero
    if (e != cudaSuccess) return fail(MVD_ERR_CUDA, "scratch set-up failed");

    float *means = reinterpret_cast<float *>(base + off_means);
    if (init_mean) {
        e = mvd::launch_plane_means(data_dev, dt == MVD_U16, views, n_planes, plane_h, plane_w, means, s);
        if (e != cudaSuccess) return fail(MVD_ERR_CUDA, "plane means kernel failed");
    }
    mvd::FusedArgs a{};
    a.means = means;
    a.psi_out = estimate_dev;
    a.phi = data_dev;
    a.phi_u16 = dt == MVD_U16;
    a.ratio = reinterpret_cast<float *>(base + off_ratio);
    a.taps = nullptr;   // the fused kernels take their taps from the parameter block
    a.taps_host = g_taps_host;
    a.ft = ft;
    a.H = plane_h;
    a.W = plane_w;
    a.P = n_planes;
    a.circular = boundary == MVD_BOUNDARY_CIRCULAR;
    a.eps = eps;
    a.view_lo = 0;
    a.view_hi = views;
    a.err = reinterpret_cast<int *>(base);
    a.wait_budget = g_wait_budget.load();
    if (iters == 0 && init_mean) {
        for (int p = 0; p < n_planes; ++p) {
            e = mvd::plain_fill(estimate_dev + p * plane_px, means, p, plane_px, s);
            if (e != cudaSuccess) return fail(MVD_ERR_CUDA, "fill kernel failed");
        }
        return MVD_OK;
    }
    for (int t = 0; t < iters; ++t) {
        a.psi_in = (t == 0 && init_mean) ? nullptr : estimate_dev;
        if ((e = mvd::launch_fused_blur_ratio(a, s)) != cudaSuccess) return fail(MVD_ERR_CUDA, "blur/ratio kernel failed");
        if ((e = mvd::launch_fused_correlate_update(a, s)) != cudaSuccess)
            return fail(MVD_ERR_CUDA, "correlate/update kernel failed");
    }
    return MVD_OK;
}

extern "C" mvd_status mvd_static_device_status(void *stream) {
    mvd::set_last_error("");
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned char *base = scratch_base();
    if (!base) return MVD_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int word = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&word, base, sizeof word, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(base, 0, sizeof word);
    if (e != cudaSuccess) {
        mvd::set_last_error(cudaGetErrorString(e));
        return MVD_ERR_CUDA;
    }
    if (word & mvd::kDevTimeout) {
        mvd::set_last_error("a tile wait of the static deconvolution timed out; its estimate is incomplete");
        return MVD_ERR_TIMEOUT;
    }
    return MVD_OK;
}

extern "C" mvd_status mvd_static_set_wait_budget(long long cycles) {
    mvd::set_last_error("");
    g_wait_budget.store(cycles == 0 ? mvd::kDefaultWaitBudget : cycles);
    return MVD_OK;
}
