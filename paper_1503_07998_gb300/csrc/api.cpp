// C ABI of the library (declared in include/mvd.h): context life cycle,
// argument checking, workspace, and the sequencing of kernels for one call.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mvd.h"
#include "mvd_internal.h"

namespace mvd {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(static_cast<uint64_t>(n), std::memory_order_relaxed); }

}  // namespace mvd

namespace {

thread_local std::string t_last_error;

}  // namespace

void mvd::set_last_error(const char *msg) { t_last_error = msg ? msg : ""; }

namespace {

mvd_status fail(mvd_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return s;
}

mvd_status cuda_fail(cudaError_t e, const char *what) {
    return fail(MVD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Tuning cache (MVD_TUNE_CACHE): lines "<key> <a> <b>".
bool tune_cache_lookup(const std::string &key, int *a, int *b, int *c);
void tune_cache_store(const std::string &key, int a, int b, int c);

struct DeviceGuard {
    int prev = -1, want;
    explicit DeviceGuard(int d) : want(d) {
        cudaGetDevice(&prev);
        if (prev != want) cudaSetDevice(want);
    }
    ~DeviceGuard() {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

// Test hook (mvd_debug_fail_allocations): this many of the next device
// allocations fail as if cudaMalloc had run out of memory.
std::atomic<int> g_fail_allocs{0};

bool take_injected_failure() {
    int n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
    return false;
}

// Device buffer that only grows.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want) {
        if (want <= bytes) return cudaSuccess;
        if (ptr) {
            cudaFree(ptr);
            ptr = nullptr;
            bytes = 0;
        }
        if (take_injected_failure()) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(&ptr, want);
        if (e == cudaSuccess) bytes = want;
        return e;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    template <typename T>
    T *as() const { return static_cast<T *>(ptr); }
};

// CUDA-event timing of every launch of a context (mvd_profile_*): an event is
// recorded before each launch, labelled with the kernel that follows it, and
// one after the last; the time between consecutive events is the labelled
// kernel's device time.
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool, all;
    std::vector<std::pair<cudaEvent_t, int>> marks;
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<uint64_t> count;
    int label(const char *name) {
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == name) return static_cast<int>(i);
        names.emplace_back(name);
        ms.push_back(0.0);
        count.push_back(0);
        return static_cast<int>(names.size() - 1);
    }
    void mark(cudaStream_t s, const char *name) {
        if (!on) return;
        cudaEvent_t e;
        if (pool.empty()) {
            if (cudaEventCreate(&e) != cudaSuccess) return;
            all.push_back(e);
        } else {
            e = pool.back();
            pool.pop_back();
        }
        cudaEventRecord(e, s);
        marks.emplace_back(e, name ? label(name) : -1);
    }
    void end(cudaStream_t s) { mark(s, nullptr); }
    void resolve() {
        if (!marks.empty()) cudaEventSynchronize(marks.back().first);
        for (size_t i = 0; i + 1 < marks.size(); ++i) {
            if (marks[i].second < 0) continue;
            float t = 0;
            if (cudaEventElapsedTime(&t, marks[i].first, marks[i + 1].first) == cudaSuccess) {
                ms[marks[i].second] += t;
                count[marks[i].second] += 1;
            }
        }
        for (auto &m : marks) pool.push_back(m.first);
        marks.clear();
    }
    void reset() {
        resolve();
        names.clear();
        ms.clear();
        count.clear();
    }
    void destroy() {
        for (auto e : all) cudaEventDestroy(e);
        all.clear();
        pool.clear();
        marks.clear();
    }
};

}  // namespace

struct mvd_ctx {
    int device = 0;
    int V = 0, K = 0, H = 0, W = 0, iters = 0;
    mvd_boundary boundary = MVD_BOUNDARY_ZERO;
    float eps = 1e-6f;
    mvd_algo algo = MVD_ALGO_FUSED;
    mvd_update_order order = MVD_ORDER_SIMULTANEOUS;
    mvd_variant variant = MVD_VARIANT_INDEPENDENT;
    double rank_tol = mvd::kDefaultRankTol;
    std::vector<float> psfs;
    std::vector<float> corr_psfs;        // a variant's flip(X_v), [V][K][K]; empty for plain MV-RL
    bool psf_dev_fresh = false;          // psf_dev holds the current psfs (+ corr_psfs)
    const float *weights = nullptr;      // caller's [V][P][H][W] per-pixel view weights, or none
    int weight_planes = 0;               // P, or 1: one plane per view used for every plane
    DevBuf wnorm, wtmp;                  // 1 / footprint per view and plane; scratch planes
    std::vector<float> axial;            // 3D route: [V][Ka] profiles along the rotation axis
    int Ka = 0;
    DevBuf axial_dev, tmp3d;
    std::vector<float> taps_host;
    mvd::FactorTable ft;
    DevBuf taps, psf_dev, means, ratio, plain;
    DevBuf psi_split;                    // split copy of the estimate (warp-specialised tensor kernels)
    // end-to-end pipeline
    DevBuf run_stack[2], run_planes, run_est[2];
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    Profiler prof;
    DevBuf status;                       // one int: device status word
    DevBuf grad_ws, grad_acc;            // PSF-gradient workspace (floats) and FP64 sums
    long long wait_budget = mvd::kDefaultWaitBudget;
    int max_ctas = 0;                    // persistent-grid cap set by a batch's tuner
    // Fourier route: padded grid, transform plans, twiddles, PSF spectra, spectra scratch
    struct {
        bool planned = false;
        int Ly = 0, Lx = 0, Lc = 0, LcP = 0;
        mvd::fftr::FftPlan1 px{}, py{};
        DevBuf tw_x, tw_y, spec, cspec, S0, T;
    } fft;
    DevBuf res_taps;                     // plane-resident route: factors padded to the size class
    bool res_taps_ready = false;         // res_taps holds the current factors
};

namespace {

// A variant's correlation kernels: the ratio is convolved with X_v, i.e.
// correlated with flip(X_v), which is what the correlation taps implement.
void build_corr_psfs(mvd_ctx *c) {
    c->corr_psfs.clear();
    if (c->variant == MVD_VARIANT_INDEPENDENT) return;
    const int K = c->K;
    const size_t KK = static_cast<size_t>(K) * K;
    std::vector<double> X(KK * c->V);
    mvd::variant_kernels(c->psfs.data(), c->V, K, c->variant, X.data());
    c->corr_psfs.resize(KK * c->V);
    for (int v = 0; v < c->V; ++v)
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j)
                c->corr_psfs[KK * v + static_cast<size_t>(i) * K + j] =
                    static_cast<float>(X[KK * v + static_cast<size_t>(K - 1 - i) * K + (K - 1 - j)]);
}

// Device copy of the PSFs followed, for a variant, by its correlation kernels.
cudaError_t upload_psf_dev(mvd_ctx *c) {
    if (c->psf_dev_fresh) return cudaSuccess;
    const size_t n = c->psfs.size() + c->corr_psfs.size();
    cudaError_t e = c->psf_dev.ensure(n * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->psf_dev.ptr, c->psfs.data(), c->psfs.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !c->corr_psfs.empty())
        e = cudaMemcpy(c->psf_dev.as<float>() + c->psfs.size(), c->corr_psfs.data(),
                       c->corr_psfs.size() * sizeof(float), cudaMemcpyHostToDevice);
    c->psf_dev_fresh = e == cudaSuccess;
    return e;
}

mvd_status upload_factors(mvd_ctx *c) {
    const int cap = mvd::max_terms(c->V, c->K) * 4 * c->K;
    std::vector<float> &taps = c->taps_host;
    taps.assign(static_cast<size_t>(cap), 0.0f);
    char msg[256] = {0};
    build_corr_psfs(c);
    c->psf_dev_fresh = false;
    c->fft.planned = false;   // the spectra follow the PSFs and the variant
    c->res_taps_ready = false;
    if (!mvd::factorise_psfs(c->psfs.data(), c->V, c->K, c->rank_tol, c->ft, taps.data(), cap, msg, sizeof msg,
                             c->corr_psfs.empty() ? nullptr : c->corr_psfs.data()))
        return fail(MVD_ERR_ARG, "PSF factorisation failed: %s", msg);
    const size_t bytes = static_cast<size_t>(c->ft.total_terms) * 4 * c->K * sizeof(float);
    cudaError_t e = c->taps.ensure(bytes);
    if (e != cudaSuccess) return fail(MVD_ERR_NOMEM, "taps: %s", cudaGetErrorString(e));
    e = cudaMemcpy(c->taps.ptr, taps.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload taps");
    return MVD_OK;
}

mvd::FusedArgs fused_args(const mvd_ctx *c, const void *data, mvd_dtype dt, float *est, int P) {
    mvd::FusedArgs a{};
    a.psi_in = est;
    a.means = c->means.as<float>();
    a.psi_out = est;
    a.phi = data;
    a.phi_u16 = dt == MVD_U16;
    a.ratio = c->ratio.as<float>();
    a.taps = c->taps.as<float>();
    a.taps_host = c->taps_host.data();
    a.ft = c->ft;
    a.H = c->H;
    a.W = c->W;
    a.P = P;
    a.circular = c->boundary == MVD_BOUNDARY_CIRCULAR;
    a.eps = c->eps;
    a.err = c->status.as<int>();
    a.weights = c->weights;
    a.wnorm = c->weights ? c->wnorm.as<float>() : nullptr;
    a.weights_bcast = c->weight_planes == 1;
    a.wait_budget = c->wait_budget;
    a.max_ctas = c->max_ctas;
    return a;
}

mvd_status fft_plan(mvd_ctx *c);

// The tensor-core routes (BF16x3, TF32): the fused kernels' schedule.
inline bool tensor_algo(mvd_algo a) { return a == MVD_ALGO_TENSOR || a == MVD_ALGO_TF32; }

// Allocate everything a deconvolution of P planes needs, so that the call
// itself allocates nothing (required while a stream is being captured).
cudaError_t prepare_workspace(mvd_ctx *c, int P) {
    const size_t plane_px = static_cast<size_t>(c->H) * c->W;
    cudaError_t e = c->means.ensure(static_cast<size_t>(P) * sizeof(float));
    if (e == cudaSuccess && c->algo == MVD_ALGO_FFT) {
        if (fft_plan(c) != MVD_OK) return cudaErrorInvalidValue;
        const size_t rows = static_cast<size_t>(P) * c->H * c->fft.LcP;
        e = c->fft.S0.ensure(rows * sizeof(float2));
        if (e == cudaSuccess) e = c->fft.T.ensure(rows * c->V * sizeof(float2));
    }
    if (e == cudaSuccess && ((c->algo == MVD_ALGO_FUSED && mvd::fused_taps_fit(c->ft)) || tensor_algo(c->algo))) {
        size_t bytes = static_cast<size_t>(c->V) * P * plane_px * sizeof(float);
        if (c->algo == MVD_ALGO_TENSOR) {   // split ratio and estimate of the warp-specialised kernels
            bytes = std::max(bytes, mvd::tcw_split_bytes(c->W, c->H, static_cast<long long>(c->V) * P));
            e = c->psi_split.ensure(mvd::tcw_split_bytes(c->W, c->H, P));
        }
        if (e == cudaSuccess) e = c->ratio.ensure(bytes);
    }
    if (e == cudaSuccess) e = c->plain.ensure(4 * plane_px * sizeof(float));
    if (e == cudaSuccess) e = upload_psf_dev(c);
    return e;
}

mvd_status run_fused(mvd_ctx *c, const void *data, mvd_dtype dt, float *est, int P, int init_mean,
                     cudaStream_t s) {
    const size_t plane_px = static_cast<size_t>(c->H) * c->W;
    // the tensor route's split ratio and estimate round each row up to 8 columns
    const bool ws_route = c->algo == MVD_ALGO_TENSOR;
    const size_t ratio_bytes =
        std::max(static_cast<size_t>(c->V) * P * plane_px * sizeof(float),
                 ws_route ? mvd::tcw_split_bytes(c->W, c->H, static_cast<long long>(c->V) * P) : size_t(0));
    cudaError_t e = c->ratio.ensure(ratio_bytes);
    if (e == cudaSuccess && ws_route) e = c->psi_split.ensure(mvd::tcw_split_bytes(c->W, c->H, P));
    if (e != cudaSuccess) return fail(MVD_ERR_NOMEM, "ratio workspace: %s", cudaGetErrorString(e));
    mvd::FusedArgs a = fused_args(c, data, dt, est, P);
    if (c->iters == 0 && init_mean) {
        for (int p = 0; p < P; ++p) {
            e = mvd::plain_fill(est + p * plane_px, a.means, p, plane_px, s);
            if (e != cudaSuccess) return cuda_fail(e, "fill");
        }
        return MVD_OK;
    }
    // simultaneous: one launch pair over all views; sequential: one per view
    const int step = c->order == MVD_ORDER_SEQUENTIAL ? 1 : c->V;
    // kernel A / kernel B of the selected route, with their profile names
    cudaError_t (*blur)(const mvd::FusedArgs &, cudaStream_t) = mvd::launch_fused_blur_ratio;
    cudaError_t (*corr)(const mvd::FusedArgs &, cudaStream_t) = mvd::launch_fused_correlate_update;
    const char *blur_name = "blur_ratio", *corr_name = "correlate_update";
    if (c->algo == MVD_ALGO_TENSOR) {
        blur = mvd::launch_tc_blur_ratio;
        corr = mvd::launch_tc_correlate_update;
        blur_name = "tc_blur_ratio";
        corr_name = "tc_correlate_update";
    } else if (c->algo == MVD_ALGO_TF32) {
        blur = mvd::launch_tf32_blur_ratio;
        corr = mvd::launch_tf32_correlate_update;
        blur_name = "tf32_blur_ratio";
        corr_name = "tf32_correlate_update";
    }
    bool first = init_mean != 0;
    // The tensor route runs a launch on its warp-specialised kernels when they
    // take it (tcw_eligible).  Between two such kernels the data travel split
    // (BF16 hi/lo, what their products use): the blur writes the ratio split
    // when the correlation that follows reads it, and the correlation writes a
    // split copy of the estimate when the next blur reads one.
    auto ws_eligible = [&](int lo, int which) {
        mvd::FusedArgs b = a;
        b.view_lo = lo;
        b.view_hi = lo + step;
        b.psi_in = est;
        return ws_route && mvd::tcw_eligible(b, which);
    };
    bool psi_split_valid = false;   // the split estimate holds the current estimate
    const int n_launch = c->iters * ((c->V + step - 1) / step);
    int li = 0;
    for (int t = 0; t < c->iters; ++t) {
        for (int v0 = 0; v0 < c->V; v0 += step, ++li) {
            a.view_lo = v0;
            a.view_hi = v0 + step;
            a.psi_in = first ? nullptr : est;
            first = false;
            const bool wa = ws_route && mvd::tcw_eligible(a, 0), wb = ws_route && mvd::tcw_eligible(a, 1);
            mvd::TcwIo io{};
            io.psi_split = c->psi_split.as<uint16_t>();
            c->prof.mark(s, wa ? "tcw_blur_ratio" : blur_name);
            if (wa) {
                io.in_mode = !a.psi_in ? mvd::kInConst : (psi_split_valid ? mvd::kInSplit : mvd::kInF32);
                io.ratio_split = wb;
                e = mvd::launch_tcw(a, 0, io, s);
            } else {
                e = blur(a, s);
            }
            if (e != cudaSuccess) return cuda_fail(e, "blur/ratio kernel");
            c->prof.mark(s, wb ? "tcw_correlate_update" : corr_name);
            if (wb) {
                // the next launch's blur reads the split estimate if it runs on the same kernels
                const int nv0 = v0 + step < c->V ? v0 + step : 0;
                io.in_mode = wa ? mvd::kInSplit : mvd::kInF32;
                io.ratio_split = 0;
                io.write_psi_split = li + 1 < n_launch && ws_eligible(nv0, 0);
                e = mvd::launch_tcw(a, 1, io, s);
                psi_split_valid = io.write_psi_split != 0;
            } else {
                e = corr(a, s);
                psi_split_valid = false;
            }
            if (e != cudaSuccess) return cuda_fail(e, "correlate/update kernel");
        }
    }
    c->prof.end(s);
    return MVD_OK;
}

// Padded grid of the Fourier route for this context; false if it has none.
bool fft_grid(const mvd_ctx *c, int *Ly, int *Lx) {
    const int R = (c->K - 1) / 2;
    int ly = c->H, lx = c->W;
    if (c->boundary == MVD_BOUNDARY_ZERO) {
        if (!mvd::fftr::smooth_size(c->H + R, &ly) || !mvd::fftr::smooth_size(c->W + R, &lx)) return false;
    }
    int r[mvd::fftr::kMaxRadices], n = 0;
    if (!mvd::fftr::radix_list(ly, r, &n) || !mvd::fftr::radix_list(lx, r, &n)) return false;
    if (ly > mvd::fftr::kMaxLen || lx > mvd::fftr::kMaxLen || ly < 2 || lx < 2) return false;
    *Ly = ly;
    *Lx = lx;
    return true;
}

// Transform plans, twiddle tables and PSF spectra (host FP64 transforms) for
// the Fourier route.
mvd_status fft_plan(mvd_ctx *c) {
    if (c->fft.planned) return MVD_OK;
    auto &f = c->fft;
    if (!fft_grid(c, &f.Ly, &f.Lx)) return fail(MVD_ERR_UNSUPPORTED, "no Fourier grid for this plane size");
    f.Lc = f.Lx / 2 + 1;
    f.LcP = (f.Lc + 7) / 8 * 8;
    std::vector<float2> tx, ty, spec, all, call;
    if (!mvd::fftr::make_plan(f.Lx, f.px, tx) || !mvd::fftr::make_plan(f.Ly, f.py, ty))
        return fail(MVD_ERR_UNSUPPORTED, "no transform plan for %d x %d", f.Ly, f.Lx);
    const size_t per = static_cast<size_t>(f.Lc) * f.Ly;
    all.resize(per * c->V);
    for (int v = 0; v < c->V; ++v) {
        mvd::fftr::psf_spectrum(c->psfs.data() + static_cast<size_t>(v) * c->K * c->K, c->K, f.Ly, f.Lx, f.Lc, spec);
        std::copy(spec.begin(), spec.end(), all.begin() + v * per);
    }
    // a variant correlates with its own kernels: spectra of their flips
    if (!c->corr_psfs.empty()) {
        call.resize(per * c->V);
        for (int v = 0; v < c->V; ++v) {
            mvd::fftr::psf_spectrum(c->corr_psfs.data() + static_cast<size_t>(v) * c->K * c->K, c->K, f.Ly, f.Lx,
                                    f.Lc, spec);
            std::copy(spec.begin(), spec.end(), call.begin() + v * per);
        }
    }
    // a plan of one stage has no twiddles: keep one entry so that the buffers exist
    if (tx.empty()) tx.push_back(make_float2(1.f, 0.f));
    if (ty.empty()) ty.push_back(make_float2(1.f, 0.f));
    cudaError_t e;
    if ((e = f.tw_x.ensure(tx.size() * sizeof(float2))) != cudaSuccess ||
        (e = f.tw_y.ensure(ty.size() * sizeof(float2))) != cudaSuccess ||
        (e = f.spec.ensure(all.size() * sizeof(float2))) != cudaSuccess ||
        (!call.empty() && (e = f.cspec.ensure(call.size() * sizeof(float2))) != cudaSuccess))
        return fail(MVD_ERR_NOMEM, "Fourier tables: %s", cudaGetErrorString(e));
    if (!call.empty() &&
        (e = cudaMemcpy(f.cspec.ptr, call.data(), call.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "upload Fourier tables");
    if ((e = cudaMemcpy(f.tw_x.ptr, tx.data(), tx.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(f.tw_y.ptr, ty.data(), ty.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(f.spec.ptr, all.data(), all.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "upload Fourier tables");
    f.planned = true;
    return MVD_OK;
}

mvd_status run_fft(mvd_ctx *c, const void *data, mvd_dtype dt, float *est, int P, int init_mean, cudaStream_t s) {
    mvd_status st = fft_plan(c);
    if (st != MVD_OK) return st;
    auto &f = c->fft;
    const size_t rows = static_cast<size_t>(P) * c->H * f.LcP;
    cudaError_t e;
    if ((e = f.S0.ensure(rows * sizeof(float2))) != cudaSuccess ||
        (e = f.T.ensure(rows * c->V * sizeof(float2))) != cudaSuccess)
        return fail(MVD_ERR_NOMEM, "Fourier workspace: %s", cudaGetErrorString(e));
    const size_t plane_px = static_cast<size_t>(c->H) * c->W;
    if (c->iters == 0 && init_mean) {
        for (int p = 0; p < P; ++p)
            if ((e = mvd::plain_fill(est + p * plane_px, c->means.as<float>(), p, plane_px, s)) != cudaSuccess)
                return cuda_fail(e, "fill");
        return MVD_OK;
    }
    mvd::fftr::FftArgs a{};
    a.Ly = f.Ly;
    a.Lx = f.Lx;
    a.Lc = f.Lc;
    a.LcP = f.LcP;
    a.px = f.px;
    a.py = f.py;
    a.tw_x = f.tw_x.as<float2>();
    a.tw_y = f.tw_y.as<float2>();
    a.spec = f.spec.as<float2>();
    a.cspec = c->corr_psfs.empty() ? a.spec : f.cspec.as<float2>();
    a.H = c->H;
    a.W = c->W;
    a.P = P;
    a.eps = c->eps;
    a.means = c->means.as<float>();
    a.psi_out = est;
    a.phi = data;
    a.u16 = dt == MVD_U16;
    a.S0 = f.S0.as<float2>();
    a.T = f.T.as<float2>();
    a.err = c->status.as<int>();
    a.wait_budget = c->wait_budget;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int step = c->order == MVD_ORDER_SEQUENTIAL ? 1 : c->V;
    bool first = init_mean != 0;
    for (int t = 0; t < c->iters; ++t) {
        for (int v0 = 0; v0 < c->V; v0 += step) {
            a.view_lo = v0;
            a.view_hi = v0 + step;
            a.psi_in = first ? nullptr : est;
            first = false;
            c->prof.mark(s, "fft_iteration");
            if ((e = mvd::fftr::launch_iteration(a, sms, s)) != cudaSuccess) return cuda_fail(e, "Fourier kernels");
        }
    }
    c->prof.end(s);
    return MVD_OK;
}

// The context's factors [terms][4][K] padded with zero taps to [terms][4][KC].
std::vector<float> padded_taps(const mvd_ctx *c, int KC) {
    const int pad = (KC - c->K) / 2;
    std::vector<float> out(static_cast<size_t>(c->ft.total_terms) * 4 * KC, 0.0f);
    for (int t = 0; t < c->ft.total_terms; ++t)
        for (int kind = 0; kind < 4; ++kind)
            for (int m = 0; m < c->K; ++m)
                out[(static_cast<size_t>(t) * 4 + kind) * KC + pad + m] =
                    c->taps_host[(static_cast<size_t>(t) * 4 + kind) * c->K + m];
    return out;
}

// Whether the plane-resident route can take this context: its cluster size,
// strip rows and shared memory.
bool resident_plan(const mvd_ctx *c, int *C, int *strip, size_t *smem) {
    const int cls = mvd::bq::size_class(c->K);
    if (cls < 0 || c->boundary != MVD_BOUNDARY_ZERO || c->weights || c->Ka != 0) return false;
    const int KC = mvd::bq::class_k(cls);
    return mvd::res::plan(c->H, c->W, cls, c->order == MVD_ORDER_SEQUENTIAL, c->ft.total_terms * 4 * KC, C, strip,
                          smem);
}

// The padded factors on the device, uploaded once per factorisation (from
// mvd_set_algo, so that a captured run does no synchronous copy).
mvd_status upload_resident_taps(mvd_ctx *c) {
    if (c->res_taps_ready) return MVD_OK;
    const std::vector<float> taps = padded_taps(c, mvd::bq::class_k(mvd::bq::size_class(c->K)));
    cudaError_t e = c->res_taps.ensure(taps.size() * sizeof(float));
    if (e != cudaSuccess) return fail(MVD_ERR_NOMEM, "resident taps: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpy(c->res_taps.ptr, taps.data(), taps.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(e, "upload resident taps");
    c->res_taps_ready = true;
    return MVD_OK;
}

mvd_status run_resident(mvd_ctx *c, const void *data, mvd_dtype dt, float *est, int P, int init_mean,
                        cudaStream_t s) {
    int C = 0, strip = 0;
    size_t smem = 0;
    if (!resident_plan(c, &C, &strip, &smem)) return fail(MVD_ERR_UNSUPPORTED, "plane does not fit on chip");
    const int cls = mvd::bq::size_class(c->K);
    const int KC = mvd::bq::class_k(cls);
    mvd_status st = upload_resident_taps(c);
    if (st != MVD_OK) return st;
    cudaError_t e;
    mvd::res::ResArgs a{};
    a.phi = data;
    a.u16 = dt == MVD_U16;
    a.psi_in = init_mean ? nullptr : est;
    a.means = c->means.as<float>();
    a.psi_out = est;
    a.taps = c->res_taps.as<float>();
    a.ntaps = c->ft.total_terms * 4 * KC;
    a.H = c->H;
    a.W = c->W;
    a.P = P;
    a.V = c->V;
    a.iters = c->iters;
    a.seq = c->order == MVD_ORDER_SEQUENTIAL;
    a.strip = strip;
    a.C = C;
    a.eps = c->eps;
    for (int v = 0; v < c->V; ++v) {
        a.rank[v] = c->ft.rank[v];
        a.tap_off[v] = c->ft.tap_off[v];
        a.crank[v] = c->ft.crank[v];
        a.ctap_off[v] = c->ft.ctap_off[v];
        a.short_mask[v] = c->ft.short_mask[v];
    }
    c->prof.mark(s, "resident");
    if ((e = mvd::res::launch(a, cls, smem, s)) != cudaSuccess) return cuda_fail(e, "plane-resident kernel");
    mvd::count_launch(1);
    c->prof.end(s);
    return MVD_OK;
}

// 3D route: in-plane blur (kernel A, blur only), the passes along the plane
// axis per view, then kernel B on the axially correlated ratios.
mvd_status run_fused3d(mvd_ctx *c, const void *data, mvd_dtype dt, float *est, int P, cudaStream_t s) {
    const size_t n = static_cast<size_t>(c->H) * c->W;
    cudaError_t e;
    if ((e = c->ratio.ensure(static_cast<size_t>(c->V) * P * n * sizeof(float))) != cudaSuccess ||
        (e = c->tmp3d.ensure(static_cast<size_t>(P) * n * sizeof(float))) != cudaSuccess)
        return fail(MVD_ERR_NOMEM, "3D workspace: %s", cudaGetErrorString(e));
    if ((e = c->axial_dev.ensure(c->axial.size() * sizeof(float))) != cudaSuccess)
        return fail(MVD_ERR_NOMEM, "axial profiles: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(c->axial_dev.ptr, c->axial.data(), c->axial.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "upload axial profiles");
    mvd::FusedArgs a = fused_args(c, data, dt, est, P);
    const int step = c->order == MVD_ORDER_SEQUENTIAL ? 1 : c->V;
    const int circ = c->boundary == MVD_BOUNDARY_CIRCULAR;
    const size_t es = dt == MVD_U16 ? 2 : 4;
    bool first = true;
    for (int t = 0; t < c->iters; ++t) {
        for (int v0 = 0; v0 < c->V; v0 += step) {
            a.view_lo = v0;
            a.view_hi = v0 + step;
            a.psi_in = first ? nullptr : est;
            first = false;
            a.store_blur = 1;
            c->prof.mark(s, "blur_ratio");
            if ((e = mvd::launch_fused_blur_ratio(a, s)) != cudaSuccess) return cuda_fail(e, "blur kernel");
            c->prof.mark(s, "axial");
            for (int v = v0; v < v0 + step; ++v) {
                float *rv = c->ratio.as<float>() + static_cast<size_t>(v) * P * n;
                const char *phi = static_cast<const char *>(data) + static_cast<size_t>(v) * P * n * es;
                const float *av = c->axial_dev.as<float>() + static_cast<size_t>(v) * c->Ka;
                if ((e = mvd::launch_axial_ratio(rv, phi, dt == MVD_U16, av, c->Ka, P, n, circ, c->eps,
                                                 c->tmp3d.as<float>(), s)) != cudaSuccess ||
                    (e = mvd::launch_axial_corr(c->tmp3d.as<float>(), av, c->Ka, P, n, circ, rv, s)) != cudaSuccess)
                    return cuda_fail(e, "axial kernels");
            }
            a.store_blur = 0;
            c->prof.mark(s, "correlate_update");
            if ((e = mvd::launch_fused_correlate_update(a, s)) != cudaSuccess) return cuda_fail(e, "correlate kernel");
        }
    }
    c->prof.end(s);
    return MVD_OK;
}

// Weighted MV-RL: 1 / (w_v (*) P_v^*) for every view and plane, before the iterations.
mvd_status prepare_weights(mvd_ctx *c, int P, cudaStream_t s) {
    const size_t n = static_cast<size_t>(c->H) * c->W * P;
    cudaError_t e;
    if ((e = c->wnorm.ensure(n * c->V * sizeof(float))) != cudaSuccess ||
        (e = c->wtmp.ensure(n * sizeof(float))) != cudaSuccess)
        return fail(MVD_ERR_NOMEM, "weight workspace: %s", cudaGetErrorString(e));
    mvd::PlainArgs a{};
    a.taps = c->taps.as<float>();
    a.ft = c->ft;
    a.H = c->H;
    a.W = c->W;
    a.circular = c->boundary == MVD_BOUNDARY_CIRCULAR;
    c->prof.mark(s, "weight_norms");
    if ((e = mvd::weight_norms(a, c->weights, P, c->wtmp.as<float>(), c->wnorm.as<float>(), s)) != cudaSuccess)
        return cuda_fail(e, "weight normaliser");
    c->prof.end(s);
    return MVD_OK;
}

mvd_status run_plain(mvd_ctx *c, const void *data, mvd_dtype dt, float *est, int P, int init_mean,
                     int direct, cudaStream_t s) {
    const size_t n = static_cast<size_t>(c->H) * c->W;
    cudaError_t e = c->plain.ensure(4 * n * sizeof(float));
    if (e != cudaSuccess) return fail(MVD_ERR_NOMEM, "plain workspace: %s", cudaGetErrorString(e));
    if (direct && (e = upload_psf_dev(c)) != cudaSuccess) return cuda_fail(e, "upload psfs");
    float *b = c->plain.as<float>(), *tmp = b + n, *cv = b + 2 * n, *prod = b + 3 * n;
    mvd::PlainArgs a{};
    a.taps = c->taps.as<float>();
    a.psf_dev = c->psf_dev.as<float>();
    a.psf_corr = c->corr_psfs.empty() ? a.psf_dev : a.psf_dev + c->psfs.size();
    a.ft = c->ft;
    a.H = c->H;
    a.W = c->W;
    a.circular = c->boundary == MVD_BOUNDARY_CIRCULAR;
    a.eps = c->eps;
    const int u16 = dt == MVD_U16;
    const size_t esz = u16 ? 2 : 4;
    const bool sequential = c->order == MVD_ORDER_SEQUENTIAL;
    for (int p = 0; p < P; ++p) {
        float *psi = est + p * n;
        if (init_mean) {
            e = mvd::plain_fill(psi, c->means.as<float>(), p, n, s);
            if (e != cudaSuccess) return cuda_fail(e, "fill");
        }
        for (int t = 0; t < c->iters; ++t) {
            c->prof.mark(s, direct ? "direct_iteration" : "plain_iteration");
            for (int v = 0; v < c->V; ++v) {
                const size_t vp = (static_cast<size_t>(v) * P + p) * n;
                const char *phi = static_cast<const char *>(data) + vp * esz;
                const size_t wp = c->weight_planes == 1 ? static_cast<size_t>(v) * n : vp;
                const float *w = c->weights ? c->weights + wp : nullptr;
                if ((e = mvd::plain_convolve(a, v, 0, direct, psi, tmp, b, s)) != cudaSuccess) return cuda_fail(e, "blur");
                if ((e = mvd::plain_ratio(phi, u16, w, b, b, n, c->eps, s)) != cudaSuccess) return cuda_fail(e, "ratio");
                if ((e = mvd::plain_convolve(a, v, 1, direct, b, tmp, cv, s)) != cudaSuccess) return cuda_fail(e, "correlate");
                if (w && (e = mvd::plain_apply_norm(cv, c->wnorm.as<float>() + wp, n, s)) != cudaSuccess)
                    return cuda_fail(e, "weight normaliser");
                if (sequential) {
                    if ((e = mvd::plain_update(psi, cv, n, s)) != cudaSuccess) return cuda_fail(e, "update");
                } else if ((e = mvd::plain_multiply(prod, cv, n, v == 0, s)) != cudaSuccess) {
                    return cuda_fail(e, "product");
                }
            }
            if (!sequential && (e = mvd::plain_update(psi, prod, n, s)) != cudaSuccess) return cuda_fail(e, "update");
        }
    }
    c->prof.end(s);
    return MVD_OK;
}

}  // namespace

extern "C" {

const char *mvd_status_string(mvd_status s) {
    switch (s) {
        case MVD_OK: return "ok";
        case MVD_ERR_ARG: return "invalid argument";
        case MVD_ERR_CUDA: return "CUDA error";
        case MVD_ERR_NOMEM: return "out of memory";
        case MVD_ERR_TIMEOUT: return "device-side wait timed out";
        case MVD_ERR_STATE: return "invalid state";
        case MVD_ERR_UNSUPPORTED: return "unsupported by the selected route";
    }
    return "unknown status";
}

const char *mvd_last_error(void) { return t_last_error.c_str(); }

mvd_status mvd_set_psfs(mvd_ctx *c, const float *psfs) {
    t_last_error.clear();
    if (!c || !psfs) return fail(MVD_ERR_ARG, "NULL argument");
    const size_t KK = static_cast<size_t>(c->K) * c->K;
    for (int v = 0; v < c->V; ++v) {
        double sum = 0;
        for (size_t i = 0; i < KK; ++i) {
            const float x = psfs[v * KK + i];
            if (!std::isfinite(x) || x < 0) return fail(MVD_ERR_ARG, "PSF %d has a negative or non-finite entry", v);
            sum += x;
        }
        if (!(sum > 0)) return fail(MVD_ERR_ARG, "PSF %d sums to zero", v);
    }
    DeviceGuard g(c->device);
    c->psfs.assign(psfs, psfs + c->V * KK);
    mvd_status st = upload_factors(c);   // also rebuilds a variant's kernels
    if (st != MVD_OK) return st;
    if (c->psf_dev.ptr) {
        cudaError_t e = upload_psf_dev(c);
        if (e != cudaSuccess) return cuda_fail(e, "upload psfs");
    }
    return MVD_OK;
}

mvd_status mvd_psf_grad(mvd_ctx *c, const void *data, mvd_dtype dt, int P, int ckpt, double *loss_host,
                        float *grad_dev, float *est_dev, void *stream) {
    t_last_error.clear();
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (!data) return fail(MVD_ERR_ARG, "NULL buffer");
    if (dt != MVD_U16 && dt != MVD_F32) return fail(MVD_ERR_ARG, "unknown dtype");
    const bool want_grad = grad_dev != nullptr;   // NULL: the loss alone (no reverse sweep)
    if (P < 1 || P > 65535 || ckpt < 1) return fail(MVD_ERR_ARG, "need 1 <= n_planes <= 65535 and checkpoint_every >= 1");
    if (c->order != MVD_ORDER_SIMULTANEOUS) return fail(MVD_ERR_UNSUPPORTED, "the gradient follows the simultaneous order");
    if (c->variant != MVD_VARIANT_INDEPENDENT || c->weights || c->Ka > 0)
        return fail(MVD_ERR_UNSUPPORTED, "the gradient follows plain MV-RL (variant INDEPENDENT, no weights)");
    if (c->K > mvd::adj::kMaxK) return fail(MVD_ERR_UNSUPPORTED, "the gradient takes K <= %d", mvd::adj::kMaxK);
    DeviceGuard g(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int V = c->V, K = c->K, H = c->H, W = c->W, T = c->iters;
    const long long plane = static_cast<long long>(H) * W, n = plane * P;
    const int u16 = dt == MVD_U16;
    const size_t es = u16 ? 2 : 4;
    const int circ = c->boundary == MVD_BOUNDARY_CIRCULAR;
    const float eps = c->eps;
    const int nck = T > 0 ? (T + ckpt - 1) / ckpt : 0;
    // float buffers, each n: checkpoints nck; psiA psiB; fb fr fc (V each);
    // segment: psi (ckpt), b r c (V*ckpt each); psibar, psibar_new; cb (V), rb, bb
    const long long nbuf = nck + 2 + 3LL * V + ckpt + 3LL * V * ckpt + 2 + V + 2;
    cudaError_t e;
    if ((e = c->grad_ws.ensure(static_cast<size_t>(nbuf * n) * sizeof(float))) != cudaSuccess ||
        (e = c->grad_acc.ensure((static_cast<size_t>(V) * K * K + 1) * sizeof(double))) != cudaSuccess ||
        (e = c->means.ensure(static_cast<size_t>(P) * sizeof(float))) != cudaSuccess)
        return fail(MVD_ERR_NOMEM, "gradient workspace: %s", cudaGetErrorString(e));
    if ((e = upload_psf_dev(c)) != cudaSuccess) return cuda_fail(e, "upload psfs");
    float *w = c->grad_ws.as<float>();
    auto take = [&](long long k) { float *p = w; w += k * n; return p; };
    float *ck = take(nck), *psiA = take(1), *psiB = take(1);
    float *fb = take(V), *fr = take(V), *fc = take(V);
    float *sp = take(ckpt), *sb = take(static_cast<long long>(V) * ckpt), *sr = take(static_cast<long long>(V) * ckpt),
          *sc = take(static_cast<long long>(V) * ckpt);
    float *pbar = take(1), *pbar2 = take(1), *cb = take(V), *rb = take(1), *bb = take(1);
    double *G = c->grad_acc.as<double>(), *loss = G + static_cast<size_t>(V) * K * K;
    const float *psf = c->psf_dev.as<float>();
    const char *phi = static_cast<const char *>(data);
    auto phi_v = [&](int v) { return static_cast<const void *>(phi + static_cast<size_t>(v) * n * es); };
    auto P_v = [&](int v) { return psf + static_cast<size_t>(v) * K * K; };
#define MVD_TRY(x)                                           \
    do {                                                     \
        if ((e = (x)) != cudaSuccess) return cuda_fail(e, #x); \
    } while (0)
    // one forward iteration; b, r, cc hold the V intermediates
    auto step = [&](const float *psi, float *next, float *b, float *r, float *cc) -> cudaError_t {
        cudaError_t e2;
        for (int v = 0; v < V; ++v) {
            if ((e2 = mvd::adj::stencil(psi, b + v * n, P_v(v), K, H, W, P, circ, 0, 0, s)) != cudaSuccess) return e2;
            if ((e2 = mvd::adj::ratio(phi_v(v), u16, b + v * n, r + v * n, n, eps, s)) != cudaSuccess) return e2;
            if ((e2 = mvd::adj::stencil(r + v * n, cc + v * n, P_v(v), K, H, W, P, circ, 1, 0, s)) != cudaSuccess) return e2;
        }
        return mvd::adj::update(psi, cc, next, V, n, s);
    };
    c->prof.mark(s, "psf_grad");
    MVD_TRY(cudaMemsetAsync(G, 0, (static_cast<size_t>(V) * K * K + 1) * sizeof(double), s));
    MVD_TRY(mvd::launch_plane_means(data, u16, V, P, H, W, c->means.as<float>(), s));
    MVD_TRY(mvd::adj::fill_means(psiA, c->means.as<float>(), plane, n, s));
    // forward sweep, keeping psi at every checkpoint
    float *cur = psiA, *nxt = psiB;
    for (int t = 0; t < T; ++t) {
        if (want_grad && t % ckpt == 0) MVD_TRY(cudaMemcpyAsync(ck + (t / ckpt) * n, cur, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        MVD_TRY(step(cur, nxt, fb, fr, fc));
        std::swap(cur, nxt);
    }
    if (est_dev) MVD_TRY(cudaMemcpyAsync(est_dev, cur, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    // terminal data fit
    MVD_TRY(cudaMemsetAsync(pbar, 0, n * sizeof(float), s));
    for (int v = 0; v < V; ++v) {
        MVD_TRY(mvd::adj::stencil(cur, rb, P_v(v), K, H, W, P, circ, 0, 0, s));                 // y_v
        MVD_TRY(mvd::adj::terminal(phi_v(v), u16, rb, bb, loss, n, eps, s));                  // ybar in bb
        if (!want_grad) continue;
        MVD_TRY(mvd::adj::stencil(bb, pbar, P_v(v), K, H, W, P, circ, 1, 1, s));              // psibar += P (*) ybar
        MVD_TRY(mvd::adj::lag_sum(bb, cur, G + static_cast<size_t>(v) * K * K, K, H, W, P, circ, -1, s));
    }
    // reverse sweep, segment by segment
    for (int sg = want_grad ? nck - 1 : -1; sg >= 0; --sg) {
        const int t0 = sg * ckpt, L = std::min(T, t0 + ckpt) - t0;
        MVD_TRY(cudaMemcpyAsync(sp, ck + sg * n, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        for (int u = 0; u < L; ++u) {
            float *next = (u + 1 < L) ? sp + (u + 1) * n : nxt;
            MVD_TRY(step(sp + u * n, next, sb + u * V * n, sr + u * V * n, sc + u * V * n));
        }
        for (int u = L - 1; u >= 0; --u) {
            const float *psi_t = sp + u * n, *b = sb + u * V * n, *r = sr + u * V * n, *cc = sc + u * V * n;
            MVD_TRY(mvd::adj::cbar(pbar, psi_t, cc, pbar2, cb, V, n, s));
            for (int v = 0; v < V; ++v) {
                double *Gv = G + static_cast<size_t>(v) * K * K;
                MVD_TRY(mvd::adj::stencil(cb + v * n, rb, P_v(v), K, H, W, P, circ, 0, 0, s));     // rbar = P * cbar
                MVD_TRY(mvd::adj::lag_sum(cb + v * n, r + v * n, Gv, K, H, W, P, circ, 1, s));
                MVD_TRY(mvd::adj::bbar(phi_v(v), u16, rb, b + v * n, bb, n, eps, s));
                MVD_TRY(mvd::adj::stencil(bb, pbar2, P_v(v), K, H, W, P, circ, 1, 1, s));           // psibar += P (*) bbar
                MVD_TRY(mvd::adj::lag_sum(bb, psi_t, Gv, K, H, W, P, circ, -1, s));
            }
            std::swap(pbar, pbar2);
        }
    }
    if (want_grad) MVD_TRY(mvd::adj::to_float(G, grad_dev, V * K * K, s));
    c->prof.end(s);
    double L_host = 0;
    MVD_TRY(cudaMemcpyAsync(&L_host, loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MVD_TRY(cudaStreamSynchronize(s));
#undef MVD_TRY
    if (loss_host) *loss_host = L_host;
    return MVD_OK;
}

mvd_status mvd_device_status(mvd_ctx *c, void *stream) {
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stream");
    int word = 0;
    if ((e = cudaMemcpy(&word, c->status.ptr, sizeof word, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "status read");
    if (word != 0) {
        if ((e = cudaMemset(c->status.ptr, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "status clear");
        if (word & mvd::kDevTimeout) return fail(MVD_ERR_TIMEOUT, "a kernel's wait for a tile copy ran out");
        return fail(MVD_ERR_CUDA, "device status word %d", word);
    }
    return MVD_OK;
}

mvd_status mvd_set_wait_budget(mvd_ctx *c, long long cycles) {
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    c->wait_budget = cycles == 0 ? mvd::kDefaultWaitBudget : cycles;
    return MVD_OK;
}

mvd_status mvd_profile_enable(mvd_ctx *c, int on) {
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    DeviceGuard g(c->device);
    c->prof.reset();
    c->prof.on = on != 0;
    return MVD_OK;
}

mvd_status mvd_profile_read(mvd_ctx *c, mvd_kernel_stat *out, int capacity, int *count) {
    if (!c || !count || (capacity > 0 && !out)) return fail(MVD_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    c->prof.resolve();
    const int n = static_cast<int>(c->prof.names.size());
    for (int i = 0; i < n && i < capacity; ++i) {
        std::memset(&out[i], 0, sizeof out[i]);
        std::snprintf(out[i].name, sizeof out[i].name, "%s", c->prof.names[i].c_str());
        out[i].total_ms = c->prof.ms[i];
        out[i].launches = c->prof.count[i];
    }
    *count = n;
    return MVD_OK;
}

mvd_status mvd_psf_factors(const float *psfs, int views, int K, double tol, int *rank_out, float *taps_out,
                           int cap) {
    t_last_error.clear();
    if (!psfs || !rank_out || !taps_out) return fail(MVD_ERR_ARG, "NULL argument");
    if (views < 1 || views > mvd::kMaxViews || K < 1 || K % 2 == 0) return fail(MVD_ERR_ARG, "bad sizes");
    if (!(tol >= 0.0)) return fail(MVD_ERR_ARG, "tolerance must be >= 0");
    mvd::FactorTable ft;
    char msg[256] = {0};
    if (!mvd::factorise_psfs(psfs, views, K, tol, ft, taps_out, cap, msg, sizeof msg))
        return fail(MVD_ERR_ARG, "%s", msg);
    for (int v = 0; v < views; ++v) rank_out[v] = ft.rank[v];
    return MVD_OK;
}

uint64_t mvd_launch_count(void) { return mvd::g_launches.load(std::memory_order_relaxed); }

mvd_status mvd_debug_fail_allocations(int n) {
    t_last_error.clear();
    if (n < 0) return fail(MVD_ERR_ARG, "n must be >= 0");
    g_fail_allocs.store(n);
    return MVD_OK;
}

mvd_status mvd_create(mvd_ctx **out, int views, const float *psfs_host, int psf_size, int plane_h, int plane_w,
                      int iters, mvd_boundary boundary, float eps) {
    t_last_error.clear();
    if (!out) return fail(MVD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (views < 1 || views > mvd::kMaxViews) return fail(MVD_ERR_ARG, "views must be in [1, %d]", mvd::kMaxViews);
    if (!psfs_host) return fail(MVD_ERR_ARG, "psfs is NULL");
    if (psf_size < 1 || psf_size % 2 == 0) return fail(MVD_ERR_ARG, "PSF size must be odd and >= 1 (got %d)", psf_size);
    if (plane_h < 1 || plane_w < 1) return fail(MVD_ERR_ARG, "plane size must be positive");
    if (iters < 0) return fail(MVD_ERR_ARG, "iters must be >= 0");
    if (!(eps > 0.0f) || !std::isfinite(eps)) return fail(MVD_ERR_ARG, "eps must be positive and finite");
    if (boundary != MVD_BOUNDARY_ZERO && boundary != MVD_BOUNDARY_CIRCULAR) return fail(MVD_ERR_ARG, "unknown boundary");
    if (boundary == MVD_BOUNDARY_CIRCULAR && (psf_size > plane_h || psf_size > plane_w))
        return fail(MVD_ERR_ARG, "circular boundary needs K <= min(H, W)");
    const size_t KK = static_cast<size_t>(psf_size) * psf_size;
    for (int v = 0; v < views; ++v) {
        double sum = 0;
        for (size_t i = 0; i < KK; ++i) {
            const float x = psfs_host[v * KK + i];
            if (!std::isfinite(x)) return fail(MVD_ERR_ARG, "PSF %d has a non-finite entry", v);
            if (x < 0) return fail(MVD_ERR_ARG, "PSF %d has a negative entry", v);
            sum += x;
        }
        if (!(sum > 0)) return fail(MVD_ERR_ARG, "PSF %d sums to zero", v);
    }
    auto *c = new (std::nothrow) mvd_ctx();
    if (!c) return fail(MVD_ERR_NOMEM, "context");
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaGetDevice");
    }
    c->V = views;
    c->K = psf_size;
    c->H = plane_h;
    c->W = plane_w;
    c->iters = iters;
    c->boundary = boundary;
    c->eps = eps;
    c->algo = mvd::fused_supported(psf_size) ? MVD_ALGO_FUSED : MVD_ALGO_PLAIN;
    c->psfs.assign(psfs_host, psfs_host + views * KK);
    if ((e = c->status.ensure(sizeof(int))) != cudaSuccess || (e = cudaMemset(c->status.ptr, 0, sizeof(int))) != cudaSuccess) {
        mvd_destroy(c);
        return fail(MVD_ERR_NOMEM, "status word: %s", cudaGetErrorString(e));
    }
    mvd_status s = upload_factors(c);
    if (s != MVD_OK) {
        mvd_destroy(c);
        return s;
    }
    // default route: the fused separable kernels when the PSFs' terms fit
    // them, else the Fourier route when the plane has a grid, else plain
    int ly, lx;
    if (!(c->algo == MVD_ALGO_FUSED && mvd::fused_taps_fit(c->ft)))
        c->algo = fft_grid(c, &ly, &lx) ? MVD_ALGO_FFT : MVD_ALGO_PLAIN;
    *out = c;
    return MVD_OK;
}

mvd_status mvd_autotune(mvd_ctx *c, const void *data, mvd_dtype dt, int n_planes, void *stream) {
    t_last_error.clear();
    if (!c || !data) return fail(MVD_ERR_ARG, "NULL argument");
    if (dt != MVD_U16 && dt != MVD_F32) return fail(MVD_ERR_ARG, "unknown dtype");
    if (n_planes < 1) return fail(MVD_ERR_ARG, "n_planes must be >= 1");
    DeviceGuard g(c->device);
    char key[256];
    std::snprintf(key, sizeof key, "route_v%d_k%d_%dx%d_t%d_b%d_o%d_r%d_x%d_w%d", c->V, c->K, c->H, c->W, c->iters,
                  static_cast<int>(c->boundary), static_cast<int>(c->order), c->ft.total_terms,
                  static_cast<int>(c->variant), c->weights ? 1 : 0);
    int cached = -1, unused = 0;
    if (tune_cache_lookup(key, &cached, &unused, &unused) && cached >= 0) {
        c->algo = static_cast<mvd_algo>(cached);
        return MVD_OK;
    }
    int ly, lx;
    std::vector<mvd_algo> cand;
    if (mvd::fused_supported(c->K) && mvd::fused_taps_fit(c->ft)) cand.push_back(MVD_ALGO_FUSED);
    if (fft_grid(c, &ly, &lx) && !c->weights && c->Ka == 0) cand.push_back(MVD_ALGO_FFT);
    if (cand.empty()) cand.push_back(MVD_ALGO_PLAIN);
    if (cand.size() == 1) {
        c->algo = cand[0];
        return MVD_OK;
    }
    const int P = std::min(n_planes, 8);
    const size_t plane_px = static_cast<size_t>(c->H) * c->W;
    DevBuf est;
    cudaError_t e = est.ensure(static_cast<size_t>(P) * plane_px * sizeof(float));
    if (e != cudaSuccess) return fail(MVD_ERR_NOMEM, "autotune buffer: %s", cudaGetErrorString(e));
    // the first P planes of every view: planes are contiguous per view, so a
    // sub-batch needs its own copy of the data
    const size_t es = dt == MVD_U16 ? 2 : 4;
    DevBuf sub;
    if ((e = sub.ensure(static_cast<size_t>(c->V) * P * plane_px * es)) != cudaSuccess) {
        est.release();
        return fail(MVD_ERR_NOMEM, "autotune buffer: %s", cudaGetErrorString(e));
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int v = 0; v < c->V; ++v)
        cudaMemcpyAsync(sub.as<char>() + static_cast<size_t>(v) * P * plane_px * es,
                        static_cast<const char *>(data) + static_cast<size_t>(v) * n_planes * plane_px * es,
                        P * plane_px * es, cudaMemcpyDeviceToDevice, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const mvd_algo keep = c->algo;
    float best = 1e30f;
    mvd_algo best_a = keep;
    mvd_status st = MVD_OK;
    for (mvd_algo a : cand) {
        c->algo = a;
        if ((st = mvd_deconvolve_planes(c, sub.ptr, dt, est.as<float>(), P, 1, s)) != MVD_OK) break;   // warm
        cudaEventRecord(e0, s);
        if ((st = mvd_deconvolve_planes(c, sub.ptr, dt, est.as<float>(), P, 1, s)) != MVD_OK) break;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_a = a;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    est.release();
    sub.release();
    if (st != MVD_OK) {
        c->algo = keep;
        return st;
    }
    c->algo = best_a;
    tune_cache_store(key, static_cast<int>(best_a), 0, 0);
    return MVD_OK;
}

mvd_status mvd_destroy(mvd_ctx *c) {
    if (!c) return MVD_OK;
    DeviceGuard g(c->device);
    c->taps.release();
    c->psf_dev.release();
    c->means.release();
    c->ratio.release();
    c->psi_split.release();
    c->plain.release();
    for (auto &b : c->run_stack) b.release();
    for (auto &b : c->run_est) b.release();
    c->run_planes.release();
    c->prof.destroy();
    c->status.release();
    c->grad_ws.release();
    c->grad_acc.release();
    c->fft.tw_x.release();
    c->fft.tw_y.release();
    c->fft.spec.release();
    c->fft.S0.release();
    c->fft.T.release();
    c->res_taps.release();
    if (c->copy_in) cudaStreamDestroy(c->copy_in);
    if (c->copy_out) cudaStreamDestroy(c->copy_out);
    delete c;
    return MVD_OK;
}

mvd_status mvd_set_algo(mvd_ctx *c, mvd_algo algo) {
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (algo != MVD_ALGO_FUSED && algo != MVD_ALGO_PLAIN && algo != MVD_ALGO_DIRECT && algo != MVD_ALGO_FFT &&
        !tensor_algo(algo) && algo != MVD_ALGO_RESIDENT)
        return fail(MVD_ERR_ARG, "unknown algo %d", static_cast<int>(algo));
    if (algo == MVD_ALGO_RESIDENT) {
        int C, strip;
        size_t smem;
        if (!resident_plan(c, &C, &strip, &smem))
            return fail(MVD_ERR_UNSUPPORTED,
                        "plane-resident route: ZERO boundary, K <= 47, no weights, planes that fit on chip");
        mvd_status st = upload_resident_taps(c);
        if (st != MVD_OK) return st;
    }
    if (tensor_algo(algo) && !mvd::tc_supported(c->K))
        return fail(MVD_ERR_UNSUPPORTED, "tensor-core route takes odd K <= 47 (got %d)", c->K);
    if (algo == MVD_ALGO_FUSED && !(mvd::fused_supported(c->K) && mvd::fused_taps_fit(c->ft)))
        return fail(MVD_ERR_UNSUPPORTED, "fused path takes K <= %d (got %d)", mvd::kFusedMaxK, c->K);
    if (algo == MVD_ALGO_FFT) {
        int ly, lx;
        if (!fft_grid(c, &ly, &lx))
            return fail(MVD_ERR_UNSUPPORTED, "no Fourier grid: padded sides must be 2^a 3^b 5^c and <= %d",
                        mvd::fftr::kMaxLen);
    }
    c->algo = algo;
    return MVD_OK;
}

mvd_status mvd_set_update_order(mvd_ctx *c, mvd_update_order order) {
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (order != MVD_ORDER_SIMULTANEOUS && order != MVD_ORDER_SEQUENTIAL)
        return fail(MVD_ERR_ARG, "unknown update order %d", static_cast<int>(order));
    c->order = order;
    return MVD_OK;
}

mvd_status mvd_set_variant(mvd_ctx *c, mvd_variant variant) {
    t_last_error.clear();
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (variant < MVD_VARIANT_INDEPENDENT || variant > MVD_VARIANT_OPTIMIZATION_2)
        return fail(MVD_ERR_ARG, "unknown variant %d", static_cast<int>(variant));
    if (variant == c->variant) return MVD_OK;
    DeviceGuard g(c->device);
    c->variant = variant;
    mvd_status st = upload_factors(c);
    if (st != MVD_OK) return st;
    if (c->psf_dev.ptr) {
        cudaError_t e = upload_psf_dev(c);
        if (e != cudaSuccess) return cuda_fail(e, "upload psfs");
    }
    return MVD_OK;
}

mvd_status mvd_set_axial_psfs(mvd_ctx *c, const float *axial_host, int axial_size) {
    t_last_error.clear();
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (!axial_host || axial_size == 0) {
        c->axial.clear();
        c->Ka = 0;
        return MVD_OK;
    }
    if (axial_size < 1 || axial_size > 127 || axial_size % 2 == 0)
        return fail(MVD_ERR_ARG, "axial profile length must be odd, 1..127");
    for (int v = 0; v < c->V; ++v) {
        double sum = 0;
        for (int i = 0; i < axial_size; ++i) {
            const float x = axial_host[v * axial_size + i];
            if (!std::isfinite(x) || x < 0) return fail(MVD_ERR_ARG, "axial profile %d has a negative or non-finite entry", v);
            sum += x;
        }
        if (!(sum > 0)) return fail(MVD_ERR_ARG, "axial profile %d sums to zero", v);
    }
    c->axial.assign(axial_host, axial_host + static_cast<size_t>(c->V) * axial_size);
    c->Ka = axial_size;
    return MVD_OK;
}

mvd_status mvd_set_weights(mvd_ctx *c, const float *weights_dev, int n_planes) {
    t_last_error.clear();
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (!weights_dev) {
        c->weights = nullptr;
        c->weight_planes = 0;
        return MVD_OK;
    }
    if (n_planes < 1 || n_planes > 65535) return fail(MVD_ERR_ARG, "need 1 <= n_planes <= 65535");
    c->weights = weights_dev;
    c->weight_planes = n_planes;
    return MVD_OK;
}

mvd_status mvd_embed_padded(const void *src, mvd_dtype dt, int views, int n_planes, int plane_h, int plane_w,
                            int pad, void *dst, float *weights, int weight_planes, void *stream) {
    t_last_error.clear();
    if (!src || !dst) return fail(MVD_ERR_ARG, "NULL buffer");
    if (dt != MVD_U16 && dt != MVD_F32) return fail(MVD_ERR_ARG, "unknown dtype");
    if (views < 1 || n_planes < 1 || plane_h < 1 || plane_w < 1 || pad < 0)
        return fail(MVD_ERR_ARG, "need views, planes, plane sides >= 1 and pad >= 0");
    if (weights && weight_planes != 1 && weight_planes != n_planes)
        return fail(MVD_ERR_ARG, "weight_planes must be 1 or n_planes");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = mvd::launch_embed_padded(src, dt == MVD_U16 ? 2 : 4, static_cast<long long>(views) * n_planes,
                                             plane_h, plane_w, pad, dst, weight_planes == n_planes ? weights : nullptr,
                                             s);
    if (e == cudaSuccess && weights && weight_planes != n_planes) {
        // one weight plane per view: embed the first plane of each view once more, keeping its mask
        const size_t pin = static_cast<size_t>(plane_h) * plane_w * (dt == MVD_U16 ? 2 : 4);
        const size_t pout = static_cast<size_t>(plane_h + 2 * pad) * (plane_w + 2 * pad);
        for (int v = 0; v < views && e == cudaSuccess; ++v) {
            const char *sv = static_cast<const char *>(src) + static_cast<size_t>(v) * n_planes * pin;
            char *dv = static_cast<char *>(dst) + static_cast<size_t>(v) * n_planes * pout * (dt == MVD_U16 ? 2 : 4);
            e = mvd::launch_embed_padded(sv, dt == MVD_U16 ? 2 : 4, 1, plane_h, plane_w, pad, dv, weights + v * pout, s);
        }
    }
    return e == cudaSuccess ? MVD_OK : cuda_fail(e, "embed kernel");
}

mvd_status mvd_crop_planes(const float *src, int n_planes, int padded_h, int padded_w, int pad, float *dst,
                           void *stream) {
    t_last_error.clear();
    if (!src || !dst) return fail(MVD_ERR_ARG, "NULL buffer");
    if (n_planes < 1 || pad < 0 || padded_h <= 2 * pad || padded_w <= 2 * pad)
        return fail(MVD_ERR_ARG, "need planes >= 1 and padded sides > 2 pad");
    const cudaError_t e = mvd::launch_crop_planes(src, n_planes, padded_h, padded_w, pad, dst,
                                                  static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MVD_OK : cuda_fail(e, "crop kernel");
}

mvd_status mvd_variant_kernels(const float *psfs, int views, int K, mvd_variant variant, float *x_out) {
    t_last_error.clear();
    if (!psfs || !x_out) return fail(MVD_ERR_ARG, "NULL argument");
    if (views < 1 || views > mvd::kMaxViews || K < 1 || K % 2 == 0) return fail(MVD_ERR_ARG, "bad sizes");
    if (variant < MVD_VARIANT_INDEPENDENT || variant > MVD_VARIANT_OPTIMIZATION_2)
        return fail(MVD_ERR_ARG, "unknown variant %d", static_cast<int>(variant));
    const size_t KK = static_cast<size_t>(K) * K;
    for (size_t i = 0; i < KK * views; ++i)
        if (!std::isfinite(psfs[i]) || psfs[i] < 0) return fail(MVD_ERR_ARG, "PSF entry %zu negative or not finite", i);
    std::vector<double> X(KK * views);
    mvd::variant_kernels(psfs, views, K, variant, X.data());
    for (int v = 0; v < views; ++v) {
        double sum = 0;
        for (size_t i = 0; i < KK; ++i) sum += X[KK * v + i];
        if (!(sum > 0)) return fail(MVD_ERR_ARG, "kernel of view %d sums to zero", v);
        // INDEPENDENT is returned at unit sum as well
        for (size_t i = 0; i < KK; ++i) x_out[KK * v + i] = static_cast<float>(X[KK * v + i] / sum);
    }
    return MVD_OK;
}

mvd_status mvd_set_rank_tolerance(mvd_ctx *c, double tol) {
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(MVD_ERR_ARG, "tolerance must be >= 0");
    DeviceGuard g(c->device);
    c->rank_tol = tol;
    return upload_factors(c);
}

mvd_status mvd_get_info(const mvd_ctx *c, mvd_info *info) {
    if (!c || !info) return fail(MVD_ERR_ARG, "NULL argument");
    std::memset(info, 0, sizeof *info);
    info->views = c->V;
    info->psf_size = c->K;
    info->plane_h = c->H;
    info->plane_w = c->W;
    info->iters = c->iters;
    info->boundary = c->boundary;
    info->algo = c->algo;
    info->order = c->order;
    for (int v = 0; v < c->V && v < 16; ++v) info->rank[v] = c->ft.rank[v];
    for (int v = 0; v < c->V && v < 16; ++v) info->corr_rank[v] = c->ft.crank[v];
    auto taps = [&](int v, unsigned bit) {
        return (!c->weights && (c->ft.short_mask[v] & bit)) ? mvd::short_tap_count(c->K) : c->K;
    };
    for (int g = 0; g < c->ft.n_groups; ++g) {
        const int lead = c->ft.group_leader[g];
        info->flops_blur += 2 * c->ft.rank[lead] * (taps(lead, 1u) + taps(lead, 2u));
    }
    for (int v = 0; v < c->V; ++v) info->flops_corr += 2 * c->ft.crank[v] * (taps(v, 4u) + taps(v, 8u));
    info->variant = c->variant;
    info->blur_groups = c->ft.n_groups;
    info->blur_terms = c->ft.total_terms;
    if (c->algo == MVD_ALGO_TENSOR)
        mvd::tc_tile_shape(c->K, &info->tile_h, &info->tile_w);
    else if (c->algo == MVD_ALGO_TF32)
        mvd::tf32_tile_shape(c->K, &info->tile_h, &info->tile_w);
    else
        mvd::fused_tile_shape(c->K, &info->tile_h, &info->tile_w);
    info->workspace_bytes = c->taps.bytes + c->psf_dev.bytes + c->means.bytes + c->ratio.bytes + c->plain.bytes +
                            c->run_stack[0].bytes + c->run_stack[1].bytes + c->run_planes.bytes +
                            c->run_est[0].bytes + c->run_est[1].bytes;
    return MVD_OK;
}

mvd_status mvd_reslice(mvd_ctx *c, const void *stacks, mvd_dtype dt, int views, int nz, int ny, int nx,
                       void *planes, void *stream) {
    t_last_error.clear();
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (!stacks || !planes) return fail(MVD_ERR_ARG, "NULL buffer");
    if (dt != MVD_U16 && dt != MVD_F32) return fail(MVD_ERR_ARG, "unknown dtype");
    if (views < 1 || nz < 0 || ny < 0 || nx < 0) return fail(MVD_ERR_ARG, "bad sizes");
    if (static_cast<long long>(nz) * ny * nx == 0) return MVD_OK;
    const size_t es = dt == MVD_U16 ? 2 : 4;
    const char *a = static_cast<const char *>(stacks), *b = static_cast<const char *>(planes);
    const size_t bytes = static_cast<size_t>(views) * nz * ny * nx * es;
    if (a < b + bytes && b < a + bytes) return fail(MVD_ERR_ARG, "stacks and planes overlap");
    DeviceGuard g(c->device);
    c->prof.mark(static_cast<cudaStream_t>(stream), "reslice");
    cudaError_t e = mvd::launch_reslice(stacks, planes, static_cast<int>(es), views, nz, ny, nx,
                                        static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "reslice kernel");
    c->prof.end(static_cast<cudaStream_t>(stream));
    return MVD_OK;
}

mvd_status mvd_deconvolve_planes(mvd_ctx *c, const void *data, mvd_dtype dt, float *est, int n_planes, int init_mean,
                                 void *stream) {
    t_last_error.clear();
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (dt != MVD_U16 && dt != MVD_F32) return fail(MVD_ERR_ARG, "unknown dtype");
    if (n_planes < 0) return fail(MVD_ERR_ARG, "n_planes must be >= 0");
    if (n_planes == 0) return MVD_OK;
    if (!data || !est) return fail(MVD_ERR_ARG, "NULL buffer");
    if (n_planes > 65535) return fail(MVD_ERR_ARG, "at most 65535 planes per call");
    const size_t n = static_cast<size_t>(c->H) * c->W;
    const size_t es = dt == MVD_U16 ? 2 : 4;
    const char *d0 = static_cast<const char *>(data), *e0 = reinterpret_cast<const char *>(est);
    const size_t dbytes = static_cast<size_t>(c->V) * n_planes * n * es, ebytes = n_planes * n * sizeof(float);
    if (d0 < e0 + ebytes && e0 < d0 + dbytes) return fail(MVD_ERR_ARG, "data and estimate overlap");
    DeviceGuard g(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (init_mean) {
        if ((e = c->means.ensure(static_cast<size_t>(n_planes) * sizeof(float))) != cudaSuccess)
            return fail(MVD_ERR_NOMEM, "means: %s", cudaGetErrorString(e));
        c->prof.mark(s, "plane_means");
        if ((e = mvd::launch_plane_means(data, dt == MVD_U16, c->V, n_planes, c->H, c->W, c->means.as<float>(), s)) !=
            cudaSuccess)
            return cuda_fail(e, "plane means kernel");
        c->prof.end(s);
    }
    if (c->Ka > 0) {
        if (c->weights || !(c->algo == MVD_ALGO_FUSED && mvd::fused_taps_fit(c->ft)))
            return fail(MVD_ERR_UNSUPPORTED, "the 3D route runs on the fused kernels, without weights");
        if (c->iters == 0) {
            for (int p = 0; p < n_planes; ++p)
                if ((e = mvd::plain_fill(est + p * n, c->means.as<float>(), p, n, s)) != cudaSuccess)
                    return cuda_fail(e, "fill");
            return MVD_OK;
        }
        if (!init_mean) return fail(MVD_ERR_UNSUPPORTED, "the 3D route starts from the plane means");
        return run_fused3d(c, data, dt, est, n_planes, s);
    }
    if (c->weights) {
        if (c->weight_planes != 1 && n_planes != c->weight_planes)
            return fail(MVD_ERR_ARG, "weights were set for %d planes, the data have %d", c->weight_planes, n_planes);
        if (c->algo == MVD_ALGO_FFT || tensor_algo(c->algo))
            return fail(MVD_ERR_UNSUPPORTED, "weights run on the fused, plain and direct routes");
        mvd_status st = prepare_weights(c, c->weight_planes, s);
        if (st != MVD_OK) return st;
    }
    // the fused kernels carry the taps in their parameter block: PSFs that need
    // more separable terms than it holds run on the plain path
    if ((c->algo == MVD_ALGO_FUSED && mvd::fused_taps_fit(c->ft)) || tensor_algo(c->algo))
        return run_fused(c, data, dt, est, n_planes, init_mean, s);
    if (c->algo == MVD_ALGO_FFT) return run_fft(c, data, dt, est, n_planes, init_mean, s);
    if (c->algo == MVD_ALGO_RESIDENT) return run_resident(c, data, dt, est, n_planes, init_mean, s);
    return run_plain(c, data, dt, est, n_planes, init_mean, c->algo == MVD_ALGO_DIRECT, s);
}

int mvd_host_chunks(int ny, long long plane_bytes, int chunk_planes, int *y0, int *n, int cap) {
    if (ny < 1 || plane_bytes < 1 || chunk_planes < 0 || !y0 || !n) return -1;
    std::vector<int> sizes;
    if (chunk_planes > 0) {
        for (int y = 0; y < ny; y += chunk_planes) sizes.push_back(std::min(chunk_planes, ny - y));
    } else {
        // about 1 GiB of input per chunk (at most a quarter of the volume):
        // every chunk's launches run long enough that their start-up and last
        // partial wave stay small
        const long long base = std::max(1LL, std::min<long long>(ny / 4, (1LL << 30) / plane_bytes));
        std::vector<int> ramp;   // base/8, base/4, base/2: the iterations start after a short copy
        for (long long d : {8LL, 4LL, 2LL})
            if (base / d >= 1) ramp.push_back(static_cast<int>(base / d));
        long long ramp_sum = 0;
        for (int r : ramp) ramp_sum += r;
        const int last = static_cast<int>(std::max(1LL, base / 4));   // short copy back at the end
        if (base >= 8 && ny >= ramp_sum + last + base && static_cast<long long>(ny) * plane_bytes >= (256LL << 20)) {
            const long long mid = ny - ramp_sum - last;
            const int parts = static_cast<int>((mid + base - 1) / base);
            sizes = ramp;
            for (int i = 0; i < parts; ++i) sizes.push_back(static_cast<int>(mid / parts + (i < mid % parts ? 1 : 0)));
            sizes.push_back(last);
        } else {
            const int cp = std::max(1, (ny + 3) / 4);
            for (int y = 0; y < ny; y += cp) sizes.push_back(std::min(cp, ny - y));
        }
    }
    if (static_cast<int>(sizes.size()) > cap) return -1;
    int y = 0;
    for (size_t i = 0; i < sizes.size(); ++i) {
        y0[i] = y;
        n[i] = sizes[i];
        y += sizes[i];
    }
    return static_cast<int>(sizes.size());
}

mvd_status mvd_run_host(mvd_ctx *c, const void *stacks_host, mvd_dtype dt, int nz, int ny, int nx, float *out_host,
                        int chunk_planes, void *stream) {
    t_last_error.clear();
    if (!c) return fail(MVD_ERR_ARG, "ctx is NULL");
    if (!stacks_host || !out_host) return fail(MVD_ERR_ARG, "NULL buffer");
    if (dt != MVD_U16 && dt != MVD_F32) return fail(MVD_ERR_ARG, "unknown dtype");
    if (nz != c->H || nx != c->W) return fail(MVD_ERR_ARG, "stack (nz, nx) must equal the context's plane (H, W)");
    if (c->weights || c->Ka > 0) return fail(MVD_ERR_UNSUPPORTED, "host pipeline without weights or axial profiles");
    if (ny < 1) return fail(MVD_ERR_ARG, "ny must be >= 1");
    if (chunk_planes < 0) return fail(MVD_ERR_ARG, "chunk_planes must be >= 0");
    DeviceGuard g(c->device);
    const size_t es = dt == MVD_U16 ? 2 : 4;
    const size_t plane_px = static_cast<size_t>(nz) * nx;
    const long long per_plane = static_cast<long long>(c->V) * plane_px * es;
    const int max_chunks = chunk_planes > 0 ? (ny + chunk_planes - 1) / chunk_planes : ny;
    std::vector<int> cy0(max_chunks), cyn(max_chunks);
    const int nchunks = mvd_host_chunks(ny, per_plane, chunk_planes, cy0.data(), cyn.data(), max_chunks);
    if (nchunks < 1) return fail(MVD_ERR_ARG, "no chunk schedule for %d planes", ny);
    const int cp = *std::max_element(cyn.begin(), cyn.begin() + nchunks);
    cudaError_t e;
    for (int i = 0; i < 2; ++i) {
        if ((e = c->run_stack[i].ensure(c->V * plane_px * cp * es)) != cudaSuccess ||
            (e = c->run_est[i].ensure(plane_px * cp * sizeof(float))) != cudaSuccess)
            return fail(MVD_ERR_NOMEM, "pipeline buffers: %s", cudaGetErrorString(e));
    }
    if ((e = c->run_planes.ensure(c->V * plane_px * cp * es)) != cudaSuccess)
        return fail(MVD_ERR_NOMEM, "pipeline buffers: %s", cudaGetErrorString(e));
    if (!c->copy_in && (e = cudaStreamCreateWithFlags(&c->copy_in, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "stream");
    if (!c->copy_out && (e = cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "stream");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<cudaEvent_t> ev(4 * static_cast<size_t>(nchunks), nullptr);
    auto evt = [&](int kind, int i) -> cudaEvent_t & { return ev[4 * static_cast<size_t>(i) + kind]; };
    enum { kH2D = 0, kResliced = 1, kComputed = 2, kD2H = 3 };
    mvd_status st = MVD_OK;
    for (auto &x : ev) {
        if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess) {
            st = cuda_fail(e, "event");
            break;
        }
    }
    const char *src = static_cast<const char *>(stacks_host);
    for (int i = 0; i < nchunks && st == MVD_OK; ++i) {
        const int y0 = cy0[i], yn = cyn[i], slot = i % 2;
        // H2D into the stack slot once the reslice of chunk i-2 has consumed it
        if (i >= 2) cudaStreamWaitEvent(c->copy_in, evt(kResliced, i - 2), 0);
        char *dst = c->run_stack[slot].as<char>();
        for (int v = 0; v < c->V && st == MVD_OK; ++v) {
            e = cudaMemcpy2DAsync(dst + static_cast<size_t>(v) * nz * yn * nx * es, yn * nx * es,
                                  src + (static_cast<size_t>(v) * nz * ny + y0) * nx * es, static_cast<size_t>(ny) * nx * es,
                                  yn * nx * es, nz, cudaMemcpyHostToDevice, c->copy_in);
            if (e != cudaSuccess) st = cuda_fail(e, "H2D copy");
        }
        if (st != MVD_OK) break;
        cudaEventRecord(evt(kH2D, i), c->copy_in);
        // reslice + deconvolve on the caller's stream
        cudaStreamWaitEvent(s, evt(kH2D, i), 0);
        if (i >= 2) cudaStreamWaitEvent(s, evt(kD2H, i - 2), 0);
        if ((st = mvd_reslice(c, dst, dt, c->V, nz, yn, nx, c->run_planes.ptr, s)) != MVD_OK) break;
        cudaEventRecord(evt(kResliced, i), s);
        float *est = c->run_est[slot].as<float>();
        if ((st = mvd_deconvolve_planes(c, c->run_planes.ptr, dt, est, yn, 1, s)) != MVD_OK) break;
        cudaEventRecord(evt(kComputed, i), s);
        // D2H: planes y0 .. y0+yn are contiguous in the [Y][Z][X] output
        cudaStreamWaitEvent(c->copy_out, evt(kComputed, i), 0);
        e = cudaMemcpyAsync(out_host + static_cast<size_t>(y0) * plane_px, est, yn * plane_px * sizeof(float),
                            cudaMemcpyDeviceToHost, c->copy_out);
        if (e != cudaSuccess) st = cuda_fail(e, "D2H copy");
        cudaEventRecord(evt(kD2H, i), c->copy_out);
    }
    cudaError_t e1 = cudaStreamSynchronize(c->copy_in);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaError_t e3 = cudaStreamSynchronize(c->copy_out);
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    if (st != MVD_OK) return st;
    if (e1 != cudaSuccess) return cuda_fail(e1, "copy stream");
    if (e2 != cudaSuccess) return cuda_fail(e2, "compute stream");
    if (e3 != cudaSuccess) return cuda_fail(e3, "copy stream");
    return MVD_OK;
}

}  // extern "C"

// ---- batches -----------------------------------------------------------------

struct mvd_batch {
    int device = 0;
    mvd_dtype dt = MVD_U16;
    std::vector<mvd_volume_desc> vols;
    std::vector<mvd_ctx *> ctx;
    std::vector<DevBuf> planes;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int concurrent = 1;
    int max_ctas = 0;
    int graph_kernels = 0;
    std::string key;
    // persistent queue schedule (MVD_BATCH_QUEUE): the fused-route volumes of
    // each PSF-size class run as one launch over a device work queue
    int schedule = MVD_BATCH_GRAPH;
    long long wait_budget = mvd::kDefaultWaitBudget;
    DevBuf status;                               // one int: the queue launches' status word
    struct Queue {
        std::vector<int> vols;                   // batch indices of the class's volumes
        DevBuf qvols, segs, taps, done, ctl;     // ctl: head (u64) + abort (int)
        mvd::bq::QParams qp{};
        long long items = 0;
    } q[mvd::bq::kClasses];
    bool queue_ready = false;
};

namespace {

void batch_drop_graph(mvd_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_kernels = 0;
}

// A volume runs on the queue when its context takes the fused separable
// route with a PSF the fused kernels cover and at least one iteration.
bool queue_volume(const mvd_ctx *c) {
    return c->algo == MVD_ALGO_FUSED && mvd::fused_supported(c->K) && mvd::bq::size_class(c->K) >= 0 &&
           c->iters > 0 && !c->weights && c->Ka == 0;
}

// Per-class tables of the queue schedule: volume descriptors with their
// factors padded to the class size, phase-major segments, per-plane counters.
mvd_status batch_queue_prepare(mvd_batch *b) {
    for (int cls = 0; cls < mvd::bq::kClasses; ++cls) {
        auto &Q = b->q[cls];
        Q.vols.clear();
        Q.items = 0;
        const int KC = mvd::bq::class_k(cls);
        std::vector<mvd::bq::QVol> qv;
        std::vector<float> taps;
        long long planes = 0;
        int max_phases = 0;
        for (size_t i = 0; i < b->vols.size(); ++i) {
            mvd_ctx *c = b->ctx[i];
            if (!queue_volume(c) || mvd::bq::size_class(c->K) != cls) continue;
            const mvd_volume_desc &d = b->vols[i];
            cudaError_t e = prepare_workspace(c, d.n_planes);
            if (e != cudaSuccess) return fail(MVD_ERR_NOMEM, "volume %zu workspace: %s", i, cudaGetErrorString(e));
            mvd::bq::QVol v{};
            v.phi = d.stacks_dev ? b->planes[i].ptr : d.planes_dev;
            v.u16 = b->dt == MVD_U16;
            v.psi = d.estimate_dev;
            v.ratio = c->ratio.as<float>();
            v.means = c->means.as<float>();
            v.H = c->H;
            v.W = c->W;
            v.P = d.n_planes;
            v.V = c->V;
            v.circular = c->boundary == MVD_BOUNDARY_CIRCULAR;
            v.seq = c->order == MVD_ORDER_SEQUENTIAL;
            v.phases = 2 * c->iters * (v.seq ? c->V : 1);
            v.tiles_x = (c->W + 127) / 128;
            v.tiles = v.tiles_x * ((c->H + 31) / 32);
            v.eps = c->eps;
            // TMA tiles on the zero boundary (zero fill outside the plane)
            int bw = 0, bh = 0;
            mvd::bq::tile_box(cls, &bw, &bh);
            v.use_tma = !v.circular &&
                        mvd::fused::encode_plane_map(&v.psi_map, v.psi, v.W, v.H, v.P, bw, bh) &&
                        mvd::fused::encode_plane_map(&v.ratio_map, v.ratio, v.W, v.H,
                                                     static_cast<long long>(v.V) * v.P, bw, bh);
            // factors [terms][4][K] -> [terms][4][KC], centred, zero taps around
            const int pad = (KC - c->K) / 2;
            const size_t base = taps.size() / (4 * KC);
            for (int t = 0; t < c->ft.total_terms; ++t)
                for (int kind = 0; kind < 4; ++kind) {
                    std::vector<float> row(KC, 0.0f);
                    for (int m = 0; m < c->K; ++m)
                        row[pad + m] = c->taps_host[(static_cast<size_t>(t) * 4 + kind) * c->K + m];
                    taps.insert(taps.end(), row.begin(), row.end());
                }
            for (int vv = 0; vv < c->V; ++vv) {
                v.rank[vv] = c->ft.rank[vv];
                v.tap_off[vv] = c->ft.tap_off[vv];
                v.crank[vv] = c->ft.crank[vv];
                v.ctap_off[vv] = c->ft.ctap_off[vv];
                v.short_mask[vv] = c->ft.short_mask[vv];
            }
            v.ntaps = c->ft.total_terms * 4 * KC;
            // taps and done are device offsets until the buffers exist
            v.taps = reinterpret_cast<const float *>(base * 4 * KC * sizeof(float));
            v.done = reinterpret_cast<int *>(planes * sizeof(int));
            planes += d.n_planes;
            max_phases = std::max(max_phases, v.phases);
            qv.push_back(v);
            Q.vols.push_back(static_cast<int>(i));
        }
        if (qv.empty()) continue;
        std::vector<mvd::bq::QSeg> segs;
        long long start = 0;
        for (int ph = 0; ph < max_phases; ++ph)
            for (size_t j = 0; j < qv.size(); ++j) {
                if (ph >= qv[j].phases) continue;
                segs.push_back({start, static_cast<int>(j), ph});
                start += static_cast<long long>(qv[j].P) * qv[j].tiles;
            }
        Q.items = start;
        cudaError_t e;
        if ((e = Q.qvols.ensure(qv.size() * sizeof(mvd::bq::QVol))) != cudaSuccess ||
            (e = Q.segs.ensure(segs.size() * sizeof(mvd::bq::QSeg))) != cudaSuccess ||
            (e = Q.taps.ensure(taps.size() * sizeof(float))) != cudaSuccess ||
            (e = Q.done.ensure(planes * sizeof(int))) != cudaSuccess ||
            (e = Q.ctl.ensure(16)) != cudaSuccess)
            return fail(MVD_ERR_NOMEM, "queue tables: %s", cudaGetErrorString(e));
        for (auto &v : qv) {
            v.taps = Q.taps.as<float>() + reinterpret_cast<size_t>(v.taps) / sizeof(float);
            v.done = Q.done.as<int>() + reinterpret_cast<size_t>(v.done) / sizeof(int);
        }
        if ((e = cudaMemcpy(Q.qvols.ptr, qv.data(), qv.size() * sizeof(mvd::bq::QVol), cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = cudaMemcpy(Q.segs.ptr, segs.data(), segs.size() * sizeof(mvd::bq::QSeg), cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = cudaMemcpy(Q.taps.ptr, taps.data(), taps.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
            return cuda_fail(e, "upload queue tables");
        auto &qp = Q.qp;
        qp.vols = Q.qvols.as<mvd::bq::QVol>();
        qp.segs = Q.segs.as<mvd::bq::QSeg>();
        qp.nseg = static_cast<int>(segs.size());
        qp.total = Q.items;
        qp.head = reinterpret_cast<unsigned long long *>(Q.ctl.ptr);
        qp.abort = reinterpret_cast<int *>(static_cast<char *>(Q.ctl.ptr) + 8);
    }
    cudaError_t e = b->status.ensure(sizeof(int));
    if (e != cudaSuccess) return fail(MVD_ERR_NOMEM, "batch status: %s", cudaGetErrorString(e));
    if ((e = cudaMemset(b->status.ptr, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "batch status");
    b->queue_ready = true;
    return MVD_OK;
}

mvd_status batch_capture(mvd_batch *b) {
    batch_drop_graph(b);
    for (auto *c : b->ctx) c->max_ctas = b->max_ctas;
    // launches made while capturing only record graph nodes: they are counted
    // when the graph runs, not now
    const uint64_t counted_before = mvd::g_launches.load();
    struct Uncount {
        uint64_t before;
        ~Uncount() { mvd::g_launches.fetch_sub(mvd::g_launches.load() - before); }
    } uncount{counted_before};
    // the queue's tables are allocated and uploaded before capturing
    if (b->schedule == MVD_BATCH_QUEUE && !b->queue_ready) {
        mvd_status qs = batch_queue_prepare(b);
        if (qs != MVD_OK) return qs;
    }
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    mvd_status st = MVD_OK;
    const bool queue = b->schedule == MVD_BATCH_QUEUE;
    std::vector<char> on_queue(b->vols.size(), 0);
    if (queue)
        for (auto &Q : b->q)
            for (int i : Q.vols) on_queue[i] = 1;
    cudaEventRecord(b->fork, b->cap);
    // queue volumes: reslice and plane means on their branches, joined before
    // the queue launches; the others: their whole schedule, joined at the end
    for (int pass = 0; pass < 2 && st == MVD_OK; ++pass) {
        for (size_t i = 0; i < b->vols.size() && st == MVD_OK; ++i) {
            if (on_queue[i] != (pass == 0)) continue;
            const mvd_volume_desc &v = b->vols[i];
            mvd_ctx *c = b->ctx[i];
            cudaStream_t s = b->concurrent ? b->streams[i] : b->cap;
            if (b->concurrent) cudaStreamWaitEvent(s, b->fork, 0);
            const void *data = v.planes_dev;
            if (v.stacks_dev) {
                st = mvd_reslice(c, v.stacks_dev, b->dt, v.views, v.plane_h, v.n_planes, v.plane_w, b->planes[i].ptr,
                                 s);
                data = b->planes[i].ptr;
            }
            if (st == MVD_OK && on_queue[i]) {
                cudaError_t e2 = mvd::launch_plane_means(data, b->dt == MVD_U16, c->V, v.n_planes, c->H, c->W,
                                                          c->means.as<float>(), s);
                if (e2 != cudaSuccess) st = cuda_fail(e2, "plane means kernel");
            } else if (st == MVD_OK) {
                st = mvd_deconvolve_planes(c, data, b->dt, v.estimate_dev, v.n_planes, 1, s);
            }
            if (b->concurrent && pass == 0) {
                cudaEventRecord(b->done[i], s);
                cudaStreamWaitEvent(b->cap, b->done[i], 0);
            }
        }
        if (pass == 0 && queue && st == MVD_OK) {
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
            for (int cls = 0; cls < mvd::bq::kClasses && st == MVD_OK; ++cls) {
                auto &Q = b->q[cls];
                if (Q.items == 0) continue;
                Q.qp.err = b->status.as<int>();
                Q.qp.wait_budget = b->wait_budget;
                cudaError_t e2 = cudaMemsetAsync(Q.done.ptr, 0, Q.done.bytes, b->cap);
                if (e2 == cudaSuccess) e2 = cudaMemsetAsync(Q.ctl.ptr, 0, 16, b->cap);
                if (e2 == cudaSuccess) e2 = mvd::bq::launch_queue(cls, Q.qp, sms, b->cap);
                if (e2 != cudaSuccess) st = cuda_fail(e2, "queue launch");
                else mvd::count_launch(1);
            }
        }
    }
    if (b->concurrent)
        for (size_t i = 0; i < b->vols.size(); ++i)
            if (!on_queue[i]) {
                cudaEventRecord(b->done[i], b->streams[i]);
                cudaStreamWaitEvent(b->cap, b->done[i], 0);
            }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (st != MVD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(g, nodes.data(), &n);
    int k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    b->graph_kernels = k;
    return MVD_OK;
}

bool tune_cache_lookup(const std::string &key, int *conc, int *ctas, int *sched) {
    const char *path = std::getenv("MVD_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[4096];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        // line: <key> <concurrent> <max_ctas> <schedule>
        int v[3];
        bool ok = true;
        for (int k = 2; k >= 0 && ok; --k) {
            char *sp = std::strrchr(line, ' ');
            if (!sp) ok = false;
            else {
                v[k] = std::atoi(sp + 1);
                *sp = 0;
            }
        }
        if (ok && key == line) {
            *conc = v[0];
            *ctas = v[1];
            *sched = v[2];
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void tune_cache_store(const std::string &key, int conc, int ctas, int sched) {
    const char *path = std::getenv("MVD_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d\n", key.c_str(), conc, ctas, sched);
    std::fclose(f);
}

}  // namespace

extern "C" {

mvd_status mvd_batch_create(mvd_batch **out, const mvd_volume_desc *vols, int n, mvd_dtype dt,
                            mvd_boundary boundary, float eps, mvd_update_order order) {
    t_last_error.clear();
    if (!out || !vols || n < 1) return fail(MVD_ERR_ARG, "need at least one volume");
    if (dt != MVD_U16 && dt != MVD_F32) return fail(MVD_ERR_ARG, "unknown dtype");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        const mvd_volume_desc &v = vols[i];
        if (!v.estimate_dev || (!v.stacks_dev && !v.planes_dev) || v.n_planes < 1)
            return fail(MVD_ERR_ARG, "volume %d: needs data, an estimate buffer and n_planes >= 1", i);
    }
    auto *b = new (std::nothrow) mvd_batch();
    if (!b) return fail(MVD_ERR_NOMEM, "batch");
    cudaGetDevice(&b->device);
    b->dt = dt;
    b->vols.assign(vols, vols + n);
    const size_t es = dt == MVD_U16 ? 2 : 4;
    char buf[128];
    b->key = "v2";
    for (int i = 0; i < n && true; ++i) {
        const mvd_volume_desc &v = vols[i];
        mvd_ctx *c = nullptr;
        mvd_status st = mvd_create(&c, v.views, v.psfs_host, v.psf_size, v.plane_h, v.plane_w, v.iters, boundary, eps);
        if (st == MVD_OK) st = mvd_set_update_order(c, order);
        if (st == MVD_OK) st = mvd_set_variant(c, static_cast<mvd_variant>(v.variant));
        if (st != MVD_OK) {
            std::string m = t_last_error;
            if (c) mvd_destroy(c);
            mvd_batch_destroy(b);
            return fail(st, "volume %d: %s", i, m.c_str());
        }
        b->ctx.push_back(c);
        b->planes.emplace_back();
        cudaError_t e = prepare_workspace(c, v.n_planes);
        if (e == cudaSuccess && v.stacks_dev)
            e = b->planes.back().ensure(static_cast<size_t>(v.views) * v.n_planes * v.plane_h * v.plane_w * es);
        if (e != cudaSuccess) {
            mvd_batch_destroy(b);
            return fail(MVD_ERR_NOMEM, "volume %d workspace: %s", i, cudaGetErrorString(e));
        }
        std::snprintf(buf, sizeof buf, "_%dx%dx%dx%dv%dk%dt%d%s", v.n_planes, v.plane_h, v.plane_w, v.variant,
                      v.views, v.psf_size, v.iters, v.stacks_dev ? "s" : "p");
        b->key += buf;
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            mvd_batch_destroy(b);
            return fail(MVD_ERR_CUDA, "streams for the batch");
        }
        b->streams.push_back(s);
        b->done.push_back(ev);
    }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        mvd_batch_destroy(b);
        return fail(MVD_ERR_CUDA, "capture stream");
    }
    *out = b;
    return MVD_OK;
}

mvd_status mvd_batch_run(mvd_batch *b, void *stream) {
    t_last_error.clear();
    if (!b) return fail(MVD_ERR_ARG, "batch is NULL");
    DeviceGuard g(b->device);
    if (!b->exec) {
        mvd_status st = batch_capture(b);
        if (st != MVD_OK) return st;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    mvd::count_launch(b->graph_kernels);
    return MVD_OK;
}

mvd_status mvd_batch_tune(mvd_batch *b, void *stream) {
    t_last_error.clear();
    if (!b) return fail(MVD_ERR_ARG, "batch is NULL");
    DeviceGuard g(b->device);
    cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    // 1. the route of every volume (fused separable kernels or Fourier route),
    //    timed on its own data; volumes given as stacks are resliced first
    {
        mvd_status st = b->exec ? MVD_OK : batch_capture(b);
        if (st != MVD_OK) return st;
        cudaGraphLaunch(b->exec, s0);
        cudaError_t e = cudaStreamSynchronize(s0);
        if (e != cudaSuccess) return cuda_fail(e, "batch run before tuning");
        for (size_t i = 0; i < b->vols.size(); ++i) {
            const mvd_volume_desc &v = b->vols[i];
            const void *data = v.stacks_dev ? b->planes[i].ptr : v.planes_dev;
            if ((st = mvd_autotune(b->ctx[i], data, b->dt, v.n_planes, stream)) != MVD_OK) return st;
            if ((e = prepare_workspace(b->ctx[i], v.n_planes)) != cudaSuccess)
                return fail(MVD_ERR_NOMEM, "volume %zu workspace: %s", i, cudaGetErrorString(e));
        }
        batch_drop_graph(b);
    }
    // 2. the schedule and launch shape
    b->queue_ready = false;
    int conc = 1, ctas = 0, sched = MVD_BATCH_GRAPH;
    if (tune_cache_lookup(b->key, &conc, &ctas, &sched)) {
        b->concurrent = conc;
        b->max_ctas = ctas;
        b->schedule = sched;
        batch_drop_graph(b);
        return MVD_OK;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    bool any_queue = false;
    for (auto *c : b->ctx) any_queue |= queue_volume(c);
    // {concurrent branches, persistent-grid cap, schedule}
    const int cand[][3] = {{1, 0, MVD_BATCH_GRAPH},
                           {0, 0, MVD_BATCH_GRAPH},
                           {1, sms > 0 ? sms : 1, MVD_BATCH_GRAPH},
                           {1, 0, MVD_BATCH_QUEUE}};
    const int n_cand = any_queue ? 4 : 3;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_i = 0;
    mvd_status st = MVD_OK;
    for (int i = 0; i < n_cand && st == MVD_OK; ++i) {
        b->concurrent = cand[i][0];
        b->max_ctas = cand[i][1];
        b->schedule = cand[i][2];
        if ((st = batch_capture(b)) != MVD_OK) break;
        cudaGraphLaunch(b->exec, s);                  // warm
        cudaEventRecord(e0, s);
        cudaGraphLaunch(b->exec, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "tuning run");
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_i = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MVD_OK) return st;
    if ((st = mvd_batch_device_status(b)) != MVD_OK) return st;
    b->concurrent = cand[best_i][0];
    b->max_ctas = cand[best_i][1];
    b->schedule = cand[best_i][2];
    batch_drop_graph(b);
    tune_cache_store(b->key, b->concurrent, b->max_ctas, b->schedule);
    return MVD_OK;
}

mvd_status mvd_batch_info(const mvd_batch *b, int *concurrent, int *max_ctas, int *graph_kernels) {
    if (!b) return fail(MVD_ERR_ARG, "batch is NULL");
    if (concurrent) *concurrent = b->concurrent;
    if (max_ctas) *max_ctas = b->max_ctas;
    if (graph_kernels) *graph_kernels = b->graph_kernels;
    return MVD_OK;
}

mvd_status mvd_batch_set_schedule(mvd_batch *b, int schedule) {
    t_last_error.clear();
    if (!b) return fail(MVD_ERR_ARG, "batch is NULL");
    if (schedule != MVD_BATCH_GRAPH && schedule != MVD_BATCH_QUEUE) return fail(MVD_ERR_ARG, "unknown schedule");
    DeviceGuard g(b->device);
    b->schedule = schedule;
    batch_drop_graph(b);
    return MVD_OK;
}

mvd_status mvd_batch_queue_info(const mvd_batch *b, int *schedule, int *queue_volumes, long long *queue_items) {
    if (!b) return fail(MVD_ERR_ARG, "batch is NULL");
    int nv = 0;
    long long items = 0;
    if (b->schedule == MVD_BATCH_QUEUE && b->queue_ready)
        for (const auto &Q : b->q) {
            nv += static_cast<int>(Q.vols.size());
            items += Q.items;
        }
    if (schedule) *schedule = b->schedule;
    if (queue_volumes) *queue_volumes = nv;
    if (queue_items) *queue_items = items;
    return MVD_OK;
}

mvd_status mvd_batch_set_wait_budget(mvd_batch *b, long long cycles) {
    t_last_error.clear();
    if (!b) return fail(MVD_ERR_ARG, "batch is NULL");
    DeviceGuard g(b->device);
    b->wait_budget = cycles == 0 ? mvd::kDefaultWaitBudget : cycles;
    batch_drop_graph(b);
    return MVD_OK;
}

mvd_status mvd_batch_device_status(mvd_batch *b) {
    t_last_error.clear();
    if (!b) return fail(MVD_ERR_ARG, "batch is NULL");
    DeviceGuard g(b->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "batch");
    if (!b->status.ptr) return MVD_OK;
    int w = 0;
    if ((e = cudaMemcpy(&w, b->status.ptr, sizeof w, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "batch status");
    if (w == 0) return MVD_OK;
    cudaMemset(b->status.ptr, 0, sizeof(int));
    return fail(MVD_ERR_TIMEOUT, "a queue wait of the batch ran out (status %d)", w);
}

mvd_status mvd_batch_destroy(mvd_batch *b) {
    if (!b) return MVD_OK;
    DeviceGuard g(b->device);
    batch_drop_graph(b);
    for (auto *c : b->ctx) mvd_destroy(c);
    for (auto &p : b->planes) p.release();
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto ev : b->done) cudaEventDestroy(ev);
    for (auto &Q : b->q) {
        Q.qvols.release();
        Q.segs.release();
        Q.taps.release();
        Q.done.release();
        Q.ctl.release();
    }
    b->status.release();
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return MVD_OK;
}

}  // extern "C"
