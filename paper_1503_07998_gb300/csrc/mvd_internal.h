// Internal declarations shared by the host side of the library and the CUDA
// translation units.  Nothing here is part of the public ABI (include/mvd.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

namespace mvd {

constexpr int kMaxViews = 64;
// 1D factors whose taps outside the short_tap_count(K) central ones carry no
// mass above the rank tolerance (narrow Gaussians) run with that many taps on
// the fused path: 17 (+-8) for K <= 31, 21 (+-10, Gaussians up to sigma of
// about 2 px) for larger K.
__host__ __device__ constexpr int short_tap_count(int K) { return K <= 17 ? K : (K <= 31 ? 17 : 21); }
constexpr int kFusedMaxK = 47;   // largest PSF side with a fused-kernel instance
// Relative Frobenius norm below which trailing SVD terms of a PSF are dropped
// by default: below the FP32 rounding of the PSF's entries.
constexpr double kDefaultRankTol = 3e-7;

// Launch accounting (mvd_launch_count).
void count_launch(int n = 1);

// Sets the calling thread's mvd_last_error() text.
void set_last_error(const char *msg);

// Per-view separable factorisation of the PSFs, laid out on the device as
//   taps[(tap_off[v] + q) * 4 * K + {0: blur vertical, 1: blur horizontal,
//                                    2: corr vertical, 3: corr horizontal}*K + m]
// Each pass computes out[i] = sum_m t[m] * in[i + m] over a window that starts
// R rows/columns before the output; the blur taps are reversed factors, the
// correlation taps the factors as they are.  The singular value is folded
// into the vertical factor.
struct FactorTable {
    int K = 0;
    int views = 0;
    int rank[kMaxViews] = {};
    int tap_off[kMaxViews] = {};     // in units of terms
    int crank[kMaxViews] = {};       // terms of the correlation step (= rank for plain MV-RL)
    // per view, the 1D factor kinds (bit k: blur vertical, blur horizontal,
    // correlation vertical, correlation horizontal) whose every term keeps
    // all but a rank-tolerance share of its mass in the short_tap_count(K) central taps
    unsigned char short_mask[kMaxViews] = {};
    int ctap_off[kMaxViews] = {};    // their offset (= tap_off for plain MV-RL)
    int group[kMaxViews] = {};       // blur group (views with identical PSFs)
    int n_groups = 0;
    int group_leader[kMaxViews] = {};
    int total_terms = 0;
};

// Host-side PSF analysis (factor.cpp).  psfs: [V][K][K] FP32.  Fills `ft` and
// the host tap array (total_terms * 4 * K floats).  With `corr` ([V][K][K],
// the kernels the ratio is correlated with) the correlation step gets terms of
// its own; without it, it uses the PSFs' terms.  Returns false with a message
// when the factorisation fails.
bool factorise_psfs(const float *psfs, int views, int K, double rank_tol,
                    FactorTable &ft, float *taps_out, int taps_capacity, char *msg, size_t msg_len,
                    const float *corr = nullptr);
int max_terms(int views, int K);

// Correlation kernels of the MV-RL variants (variants.cpp): X_v, [V][K][K],
// unit sum, FP64 (Supp. Note 2 sec. 1).  variant: an mvd_variant value.
void variant_kernels(const float *psfs, int views, int K, int variant, double *X);

// ---- kernel launchers (return cudaGetLastError after the launch) ---------

// stacks [V][Z][Y][X] -> planes [V][Y][Z][X]
cudaError_t launch_reslice(const void *src, void *dst, int elem_bytes, int views,
                           int nz, int ny, int nx, cudaStream_t s);

// [planes][H][W] -> [planes][H+2pad][W+2pad] with zeros around; weights
// (optional) 1 on the data and 0 in the padding.
cudaError_t launch_embed_padded(const void *src, int elem_bytes, long long planes, int H, int W, int pad, void *dst,
                                float *weights, cudaStream_t s);
// [planes][Hp][Wp] -> [planes][Hp-2pad][Wp-2pad] (the centre).
cudaError_t launch_crop_planes(const float *src, long long planes, int Hp, int Wp, int pad, float *dst,
                               cudaStream_t s);

// means[p] = (sum over views and pixels of plane p) / (V*H*W), FP64 sum.
cudaError_t launch_plane_means(const void *data, int u16, int views, int planes, int H,
                               int W, float *means, cudaStream_t s);

struct FusedArgs {
    const float *psi_in;     // [P][H][W], or nullptr -> use means (iteration 0)
    const float *means;      // [P]
    float *psi_out;          // [P][H][W]
    const void *phi;         // [V][P][H][W]
    int phi_u16;
    float *ratio;            // [V][P][H][W] scratch
    const float *taps;       // device factor taps (see FactorTable)
    const float *taps_host;  // the same table on the host (copied into each launch)
    FactorTable ft;
    int H, W, P;
    int circular;
    float eps;
    int view_lo, view_hi;    // views [lo, hi) take part in this launch
    const float *weights;    // [V][P][H][W] per-pixel view weights, or nullptr (plain MV-RL)
    const float *wnorm;      // [V][P][H][W] 1 / (w_v (*) P_v^*), negative where that is below the floor
    int weights_bcast;       // weights and wnorm hold one plane per view, used for every plane
    int store_blur;          // kernel A writes the in-plane blur instead of the ratio (3D route)
    int *err;                // device status word (kDevTimeout set on an expired wait)
    long long wait_budget;   // clock cycles a tile wait may spin before it reports a timeout
    int max_ctas;            // cap on the persistent grid (0: one resident wave)
};

constexpr int kDevTimeout = 1;
constexpr float kNormFloor = 1e-6f;      // weighted MV-RL: a view leaves psi unchanged below this footprint
constexpr long long kDefaultWaitBudget = 2000000000LL;   // about one second at 2 GHz

bool fused_supported(int K);
// The fused kernels carry the taps in their parameter block; false if they do not fit.
bool fused_taps_fit(const FactorTable &ft);
void fused_tile_shape(int K, int *tile_h, int *tile_w);
cudaError_t launch_fused_blur_ratio(const FusedArgs &a, cudaStream_t s);
cudaError_t launch_fused_correlate_update(const FusedArgs &a, cudaStream_t s);

// 3D route (vol3d.cu): passes along the plane axis with the profile a [Ka].
// blur, phi, r, c: one view's [P][plane] planes.
cudaError_t launch_axial_ratio(const float *blur, const void *phi, int u16, const float *a, int Ka, int P,
                               long long plane, int circular, float eps, float *r, cudaStream_t s);
cudaError_t launch_axial_corr(const float *r, const float *a, int Ka, int P, long long plane, int circular, float *c,
                              cudaStream_t s);

// Tensor-core route (tc.cu): the same two kernels with BF16x3 tcgen05 passes.
bool tc_supported(int K);
void tc_tile_shape(int K, int *tile_h, int *tile_w);
cudaError_t launch_tc_blur_ratio(const FusedArgs &a, cudaStream_t s);
cudaError_t launch_tc_correlate_update(const FusedArgs &a, cudaStream_t s);
// Warp-specialised BF16x3 tensor-core kernels (tcw.cu) for launches whose
// views share one rank-1 factorisation on the zero boundary; the tensor
// route runs a launch on them whenever tcw_eligible says so.
constexpr int kInConst = 0;   // input: the constant first estimate (the plane means)
constexpr int kInF32 = 1;     // input: FP32 planes, split by the kernel
constexpr int kInSplit = 2;   // input: planes written already split (hi, lo BF16, column-blocked)
struct TcwIo {
    int in_mode;              // kInConst / kInF32 / kInSplit (blur: the estimate; correlation: the ratio)
    int ratio_split;          // blur: write the ratio split (for a split-input correlation), else FP32
    uint16_t *psi_split;      // split copy of the estimate, [P][2][G][H][8] (G = W rounded up to 8, / 8)
    int write_psi_split;      // correlation: also write the split estimate (for a split-input blur)
};
bool tcw_eligible(const FusedArgs &a, int which);   // which: 0 blur/ratio, 1 correlate/update
// Bytes of `planes` split planes (hi and lo, columns rounded up to 8).
size_t tcw_split_bytes(int W, int H, long long planes);
cudaError_t launch_tcw(const FusedArgs &a, int which, const TcwIo &io, cudaStream_t s);
// TF32 variant of the tensor-core kernels (same K range and tile rule).
void tf32_tile_shape(int K, int *tile_h, int *tile_w);
cudaError_t launch_tf32_blur_ratio(const FusedArgs &a, cudaStream_t s);
cudaError_t launch_tf32_correlate_update(const FusedArgs &a, cudaStream_t s);

// Persistent batched launch of the fused path (batchq.cu).
namespace bq {
// One volume of the queue: its planes, estimate, ratio scratch, plane means,
// factor taps padded to the launch's PSF-size class ([terms][4][KC], the
// FactorTable layout) and one counter of finished tiles per plane.
struct QVol {
    CUtensorMap psi_map;      // TMA maps of the estimate [P][H][W] and the ratios [V*P][H][W]
    CUtensorMap ratio_map;    // (boxes of the launch's tile), valid if use_tma
    int use_tma;
    const void *phi;          // [V][P][H][W]
    int u16;
    float *psi;               // [P][H][W]
    float *ratio;             // [V][P][H][W]
    const float *means;       // [P]
    const float *taps;        // this volume's factors
    int ntaps;                // their floats (terms * 4 * KC)
    int *done;                // [P]
    int H, W, P, V, circular, seq, phases, tiles_x, tiles;
    float eps;
    int rank[kMaxViews], tap_off[kMaxViews], crank[kMaxViews], ctap_off[kMaxViews];
    unsigned char short_mask[kMaxViews];
};
// Items [start, start + P * tiles) are phase `phase` of volume `vol`.
struct QSeg {
    long long start;
    int vol, phase;
};
struct QParams {
    const QVol *vols;
    const QSeg *segs;
    int nseg;
    long long total;                  // items
    unsigned long long *head;         // queue counter (zero before the launch)
    int *abort;                       // set when a wait expires: every CTA leaves
    int *err;                         // device status word
    long long wait_budget;            // clock cycles per wait; < 0: report a timeout (test hook)
};
constexpr int kClasses = 3;
// PSF-size class of K (0: 17, 1: 31, 2: 47), -1 beyond the fused kernels.
int size_class(int K);
int class_k(int cls);
// Items, grid and shared memory of a class's launch.
cudaError_t launch_queue(int cls, const QParams &qp, int sms, cudaStream_t s);
// TMA box (width, height) of a class's tiles.
void tile_box(int cls, int *box_w, int *box_h);
}  // namespace bq
namespace fused {
bool encode_plane_map(CUtensorMap *m, const void *base, int W, int H, long long D, int box_w, int box_h);
}  // namespace fused

// Plane-resident route (resident.cu): a cluster of CTAs keeps one plane's
// estimate, ratio and running product in shared memory for all iterations.
namespace res {
struct ResArgs {
    const void *phi;          // [V][P][H][W]
    int u16;
    const float *psi_in;      // [P][H][W], or nullptr: start from the plane means
    const float *means;       // [P]
    float *psi_out;           // [P][H][W]
    const float *taps;        // [terms][4][KC] (factors padded to the size class)
    int ntaps;
    int H, W, P, V, iters, seq, strip, C;
    float eps;
    int rank[kMaxViews], tap_off[kMaxViews], crank[kMaxViews], ctap_off[kMaxViews];
    unsigned char short_mask[kMaxViews];
};
// Cluster size C, strip rows and dynamic shared memory for planes H x W with
// PSF-size class cls; false if a plane does not fit on chip.
bool plan(int H, int W, int cls, int seq, int ntaps, int *C, int *strip, size_t *smem);
cudaError_t launch(const ResArgs &a, int cls, size_t smem, cudaStream_t s);
}  // namespace res

// Fourier route (fft.cu, fft_rows.cu, fft_cols.cu).
namespace fftr {
constexpr int kMaxRadices = 16;
constexpr int kMaxLen = 2048;          // largest padded side
constexpr int kMaxStages = 5;
// One Stockham stage of a warp transform: radix R after stages whose radices
// multiply to p; M = N / R butterflies; its twiddles start at tw_off of the
// axis's table ((R - 1) p entries exp(+2 pi i q k / (p R)), q >= 1, k < p),
// none when p == 1; rp = 1 / p.
struct FftStage {
    int R, p, M, tw_off;
    float rp;
};
struct FftPlan1 {
    int N, nst, tw_len;                // length, stages, twiddle entries of all stages
    FftStage st[kMaxStages];
};
struct FftArgs {
    int Ly, Lx, Lc, LcP;               // padded grid, half-spectrum columns and their pitch
    FftPlan1 px, py;                   // row (length Lx) and column (length Ly) transforms
    const float2 *tw_x, *tw_y;         // their stage twiddle tables
    const float2 *spec;                // [V][Lc][Ly] PSF spectra / (Ly Lx), column by column
    const float2 *cspec;               // spectra the correlation uses (= spec for plain MV-RL)
    int H, W, P, view_lo, view_hi;
    float eps;
    const float *psi_in;               // nullptr: constant first estimate (means)
    const float *means;
    float *psi_out;
    const void *phi;
    int u16;
    float2 *S0;                        // [P][H][LcP]
    float2 *T;                         // [V][P][H][LcP]
    int *err;                          // device status word (kDevTimeout on an expired copy wait)
    long long wait_budget;             // clock cycles a copy wait may spin
};
bool smooth_size(int n, int *out);
bool radix_list(int n, int *rad, int *nrad);
// Stages of a warp transform of length N (2 <= N <= kMaxLen, factors 2, 3, 5)
// and their twiddle table; false if N has another factor.
bool make_plan(int N, FftPlan1 &plan, std::vector<float2> &tw);
void psf_spectrum(const float *psf, int K, int Ly, int Lx, int Lc, std::vector<float2> &out);
cudaError_t launch_rows(int mode, const FftArgs &a, int sms, cudaStream_t s);   // 0 estimate, 1 ratio, 2 update
cudaError_t launch_cols(int mode, const FftArgs &a, int sms, cudaStream_t s);   // 0 blur, 1 correlation
cudaError_t launch_iteration(const FftArgs &a, int sms, cudaStream_t s);
}  // namespace fftr

// PSF-gradient building blocks (adjoint.cu); every call covers P planes.
namespace adj {
constexpr int kMaxK = 63;
cudaError_t stencil(const float *in, float *out, const float *psf, int K, int H, int W, int P, int circular,
                    int correlate, int accumulate, cudaStream_t s);
cudaError_t lag_sum(const float *g, const float *img, double *G, int K, int H, int W, int P, int circular, int sign,
                    cudaStream_t s);
cudaError_t fill_means(float *psi, const float *means, long long plane, long long n, cudaStream_t s);
cudaError_t ratio(const void *phi, int u16, const float *b, float *r, long long n, float eps, cudaStream_t s);
cudaError_t update(const float *psi, const float *c, float *psi_next, int V, long long n, cudaStream_t s);
cudaError_t terminal(const void *phi, int u16, const float *y, float *ybar, double *loss, long long n, float eps,
                     cudaStream_t s);
cudaError_t cbar(const float *psibar, const float *psi_t, const float *c, float *psibar_new, float *cb, int V,
                 long long n, cudaStream_t s);
cudaError_t bbar(const void *phi, int u16, const float *rbar, const float *b, float *bb, long long n, float eps,
                 cudaStream_t s);
cudaError_t to_float(const double *G, float *out, int n, cudaStream_t s);
}  // namespace adj

// Plain per-plane path (one plane, one step per launch).
struct PlainArgs {
    const float *taps;       // device factor taps
    const float *psf_dev;    // [V][K][K] raw PSFs (direct route)
    const float *psf_corr;   // [V][K][K] kernels the direct correlation uses (= psf_dev for plain MV-RL)
    FactorTable ft;
    int H, W, circular;
    float eps;
};
// out = conv/corr of `in` (one plane) with view v's PSF. `direct` uses K^2 taps.
cudaError_t plain_convolve(const PlainArgs &a, int v, int correlate, int direct,
                           const float *in, float *tmp, float *out, cudaStream_t s);
cudaError_t plain_fill(float *dst, const float *means, int plane, size_t n, cudaStream_t s);
cudaError_t plain_ratio(const void *phi, int u16, const float *weights, const float *blur, float *ratio,
                        size_t n, float eps, cudaStream_t s);
// Weighted MV-RL: c = c * m where m >= 0, else 1 (m = 1 / n_v from weight_norms).
cudaError_t plain_apply_norm(float *c, const float *wnorm, size_t n, cudaStream_t s);
// m_v = 1 / (w_v (*) P_v^*) (correlation factors of view v), or -1 below
// kNormFloor, for the P planes of every view: weights and wnorm [V][P][H][W];
// tmp holds P planes.
cudaError_t weight_norms(const PlainArgs &a, const float *weights, int P, float *tmp, float *wnorm, cudaStream_t s);
cudaError_t plain_multiply(float *acc, const float *c, size_t n, int first, cudaStream_t s);
cudaError_t plain_update(float *psi, const float *prod, size_t n, cudaStream_t s);

}  // namespace mvd
