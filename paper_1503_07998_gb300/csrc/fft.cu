// Fourier route of the MV-RL iteration (Supp. Note 2 sec. 4: the
// convolutions are products of spectra): host side.  Padded grid sizes,
// transform plans, FP64 PSF spectra and the launch sequence of one update.
//
// The update runs as five passes over the planes (fft_rows.cu, fft_cols.cu):
//
//   rows  F   real rows of psi (zero beyond the plane) -> half spectra S0
//   cols  FM  S0 -> column FFT -> Psi; per view: Psi . H_v -> inverse column FFT -> T_v
//   rows  R   per view: T_v -> inverse row FFT -> blur b_v -> r_v = phi_v / max(b_v, eps)
//             (zero beyond the plane) -> forward row FFT -> T_v
//   cols  C   per view: T_v -> column FFT -> . conj(H_v) -> inverse column FFT -> T_v
//   rows  U   per view: T_v -> inverse row FFT -> c_v; psi <- psi * prod_v c_v
//
// H_v is the spectrum of view v's PSF wrapped onto the padded grid with its
// centre at the origin, scaled by 1 / (Ly Lx) so that both inverse
// transforms come out normalised; the correlation uses its conjugate.  For
// the ZERO boundary the grid is padded to Ly >= H + R, Lx >= W + R (enough
// for the cyclic product to equal the linear convolution on the plane); for
// CIRCULAR it is the plane itself.  Two real rows travel as one complex row
// (a + i b) and are separated by Hermitian symmetry.  Only the H rows of the
// plane are stored between passes: the padding rows of every real-space
// input are zero, so the column kernels fill them in shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <vector>

#include "mvd_internal.h"

namespace mvd {
namespace fftr {

namespace {

bool is_pow2(long long n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

// Smallest 2^a 3^b 5^c >= n.  A power of two of 64 or more is passed over
// for a size with an odd factor up to 10 % larger: the first stage of a warp
// transform writes at a stride of its radix, which is free of shared-memory
// bank conflicts only when that radix is odd.
bool smooth_size(int n, int *out) {
    std::vector<long long> c;
    for (long long a = 1; a <= 8192; a *= 2)
        for (long long b = a; b <= 8192; b *= 3)
            for (long long d = b; d <= 8192; d *= 5)
                if (d >= n) c.push_back(d);
    if (c.empty()) return false;
    std::sort(c.begin(), c.end());
    long long best = c[0];
    if (is_pow2(best) && best >= 64) {
        for (long long d : c)
            if (!is_pow2(d) && d <= best + best / 10 && d <= kMaxLen) {
                best = d;
                break;
            }
    }
    *out = static_cast<int>(best);
    return true;
}

bool radix_list(int n, int *rad, int *nrad) {
    int k = 0;
    while (n % 4 == 0 && k < kMaxRadices) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < kMaxRadices) { rad[k++] = 2; n /= 2; }
    while (n % 3 == 0 && k < kMaxRadices) { rad[k++] = 3; n /= 3; }
    while (n % 5 == 0 && k < kMaxRadices) { rad[k++] = 5; n /= 5; }
    *nrad = k;
    return n == 1;
}

// ---- transform plans ---------------------------------------------------------

namespace {

// radices with a device instance (fft_engine.cuh, stage_any)
const int kRadices[] = {2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40};

int split_factor(int R) { return (R % 4 == 0 && R != 8) ? 4 : (R % 5 == 0 ? 5 : (R % 3 == 0 ? 3 : 2)); }

// Arithmetic of an R-point DFT as the device nests it (real operations).
double dft_ops(int R) {
    switch (R) {
        case 2: return 4;
        case 3: return 16;
        case 4: return 16;
        case 5: return 40;
        default: break;
    }
    const int R1 = split_factor(R), R2 = R / R1;
    int nontrivial = 0;
    for (int n2 = 0; n2 < R2; ++n2)
        for (int k1 = 0; k1 < R1; ++k1) {
            const int e = (n2 * k1) % R;
            if (e != 0 && 2 * e != R && 4 * e != R && 4 * e != 3 * R) ++nontrivial;
        }
    return R2 * dft_ops(R1) + R1 * dft_ops(R2) + 6.0 * nontrivial;
}

// Shared-memory wavefronts of one warp access to 8-byte words at addr[0..n)
// (lane l at addr[l]; lanes >= n inactive): each half-warp is one 128-byte
// request, split by the most-used bank pair.
int wavefronts(const int *addr, int n) {
    int total = 0;
    for (int h = 0; h < 2; ++h) {
        int cnt[16] = {}, seen[16][16], ns[16] = {};
        int worst = 0;
        for (int l = 16 * h; l < std::min(n, 16 * h + 16); ++l) {
            const int b = addr[l] & 15;
            bool dup = false;
            for (int j = 0; j < ns[b]; ++j) dup |= seen[b][j] == addr[l];
            if (!dup) {
                seen[b][ns[b]++] = addr[l];
                worst = std::max(worst, ++cnt[b]);
            }
        }
        total += worst;
    }
    return total;
}

// Issue-slot estimate of one stage over one transform: per round of 32
// butterflies the DFT, twiddle and index arithmetic plus the shared-memory
// wavefronts (weighted 2: one wavefront per clock against four issues).
double stage_cost(int N, int R, int p) {
    const int M = N / R;
    double cost = 0;
    int addr[32];
    for (int i0 = 0; i0 < M; i0 += 32) {
        const int n = std::min(32, M - i0);
        int wf = 0;
        for (int q = 0; q < R; ++q) {
            for (int l = 0; l < n; ++l) addr[l] = i0 + l + q * M;
            wf += wavefronts(addr, n);
            if (p > 1 && q > 0) {
                for (int l = 0; l < n; ++l) addr[l] = (q - 1) * p + (i0 + l) % p;
                wf += wavefronts(addr, n);
            }
            for (int l = 0; l < n; ++l) {
                const int i = i0 + l, k = i % p;
                addr[l] = (i - k) * R + k + q * p;
            }
            wf += wavefronts(addr, n);
        }
        cost += dft_ops(R) / 2 + (p > 1 ? 4.0 * (R - 1) : 0.0) + 16 + 2.0 * wf;
    }
    return cost;
}

struct Search {
    int N;
    std::map<std::pair<int, int>, double> memo;
    double best = 1e300;
    int best_r[kMaxStages], best_n = 0;
    int cur[kMaxStages];
    double cost(int R, int p) {
        auto key = std::make_pair(R, p);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
        const double c = stage_cost(N, R, p);
        memo[key] = c;
        return c;
    }
    void go(int depth, int p, double acc) {
        if (acc >= best) return;
        if (p == N) {
            best = acc;
            best_n = depth;
            std::copy(cur, cur + depth, best_r);
            return;
        }
        if (depth == kMaxStages) return;
        for (int R : kRadices) {
            if ((N / p) % R != 0) continue;
            cur[depth] = R;
            go(depth + 1, p * R, acc + cost(R, p) + 24.0);   // + a stage's fixed cost (sync, loop)
        }
    }
};

}  // namespace

bool make_plan(int N, FftPlan1 &plan, std::vector<float2> &tw) {
    if (N < 2 || N > kMaxLen) return false;
    Search s;
    s.N = N;
    s.go(0, 1, 0.0);
    if (s.best_n == 0) return false;
    plan = FftPlan1{};
    plan.N = N;
    plan.nst = s.best_n;
    tw.clear();
    int p = 1;
    for (int k = 0; k < s.best_n; ++k) {
        FftStage &st = plan.st[k];
        st.R = s.best_r[k];
        st.p = p;
        st.M = N / st.R;
        st.rp = 1.0f / static_cast<float>(p);
        st.tw_off = p > 1 ? static_cast<int>(tw.size()) : 0;
        if (p > 1)
            for (int q = 1; q < st.R; ++q)
                for (int kk = 0; kk < p; ++kk) {
                    const double th = 2.0 * M_PI * static_cast<double>(q * kk) / (static_cast<double>(p) * st.R);
                    tw.push_back(make_float2(static_cast<float>(std::cos(th)), static_cast<float>(std::sin(th))));
                }
        p *= st.R;
    }
    plan.tw_len = static_cast<int>(tw.size());
    return true;
}

// ---- PSF spectra ---------------------------------------------------------------

namespace {

// FP64 host transform (radix 4, 2, 3, 5 Stockham stages), used once per
// context for the PSF spectra.
void host_fft(std::vector<double> &re, std::vector<double> &im, int N, int sign) {
    int rad[kMaxRadices], nrad = 0;
    radix_list(N, rad, &nrad);
    std::vector<double> yr(N), yi(N), c(N), sn(N);
    for (int k = 0; k < N; ++k) {
        c[k] = std::cos(2.0 * M_PI * k / N);
        sn[k] = sign * std::sin(2.0 * M_PI * k / N);
    }
    int p = 1;
    for (int s = 0; s < nrad; ++s) {
        const int R = rad[s], M = N / R, stride = N / (p * R);
        for (int i = 0; i < M; ++i) {
            const int k = i % p;
            double ar[5], ai[5];
            for (int q = 0; q < R; ++q) {
                const double xr = re[i + q * M], xi = im[i + q * M];
                const int e = static_cast<int>((static_cast<long long>(q) * k * stride) % N);
                ar[q] = xr * c[e] - xi * sn[e];
                ai[q] = xr * sn[e] + xi * c[e];
            }
            const int j = (i / p) * p * R + k;
            for (int m = 0; m < R; ++m) {
                double sr = 0, si = 0;
                for (int q = 0; q < R; ++q) {
                    const int e = (q * m * (N / R)) % N;
                    sr += ar[q] * c[e] - ai[q] * sn[e];
                    si += ar[q] * sn[e] + ai[q] * c[e];
                }
                yr[j + m * p] = sr;
                yi[j + m * p] = si;
            }
        }
        re.swap(yr);
        im.swap(yi);
        p *= R;
    }
}

}  // namespace

// Spectrum of a K x K PSF wrapped onto Ly x Lx with its centre at the origin,
// scaled by 1 / (Ly Lx): columns 0 .. Lc-1, each column's Ly values
// contiguous (out[x * Ly + y]), the order in which a warp of the column
// kernels reads them.
void psf_spectrum(const float *psf, int K, int Ly, int Lx, int Lc, std::vector<float2> &out) {
    const int R = (K - 1) / 2;
    std::vector<double> re(static_cast<size_t>(Ly) * Lx, 0.0), im(static_cast<size_t>(Ly) * Lx, 0.0);
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            const int y = ((i - R) % Ly + Ly) % Ly, x = ((j - R) % Lx + Lx) % Lx;
            re[static_cast<size_t>(y) * Lx + x] += psf[i * K + j];
        }
    std::vector<double> r(Lx), m(Lx);
    for (int y = 0; y < Ly; ++y) {       // rows
        for (int x = 0; x < Lx; ++x) {
            r[x] = re[static_cast<size_t>(y) * Lx + x];
            m[x] = im[static_cast<size_t>(y) * Lx + x];
        }
        host_fft(r, m, Lx, -1);
        for (int x = 0; x < Lx; ++x) {
            re[static_cast<size_t>(y) * Lx + x] = r[x];
            im[static_cast<size_t>(y) * Lx + x] = m[x];
        }
    }
    std::vector<double> cr(Ly), ci(Ly);
    out.assign(static_cast<size_t>(Lc) * Ly, make_float2(0.f, 0.f));
    const double scale = 1.0 / (static_cast<double>(Ly) * Lx);
    for (int x = 0; x < Lc; ++x) {       // columns
        for (int y = 0; y < Ly; ++y) {
            cr[y] = re[static_cast<size_t>(y) * Lx + x];
            ci[y] = im[static_cast<size_t>(y) * Lx + x];
        }
        host_fft(cr, ci, Ly, -1);
        for (int y = 0; y < Ly; ++y)
            out[static_cast<size_t>(x) * Ly + y] =
                make_float2(static_cast<float>(cr[y] * scale), static_cast<float>(ci[y] * scale));
    }
}

cudaError_t launch_iteration(const FftArgs &a, int sms, cudaStream_t s) {
    cudaError_t e;
    if ((e = launch_rows(0, a, sms, s)) != cudaSuccess || (e = launch_cols(0, a, sms, s)) != cudaSuccess ||
        (e = launch_rows(1, a, sms, s)) != cudaSuccess || (e = launch_cols(1, a, sms, s)) != cudaSuccess ||
        (e = launch_rows(2, a, sms, s)) != cudaSuccess)
        return e;
    count_launch(5);
    return cudaSuccess;
}

}  // namespace fftr
}  // namespace mvd
