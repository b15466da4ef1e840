// Host-side PSF analysis: an FP64 singular value decomposition of every
// view's K x K PSF, P = sum_q s_q u_q w_q^T, so that each 2D convolution of
// the RL update (Supp. Note 1) runs as a sum of vertical-then-horizontal 1D
// passes.  A sampled axis-aligned Gaussian (the PSFs of the paper's
// light-sheet views, Supp. Fig. 2 and 4) has one term; any PSF is exact with
// K terms.  Terms are dropped only while the dropped part stays below
// `rank_tol` of the PSF's Frobenius norm.
//
// The SVD is the one-sided Jacobi method (Hestenes): plane rotations of
// column pairs until all columns are mutually orthogonal; the column norms
// are then the singular values.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "mvd_internal.h"

namespace mvd {

namespace {

// A is K x K, column-major: A[i + K*j].  On return A's columns are s_j u_j and
// Vm's columns are the right singular vectors.
void jacobi_svd(std::vector<double> &A, std::vector<double> &Vm, int K) {
    Vm.assign(static_cast<size_t>(K) * K, 0.0);
    for (int i = 0; i < K; ++i) Vm[i + K * i] = 1.0;
    for (int sweep = 0; sweep < 80; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < K - 1; ++p) {
            for (int q = p + 1; q < K; ++q) {
                double alpha = 0, beta = 0, gamma = 0;
                for (int i = 0; i < K; ++i) {
                    const double ap = A[i + K * p], aq = A[i + K * q];
                    alpha += ap * ap;
                    beta += aq * aq;
                    gamma += ap * aq;
                }
                if (alpha == 0.0 || beta == 0.0) continue;
                const double rel = std::fabs(gamma) / std::sqrt(alpha * beta);
                off = std::max(off, rel);
                if (rel < 1e-15) continue;
                const double zeta = (beta - alpha) / (2.0 * gamma);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t);
                const double s = c * t;
                for (int i = 0; i < K; ++i) {
                    const double ap = A[i + K * p], aq = A[i + K * q];
                    A[i + K * p] = c * ap - s * aq;
                    A[i + K * q] = s * ap + c * aq;
                    const double vp = Vm[i + K * p], vq = Vm[i + K * q];
                    Vm[i + K * p] = c * vp - s * vq;
                    Vm[i + K * q] = s * vp + c * vq;
                }
            }
        }
        if (off < 1e-15) break;
    }
}

}  // namespace

int max_terms(int views, int K) { return 2 * views * K; }

namespace {

// Separable factors of one K x K kernel (row-major, FP64): on return r terms
// with kernel ~= sum_q u_q w_q^T, u_q (scaled by the singular value) in
// U[q*K .. q*K+K) and w_q in Wv likewise; r = 0 if the kernel is zero.
int factor_kernel(const double *kernel, int K, double rank_tol, std::vector<double> &U, std::vector<double> &Wv) {
    const size_t KK = static_cast<size_t>(K) * K;
    std::vector<double> A(KK), Vm;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) A[i + static_cast<size_t>(K) * j] = kernel[static_cast<size_t>(i) * K + j];
    jacobi_svd(A, Vm, K);
    std::vector<double> sig(K);
    for (int j = 0; j < K; ++j) {
        double s = 0;
        for (int i = 0; i < K; ++i) s += A[i + static_cast<size_t>(K) * j] * A[i + static_cast<size_t>(K) * j];
        sig[j] = std::sqrt(s);
    }
    std::vector<int> order(K);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return sig[a] > sig[b]; });
    double total = 0;
    for (double s : sig) total += s * s;
    if (!(total > 0)) return 0;
    // smallest r whose dropped tail is within tolerance
    int r = K;
    double tail = 0;
    for (int q = K - 1; q >= 0; --q) {
        const double s = sig[order[q]];
        if (rank_tol > 0) {
            if (std::sqrt(tail + s * s) <= rank_tol * std::sqrt(total)) {
                tail += s * s;
                r = q;
                continue;
            }
        } else if (s == 0.0) {
            r = q;
            continue;
        }
        break;
    }
    if (r < 1) r = 1;
    U.assign(static_cast<size_t>(r) * K, 0.0);
    Wv.assign(static_cast<size_t>(r) * K, 0.0);
    for (int q = 0; q < r; ++q) {
        const int j = order[q];
        for (int m = 0; m < K; ++m) {
            U[static_cast<size_t>(q) * K + m] = A[m + static_cast<size_t>(K) * j];
            Wv[static_cast<size_t>(q) * K + m] = Vm[m + static_cast<size_t>(K) * j];
        }
    }
    return r;
}

}  // namespace

bool factorise_psfs(const float *psfs, int views, int K, double rank_tol, FactorTable &ft,
                    float *taps_out, int taps_capacity, char *msg, size_t msg_len, const float *corr) {
    ft = FactorTable{};
    ft.K = K;
    ft.views = views;
    const size_t KK = static_cast<size_t>(K) * K;
    // blur groups: views whose PSFs are bitwise identical share one blur
    for (int v = 0; v < views; ++v) {
        int g = -1;
        for (int u = 0; u < v; ++u) {
            if (std::memcmp(psfs + KK * v, psfs + KK * u, KK * sizeof(float)) == 0) {
                g = ft.group[u];
                break;
            }
        }
        if (g < 0) {
            g = ft.n_groups++;
            ft.group_leader[g] = v;
        }
        ft.group[v] = g;
    }
    int off = 0;
    std::vector<double> kern(KK), U, Wv;
    auto reserve = [&](int r) {
        if ((off + r) * 4 * K > taps_capacity) {
            std::snprintf(msg, msg_len, "factor table overflow");
            return false;
        }
        return true;
    };
    for (int v = 0; v < views; ++v) {
        const int leader = ft.group_leader[ft.group[v]];
        if (leader != v) {            // identical PSF: reuse the leader's terms
            ft.rank[v] = ft.rank[leader];
            ft.tap_off[v] = ft.tap_off[leader];
            continue;
        }
        for (size_t i = 0; i < KK; ++i) kern[i] = psfs[KK * v + i];
        const int r = factor_kernel(kern.data(), K, rank_tol, U, Wv);
        if (r == 0) {
            std::snprintf(msg, msg_len, "PSF of view %d is zero", v);
            return false;
        }
        if (!reserve(r)) return false;
        ft.rank[v] = r;
        ft.tap_off[v] = off;
        for (int q = 0; q < r; ++q) {
            const double *u = U.data() + static_cast<size_t>(q) * K, *w = Wv.data() + static_cast<size_t>(q) * K;
            float *t = taps_out + static_cast<size_t>(off + q) * 4 * K;
            for (int m = 0; m < K; ++m) {
                t[0 * K + m] = static_cast<float>(u[K - 1 - m]);   // blur vertical
                t[1 * K + m] = static_cast<float>(w[K - 1 - m]);   // blur horizontal
                t[2 * K + m] = static_cast<float>(u[m]);           // correlation vertical
                t[3 * K + m] = static_cast<float>(w[m]);           // correlation horizontal
            }
        }
        off += r;
    }
    for (int v = 0; v < views; ++v) {
        ft.crank[v] = ft.rank[v];
        ft.ctap_off[v] = ft.tap_off[v];
    }
    // a variant's correlation kernels: terms of their own, correlation taps only
    for (int v = 0; corr && v < views; ++v) {
        for (size_t i = 0; i < KK; ++i) kern[i] = corr[KK * v + i];
        const int r = factor_kernel(kern.data(), K, rank_tol, U, Wv);
        if (r == 0) {
            std::snprintf(msg, msg_len, "correlation kernel of view %d is zero", v);
            return false;
        }
        if (!reserve(r)) return false;
        ft.crank[v] = r;
        ft.ctap_off[v] = off;
        for (int q = 0; q < r; ++q) {
            const double *u = U.data() + static_cast<size_t>(q) * K, *w = Wv.data() + static_cast<size_t>(q) * K;
            float *t = taps_out + static_cast<size_t>(off + q) * 4 * K;
            for (int m = 0; m < K; ++m) {
                t[0 * K + m] = 0.0f;
                t[1 * K + m] = 0.0f;
                t[2 * K + m] = static_cast<float>(u[m]);
                t[3 * K + m] = static_cast<float>(w[m]);
            }
        }
        off += r;
    }
    ft.total_terms = off;
    // short factors: the mass outside the short_tap_count(K) central taps is within the tolerance
    const int KS = short_tap_count(K);
    if (K > KS && rank_tol > 0) {
        const int OFF = (K - KS) / 2;
        auto trimmable = [&](int term, int kind) {
            const float *t = taps_out + static_cast<size_t>(term) * 4 * K + static_cast<size_t>(kind) * K;
            double all = 0, tail = 0;
            for (int m = 0; m < K; ++m) {
                all += std::fabs(t[m]);
                if (m < OFF || m >= OFF + KS) tail += std::fabs(t[m]);
            }
            return all > 0 && tail <= rank_tol * all;
        };
        for (int v = 0; v < views; ++v) {
            unsigned char mask = 0;
            for (int kind = 0; kind < 4; ++kind) {
                const int n = kind < 2 ? ft.rank[v] : ft.crank[v];
                const int t0 = kind < 2 ? ft.tap_off[v] : ft.ctap_off[v];
                bool ok = n > 0;
                for (int q = 0; q < n && ok; ++q) ok = trimmable(t0 + q, kind);
                if (ok) mask |= static_cast<unsigned char>(1u << kind);
            }
            ft.short_mask[v] = mask;
        }
    }
    return true;
}

}  // namespace mvd
