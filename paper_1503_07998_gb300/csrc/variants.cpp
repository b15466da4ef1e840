// Correlation kernels X_v of the multi-view RL variants (Supp. Note 2 sec. 1).
//
// Every variant keeps the update psi <- psi * prod_v [(phi_v / (psi * P_v)) * X_v]
// and differs only in the kernel the ratio of view v is convolved with:
//   independent          X_v = P_v^*
//   efficient Bayesian   X_v = P_v^* . prod_{w != v} (P_v^* * P_w * P_w^*)
//   optimization I       X_v = P_v^* . prod_{w != v} (P_v^* * P_w)
//   optimization II      X_v = P_v^* . prod_{w != v} P_w^*
// where '.' multiplies kernels entry by entry over the K x K support of P_v^*,
// '*' is a convolution of two K x K kernels cropped to the K x K centre, and
// every X_v is scaled to unit sum.  Built once per PSF set on the host in
// FP64; the device only ever sees the separable factors of flip(X_v).
#include <cstddef>
#include <vector>

#include "mvd.h"
#include "mvd_internal.h"

namespace mvd {

namespace {

// out[i][j] = sum_{a,b} A[a][b] B[i+R-a][j+R-b] over in-range indices: the
// full (2K-1)^2 convolution of two K x K kernels, centre K x K window.
void conv_centre(const double *A, const double *B, int K, double *out) {
    const int R = (K - 1) / 2;
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
            for (int a = 0; a < K; ++a) {
                const int m = i + R - a;
                if (m < 0 || m >= K) continue;
                for (int b = 0; b < K; ++b) {
                    const int n = j + R - b;
                    if (n < 0 || n >= K) continue;
                    s += A[a * K + b] * B[m * K + n];
                }
            }
            out[i * K + j] = s;
        }
    }
}

}  // namespace

void variant_kernels(const float *psfs, int views, int K, int variant, double *X) {
    const size_t KK = static_cast<size_t>(K) * K;
    std::vector<double> P(KK * views), F(KK * views), t1(KK), t2(KK);
    for (int v = 0; v < views; ++v) {
        for (int i = 0; i < K; ++i) {
            for (int j = 0; j < K; ++j) {
                const double p = psfs[KK * v + static_cast<size_t>(i) * K + j];
                P[KK * v + static_cast<size_t>(i) * K + j] = p;
                F[KK * v + static_cast<size_t>(K - 1 - i) * K + (K - 1 - j)] = p;   // P_v^*
            }
        }
    }
    for (int v = 0; v < views; ++v) {
        double *x = X + KK * v;
        const double *Fv = F.data() + KK * v;
        for (size_t i = 0; i < KK; ++i) x[i] = Fv[i];
        for (int w = 0; w < views && variant != MVD_VARIANT_INDEPENDENT; ++w) {
            if (w == v) continue;
            const double *Pw = P.data() + KK * w, *Fw = F.data() + KK * w;
            const double *factor = Fw;                 // optimization II
            if (variant == MVD_VARIANT_OPTIMIZATION_1) {
                conv_centre(Fv, Pw, K, t1.data());
                factor = t1.data();
            } else if (variant == MVD_VARIANT_EFFICIENT_BAYESIAN) {
                conv_centre(Fv, Pw, K, t1.data());
                conv_centre(t1.data(), Fw, K, t2.data());
                factor = t2.data();
            }
            for (size_t i = 0; i < KK; ++i) x[i] *= factor[i];
        }
        double sum = 0.0;
        for (size_t i = 0; i < KK; ++i) sum += x[i];
        if (sum > 0.0)
            for (size_t i = 0; i < KK; ++i) x[i] /= sum;
    }
}

}  // namespace mvd
