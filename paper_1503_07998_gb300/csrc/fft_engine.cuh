// Warp-level mixed-radix Stockham FFT for the Fourier route (Supp. Note 2
// sec. 4: the convolutions of the update are products of spectra).
//
// One warp owns one transform of length N held in shared memory (two
// ping-pong buffers).  N is split into a few stages of composite radix R
// (2 .. 40, products of 2, 3, 4 and 5; the host's list in fft.cu); a stage is one pass over the buffer:
// every lane takes whole butterflies, reads R inputs, multiplies them by the
// stage's twiddles (a per-stage table laid out so that the lanes of a warp hit
// distinct banks), runs an R-point DFT in registers and writes R outputs.
// The R-point DFTs are nested Cooley-Tukey splits R = R1 * R2 down to 2, 3, 4
// and 5 points; their inner twiddles are compile-time constants.  Stages of
// one transform are separated by __syncwarp only.
//
// Stockham stage with radix R after stages whose radices multiply to p
// (M = N / R butterflies, k = i mod p):
//   a_q = x[i + q M] * w_N^(q k N / (p R))      q = 0 .. R-1
//   y[(i - k) R + k + m p] = sum_q a_q w_R^(q m)  m = 0 .. R-1
// with w_L = exp(-2 pi i / L) forward and exp(+2 pi i / L) inverse.
#pragma once

#include <cuda_runtime.h>

#include "mvd_internal.h"

namespace mvd {
namespace fftr {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// -i*d (forward) or +i*d (inverse): d times w_4
template <bool INV>
__device__ __forceinline__ float2 rot(float2 d) {
    return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
}

// cos and sin of 2 pi e / R at compile time: Taylor series on the angle
// reduced to [-pi, pi] (30 terms are far below double rounding there).
constexpr double kPi = 3.14159265358979323846;
__host__ __device__ constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 30; ++n) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n < 30; ++n) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double root_angle(int R, int e) {   // 2 pi e / R reduced to (-pi, pi]
    const int m = ((e % R) + R) % R;
    const int s = 2 * m > R ? m - R : m;
    return 2.0 * kPi * s / R;
}

// v * w_R^E (forward) or v * conj(w_R^E)... i.e. v * exp(-+2 pi i E / R)
template <int R, int E, bool INV>
__device__ __forceinline__ float2 twc(float2 v) {
    constexpr int e = E % R;
    if constexpr (e == 0) {
        return v;
    } else if constexpr (2 * e == R) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (4 * e == R) {
        return rot<INV>(v);
    } else if constexpr (4 * e == 3 * R) {
        return rot<!INV>(v);
    } else {
        constexpr float c = static_cast<float>(taylor_cos(root_angle(R, e)));
        constexpr float s = static_cast<float>(INV ? taylor_sin(root_angle(R, e)) : -taylor_sin(root_angle(R, e)));
        return make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
    }
}

template <int V> struct IC { static constexpr int value = V; };
template <int B, int E, class F>
__device__ __forceinline__ void sfor(F &&f) {
    if constexpr (B < E) {
        f(IC<B>{});
        sfor<B + 1, E>(f);
    }
}

template <int R> struct Split {   // first factor of a composite R
    static constexpr int f = (R % 4 == 0 && R != 8) ? 4 : (R % 5 == 0 ? 5 : (R % 3 == 0 ? 3 : 2));
};

template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2 (&a)[2]) {
        const float2 s = cadd(a[0], a[1]), d = csub(a[0], a[1]);
        a[0] = s;
        a[1] = d;
    }
};
template <bool INV> struct Dft<3, INV> {
    __device__ __forceinline__ static void run(float2 (&a)[3]) {
        constexpr float s3 = 0.8660254037844386f;   // sin(2 pi / 3)
        const float2 t1 = cadd(a[1], a[2]);
        const float2 t2 = rot<INV>(csub(a[1], a[2]));
        const float2 m = make_float2(a[0].x - 0.5f * t1.x, a[0].y - 0.5f * t1.y);
        a[0] = cadd(a[0], t1);
        a[1] = make_float2(m.x + s3 * t2.x, m.y + s3 * t2.y);
        a[2] = make_float2(m.x - s3 * t2.x, m.y - s3 * t2.y);
    }
};
template <bool INV> struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2 (&a)[4]) {
        const float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
        const float2 s13 = cadd(a[1], a[3]), d13 = rot<INV>(csub(a[1], a[3]));
        a[0] = cadd(s02, s13);
        a[1] = cadd(d02, d13);
        a[2] = csub(s02, s13);
        a[3] = csub(d02, d13);
    }
};
template <bool INV> struct Dft<5, INV> {
    __device__ __forceinline__ static void run(float2 (&a)[5]) {
        constexpr float c1 = 0.30901699437494745f, c2 = -0.8090169943749475f;   // cos(2 pi/5), cos(4 pi/5)
        constexpr float s1 = 0.9510565162951535f, s2 = 0.5877852522924731f;     // sin(2 pi/5), sin(4 pi/5)
        const float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
        const float2 t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
        const float2 b1 = make_float2(a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y);
        const float2 b2 = make_float2(a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y);
        const float2 d1 = rot<INV>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
        const float2 d2 = rot<INV>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
        a[0] = cadd(a[0], cadd(t1, t2));
        a[1] = cadd(b1, d1);
        a[4] = csub(b1, d1);
        a[2] = cadd(b2, d2);
        a[3] = csub(b2, d2);
    }
};

// Composite R = R1 R2 (R1 = Split<R>::f): input index n = R2 n1 + n2, output
// index k = k1 + R1 k2;  X_k = sum_n2 w_R2^(n2 k2) [w_R^(n2 k1) sum_n1 x_n w_R1^(n1 k1)].
template <int R, bool INV> struct Dft {
    static constexpr int R1 = Split<R>::f, R2 = R / R1;
    __device__ __forceinline__ static void run(float2 (&a)[R]) {
        float2 b[R];
        sfor<0, R2>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            float2 t[R1];
            sfor<0, R1>([&](auto n1c) { t[decltype(n1c)::value] = a[R2 * decltype(n1c)::value + n2]; });
            Dft<R1, INV>::run(t);
            sfor<0, R1>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                b[R2 * k1 + n2] = twc<R, n2 * k1, INV>(t[k1]);
            });
        });
        sfor<0, R1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            float2 u[R2];
            sfor<0, R2>([&](auto n2c) { u[decltype(n2c)::value] = b[R2 * k1 + decltype(n2c)::value]; });
            Dft<R2, INV>::run(u);
            sfor<0, R2>([&](auto k2c) { a[k1 + R1 * decltype(k2c)::value] = u[decltype(k2c)::value]; });
        });
    }
};

// One stage over the warp's buffer x -> y.  st: radix, p, M and the offset of
// the stage's twiddles in `tw` (entries (q - 1) p + k = exp(+2 pi i q k / (p R))).
template <int R, bool INV>
__device__ __forceinline__ void stage(const float2 *__restrict__ x, float2 *__restrict__ y, const FftStage &st,
                                      const float2 *__restrict__ tw, int lane) {
    const int M = st.M, p = st.p;
    const float rp = st.rp;
    for (int i = lane; i < M; i += 32) {
        // i / p exactly: i < 2^16, and (i + 1/2) / p is at least 1/(2p) from an integer
        const int k = p == 1 ? 0 : i - p * __float2int_rz((static_cast<float>(i) + 0.5f) * rp);
        float2 a[R];
        sfor<0, R>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            a[q] = x[i + q * M];
        });
        if (p > 1) {
            const float2 *t = tw + st.tw_off + k;
            sfor<1, R>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                const float2 w = t[(q - 1) * p];
                a[q] = INV ? cmul(a[q], w) : cmulc(a[q], w);
            });
        }
        Dft<R, INV>::run(a);
        float2 *o = y + (i - k) * R + k;
        sfor<0, R>([&](auto mc) {
            constexpr int m = decltype(mc)::value;
            o[m * p] = a[m];
        });
    }
}

template <bool INV>
__device__ __forceinline__ void stage_any(const float2 *x, float2 *y, const FftStage &st, const float2 *tw,
                                          int lane) {
    switch (st.R) {
        case 2: stage<2, INV>(x, y, st, tw, lane); break;
        case 3: stage<3, INV>(x, y, st, tw, lane); break;
        case 4: stage<4, INV>(x, y, st, tw, lane); break;
        case 5: stage<5, INV>(x, y, st, tw, lane); break;
        case 6: stage<6, INV>(x, y, st, tw, lane); break;
        case 8: stage<8, INV>(x, y, st, tw, lane); break;
        case 9: stage<9, INV>(x, y, st, tw, lane); break;
        case 10: stage<10, INV>(x, y, st, tw, lane); break;
        case 12: stage<12, INV>(x, y, st, tw, lane); break;
        case 15: stage<15, INV>(x, y, st, tw, lane); break;
        case 16: stage<16, INV>(x, y, st, tw, lane); break;
        case 18: stage<18, INV>(x, y, st, tw, lane); break;
        case 20: stage<20, INV>(x, y, st, tw, lane); break;
        case 24: stage<24, INV>(x, y, st, tw, lane); break;
        case 25: stage<25, INV>(x, y, st, tw, lane); break;
        case 27: stage<27, INV>(x, y, st, tw, lane); break;
        case 30: stage<30, INV>(x, y, st, tw, lane); break;
        case 32: stage<32, INV>(x, y, st, tw, lane); break;
        case 36: stage<36, INV>(x, y, st, tw, lane); break;
        default: stage<40, INV>(x, y, st, tw, lane); break;
    }
}

// The warp's transform of x (scratch y); returns the buffer holding the result.
template <bool INV>
__device__ __forceinline__ float2 *fft_warp(float2 *x, float2 *y, const FftPlan1 &pl, const float2 *tw, int lane) {
    for (int s = 0; s < pl.nst; ++s) {
        stage_any<INV>(x, y, pl.st[s], tw, lane);
        __syncwarp();
        float2 *t = x;
        x = y;
        y = t;
    }
    return x;
}

}  // namespace fftr
}  // namespace mvd
