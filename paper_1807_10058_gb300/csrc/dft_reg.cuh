// Small DFTs held entirely in registers, fully unrolled at compile time.
//
//   Dft<R, S>::run(re, im):  X[k] = sum_a x[a] exp(S * 2 pi i a k / R),  S = +1 or -1,
//
// in natural order in and out.  Composite lengths use one Cooley-Tukey
// split R = R1 * R2 (a = a2 + R2 a1, k = k1 + R1 k2) with the twiddles as
// compile-time constants; prime lengths use the direct sum.  The constants
// cos/sin(2 pi m / R) are evaluated at compile time from their Taylor series
// in double precision (no math-library call).
#pragma once

#if defined(__CUDACC__)
#define FCC_HD __host__ __device__ __forceinline__
#else
#define FCC_HD inline
#endif

namespace fcc {
namespace reg {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// sin(x) and cos(x) for |x| <= pi/4 by Taylor series (terms up to x^27).
constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}

// cos and sin of 2 pi m / R, reduced by octant so the series argument stays
// within pi/4 (exact symmetries of the circle).
constexpr void unit_root(long m, long R, double& c, double& s) {
    m %= R;
    if (m < 0) m += R;
    // angle = 2 pi m / R = (pi/4) * (8 m / R); octant o = floor(8m/R)
    const long o = (8 * m) / R;
    const double frac = (double)(8 * m - o * R) / (double)R;  // in [0, 1)
    const double t = frac * (kTwoPi / 8.0);                    // in [0, pi/4)
    const double st = taylor_sin(t), ct = taylor_cos(t);
    const double u = kTwoPi / 8.0 - t;                         // complementary angle
    const double su = taylor_sin(u), cu = taylor_cos(u);
    switch (o) {
        case 0: c = ct; s = st; break;
        case 1: c = su; s = cu; break;
        case 2: c = -st; s = ct; break;
        case 3: c = -cu; s = su; break;
        case 4: c = -ct; s = -st; break;
        case 5: c = -su; s = -cu; break;
        case 6: c = st; s = -ct; break;
        default: c = cu; s = -su; break;
    }
}
constexpr double root_cos(long m, long R) { double c = 0, s = 0; unit_root(m, R, c, s); return c; }
constexpr double root_sin(long m, long R) { double c = 0, s = 0; unit_root(m, R, c, s); return s; }

constexpr int smallest_factor(int R) {
    for (int p = 2; p * p <= R; ++p)
        if (R % p == 0) return p;
    return R;
}
// split of a composite length: prefer 4, then the smallest prime factor
constexpr int split_of(int R) {
    return (R % 4 == 0 && R > 4) ? 4 : smallest_factor(R);
}

// multiply (xr, xi) by exp(S 2 pi i m / R), a compile-time constant
template <long M, long R, int S, typename T>
FCC_HD void twiddle(T& xr, T& xi) {
    constexpr long m = ((M % R) + R) % R;
    if constexpr (m == 0) {
        return;
    } else if constexpr (4 * m == R) {          // S i
        const T t = xr;
        xr = -T(S) * xi;
        xi = T(S) * t;
    } else if constexpr (2 * m == R) {          // -1
        xr = -xr;
        xi = -xi;
    } else if constexpr (4 * m == 3 * R) {      // -S i
        const T t = xr;
        xr = T(S) * xi;
        xi = -T(S) * t;
    } else {
        constexpr T c = T(root_cos(m, R));
        constexpr T s = T(S) * T(root_sin(m, R));
        const T t = xr * c - xi * s;
        xi = xr * s + xi * c;
        xr = t;
    }
}

template <int R, int S, typename T, int Split = split_of(R)>
struct Dft;

// direct sum for prime lengths (and the split-free base cases)
template <int R, int S, typename T>
struct DftDirect {
    FCC_HD static void run(T* re, T* im) {
        T outr[R], outi[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            outr[k] = re[0];
            outi[k] = im[0];
        }
        run_terms<1>(re, im, outr, outi);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            re[k] = outr[k];
            im[k] = outi[k];
        }
    }
    template <int A>
    FCC_HD static void run_terms(const T* re, const T* im, T* outr, T* outi) {
        if constexpr (A < R) {
            add_k<A, 0>(re, im, outr, outi);
            run_terms<A + 1>(re, im, outr, outi);
        }
    }
    template <int A, int K>
    FCC_HD static void add_k(const T* re, const T* im, T* outr, T* outi) {
        if constexpr (K < R) {
            T xr = re[A], xi = im[A];
            twiddle<(long)A * K, R, S>(xr, xi);
            outr[K] += xr;
            outi[K] += xi;
            add_k<A, K + 1>(re, im, outr, outi);
        }
    }
};

template <int S, typename T>
struct Dft<1, S, T, 1> {
    FCC_HD static void run(T*, T*) {}
};

template <int S, typename T>
struct Dft<2, S, T, 2> {
    FCC_HD static void run(T* re, T* im) {
        const T ar = re[0], ai = im[0];
        re[0] = ar + re[1];
        im[0] = ai + im[1];
        re[1] = ar - re[1];
        im[1] = ai - im[1];
    }
};

template <int S, typename T>
struct Dft<4, S, T, 2> {
    FCC_HD static void run(T* re, T* im) {
        const T ar = re[0] + re[2], ai = im[0] + im[2];
        const T br = re[0] - re[2], bi = im[0] - im[2];
        const T cr = re[1] + re[3], ci = im[1] + im[3];
        const T dr = re[1] - re[3], di = im[1] - im[3];
        re[0] = ar + cr;
        im[0] = ai + ci;
        re[2] = ar - cr;
        im[2] = ai - ci;
        // X1 = b + S i d, X3 = b - S i d
        re[1] = br - T(S) * di;
        im[1] = bi + T(S) * dr;
        re[3] = br + T(S) * di;
        im[3] = bi - T(S) * dr;
    }
};

// prime (or otherwise unsplit) length
template <int R, int S, typename T>
struct Dft<R, S, T, R> : DftDirect<R, S, T> {};

// Cooley-Tukey split R = R1 * R2, a = a2 + R2 a1, k = k1 + R1 k2
template <int R, int S, typename T, int R1>
struct Dft {
    static constexpr int R2 = R / R1;
    FCC_HD static void run(T* re, T* im) {
        T yr[R2][R1], yi[R2][R1];
#pragma unroll
        for (int a2 = 0; a2 < R2; ++a2) {
#pragma unroll
            for (int a1 = 0; a1 < R1; ++a1) {
                yr[a2][a1] = re[a2 + R2 * a1];
                yi[a2][a1] = im[a2 + R2 * a1];
            }
            Dft<R1, S, T>::run(yr[a2], yi[a2]);
        }
        apply_twiddles<1, 1>(yr, yi);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            T zr[R2], zi[R2];
#pragma unroll
            for (int a2 = 0; a2 < R2; ++a2) {
                zr[a2] = yr[a2][k1];
                zi[a2] = yi[a2][k1];
            }
            Dft<R2, S, T>::run(zr, zi);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                re[k1 + R1 * k2] = zr[k2];
                im[k1 + R1 * k2] = zi[k2];
            }
        }
    }
    template <int A2, int K1>
    FCC_HD static void apply_twiddles(T (&yr)[R2][R1], T (&yi)[R2][R1]) {
        if constexpr (A2 < R2) {
            if constexpr (K1 < R1) {
                twiddle<(long)A2 * K1, R, S>(yr[A2][K1], yi[A2][K1]);
                apply_twiddles<A2, K1 + 1>(yr, yi);
            } else {
                apply_twiddles<A2 + 1, 1>(yr, yi);
            }
        }
    }
};

}  // namespace reg
}  // namespace fcc
