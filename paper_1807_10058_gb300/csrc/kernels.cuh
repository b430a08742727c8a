// CUDA kernels of the FCC cosine transform, generic (any supported order).
//
//   orbit_mix_kernel  -- the block-diagonal orbit mixing S, S^{-1} or S^H of
//                        the factorisation DCT_n = F S (see plan.h), one
//                        thread per W-orbit, 24 slots per thread.
//   fft_axis_kernel   -- length-n DFT along one axis of every volume
//                        (Stockham autosort in shared memory, mixed radix).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fcc {

static __constant__ int c_W[24][9];  // group matrices, row-major
static __constant__ int c_u[24][3];  // W_g^T (1,0,3)

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

enum { MODE_FWD = 0, MODE_INV = 1, MODE_ADJ = 2 };

template <typename T>
struct MixArgs {
    const uint32_t* reps;       // [n_orbits]
    const uint8_t* cls;         // [n_orbits]
    const T* mats;              // [n_classes][24][24][2] (re, im) for this mode
    const int8_t* wrap;         // [n_classes][24][3]
    const uint32_t* canon_mask; // [n_classes]
    const T* phase;             // [M][2]: exp(2 pi i e / M), M = d n for the shift c = v / d
    int u[24][3];               // W_h^T v: the row-phase exponent of slot h is u_h . kO mod M
    int M;
    int n;
    int64_t n_orbits;
    int64_t n3;                 // points per volume
    T scale;
};

// One thread per orbit.  FWD: Z[kappa_g] = scale * R_g * sum_h M[g][h] x[kappa_h]
// INV/ADJ: x[kappa_h] = scale * sum_g M[h][g] conj(R_g) Z[kappa_g].
template <typename T, int MODE, bool RIN, bool ROUT>
__global__ void __launch_bounds__(128) orbit_mix_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                        MixArgs<T> a) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= a.n_orbits) return;
    const int64_t vol = blockIdx.y;
    const uint32_t rp = a.reps[o];
    const int k0 = rp & 1023, k1 = (rp >> 10) & 1023, k2 = (rp >> 20) & 1023;
    const int c = a.cls[o];
    const int8_t* wr = a.wrap + c * 72;
    const uint32_t cm = a.canon_mask[c];
    const T* M = a.mats + (size_t)c * 1152;
    const int n = a.n;
    const int PM = a.M;   // phase-table length d n
    int idx[24];
    int ph[24];
#pragma unroll
    for (int h = 0; h < 24; ++h) {
        const int p0 = c_W[h][0] * k0 + c_W[h][1] * k1 + c_W[h][2] * k2 - n * wr[3 * h + 0];
        const int p1 = c_W[h][3] * k0 + c_W[h][4] * k1 + c_W[h][5] * k2 - n * wr[3 * h + 1];
        const int p2 = c_W[h][6] * k0 + c_W[h][7] * k1 + c_W[h][8] * k2 - n * wr[3 * h + 2];
        idx[h] = (p0 * n + p1) * n + p2;
        int e = (a.u[h][0] * k0 + a.u[h][1] * k1 + a.u[h][2] * k2) % PM;
        ph[h] = e < 0 ? e + PM : e;
    }
    if (MODE == MODE_FWD) {
        const T* src = in + vol * a.n3 * (RIN ? 1 : 2);
        T xr[24], xi[24];
#pragma unroll
        for (int h = 0; h < 24; ++h) {
            if (RIN) {
                xr[h] = src[idx[h]];
                xi[h] = T(0);
            } else {
                xr[h] = src[2 * (int64_t)idx[h]];
                xi[h] = src[2 * (int64_t)idx[h] + 1];
            }
        }
        T* dst = out + vol * a.n3 * 2;
#pragma unroll
        for (int g = 0; g < 24; ++g) {
            if (!((cm >> g) & 1u)) continue;
            T ar = T(0), ai = T(0);
#pragma unroll
            for (int h = 0; h < 24; ++h) {
                const T mr = __ldg(M + 2 * (g * 24 + h)), mi = __ldg(M + 2 * (g * 24 + h) + 1);
                ar = fma(mr, xr[h], ar);
                ai = fma(mi, xr[h], ai);
                if (!RIN) {
                    ar = fma(-mi, xi[h], ar);
                    ai = fma(mr, xi[h], ai);
                }
            }
            const T rr = __ldg(a.phase + 2 * ph[g]), ri = __ldg(a.phase + 2 * ph[g] + 1);
            dst[2 * (int64_t)idx[g]] = a.scale * (rr * ar - ri * ai);
            dst[2 * (int64_t)idx[g] + 1] = a.scale * (rr * ai + ri * ar);
        }
    } else {
        const T* src = in + vol * a.n3 * 2;
        T tr[24], ti[24];
#pragma unroll
        for (int g = 0; g < 24; ++g) {
            if ((cm >> g) & 1u) {
                const T zr = src[2 * (int64_t)idx[g]], zi = src[2 * (int64_t)idx[g] + 1];
                const T rr = __ldg(a.phase + 2 * ph[g]), ri = __ldg(a.phase + 2 * ph[g] + 1);
                tr[g] = rr * zr + ri * zi;  // conj(R) * Z
                ti[g] = rr * zi - ri * zr;
            } else {
                tr[g] = T(0);
                ti[g] = T(0);
            }
        }
        T* dst = out + vol * a.n3 * (ROUT ? 1 : 2);
#pragma unroll
        for (int h = 0; h < 24; ++h) {
            if (!((cm >> h) & 1u)) continue;
            T ar = T(0), ai = T(0);
#pragma unroll
            for (int g = 0; g < 24; ++g) {
                const T mr = __ldg(M + 2 * (h * 24 + g)), mi = __ldg(M + 2 * (h * 24 + g) + 1);
                ar = fma(mr, tr[g], ar);
                ar = fma(-mi, ti[g], ar);
                if (!ROUT) {
                    ai = fma(mr, ti[g], ai);
                    ai = fma(mi, tr[g], ai);
                }
            }
            if (ROUT) {
                dst[idx[h]] = a.scale * ar;
            } else {
                dst[2 * (int64_t)idx[h]] = a.scale * ar;
                dst[2 * (int64_t)idx[h] + 1] = a.scale * ai;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// DFT along one axis.  X[k] = sum_j x[j] exp(sign * 2 pi i j k / n).
// ---------------------------------------------------------------------------

constexpr int kMaxStages = 12;

struct FftArgs {
    int n;
    int nstages;
    int radix[kMaxStages];
    int axis;      // 0: slowest (stride n^2), 1: middle (stride n), 2: fastest
    int P;         // pencils per block
    int64_t nvol;
    int64_t vstride;   // complex values from one volume to the next (>= n^3)
    int sign;      // +1 or -1
};

template <typename T>
__device__ __forceinline__ void cmul(T ar, T ai, T br, T bi, T& cr, T& ci) {
    cr = ar * br - ai * bi;
    ci = ar * bi + ai * br;
}

// One radix-R Stockham stage over all pencils of the block.
template <typename T, int R>
__device__ __forceinline__ void fft_stage(const T* __restrict__ src, T* __restrict__ dst,
                                          const T* __restrict__ tw, int n, int P, int Ns,
                                          int sign, int pstride) {
    const int m = n / R;
    const int twstep = n / (Ns * R);  // twiddle index unit: exp(2 pi i k q / (Ns R))
    const int rstep = n / R;          // exp(2 pi i / R) = tw[n/R]
    for (int i = threadIdx.x; i < P * m; i += blockDim.x) {
        const int p = i / m;
        const int t = i - p * m;
        const int k = t % Ns;
        T vr[R], vi[R];
        const T* s = src + 2 * (p * pstride);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            vr[q] = s[2 * (t + q * m)];
            vi[q] = s[2 * (t + q * m) + 1];
        }
#pragma unroll
        for (int q = 1; q < R; ++q) {
            const int e = (q * k * twstep) % n;
            const T wr = tw[2 * e], wi = sign * tw[2 * e + 1];
            T xr, xi;
            cmul(vr[q], vi[q], wr, wi, xr, xi);
            vr[q] = xr;
            vi[q] = xi;
        }
        T Vr[R], Vi[R];
        if (R == 2) {
            Vr[0] = vr[0] + vr[1]; Vi[0] = vi[0] + vi[1];
            Vr[1] = vr[0] - vr[1]; Vi[1] = vi[0] - vi[1];
        } else if (R == 4) {
            const T ar = vr[0] + vr[2], ai = vi[0] + vi[2];
            const T br = vr[0] - vr[2], bi = vi[0] - vi[2];
            const T cr = vr[1] + vr[3], ci = vi[1] + vi[3];
            const T dr = vr[1] - vr[3], di = vi[1] - vi[3];
            // j = sign * i ; X1 = b + j d, X3 = b - j d
            Vr[0] = ar + cr; Vi[0] = ai + ci;
            Vr[2] = ar - cr; Vi[2] = ai - ci;
            Vr[1] = br - sign * di; Vi[1] = bi + sign * dr;
            Vr[3] = br + sign * di; Vi[3] = bi - sign * dr;
        } else {
#pragma unroll
            for (int pp = 0; pp < R; ++pp) {
                T ar = vr[0], ai = vi[0];
#pragma unroll
                for (int q = 1; q < R; ++q) {
                    const int e = ((pp * q) % R) * rstep;
                    const T wr = tw[2 * e], wi = sign * tw[2 * e + 1];
                    ar += vr[q] * wr - vi[q] * wi;
                    ai += vr[q] * wi + vi[q] * wr;
                }
                Vr[pp] = ar;
                Vi[pp] = ai;
            }
        }
        const int base = (t / Ns) * Ns * R + k;
        T* d = dst + 2 * (p * pstride);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            d[2 * (base + q * Ns)] = Vr[q];
            d[2 * (base + q * Ns) + 1] = Vi[q];
        }
    }
}

template <typename T>
__device__ __forceinline__ int64_t fft_global_index(const FftArgs& a, int64_t tile, int p, int e, bool& ok) {
    const int n = a.n;
    const int64_t n2 = (int64_t)n * n;
    if (a.axis == 2) {
        const int64_t row = tile * a.P + p;
        ok = row < a.nvol * n2;
        const int64_t vol = row / n2;
        return vol * a.vstride + (row - vol * n2) * n + e;
    }
    const int ctiles = (n + a.P - 1) / a.P;
    const int64_t vol = tile / ((int64_t)n * ctiles);
    const int64_t rem = tile - vol * n * ctiles;
    const int fixed = (int)(rem / ctiles);
    const int c = (int)(rem % ctiles) * a.P + p;
    ok = c < n;
    if (a.axis == 1) return vol * a.vstride + ((int64_t)fixed * n + e) * n + c;
    return vol * a.vstride + ((int64_t)e * n + fixed) * n + c;
}

template <typename T>
__global__ void __launch_bounds__(256) fft_axis_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                       const T* __restrict__ twg, FftArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int n = a.n;
    const int P = a.P;
    const int pstride = n + 1;
    T* buf0 = sm;
    T* buf1 = sm + 2 * P * pstride;
    T* tw = sm + 4 * P * pstride;
    for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) tw[j] = twg[j];
    const int64_t tile = blockIdx.x;
    const int total = P * n;
    for (int j = threadIdx.x; j < total; j += blockDim.x) {
        int p, e;
        if (a.axis == 2) { p = j / n; e = j - p * n; }
        else { e = j / P; p = j - e * P; }
        bool ok;
        const int64_t g = fft_global_index<T>(a, tile, p, e, ok);
        T vr = T(0), vi = T(0);
        if (ok) { vr = in[2 * g]; vi = in[2 * g + 1]; }
        buf0[2 * (p * pstride + e)] = vr;
        buf0[2 * (p * pstride + e) + 1] = vi;
    }
    __syncthreads();
    T* src = buf0;
    T* dst = buf1;
    int Ns = 1;
    for (int s = 0; s < a.nstages; ++s) {
        const int R = a.radix[s];
        switch (R) {
            case 2: fft_stage<T, 2>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 3: fft_stage<T, 3>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 4: fft_stage<T, 4>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 5: fft_stage<T, 5>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 7: fft_stage<T, 7>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 11: fft_stage<T, 11>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 13: fft_stage<T, 13>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 17: fft_stage<T, 17>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 19: fft_stage<T, 19>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 23: fft_stage<T, 23>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 29: fft_stage<T, 29>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            case 31: fft_stage<T, 31>(src, dst, tw, n, P, Ns, a.sign, pstride); break;
            default: break;  // rejected on the host
        }
        __syncthreads();
        T* t = src; src = dst; dst = t;
        Ns *= R;
    }
    for (int j = threadIdx.x; j < total; j += blockDim.x) {
        int p, e;
        if (a.axis == 2) { p = j / n; e = j - p * n; }
        else { e = j / P; p = j - e * P; }
        bool ok;
        const int64_t g = fft_global_index<T>(a, tile, p, e, ok);
        if (ok) {
            out[2 * g] = src[2 * (p * pstride + e)];
            out[2 * g + 1] = src[2 * (p * pstride + e) + 1];
        }
    }
}

}  // namespace fcc
