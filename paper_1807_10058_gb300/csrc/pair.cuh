// Pairing of two real volumes through the conjugate symmetry of DCT_n.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fcc {

// --- pairing of two real volumes ------------------------------------------
//
// For real x the rows of DCT_n come in conjugate pairs: (D x)[pi(i,l,q)] =
// conj((D x)[i,l,q]) with pi(i,l,q) = (i-l, -l, q-l) mod n, an involution.
// Hence one complex transform Y = D (x1 + i x2) gives
//   D x1 = (Y + conj(Y o pi)) / 2,   D x2 = (Y - conj(Y o pi)) / (2i),
// and with P(v) = (v + conj(v o pi)) / 2 one has Re(D^-1 v) = D^-1 P(v) and
// Re(D^H v) = D^H P(v), so P(v1) + i P(v2) pairs the inverse and adjoint.

// Threads enumerate (i, l, q) with 0 <= l <= n/2; each handles one point a
// and its partner b = pi(a) (a alone when l = 0, only i < n/2 when 2l = n).
__device__ __forceinline__ bool pair_point(int64_t t, int n, int& a, int& b) {
    const int q = (int)(t % n);
    const int i = (int)((t / n) % n);
    const int l = (int)(t / ((int64_t)n * n));
    if (2 * l == n && i >= n / 2) return false;
    a = (i * n + l) * n + q;
    const int i2 = (i - l + n) % n, l2 = (n - l) % n, q2 = (q - l + n) % n;
    b = (i2 * n + l2) * n + q2;
    return true;
}

// Y (complex) at volume 2p of y -> D x1 into volume 2p, D x2 into 2p+1.
__global__ void pair_split_kernel(float2* y, int n, int64_t n3, int64_t per_pair) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= per_pair) return;
    int a, b;
    if (!pair_point(t, n, a, b)) return;
    float2* Y = y + (int64_t)blockIdx.y * 2 * n3;
    float2* Y2 = Y + n3;
    const float2 ya = Y[a], yb = Y[b];
    // y1[a] = (ya + conj(yb))/2, y2[a] = (ya - conj(yb))/(2i) = -i (ya - conj(yb))/2
    const float2 s1a = make_float2(0.5f * (ya.x + yb.x), 0.5f * (ya.y - yb.y));
    const float2 d1a = make_float2(0.5f * (ya.x - yb.x), 0.5f * (ya.y + yb.y));
    const float2 s1b = make_float2(s1a.x, -s1a.y);                    // (yb + conj(ya))/2 = conj(s1a)
    const float2 d1b = make_float2(-d1a.x, d1a.y);                    // (yb - conj(ya))/2 = -conj(d1a)
    Y[a] = s1a;
    Y[b] = s1b;
    Y2[a] = make_float2(d1a.y, -d1a.x);
    Y2[b] = make_float2(d1b.y, -d1b.x);
}

// v1, v2 (complex, volumes 2p and 2p+1 of y) -> W = P(v1) + i P(v2) at
// volume p of w.
__global__ void pair_merge_kernel(const float2* __restrict__ y, float2* __restrict__ w, int n, int64_t n3,
                                  int64_t per_pair) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= per_pair) return;
    int a, b;
    if (!pair_point(t, n, a, b)) return;
    const float2* V1 = y + (int64_t)blockIdx.y * 2 * n3;
    const float2* V2 = V1 + n3;
    float2* W = w + (int64_t)blockIdx.y * n3;
    const float2 pa = V1[a], pb = V1[b], qa = V2[a], qb = V2[b];
    const float2 P1 = make_float2(0.5f * (pa.x + pb.x), 0.5f * (pa.y - pb.y));   // P(v1)[a]
    const float2 P2 = make_float2(0.5f * (qa.x + qb.x), 0.5f * (qa.y - qb.y));   // P(v2)[a]
    // W[a] = P1 + i P2 ; W[b] = conj(P1) + i conj(P2)
    W[a] = make_float2(P1.x - P2.y, P1.y + P2.x);
    W[b] = make_float2(P1.x + P2.y, -P1.y + P2.x);
}

// --- Hermitian-packed layout of real-input transforms ----------------------
//
// For real x the n^3 complex values y = D x are determined by n^3 reals: on
// each pair {a, pi(a)} y[pi(a)] = conj(y[a]), and at the fixed points of pi
// (the row l = 0) y is real.  The packed volume stores, at every point
// a = (i, l, q),
//   Re y[a]   if a is primary: 2l < n, or 2l = n and 2q < n (this includes
//             the fixed points, l = 0),
//   -Im y[a]  otherwise (= Im y at its primary partner pi(a)).
// Unpacking: at a primary a, y[a] = pk[a] + i pk[pi(a)] (l = 0: pk[a]); at
// any other point y[a] = pk[pi(a)] - i pk[a].  The fast DFT passes use the
// same split into primary and partner pencils (fft_pencil_pair_kernel,
// fft_pencil_merge_kernel).
__host__ __device__ __forceinline__ bool packed_primary(int l, int q, int n) {
    return 2 * l < n || (2 * l == n && 2 * q < n);
}

// complex y (nvol volumes of n^3) -> packed reals pk
template <typename T>
__global__ void pack_hermitian_kernel(const T* __restrict__ y, T* __restrict__ pk, int n, int64_t total) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int q = (int)(t % n);
    const int l = (int)((t / n) % n);
    pk[t] = packed_primary(l, q, n) ? y[2 * t] : -y[2 * t + 1];
}

// packed reals pk -> complex y (nvol volumes of n^3)
template <typename T>
__global__ void unpack_hermitian_kernel(const T* __restrict__ pk, T* __restrict__ y, int n, int64_t total) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t r = t % n3, vb = t - r;
    const int q = (int)(r % n);
    const int l = (int)((r / n) % n);
    const int i = (int)(r / ((int64_t)n * n));
    const int i2 = (i - l + n) % n, l2 = (n - l) % n, q2 = (q - l + n) % n;
    const T own = pk[t], other = pk[vb + ((int64_t)i2 * n + l2) * n + q2];
    if (packed_primary(l, q, n)) {
        y[2 * t] = own;
        y[2 * t + 1] = l == 0 ? T(0) : other;
    } else {
        y[2 * t] = other;
        y[2 * t + 1] = -own;
    }
}

}  // namespace fcc
