// Fast 3-D DFT passes for orders with a register-resident factorisation
// n = R1 * G (G threads per pencil, R1 values per thread):
//
//   fft_slab_kernel    DFT along the two fast axes of one n x n slab:
//                      rows straight from global memory into registers,
//                      columns from a padded shared-memory copy of the slab.
//   fft_pencil_kernel  DFT along the slow axis, 32/G pencils per warp,
//                      straight from and back to global memory.
//
// Within a pencil: a = j + G m (j = thread, m < R1); step 1 is a length-R1
// DFT over m in registers, then the twiddle exp(S 2 pi i j k2 / n), then an
// exchange through a small per-warp buffer (__syncwarp only) and a length-G
// DFT over j, giving X[k2 + R1 k1].  Every global access of a warp touches
// whole 32-byte sectors.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dft_reg.cuh"

namespace fcc {

template <int N> struct FftShape { static constexpr bool ok = false; static constexpr int R1 = 1, G = 1; };
#define FCC_SHAPE(NN, RR, GG) \
    template <> struct FftShape<NN> { static constexpr bool ok = true; static constexpr int R1 = RR, G = GG; };
FCC_SHAPE(128, 16, 8)
FCC_SHAPE(96, 24, 4)
FCC_SHAPE(64, 8, 8)
FCC_SHAPE(32, 8, 4)
FCC_SHAPE(16, 4, 4)
#undef FCC_SHAPE

constexpr int kFastThreads = 256;            // pencil kernel
constexpr int kFastWarps = kFastThreads / 32;
constexpr int kSlabThreads = 512;            // slab kernel: one block per SM, 16 warps
constexpr int kSlabWarps = kSlabThreads / 32;

template <int N>
struct FastLayout {
    static constexpr int R1 = FftShape<N>::R1;
    static constexpr int G = FftShape<N>::G;
    static constexpr int PPW = 32 / G;                 // pencils per warp
    static constexpr int LD = N + 4;                   // slab row stride (complex)
    static constexpr int EXP = G * (R1 + 1);           // exchange stride per pencil
    static constexpr int EXW = PPW * EXP;              // exchange per warp
    static constexpr size_t slab_smem = (size_t)(N * LD + kSlabWarps * EXW + N) * sizeof(float2);
    static constexpr size_t pencil_smem = (size_t)(kFastWarps * EXW + N) * sizeof(float2);
};

// One pencil step for the thread holding v[m] = x[j + G m]: DFT over m,
// twiddle, exchange, DFT over j.  On return the thread owns outputs
// X[k2 + R1 k1] for k2 = q + G e (e < R1/G... handled by the caller via emit).
template <int N, int S>
struct PencilFft {
    using L = FastLayout<N>;
    static constexpr int R1 = L::R1, G = L::G;
    static_assert(R1 % G == 0, "R1 must be a multiple of G");

    // ex: this pencil's exchange area (G * (R1+1) complex); tw: exp(+2 pi i m / N)
    template <typename Emit>
    __device__ __forceinline__ static void run(float (&vr)[R1], float (&vi)[R1], int j, float2* ex,
                                               const float2* tw, Emit emit) {
        reg::Dft<R1, S, float>::run(vr, vi);
#pragma unroll
        for (int k2 = 1; k2 < R1; ++k2) {
            const float2 w = tw[(j * k2) % N];
            const float wi = S > 0 ? w.y : -w.y;
            const float t = vr[k2] * w.x - vi[k2] * wi;
            vi[k2] = vr[k2] * wi + vi[k2] * w.x;
            vr[k2] = t;
        }
#pragma unroll
        for (int k2 = 0; k2 < R1; ++k2) ex[j * (R1 + 1) + k2] = make_float2(vr[k2], vi[k2]);
        __syncwarp();
        const int q = j;
#pragma unroll
        for (int e = 0; e < R1 / G; ++e) {
            const int k2 = q + G * e;
            float ur[G], ui[G];
#pragma unroll
            for (int jj = 0; jj < G; ++jj) {
                const float2 t = ex[jj * (R1 + 1) + k2];
                ur[jj] = t.x;
                ui[jj] = t.y;
            }
            reg::Dft<G, S, float>::run(ur, ui);
#pragma unroll
            for (int k1 = 0; k1 < G; ++k1) emit(k2 + R1 * k1, ur[k1], ui[k1]);
        }
        __syncwarp();
    }
};

// grid.x = number of slabs (volumes * N); volume v starts at v * vstride
// complex values; in and out may alias.
template <int N, int S>
__global__ void __launch_bounds__(kSlabThreads, 1)
fft_slab_kernel(const float2* in, float2* out, const float2* __restrict__ twg, int64_t vstride) {
    using L = FastLayout<N>;
    constexpr int R1 = L::R1, G = L::G, PPW = L::PPW, LD = L::LD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* slab = reinterpret_cast<float2*>(smem_raw);
    float2* exall = slab + N * LD;
    float2* tw = exall + kSlabWarps * L::EXW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < N; t += kSlabThreads) tw[t] = twg[t];
    __syncthreads();
    const int64_t base = (int64_t)(blockIdx.x / N) * vstride + (int64_t)(blockIdx.x % N) * N * N;

    // rows (fastest axis)
    {
        const int p = lane / G, j = lane % G;
        float2* ex = exall + warp * L::EXW + p * L::EXP;
        for (int r0 = 0; r0 < N; r0 += kSlabWarps * PPW) {
            const int r = r0 + warp * PPW + p;
            const bool act = r < N;   // warp-uniform: N is a multiple of PPW
            if (act) {
                float vr[R1], vi[R1];
                const float2* src = in + base + (int64_t)r * N + j;
#pragma unroll
                for (int m = 0; m < R1; ++m) {
                    const float2 t = src[G * m];
                    vr[m] = t.x;
                    vi[m] = t.y;
                }
                float2* row = slab + r * LD;
                PencilFft<N, S>::run(vr, vi, j, ex, tw, [&](int c, float xr, float xi) {
                    row[c] = make_float2(xr, xi);
                });
            }
        }
    }
    __syncthreads();
    // columns (middle axis), results straight to global memory
    {
        const int cl = lane % PPW, j = lane / PPW;
        float2* ex = exall + warp * L::EXW + cl * L::EXP;
        for (int c0 = 0; c0 < N; c0 += kSlabWarps * PPW) {
            const int c = c0 + warp * PPW + cl;
            if (c0 + warp * PPW < N) {
                float vr[R1], vi[R1];
#pragma unroll
                for (int m = 0; m < R1; ++m) {
                    const float2 t = slab[(j + G * m) * LD + c];
                    vr[m] = t.x;
                    vi[m] = t.y;
                }
                float2* dst = out + base + c;
                PencilFft<N, S>::run(vr, vi, j, ex, tw, [&](int b, float xr, float xi) {
                    dst[(int64_t)b * N] = make_float2(xr, xi);
                });
            }
        }
    }
}

// Two pencils (adjacent columns c, c+1) per thread, 16-byte accesses.
// grid.x = volumes * N (b) * ceil(N / CPB) column blocks; pencils along the
// slowest axis.  in and out may alias.
template <int N, int S>
__global__ void __launch_bounds__(kFastThreads)
fft_pencil_kernel(const float2* in, float2* out, const float2* __restrict__ twg, int64_t vstride) {
    using L = FastLayout<N>;
    constexpr int R1 = L::R1, G = L::G, PPW = L::PPW;
    constexpr int CPB = kFastWarps * PPW * 2;
    constexpr int CBLK = (N + CPB - 1) / CPB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* exall = reinterpret_cast<float2*>(smem_raw);
    float2* tw = exall + kFastWarps * L::EXW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < N; t += kFastThreads) tw[t] = twg[t];
    __syncthreads();
    const int64_t blk = blockIdx.x;
    const int64_t vol = blk / ((int64_t)N * CBLK);
    const int rem = (int)(blk - vol * N * CBLK);
    const int b = rem / CBLK;
    const int cb = rem % CBLK;
    const int cl = lane % PPW, j = lane / PPW;
    const int c = cb * CPB + 2 * (warp * PPW + cl);
    if (cb * CPB + 2 * warp * PPW >= N) return;   // warp-uniform (N is a multiple of 2 PPW)
    float2* ex = exall + warp * L::EXW + cl * L::EXP;
    const int64_t NN = (int64_t)N * N;
    const int64_t base = vol * vstride + (int64_t)b * N + c;
    float ar[R1], ai[R1], br[R1], bi[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) {
        const float4 t = *reinterpret_cast<const float4*>(in + base + (int64_t)(j + G * m) * NN);
        ar[m] = t.x;
        ai[m] = t.y;
        br[m] = t.z;
        bi[m] = t.w;
    }
    // pencil c, then pencil c+1 through the same exchange slot; keep the
    // length-G inputs of both, then emit 16-byte stores
    constexpr int E = R1 / G;
    float ur[2][E][G], ui[2][E][G];
#pragma unroll
    for (int pz = 0; pz < 2; ++pz) {
        float* vr = pz ? br : ar;
        float* vi = pz ? bi : ai;
        reg::Dft<R1, S, float>::run(vr, vi);
#pragma unroll
        for (int k2 = 1; k2 < R1; ++k2) {
            const float2 w = tw[(j * k2) % N];
            const float wi = S > 0 ? w.y : -w.y;
            const float t = vr[k2] * w.x - vi[k2] * wi;
            vi[k2] = vr[k2] * wi + vi[k2] * w.x;
            vr[k2] = t;
        }
#pragma unroll
        for (int k2 = 0; k2 < R1; ++k2) ex[j * (R1 + 1) + k2] = make_float2(vr[k2], vi[k2]);
        __syncwarp();
#pragma unroll
        for (int e = 0; e < E; ++e) {
#pragma unroll
            for (int jj = 0; jj < G; ++jj) {
                const float2 t = ex[jj * (R1 + 1) + j + G * e];
                ur[pz][e][jj] = t.x;
                ui[pz][e][jj] = t.y;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        reg::Dft<G, S, float>::run(ur[0][e], ui[0][e]);
        reg::Dft<G, S, float>::run(ur[1][e], ui[1][e]);
        const int k2 = j + G * e;
#pragma unroll
        for (int k1 = 0; k1 < G; ++k1) {
            *reinterpret_cast<float4*>(out + base + (int64_t)(k2 + R1 * k1) * NN) =
                make_float4(ur[0][e][k1], ui[0][e][k1], ur[1][e][k1], ui[1][e][k1]);
        }
    }
}

}  // namespace fcc

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

}  // namespace fcc
