// Fast 3-D DFT passes for orders with a register-resident factorisation
// n = R1 * G (G threads per pencil, R1 values per thread):
//
//   fft_slab_kernel    DFT along the two fast axes of one n x n slab:
//                      rows straight from global memory into registers,
//                      columns from a padded shared-memory copy of the slab.
//   fft_pencil_kernel  DFT along the slow axis, 32/G pencils per warp (one or
//                      two per thread), straight from and back to global memory.
//
// Within a pencil: a = j + G m (j = thread, m < R1); step 1 is a length-R1
// DFT over m in registers, then the twiddle exp(S 2 pi i j k2 / n), then an
// exchange through a small per-warp buffer (__syncwarp only) and a length-G
// DFT over j, giving X[k2 + R1 k1].  Lanes past the end of the data run the
// same arithmetic on zeros with their memory accesses switched off, so every
// __syncwarp sees the whole warp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "dft_reg.cuh"

namespace fcc {

template <int N> struct FftShape { static constexpr bool ok = false; static constexpr int R1 = 1, G = 1; };
#define FCC_SHAPE(NN, RR, GG) \
    template <> struct FftShape<NN> { static constexpr bool ok = true; static constexpr int R1 = RR, G = GG; };
FCC_SHAPE(128, 16, 8)
FCC_SHAPE(96, 24, 4)
FCC_SHAPE(88, 44, 2)
FCC_SHAPE(80, 20, 4)
FCC_SHAPE(72, 36, 2)
FCC_SHAPE(64, 8, 8)
FCC_SHAPE(56, 28, 2)
FCC_SHAPE(48, 12, 4)
FCC_SHAPE(40, 20, 2)
FCC_SHAPE(32, 8, 4)
FCC_SHAPE(24, 12, 2)
FCC_SHAPE(16, 4, 4)
FCC_SHAPE(8, 4, 2)
#undef FCC_SHAPE

// Kernel attributes (dynamic shared-memory limits) are per device: a bit per
// device id records that they are set.  Concurrent first calls may set them
// twice (harmless); none launches before its own device's bit is set.
struct DeviceOnce {
    std::atomic<unsigned long long> bits{0};
    static int dev() {
        int d = 0;
        cudaGetDevice(&d);
        return d & 63;
    }
    bool done() const { return (bits.load() >> dev()) & 1ull; }
    void mark() { bits.fetch_or(1ull << dev()); }
};

constexpr int kFastThreads = 256;            // pencil kernel
constexpr int kFastWarps = kFastThreads / 32;

// Smallest stride >= e at which the 8-byte exchange accesses of the pencil
// layout are free of bank conflicts: PPW = 32 / g pencils per warp must land
// 32 / PPW banks apart within a 16-lane phase.
constexpr int pencil_stride(int g, int e) {
    while (!(g == 8 ? (e % 16 == 4 || e % 16 == 12) : g == 4 ? e % 4 == 2 : g == 2 ? e % 2 == 1 : true)) ++e;
    return e;
}

template <int N>
struct FastLayout {
    static constexpr int R1 = FftShape<N>::R1;
    static constexpr int G = FftShape<N>::G;
    static constexpr int PPW = 32 / G;                 // pencils per warp
    static constexpr int LD = N + 4;                   // slab row stride (complex)
    static constexpr int EXP = G * (R1 + 1);           // exchange stride per pencil (lane = p G + j)
    // stride for the pencil layout (lane = j PPW + cl): padded so that the
    // PPW pencils of a half-warp fall into distinct shared-memory banks
    static constexpr int EXPC = pencil_stride(G, EXP);
    static constexpr int EXW = PPW * EXPC;             // exchange per warp
    // slab kernel: 16 warps when the slab and 16 exchange buffers fit in
    // ~200 KB (leaving room on the SM for a block of another kernel)
    static constexpr int SW = ((size_t)(N * LD + 16 * EXW + N) * 8 <= 200 * 1024) ? 16 : 8;
    static constexpr int SLAB_THREADS = 32 * SW;
    static constexpr size_t slab_smem = (size_t)(N * LD + SW * EXW + N) * sizeof(float2);
    static constexpr int NP = R1 <= 24 ? 2 : 1;        // pencils per thread in the pencil kernel
    static constexpr int CPB = kFastWarps * PPW * NP;  // columns per pencil block
    static constexpr size_t pencil_smem = (size_t)(kFastWarps * EXW + N) * sizeof(float2);
};

// Step 1 (DFT over m), twiddle and exchange for the thread holding
// v[m] = x[j + G m]; afterwards the thread reads its length-G inputs.
template <int N, int S>
__device__ __forceinline__ void pencil_stage1(float* vr, float* vi, int j, float2* ex, const float2* tw) {
    constexpr int R1 = FastLayout<N>::R1;
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
}

// Order 128 (R1 = 16, G = 8): stage 1 of thread j with the exchange done by
// warp shuffles instead of shared memory.  The 8 threads of a pencil are
// lanes j * lstride + c; thread j holds A[j][k2] (k2 < 16) after the
// length-16 DFT and the twiddle.  Viewing (A[j][e], A[j][e + 8]) as element
// (j, e) of an 8 x 8 matrix, three butterfly stages (lane distance m lstride,
// m = 1, 2, 4) transpose it: at stage m, of each position pair (e, e | m)
// the thread whose bit m of j is set keeps e | m and sends e, the other keeps
// e and sends e | m.  Afterwards thread q holds (ur[0][jj], ur[1][jj]) =
// (A[jj][q], A[jj][q + 8]), the inputs of its two length-8 DFTs.
template <int S>
__device__ __forceinline__ void pencil128_stage1_shfl(float (&vr)[16], float (&vi)[16], int j, int lstride,
                                                      const float2* tw, float (&ur)[2][8], float (&ui)[2][8]) {
    reg::Dft<16, S, float>::run(vr, vi);
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) {
        const float2 w = tw[(j * k2) & 127];
        const float wi = S > 0 ? w.y : -w.y;
        const float t = vr[k2] * w.x - vi[k2] * wi;
        vi[k2] = vr[k2] * wi + vi[k2] * w.x;
        vr[k2] = t;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        ur[0][e] = vr[e];
        ui[0][e] = vi[e];
        ur[1][e] = vr[e + 8];
        ui[1][e] = vi[e + 8];
    }
#pragma unroll
    for (int m = 1; m < 8; m <<= 1) {
        const bool hi = (j & m) != 0;
#pragma unroll
        for (int e0 = 0; e0 < 8; ++e0) {
            if (e0 & m) continue;
            const int e1 = e0 | m;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float sr = hi ? ur[h][e0] : ur[h][e1];
                float si = hi ? ui[h][e0] : ui[h][e1];
                sr = __shfl_xor_sync(0xffffffffu, sr, m * lstride);
                si = __shfl_xor_sync(0xffffffffu, si, m * lstride);
                if (hi) {
                    ur[h][e0] = sr;
                    ui[h][e0] = si;
                } else {
                    ur[h][e1] = sr;
                    ui[h][e1] = si;
                }
            }
        }
    }
}

template <int N, int S>
struct PencilFft {
    using L = FastLayout<N>;
    static constexpr int R1 = L::R1, G = L::G;
    static_assert(R1 % G == 0, "R1 must be a multiple of G");

    // whole pencil; emit(index, re, im) receives X[k2 + R1 k1]
    template <typename Emit>
    __device__ __forceinline__ static void run(float (&vr)[R1], float (&vi)[R1], int j, float2* ex,
                                               const float2* tw, Emit emit) {
        pencil_stage1<N, S>(vr, vi, j, ex, tw);
        __syncwarp();
        const int q = j;
        float ur[R1 / G][G], ui[R1 / G][G];
#pragma unroll
        for (int e = 0; e < R1 / G; ++e) {
#pragma unroll
            for (int jj = 0; jj < G; ++jj) {
                const float2 t = ex[jj * (R1 + 1) + q + G * e];
                ur[e][jj] = t.x;
                ui[e][jj] = t.y;
            }
        }
        __syncwarp();   // the exchange slot may be reused right after
#pragma unroll
        for (int e = 0; e < R1 / G; ++e) {
            reg::Dft<G, S, float>::run(ur[e], ui[e]);
#pragma unroll
            for (int k1 = 0; k1 < G; ++k1) emit(q + G * e + R1 * k1, ur[e][k1], ui[e][k1]);
        }
    }

    // two independent pencils in lockstep (more independent work per warp);
    // they share the exchange slot one after the other.  emit(p, index, re, im)
    template <typename Emit>
    __device__ __forceinline__ static void run2(float (&ar)[R1], float (&ai)[R1], float (&br)[R1], float (&bi)[R1],
                                                int j, float2* ex, const float2* tw, Emit emit) {
        constexpr int E = R1 / G;
        reg::Dft<R1, S, float>::run(ar, ai);
        reg::Dft<R1, S, float>::run(br, bi);
#pragma unroll
        for (int k2 = 1; k2 < R1; ++k2) {
            const float2 w = tw[(j * k2) % N];
            const float wi = S > 0 ? w.y : -w.y;
            float t = ar[k2] * w.x - ai[k2] * wi;
            ai[k2] = ar[k2] * wi + ai[k2] * w.x;
            ar[k2] = t;
            t = br[k2] * w.x - bi[k2] * wi;
            bi[k2] = br[k2] * wi + bi[k2] * w.x;
            br[k2] = t;
        }
        float ur[2][E][G], ui[2][E][G];
#pragma unroll
        for (int pz = 0; pz < 2; ++pz) {
#pragma unroll
            for (int k2 = 0; k2 < R1; ++k2)
                ex[j * (R1 + 1) + k2] = pz ? make_float2(br[k2], bi[k2]) : make_float2(ar[k2], ai[k2]);
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
#pragma unroll
            for (int k1 = 0; k1 < G; ++k1) {
                emit(0, j + G * e + R1 * k1, ur[0][e][k1], ui[0][e][k1]);
                emit(1, j + G * e + R1 * k1, ur[1][e][k1], ui[1][e][k1]);
            }
        }
    }
};

__device__ __forceinline__ int64_t vol_base(const int64_t* voff, int64_t v, int64_t vstride) {
    return voff ? voff[v] : v * vstride;
}

// Shared memory of the slab transform with SW warps.
template <int N>
constexpr size_t slab_smem_for(int sw) {
    return (size_t)(N * FastLayout<N>::LD + sw * FastLayout<N>::EXW + N) * sizeof(float2);
}

// DFT along the two fast axes of the n x n slab starting at `base` (complex
// values), by a block of SW warps; in and out may alias.  PRE: every input
// value is first multiplied by preg[c], c its index along the fastest axis
// (a separable modulation of the input; N more complex values of shared
// memory).
template <int N, int S, int SW, bool PRE = false>
__device__ __forceinline__ void fft_slab_body(const float2* in, float2* out, const float2* __restrict__ twg,
                                              int64_t base, unsigned char* smem_raw,
                                              const float2* __restrict__ preg = nullptr) {
    using L = FastLayout<N>;
    constexpr int R1 = L::R1, G = L::G, PPW = L::PPW, LD = L::LD;
    float2* slab = reinterpret_cast<float2*>(smem_raw);
    float2* exall = slab + N * LD;
    float2* tw = exall + SW * L::EXW;
    float2* pre = tw + N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < N; t += 32 * SW) {
        tw[t] = twg[t];
        if (PRE) pre[t] = preg[t];
    }
    __syncthreads();
    // input value at fast index c, modulated when PRE
    auto modulate = [&](float2 t, int c) -> float2 {
        if (!PRE) return t;
        const float2 w = pre[c];
        return make_float2(t.x * w.x - t.y * w.y, t.x * w.y + t.y * w.x);
    };

    // rows (fastest axis)
    {
        const int p = lane / G, j = lane % G;
        float2* ex = exall + warp * L::EXW + p * L::EXP;
        constexpr int RR = SW * PPW;                    // rows per round
        constexpr int NR = (N + RR - 1) / RR;           // rounds
        if (NR > 1 && NR * R1 * 2 <= (SW == 8 ? 128 : 64)) {
            // every round's loads in flight before the first transform
            float vr[NR][R1], vi[NR][R1];
#pragma unroll
            for (int rd = 0; rd < NR; ++rd) {
                const int r = rd * RR + warp * PPW + p;
                const bool act = r < N;
                const float2* src = in + base + (int64_t)r * N + j;
#pragma unroll
                for (int m = 0; m < R1; ++m) {
                    const float2 t = modulate(act ? src[G * m] : make_float2(0.f, 0.f), j + G * m);
                    vr[rd][m] = t.x;
                    vi[rd][m] = t.y;
                }
            }
            // two rounds in lockstep where every row of both exists
            constexpr int NP2 = N % RR == 0 ? NR / 2 * 2 : 0;
#pragma unroll
            for (int rd = 0; rd < NP2; rd += 2) {
                const int r0 = rd * RR + warp * PPW + p, r1 = r0 + RR;
                float2* row0 = slab + r0 * LD;
                float2* row1 = slab + r1 * LD;
                PencilFft<N, S>::run2(vr[rd], vi[rd], vr[rd + 1], vi[rd + 1], j, ex, tw,
                                      [&](int pz, int c, float xr, float xi) {
                                          (pz ? row1 : row0)[c] = make_float2(xr, xi);
                                      });
            }
#pragma unroll
            for (int rd = NP2; rd < NR; ++rd) {
                if (rd * RR + warp * PPW >= N) continue;   // warp-uniform
                const int r = rd * RR + warp * PPW + p;
                const bool act = r < N;
                float2* row = slab + r * LD;
                PencilFft<N, S>::run(vr[rd], vi[rd], j, ex, tw, [&](int c, float xr, float xi) {
                    if (act) row[c] = make_float2(xr, xi);
                });
            }
        } else {
            for (int r0 = 0; r0 < N; r0 += RR) {
                if (r0 + warp * PPW >= N) continue;   // warp-uniform
                const int r = r0 + warp * PPW + p;
                const bool act = r < N;
                float vr[R1], vi[R1];
                const float2* src = in + base + (int64_t)r * N + j;
#pragma unroll
                for (int m = 0; m < R1; ++m) {
                    const float2 t = modulate(act ? src[G * m] : make_float2(0.f, 0.f), j + G * m);
                    vr[m] = t.x;
                    vi[m] = t.y;
                }
                float2* row = slab + r * LD;
                PencilFft<N, S>::run(vr, vi, j, ex, tw, [&](int c, float xr, float xi) {
                    if (act) row[c] = make_float2(xr, xi);
                });
            }
        }
    }
    __syncthreads();
    // columns (middle axis), results straight to global memory
    {
        const int cl = lane % PPW, j = lane / PPW;
        float2* ex = exall + warp * L::EXW + cl * L::EXPC;
        constexpr int CR = SW * PPW;   // columns per round
        if (N % (2 * CR) == 0 && R1 <= 16) {
            // two column rounds in lockstep (every column exists)
            for (int c0 = 0; c0 < N; c0 += 2 * CR) {
                const int c = c0 + warp * PPW + cl;
                float ar[R1], ai[R1], br[R1], bi[R1];
#pragma unroll
                for (int m = 0; m < R1; ++m) {
                    const float2 t = slab[(j + G * m) * LD + c];
                    const float2 u = slab[(j + G * m) * LD + c + CR];
                    ar[m] = t.x;
                    ai[m] = t.y;
                    br[m] = u.x;
                    bi[m] = u.y;
                }
                float2* dst = out + base + c;
                PencilFft<N, S>::run2(ar, ai, br, bi, j, ex, tw, [&](int pz, int b, float xr, float xi) {
                    dst[(int64_t)b * N + (pz ? CR : 0)] = make_float2(xr, xi);
                });
            }
        } else {
            for (int c0 = 0; c0 < N; c0 += CR) {
                if (c0 + warp * PPW >= N) continue;   // warp-uniform
                const int c = c0 + warp * PPW + cl;
                const bool act = c < N;
                float vr[R1], vi[R1];
#pragma unroll
                for (int m = 0; m < R1; ++m) {
                    const float2 t = act ? slab[(j + G * m) * LD + c] : make_float2(0.f, 0.f);
                    vr[m] = t.x;
                    vi[m] = t.y;
                }
                float2* dst = out + base + c;
                PencilFft<N, S>::run(vr, vi, j, ex, tw, [&](int b, float xr, float xi) {
                    if (act) dst[(int64_t)b * N] = make_float2(xr, xi);
                });
            }
        }
    }
}

// grid.x = number of slabs (volumes * N); volume v starts at voff[v] (or
// v * vstride) complex values; in and out may alias.  PRE: inputs modulated
// by pre[c] along the fastest axis (dynamic shared memory slab_smem + N
// complex values).
template <int N, int S, bool PRE = false>
__global__ void __launch_bounds__(FastLayout<N>::SLAB_THREADS, 1)
fft_slab_kernel(const float2* in, float2* out, const float2* __restrict__ twg, int64_t vstride, const int64_t* voff,
                const float2* __restrict__ pre = nullptr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t base = vol_base(voff, blockIdx.x / N, vstride) + (int64_t)(blockIdx.x % N) * N * N;
    fft_slab_body<N, S, FastLayout<N>::SW, PRE>(in, out, twg, base, smem_raw, pre);
}

// NP adjacent pencils (columns c, c+1) per thread.  grid.x = volumes * N (b)
// * ceil(N / CPB) column blocks; pencils along the slowest axis.
// Pencils along the slowest axis of the volume at `vbase` (complex values):
// middle index b, column block cb; block of kFastThreads threads.
template <int N, int S>
__device__ __forceinline__ void fft_pencil_body(const float2* in, float2* out, const float2* __restrict__ twg,
                                                int64_t vbase, int b, int cb, unsigned char* smem_raw) {
    using L = FastLayout<N>;
    constexpr int R1 = L::R1, G = L::G, PPW = L::PPW, NP = L::NP, CPB = L::CPB;
    float2* exall = reinterpret_cast<float2*>(smem_raw);
    float2* tw = exall + kFastWarps * L::EXW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < N; t += kFastThreads) tw[t] = twg[t];
    __syncthreads();
    const int cl = lane % PPW, j = lane / PPW;
    if (cb * CPB + NP * warp * PPW >= N) return;   // warp-uniform; no block barrier below
    const int c = cb * CPB + NP * (warp * PPW + cl);
    const bool act = c < N;
    float2* ex = exall + warp * L::EXW + cl * L::EXPC;
    const int64_t NN = (int64_t)N * N;
    const int64_t base = vbase + (int64_t)b * N + c;
    float ar[R1], ai[R1], br[R1], bi[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) {
        if (NP == 2) {
            const float4 t = act ? *reinterpret_cast<const float4*>(in + base + (int64_t)(j + G * m) * NN)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            ar[m] = t.x;
            ai[m] = t.y;
            br[m] = t.z;
            bi[m] = t.w;
        } else {
            const float2 t = act ? in[base + (int64_t)(j + G * m) * NN] : make_float2(0.f, 0.f);
            ar[m] = t.x;
            ai[m] = t.y;
            br[m] = 0.f;
            bi[m] = 0.f;
        }
    }
    constexpr int E = R1 / G;
    float ur[NP][E][G], ui[NP][E][G];
#pragma unroll
    for (int pz = 0; pz < NP; ++pz) {
        float* vr = pz ? br : ar;
        float* vi = pz ? bi : ai;
        pencil_stage1<N, S>(vr, vi, j, ex, tw);
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
#pragma unroll
        for (int pz = 0; pz < NP; ++pz) reg::Dft<G, S, float>::run(ur[pz][e], ui[pz][e]);
        const int k2 = j + G * e;
#pragma unroll
        for (int k1 = 0; k1 < G; ++k1) {
            if (!act) continue;
            if (NP == 2) {
                *reinterpret_cast<float4*>(out + base + (int64_t)(k2 + R1 * k1) * NN) =
                    make_float4(ur[0][e][k1], ui[0][e][k1], ur[NP - 1][e][k1], ui[NP - 1][e][k1]);
            } else {
                out[base + (int64_t)(k2 + R1 * k1) * NN] = make_float2(ur[0][e][k1], ui[0][e][k1]);
            }
        }
    }
}

template <int N, int S>
__global__ void __launch_bounds__(kFastThreads)
fft_pencil_kernel(const float2* in, float2* out, const float2* __restrict__ twg, int64_t vstride, const int64_t* voff) {
    using L = FastLayout<N>;
    constexpr int CBLK = (N + L::CPB - 1) / L::CPB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t blk = blockIdx.x;
    const int64_t vol = blk / ((int64_t)N * CBLK);
    const int rem = (int)(blk - vol * N * CBLK);
    fft_pencil_body<N, S>(in, out, twg, vol_base(voff, vol, vstride), rem / CBLK, rem % CBLK, smem_raw);
}

// Last pass of the forward transform of paired real volumes, fused with the
// split of Y = D (x1 + i x2) into D x1 and D x2.  The pairing map
// pi(i, l, q) = (i - l, -l, q - l) sends the pencil (l, q) along the slow
// axis onto the pencil (n - l, q - l) with its index shifted by -l.  Warps
// 0-3 of a block transform primary pencils (l, q), warps 4-7 their partners;
// both stage their outputs in shared memory, and every thread forms, for
// each output index k of its own pencil with counterpart index k' (k - l on
// a primary pencil, k + l on a partner),
//   y1 = (Y[k] + conj(Y'[k'])) / 2,   y2 = (Y[k] - conj(Y'[k'])) / (2i),
// written into volumes 2p and 2p + 1 at its own pencil.  Primary rows
// l = 0 .. n/2: row 0 is its own partner (warps 4-7 idle), in row n/2 only
// columns q < n/2 are primary, so every pencil is written exactly once.
// grid.x = pairs * (n/2 + 1) * ceil(n / CPB2); Y of pair p sits at
// p * vstride (vstride >= 2 n^3), y2 at p * vstride + n^3.
//
// PACKED: out holds real volumes (pair p at p * 2 n^3 floats, volume 2p + 1
// n^3 floats after volume 2p) in the Hermitian-packed layout: a point of a
// primary pencil stores Re y, a point of a partner pencil stores -Im y (the
// imaginary part at its primary partner), so each of the n^3 reals of a
// volume is written by the thread that owns its point.
template <int N>
struct PairLayout {
    static constexpr int PPW = FastLayout<N>::PPW;
    static constexpr int CPB2 = (kFastWarps / 2) * PPW;   // primary columns per block
    static constexpr int CBLK = (N + CPB2 - 1) / CPB2;
};

// PRE: the pencil's inputs are first multiplied by pre[k], k their index
// along the slow axis (dynamic shared memory pencil_smem + N complex values).
template <int N, bool PACKED = false, bool PRE = false>
__global__ void __launch_bounds__(kFastThreads)
fft_pencil_pair_kernel(const float2* in, float2* out, const float2* __restrict__ twg, int64_t vstride,
                       const float2* __restrict__ preg = nullptr, const int64_t* __restrict__ poff = nullptr) {
    using L = FastLayout<N>;
    using P = PairLayout<N>;
    constexpr int R1 = L::R1, G = L::G, PPW = L::PPW, E = R1 / G;
    constexpr int ROWS = N / 2 + 1;
    constexpr int64_t NN = (int64_t)N * N, N3 = NN * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* exall = reinterpret_cast<float2*>(smem_raw);
    float2* tw = exall + kFastWarps * L::EXW;
    float2* pre = tw + N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < N; t += kFastThreads) {
        tw[t] = twg[t];
        if (PRE) pre[t] = preg[t];
    }
    __syncthreads();
    const int64_t blk = blockIdx.x;
    const int64_t pr = blk / (ROWS * P::CBLK);
    const int rem = (int)(blk - pr * ROWS * P::CBLK);
    const int l = rem / P::CBLK, cb = rem % P::CBLK;
    const int qlim = 2 * l == N ? N / 2 : N;
    const bool partner = warp >= kFastWarps / 2;
    const int wq = partner ? warp - kFastWarps / 2 : warp;
    const int cl = lane % PPW, j = lane / PPW;
    const int c = cb * P::CPB2 + wq * PPW + cl;                     // primary column
    // warp-uniform: the whole primary warp is past the end, or row 0's partner warps
    const bool idle = cb * P::CPB2 + wq * PPW >= qlim || (partner && l == 0);
    const bool act = !idle && c < qlim;
    const int lo = partner ? (N - l) % N : l;
    const int co = partner ? (c - l + N) % N : c;
    // Y of pair pr and D x1 at y0, D x2 at y1 (ragged batches: a table of two
    // complex offsets per pair; else consecutive volumes)
    const int64_t y0 = poff ? poff[2 * pr] : pr * vstride;
    const int64_t y1 = poff ? poff[2 * pr + 1] : y0 + N3;
    const int64_t base = y0 + (int64_t)lo * N + co;                // own pencil; + k * NN
    const int64_t base2 = y1 + (int64_t)lo * N + co;
    const int64_t pbase = pr * 2 * N3 + (int64_t)lo * N + co;      // PACKED: own pencil of volume 2p
    float2* ex = exall + warp * L::EXW + cl * L::EXPC;
    float ur[E][G], ui[E][G];
    if (!idle) {
        float vr[R1], vi[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) {
            const float2 t = act ? in[base + (int64_t)(j + G * m) * NN] : make_float2(0.f, 0.f);
            if (PRE) {
                const float2 w = pre[j + G * m];
                vr[m] = t.x * w.x - t.y * w.y;
                vi[m] = t.x * w.y + t.y * w.x;
            } else {
                vr[m] = t.x;
                vi[m] = t.y;
            }
        }
        if constexpr (N == 128) {
            static_assert(R1 == 16 && G == 8 && PPW == 4, "order-128 shuffle exchange");
            pencil128_stage1_shfl<1>(vr, vi, j, PPW, tw, ur, ui);   // exchange by warp shuffles
        } else {
            pencil_stage1<N, 1>(vr, vi, j, ex, tw);
            __syncwarp();
#pragma unroll
            for (int e = 0; e < E; ++e) {
#pragma unroll
                for (int jj = 0; jj < G; ++jj) {
                    const float2 t = ex[jj * (R1 + 1) + j + G * e];
                    ur[e][jj] = t.x;
                    ui[e][jj] = t.y;
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            reg::Dft<G, 1, float>::run(ur[e], ui[e]);
#pragma unroll
            for (int k1 = 0; k1 < G; ++k1) ex[j + G * e + R1 * k1] = make_float2(ur[e][k1], ui[e][k1]);
        }
    }
    __syncthreads();
    if (idle) return;
    // counterpart pencil: the other half of the block, same slot (row 0: itself)
    const float2* cx = l == 0 ? ex : exall + (partner ? warp - kFastWarps / 2 : warp + kFastWarps / 2) * L::EXW + cl * L::EXPC;
    const int sh = partner ? l : N - l;   // k' = k - l (primary) or k + l (partner), mod N
#pragma unroll
    for (int e = 0; e < E; ++e) {
#pragma unroll
        for (int k1 = 0; k1 < G; ++k1) {
            const int k = j + G * e + R1 * k1;
            int kc = k + sh;
            kc -= kc >= N ? N : 0;
            const float2 B = cx[kc];
            const float Ar = ur[e][k1], Ai = ui[e][k1];
            const float dr = 0.5f * (Ar - B.x), di = 0.5f * (Ai + B.y);   // y2 = -i d
            if (act && PACKED) {   // primary: Re y1, Re y2; partner: -Im y1, -Im y2
                float* o = reinterpret_cast<float*>(out);
                o[pbase + k * NN] = partner ? 0.5f * (B.y - Ai) : 0.5f * (Ar + B.x);
                o[pbase + N3 + k * NN] = partner ? dr : di;
            } else if (act) {
                out[base + k * NN] = make_float2(0.5f * (Ar + B.x), 0.5f * (Ai - B.y));
                out[base2 + k * NN] = make_float2(di, -dr);
            }
        }
    }
}

// First pass of the inverse / adjoint of paired real volumes, fused with the
// merge W = P(v1) + i P(v2), P(v)[a] = (v[a] + conj(v[pi(a)])) / 2 (see
// pair.cuh): the same primary / partner pencils as fft_pencil_pair_kernel.
// Each half of the block loads its pencil of v1 and v2 (volumes 2p, 2p + 1
// at p * in_vstride), the raw pencils meet in shared memory (v1, then v2),
// every thread forms W at its own pencil and transforms it along the slow
// axis with the - sign, written to the compact volume p at p * out_vstride.
// Row 0's partner warps idle; in row n/2 only columns q < n/2 are primary.
//
// PACKED: in holds Hermitian-packed real volumes (pair p at p * in_vstride
// floats, volume 2p + 1 n^3 floats later; the layout of the packed forward).
// A packed volume stands for a v with v o pi = conj v, so P(v) = v: at a
// primary point v = (own, counterpart) (row 0: (own, 0)), at a partner point
// v = (counterpart, -own); the two volumes' raw values meet in shared memory
// together.
template <int N, bool PACKED = false>
__global__ void __launch_bounds__(kFastThreads)
fft_pencil_merge_kernel(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ twg,
                        int64_t in_vstride, int64_t out_vstride, const int64_t* __restrict__ poff = nullptr) {
    using L = FastLayout<N>;
    using P = PairLayout<N>;
    constexpr int R1 = L::R1, G = L::G, PPW = L::PPW;
    constexpr int ROWS = N / 2 + 1;
    constexpr int64_t NN = (int64_t)N * N, N3 = NN * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* exall = reinterpret_cast<float2*>(smem_raw);
    float2* tw = exall + kFastWarps * L::EXW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < N; t += kFastThreads) tw[t] = twg[t];
    const int64_t blk = blockIdx.x;
    const int64_t pr = blk / (ROWS * P::CBLK);
    const int rem = (int)(blk - pr * ROWS * P::CBLK);
    const int l = rem / P::CBLK, cb = rem % P::CBLK;
    const int qlim = 2 * l == N ? N / 2 : N;
    const bool partner = warp >= kFastWarps / 2;
    const int wq = partner ? warp - kFastWarps / 2 : warp;
    const int cl = lane % PPW, j = lane / PPW;
    const int c = cb * P::CPB2 + wq * PPW + cl;
    const bool idle = cb * P::CPB2 + wq * PPW >= qlim || (partner && l == 0);   // warp-uniform
    const bool act = !idle && c < qlim;
    const int lo = partner ? (N - l) % N : l;
    const int co = partner ? (c - l + N) % N : c;
    // v1 at pin, v2 at pin2 (+ k * NN); ragged pairs: two complex offsets per pair
    const int64_t pin = (poff ? poff[2 * pr] : pr * in_vstride) + (int64_t)lo * N + co;
    const int64_t pin2 = (poff ? poff[2 * pr + 1] : pr * in_vstride + N3) + (int64_t)lo * N + co;
    const int64_t pout = pr * out_vstride + (int64_t)lo * N + co;
    float2* ex = exall + warp * L::EXW + cl * L::EXPC;
    const float2* cx = l == 0 ? ex : exall + (partner ? warp - kFastWarps / 2 : warp + kFastWarps / 2) * L::EXW + cl * L::EXPC;
    const int sh = partner ? l : N - l;   // counterpart index k + sh (mod N)
    float wr[R1], wi[R1];
    if (PACKED) {
        const float* inf = reinterpret_cast<const float*>(in);
        float p1[R1], p2[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) {
            const int64_t o = (int64_t)(j + G * m) * NN;
            p1[m] = act ? inf[pin + o] : 0.f;
            p2[m] = act ? inf[pin2 + o] : 0.f;
        }
        if (!idle) {
#pragma unroll
            for (int m = 0; m < R1; ++m) ex[j + G * m] = make_float2(p1[m], p2[m]);
        }
        __syncthreads();
        if (!idle) {
#pragma unroll
            for (int m = 0; m < R1; ++m) {
                int kc = j + G * m + sh;
                kc -= kc >= N ? N : 0;
                const float2 C = cx[kc];
                const float c1 = l == 0 ? 0.f : C.x, c2 = l == 0 ? 0.f : C.y;
                const float v1r = partner ? C.x : p1[m], v1i = partner ? -p1[m] : c1;
                const float v2r = partner ? C.y : p2[m], v2i = partner ? -p2[m] : c2;
                wr[m] = v1r - v2i;   // W = v1 + i v2
                wi[m] = v1i + v2r;
            }
        }
        __syncthreads();   // counterpart reads done before the exchange buffers are reused
    } else {
        float v1r[R1], v1i[R1], v2r[R1], v2i[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) {
            const int64_t o = (int64_t)(j + G * m) * NN;
            const float2 a = act ? in[pin + o] : make_float2(0.f, 0.f);
            const float2 b = act ? in[pin2 + o] : make_float2(0.f, 0.f);
            v1r[m] = a.x;
            v1i[m] = a.y;
            v2r[m] = b.x;
            v2i[m] = b.y;
        }
#pragma unroll
        for (int vv = 0; vv < 2; ++vv) {
            const float* vr = vv ? v2r : v1r;
            const float* vi = vv ? v2i : v1i;
            if (!idle) {
#pragma unroll
                for (int m = 0; m < R1; ++m) ex[j + G * m] = make_float2(vr[m], vi[m]);
            }
            __syncthreads();
            if (!idle) {
#pragma unroll
                for (int m = 0; m < R1; ++m) {
                    int kc = j + G * m + sh;
                    kc -= kc >= N ? N : 0;
                    const float2 B = cx[kc];
                    const float pr_ = 0.5f * (vr[m] + B.x), pi_ = 0.5f * (vi[m] - B.y);   // P(v) at this point
                    if (vv == 0) {
                        wr[m] = pr_;
                        wi[m] = pi_;
                    } else {   // W = P(v1) + i P(v2)
                        wr[m] -= pi_;
                        wi[m] += pr_;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (idle) return;   // no block barrier below
    PencilFft<N, -1>::run(wr, wi, j, ex, tw, [&](int k, float xr, float xi) {
        if (act) out[pout + (int64_t)k * NN] = make_float2(xr, xi);
    });
}

// Host launchers (fft_fast.cu).
bool has_fast_fft(int n);
cudaError_t launch_fast_fft(int n, bool slab, int sign, const float2* in, float2* out, int64_t nvol,
                            const float2* tw, int64_t vstride, const int64_t* voff, cudaStream_t st);
// inverse / adjoint: pair merge + first (pencil) pass, pairs at p * 2 n^3 of in,
// compact results at p * n^3 of out
// (packed: in holds Hermitian-packed real volumes, pair p at p * 2 n^3 floats)
cudaError_t launch_fast_pencil_merge(int n, const float2* in, float2* out, int64_t npairs, const float2* tw,
                                     cudaStream_t st, bool packed = false, const int64_t* poff = nullptr);
// forward pencil pass + pair split over `npairs` pairs (Y of pair p at p * vstride)
// (packed: out receives Hermitian-packed real volumes, pair p at p * 2 n^3 floats;
// pre: n complex factors the inputs are multiplied by along the slow axis, or null;
// poff: ragged pairs, two even complex offsets per pair -- Y and D x1 at the
// first, D x2 at the second; not with packed)
cudaError_t launch_fast_pencil_pair(int n, const float2* in, float2* out, int64_t npairs, const float2* tw,
                                    int64_t vstride, cudaStream_t st, bool packed = false,
                                    const float2* pre = nullptr, const int64_t* poff = nullptr);
// forward slab pass (+ sign) with the inputs multiplied by pre[c] along the fastest axis
cudaError_t launch_fast_slab_pre(int n, const float2* in, float2* out, int64_t nvol, const float2* tw,
                                 const float2* pre, int64_t vstride, cudaStream_t st);

}  // namespace fcc
