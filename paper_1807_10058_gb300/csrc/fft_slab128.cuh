// DFT along the two fast axes of 128 x 128 slabs with 16 warps per slab and no
// exchange buffers: the intra-pencil exchange of each length-128 DFT goes
// through the pencil's own row (or column) of the shared-memory slab.
//
// A pencil is transformed by 8 threads (j = 0..7) holding x[j + 8 m],
// m = 0..15: a length-16 DFT over m in registers, the twiddle
// exp(S 2 pi i j k2 / 128), then the exchange and a length-8 DFT over j giving
// X[k2 + 16 k1].  The exchange value (j, k2) is stored at position
//   xpos(j, k2) = 16 j + ((k2 + t(j)) mod 16),   t(j) = (j & 3) + 8 (j >> 2),
// of the pencil's row (columns: row index, same column), and in the second
// stage thread q owns k2 in {u(q), u(q) + 4}, u(q) = (q & 3) + 8 (q >> 2).
// With the slab row stride of 132 complex values (8 banks between
// consecutive rows) every shared-memory access of a half-warp then touches
// 16 distinct bank pairs: rows, 2 pencils per half-warp: positions mod 16
// form a set S with S + 4 its complement; columns, 4 columns x 4 threads per
// half-warp: row indices distinct mod 4.  The row phase writes its results
// back into the row in natural order; the column phase writes to global
// memory.  Shared memory is the slab alone (plus twiddles), so 16 warps fit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dft_reg.cuh"

namespace fcc {

constexpr int kSlab128Warps = 16;
constexpr int kSlab128Threads = 32 * kSlab128Warps;
constexpr int kSlab128LD = 132;   // complex values per slab row in shared memory
constexpr size_t kSlab128Smem = (size_t)(128 * kSlab128LD + 2 * 128) * sizeof(float2);

__device__ __forceinline__ int slab128_xpos(int j, int k2) { return 16 * j + ((k2 + (j & 3) + 8 * (j >> 2)) & 15); }
__device__ __forceinline__ int slab128_u(int q) { return (q & 3) + 8 * (q >> 2); }

// Length-16 DFT of (vr, vi) and the twiddle of stage 1 for thread j.
template <int S>
__device__ __forceinline__ void slab128_stage1(float* vr, float* vi, int j, const float2* tw) {
    reg::Dft<16, S, float>::run(vr, vi);
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) {
        const float2 w = tw[(j * k2) & 127];
        const float wi = S > 0 ? w.y : -w.y;
        const float t = vr[k2] * w.x - vi[k2] * wi;
        vi[k2] = vr[k2] * wi + vi[k2] * w.x;
        vr[k2] = t;
    }
}

// grid.x = volumes * 128 slabs; volume v at voff[v] (or v * vstride) complex
// values; in and out may alias (a block reads its whole slab before it
// writes).  PRE: inputs multiplied by pre[c], c the index along the fastest
// axis.
template <int S, bool PRE>
__global__ void __launch_bounds__(kSlab128Threads, 1)
fft_slab128_kernel(const float2* in, float2* out, const float2* __restrict__ twg, int64_t vstride,
                   const int64_t* voff, const float2* __restrict__ preg) {
    constexpr int N = 128, LD = kSlab128LD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* slab = reinterpret_cast<float2*>(smem_raw);
    float2* tw = slab + N * LD;
    float2* pre = tw + N;
    const int64_t vol = blockIdx.x / N;
    const int64_t base = (voff ? voff[vol] : vol * vstride) + (int64_t)(blockIdx.x % N) * N * N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < N; t += kSlab128Threads) {
        tw[t] = twg[t];
        if (PRE) pre[t] = preg[t];
    }
    // rows: 4 pencils per warp (lane = 8 p + j), 64 rows per round, both
    // rounds' loads in flight before the first transform
    {
        const int p = lane >> 3, j = lane & 7;
        float vr[2][16], vi[2][16];
#pragma unroll
        for (int rd = 0; rd < 2; ++rd) {
            const float2* src = in + base + (int64_t)(rd * 64 + warp * 4 + p) * N + j;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const float2 t = src[8 * m];
                vr[rd][m] = t.x;
                vi[rd][m] = t.y;
            }
        }
        __syncthreads();   // twiddles and modulation staged
#pragma unroll
        for (int rd = 0; rd < 2; ++rd) {
            float2* row = slab + (rd * 64 + warp * 4 + p) * LD;
            if (PRE) {
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    const float2 w = pre[j + 8 * m];
                    const float t = vr[rd][m] * w.x - vi[rd][m] * w.y;
                    vi[rd][m] = vr[rd][m] * w.y + vi[rd][m] * w.x;
                    vr[rd][m] = t;
                }
            }
            slab128_stage1<S>(vr[rd], vi[rd], j, tw);
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) row[slab128_xpos(j, k2)] = make_float2(vr[rd][k2], vi[rd][k2]);
            __syncwarp();
            float ur[2][8], ui[2][8];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const float2 t = row[slab128_xpos(jj, slab128_u(j) + 4 * e)];
                    ur[e][jj] = t.x;
                    ui[e][jj] = t.y;
                }
            }
            __syncwarp();   // every exchange read done before the row is overwritten
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                reg::Dft<8, S, float>::run(ur[e], ui[e]);
#pragma unroll
                for (int k1 = 0; k1 < 8; ++k1) row[slab128_u(j) + 4 * e + 16 * k1] = make_float2(ur[e][k1], ui[e][k1]);
            }
        }
    }
    __syncthreads();
    // columns: 4 columns per warp (lane = 4 j + cl), 64 columns per round
    {
        const int cl = lane & 3, j = lane >> 2;
#pragma unroll 1
        for (int rd = 0; rd < 2; ++rd) {
            const int c = rd * 64 + warp * 4 + cl;
            float2* col = slab + c;
            float vr[16], vi[16];
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const float2 t = col[(j + 8 * m) * LD];
                vr[m] = t.x;
                vi[m] = t.y;
            }
            __syncwarp();   // every input of the column read before the exchange overwrites it
            slab128_stage1<S>(vr, vi, j, tw);
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) col[slab128_xpos(j, k2) * LD] = make_float2(vr[k2], vi[k2]);
            __syncwarp();
            float ur[2][8], ui[2][8];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const float2 t = col[slab128_xpos(jj, slab128_u(j) + 4 * e) * LD];
                    ur[e][jj] = t.x;
                    ui[e][jj] = t.y;
                }
            }
            float2* dst = out + base + c;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                reg::Dft<8, S, float>::run(ur[e], ui[e]);
#pragma unroll
                for (int k1 = 0; k1 < 8; ++k1)
                    dst[(int64_t)(slab128_u(j) + 4 * e + 16 * k1) * N] = make_float2(ur[e][k1], ui[e][k1]);
            }
        }
    }
}

}  // namespace fcc
