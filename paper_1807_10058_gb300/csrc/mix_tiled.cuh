// Orbit mixing S, S^{-1}, S^H over tiles of representatives (FP32).
//
// One block per tile (<= kTileMax orbits) and volume, three phases:
//   gather   for each slot g, warp lanes walk the tile along the direction
//            that slot g maps to contiguous memory (c_dir[g]) and stage the
//            24 slot values of every orbit in shared memory;
//   core     one thread per orbit: the class core (free orbits: c_core in
//            constant memory, indices known at compile time) and the row
//            phases R_g = exp(2 pi i (W_g kO).v / (8n));
//   scatter  same walk as the gather, canonical slots only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "plan.h"

namespace fcc {

__constant__ float2 c_core[3][24][24];  // free-orbit cores: forward, inverse, adjoint
__constant__ int c_dir[24];

struct TiledMixArgs {
    const int32_t* tile_off;
    const uint32_t* reps;
    const uint8_t* cls;
    const uint16_t* permb;
    const uint16_t* permc;
    const float* mats;          // [ncls][24][24][2] core of this mode for every class
    const int8_t* wrap;         // [ncls][24][3]
    const uint32_t* canon_mask; // [ncls]
    const float2* phase;        // [8n]
    int n;
    int free_class;
    int64_t n3;
    float scale;
};

constexpr int kMixRow = 50;  // floats per orbit row in shared memory (24 complex + pad)

__device__ __forceinline__ int tile_pick(int dir, int t, const uint16_t* pb, const uint16_t* pc) {
    return dir == 1 ? (int)pb[t] : dir == 2 ? (int)pc[t] : t;
}

__device__ __forceinline__ int slot_index(int g, uint32_t rp, const int8_t* wr, int n) {
    const int k0 = rp & 1023, k1 = (rp >> 10) & 1023, k2 = (rp >> 20) & 1023;
    const int p0 = c_W[g][0] * k0 + c_W[g][1] * k1 + c_W[g][2] * k2 - n * wr[3 * g + 0];
    const int p1 = c_W[g][3] * k0 + c_W[g][4] * k1 + c_W[g][5] * k2 - n * wr[3 * g + 1];
    const int p2 = c_W[g][6] * k0 + c_W[g][7] * k1 + c_W[g][8] * k2 - n * wr[3 * g + 2];
    return (p0 * n + p1) * n + p2;
}

__device__ __forceinline__ int phase_exp(int g, uint32_t rp, int M8) {
    const int k0 = rp & 1023, k1 = (rp >> 10) & 1023, k2 = (rp >> 20) & 1023;
    int e = (c_u[g][0] * k0 + c_u[g][1] * k1 + c_u[g][2] * k2) % M8;
    return e < 0 ? e + M8 : e;
}

template <int MODE, bool RIN, bool ROUT>
__global__ void __launch_bounds__(kTileMax) mix_tiled_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                             TiledMixArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* rows = reinterpret_cast<float*>(smem_raw);                 // [kTileMax][kMixRow]
    float2* ph = reinterpret_cast<float2*>(rows + kTileMax * kMixRow);  // [8n]
    uint32_t* s_rep = reinterpret_cast<uint32_t*>(ph + 8 * a.n);
    uint16_t* s_pb = reinterpret_cast<uint16_t*>(s_rep + kTileMax);
    uint16_t* s_pc = s_pb + kTileMax;
    uint8_t* s_cls = reinterpret_cast<uint8_t*>(s_pc + kTileMax);

    const int tile = blockIdx.x;
    const int64_t vol = blockIdx.y;
    const int o0 = a.tile_off[tile];
    const int cnt = a.tile_off[tile + 1] - o0;
    const int t = threadIdx.x;
    const int n = a.n, M8 = 8 * n;
    if (t < cnt) {
        s_rep[t] = a.reps[o0 + t];
        s_cls[t] = a.cls[o0 + t];
        s_pb[t] = a.permb[o0 + t];
        s_pc[t] = a.permc[o0 + t];
    }
    for (int e = t; e < M8; e += blockDim.x) ph[e] = a.phase[e];
    __syncthreads();

    // gather: forward reads x (real or complex); inverse/adjoint read Z (complex)
    constexpr bool CIN = (MODE != MODE_FWD) || !RIN;
    const int64_t in_base = vol * a.n3;
    if (t < cnt) {
        for (int g = 0; g < 24; ++g) {
            const int r = tile_pick(c_dir[g], t, s_pb, s_pc);
            const uint32_t rp = s_rep[r];
            const int idx = slot_index(g, rp, a.wrap + 72 * s_cls[r], n);
            if (CIN) {
                const float2 v = reinterpret_cast<const float2*>(in)[in_base + idx];
                *reinterpret_cast<float2*>(rows + r * kMixRow + 2 * g) = v;
            } else {
                rows[r * kMixRow + 2 * g] = in[in_base + idx];
            }
        }
    }
    __syncthreads();

    // core: one thread per orbit, in place in its own row
    if (t < cnt) {
        float* row = rows + t * kMixRow;
        const uint32_t rp = s_rep[t];
        const int c = s_cls[t];
        float xr[24], xi[24];
#pragma unroll
        for (int h = 0; h < 24; ++h) {
            if (CIN) {
                const float2 v = *reinterpret_cast<const float2*>(row + 2 * h);
                xr[h] = v.x;
                xi[h] = v.y;
            } else {
                xr[h] = row[2 * h];
                xi[h] = 0.f;
            }
        }
        if (MODE != MODE_FWD) {
            // t_g = conj(R_g) Z_g
#pragma unroll
            for (int g = 0; g < 24; ++g) {
                const float2 R = ph[phase_exp(g, rp, M8)];
                const float zr = xr[g], zi = xi[g];
                xr[g] = R.x * zr + R.y * zi;
                xi[g] = R.x * zi - R.y * zr;
            }
        }
        const bool fast = c == a.free_class;
        const float* M = a.mats + (size_t)c * 1152;
#pragma unroll
        for (int g = 0; g < 24; ++g) {
            float ar = 0.f, ai = 0.f;
            if (fast) {
#pragma unroll
                for (int h = 0; h < 24; ++h) {
                    const float2 m = c_core[MODE][g][h];
                    ar = fmaf(m.x, xr[h], ar);
                    ai = fmaf(m.y, xr[h], ai);
                    if (CIN) {
                        ar = fmaf(-m.y, xi[h], ar);
                        ai = fmaf(m.x, xi[h], ai);
                    }
                }
            } else {
                for (int h = 0; h < 24; ++h) {
                    const float mr = __ldg(M + 2 * (g * 24 + h)), mi = __ldg(M + 2 * (g * 24 + h) + 1);
                    ar = fmaf(mr, xr[h], ar);
                    ai = fmaf(mi, xr[h], ai);
                    if (CIN) {
                        ar = fmaf(-mi, xi[h], ar);
                        ai = fmaf(mr, xi[h], ai);
                    }
                }
            }
            if (MODE == MODE_FWD) {
                const float2 R = ph[phase_exp(g, rp, M8)];
                const float zr = R.x * ar - R.y * ai, zi = R.x * ai + R.y * ar;
                *reinterpret_cast<float2*>(row + 2 * g) = make_float2(a.scale * zr, a.scale * zi);
            } else if (ROUT) {
                row[2 * g] = a.scale * ar;
            } else {
                *reinterpret_cast<float2*>(row + 2 * g) = make_float2(a.scale * ar, a.scale * ai);
            }
        }
    }
    __syncthreads();

    // scatter canonical slots
    const bool COUT = (MODE == MODE_FWD) || !ROUT;
    if (t < cnt) {
        for (int g = 0; g < 24; ++g) {
            const int r = tile_pick(c_dir[g], t, s_pb, s_pc);
            const int c = s_cls[r];
            if (!((a.canon_mask[c] >> g) & 1u)) continue;
            const int idx = slot_index(g, s_rep[r], a.wrap + 72 * c, n);
            if (COUT) {
                reinterpret_cast<float2*>(out)[in_base + idx] = *reinterpret_cast<const float2*>(rows + r * kMixRow + 2 * g);
            } else {
                out[in_base + idx] = rows[r * kMixRow + 2 * g];
            }
        }
    }
}

inline size_t mix_tiled_smem(int n) {
    return (size_t)kTileMax * kMixRow * 4 + (size_t)8 * n * 8 + kTileMax * (4 + 2 + 2 + 1) + 16;
}

}  // namespace fcc
