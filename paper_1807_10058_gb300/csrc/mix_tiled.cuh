// Orbit mixing S, S^{-1}, S^H over tiles of representatives (FP32).
//
// One warp per tile (<= 32 orbits forming a 4 x 4 x 2 box of
// representatives); warps are independent (no block barrier).  Three phases:
//   gather   for every slot g (unrolled, geometry known at compile time) each
//            thread loads one value; lanes walk the tile along the direction
//            slot g maps onto contiguous memory (wc::K::t.dir[g]).  All 24
//            loads are in flight before the first shared-memory store;
//   core     one thread per orbit: the class core (free orbits: c_core in
//            constant memory) and the row phases R_g = w_{8n}^{(W_g kO).v};
//   scatter  the same walk back to global memory, canonical slots only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "kernels.cuh"
#include "plan.h"
#include "weyl_const.h"

namespace fcc {

static __constant__ float2 c_core[3][24][24];  // free-orbit cores: forward, inverse, adjoint

constexpr int kMaxClasses = 16;

struct TiledMixArgs {
    const int32_t* tile_off;
    const uint32_t* reps;
    const uint8_t* cls;
    const uint8_t* permb;
    const uint8_t* permc;
    const float* mats;          // [ncls][24][24][2] core of this mode for every class
    const int8_t* wrap;         // [ncls][24][3]
    const uint32_t* canon_mask; // [ncls]
    const float2* phase;        // [M]: exp(2 pi i e / M)
    const int* uv;              // [24][3] W_g^T v of the plan's shift c = v / d (device)
    int M;                      // d n
    // flat index of slot g of a free orbit: k . lin[g] + lin[g][3]; lin[g][0..2]
    // are the columns of W_g weighted by (n^2, n, 1), lin[g][3] the wrap offset
    int lin[24][4];
    int n;
    int ncls;
    int free_class;
    int64_t n3;
    float scale;
};

constexpr int kMixRow = 50;  // floats per orbit row in shared memory (24 complex + pad)

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// Compile-time entries of W (read only in constant expressions).
template <int G, int I> struct WU { static constexpr int v = wc::K::t.u[G][I]; };
template <int G> struct WD { static constexpr int v = wc::K::t.dir[G]; };


constexpr int kMixWarps = 8;                 // warps (= independent tiles) per block
constexpr int kMixThreads = 32 * kMixWarps;

__device__ __forceinline__ int rep_dot(uint32_t rp, int a0, int a1, int a2) {
    return (int)(rp & 1023) * a0 + (int)((rp >> 10) & 1023) * a1 + (int)((rp >> 20) & 1023) * a2;
}

// flat index of slot G: affine in the representative; non-free orbits take
// their class's wrap vector instead of the free one
template <int G>
__device__ __forceinline__ int slot_flat(const TiledMixArgs& a, uint32_t rp, bool free_orbit, int cls) {
    const int lin = rep_dot(rp, a.lin[G][0], a.lin[G][1], a.lin[G][2]);
    if (free_orbit) return lin + a.lin[G][3];
    const int8_t* wr = a.wrap + 72 * cls + 3 * G;
    const int n = a.n;
    return lin - n * ((int)__ldg(wr) * n * n + (int)__ldg(wr + 1) * n + (int)__ldg(wr + 2));
}

// row-phase exponent (W_G kO).v mod 8n, v = (1, 0, 3)
template <int G>
__device__ __forceinline__ int slot_exp(uint32_t rp, int M8) {
    const int q = rep_dot(rp, WU<G, 0>::v, WU<G, 1>::v, WU<G, 2>::v);
    return q < 0 ? q + M8 : q;
}

// The free-orbit core of one mode and the row-phase weights of a skew plan,
// passed to its kernels as a __grid_constant__ parameter: with compile-time
// slot indices they are read from the constant bank, as c_core and the
// compile-time weights are for the shift (1/8, 0, 3/8).
struct SkewCore {
    float2 m[24][24];
    int u[24][3];
};

// row-phase exponent of slot g for any shift: (W_g kO).v mod M from the
// plan's weights (skew plans; the canonical kernels use slot_exp)
__device__ __forceinline__ int skew_exp(const TiledMixArgs& a, uint32_t rp, int g) {
    const int* u = a.uv + 3 * g;
    const int q = rep_dot(rp, __ldg(u), __ldg(u + 1), __ldg(u + 2)) % a.M;
    return q < 0 ? q + a.M : q;
}

// grid.x covers the tiles (kMixWarps per block), grid.y the volumes (pairs
// of real volumes when PAIR: forward reads x1 + i x2 from volumes 2p, 2p+1
// and writes Z to volume 2p of the complex output; inverse / adjoint read a
// compact complex volume p and write Re / Im to real volumes 2p, 2p+1).
// One warp's tile `tile` of volume `vol` (warp = threadIdx.x / 32 < kMixWarps
// selects its shared-memory slot); a warp past ntiles returns at once.
// SKEW: a shifted transform DCT_n(r,s,t); free orbits take the core and
// the row-phase weights of `sc`, boundary tiles their staged class core and
// the plan's weights (the constant-memory free core and the compile-time
// weights belong to the shift (1/8, 0, 3/8)).
template <int MODE, bool RIN, bool ROUT, bool PAIR = false, bool SKEW = false>
__device__ __forceinline__ void mix_tiled_body(const float* __restrict__ in, float* __restrict__ out,
                                               const TiledMixArgs& a, int ntiles, int tile, int64_t vol,
                                               int core_in_smem, const int64_t* voff, unsigned char* smem_raw,
                                               const SkewCore* sc = nullptr) {
    constexpr bool CIN = (MODE != MODE_FWD) || !RIN || PAIR;    // complex values in the core
    constexpr bool COUT = (MODE == MODE_FWD) || !ROUT || PAIR;  // complex values out of the core
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* rows = reinterpret_cast<float*>(smem_raw) + warp * (32 * kMixRow);   // this warp's [32][kMixRow]
    if (tile >= ntiles) return;                      // warp-uniform; no block barrier below
    // unpaired volume offset (values): ragged batches pass a table of point
    // offsets; paired: the two volumes of the pair (ragged batches: a table of
    // two point offsets per pair), Z in the first volume's complex region
    const int64_t base = voff && !PAIR ? voff[vol] : vol * a.n3;
    const int64_t pb = PAIR && voff ? voff[2 * vol] : vol * 2 * a.n3;
    const int64_t pb1 = PAIR && voff ? voff[2 * vol + 1] : pb + a.n3;
    const int o0 = a.tile_off[tile];
    const int cnt = a.tile_off[tile + 1] - o0;
    const int M8 = 8 * a.n;
    const bool act = lane < cnt;
    uint32_t myrep = 0;
    int mycls = a.free_class < 0 ? 0 : a.free_class;
    int rsel[4] = {lane, lane, lane, lane};
    if (act) {
        myrep = __ldg(a.reps + o0 + lane);
        mycls = __ldg(a.cls + o0 + lane);
        rsel[1] = __ldg(a.permb + o0 + lane);
        rsel[2] = __ldg(a.permc + o0 + lane);
    }
    const bool free_orbit = mycls == a.free_class;
    const uint32_t mycanon = free_orbit ? 0xffffffu : __ldg(a.canon_mask + mycls);
    const float2* __restrict__ ph = a.phase;

    // ---- gather: lanes walk the tile in the order slot g maps to memory;
    // the owning lane computes each index and shuffles it over
    {
        float vr[24], vi[24];
        static_for<0, 24>([&](auto Gc) {
            constexpr int g = decltype(Gc)::value;
            const int r = rsel[WD<g>::v];
            const int gi = __shfl_sync(0xffffffffu, slot_flat<g>(a, myrep, free_orbit, mycls), r);
            vr[g] = 0.f;
            vi[g] = 0.f;
            if (act) {
                if (PAIR && MODE == MODE_FWD) {
                    vr[g] = __ldg(in + pb + gi);
                    vi[g] = __ldg(in + pb1 + gi);
                } else if (CIN) {
                    const float2 v = __ldg(reinterpret_cast<const float2*>(in) + base + gi);
                    vr[g] = v.x;
                    vi[g] = v.y;
                } else {
                    vr[g] = __ldg(in + base + gi);
                }
            }
        });
        if (act) {
            static_for<0, 24>([&](auto Gc) {
                constexpr int g = decltype(Gc)::value;
                const int r = rsel[WD<g>::v];
                if (CIN) *reinterpret_cast<float2*>(rows + r * kMixRow + 2 * g) = make_float2(vr[g], vi[g]);
                else rows[r * kMixRow + 2 * g] = vr[g];
            });
        }
    }
    // boundary tiles (one class per tile): all 32 lanes stage the class core
    if (core_in_smem) {
        const int tcls = __shfl_sync(0xffffffffu, mycls, 0);
        if (tcls != a.free_class) {
            float* Ms = reinterpret_cast<float*>(smem_raw) + kMixWarps * 32 * kMixRow + warp * 1152;
            const float4* src = reinterpret_cast<const float4*>(a.mats + (size_t)tcls * 1152);
            for (int e = lane; e < 1152 / 4; e += 32) reinterpret_cast<float4*>(Ms)[e] = __ldg(src + e);
        }
    }
    __syncwarp();
    // ---- core: lane = orbit, in place in its own row
    if (act) {
        float* row = rows + lane * kMixRow;
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
            static_for<0, 24>([&](auto Gc) {
                constexpr int g = decltype(Gc)::value;
                int q;
                if constexpr (SKEW) {
                    q = rep_dot(myrep, sc->u[g][0], sc->u[g][1], sc->u[g][2]) % a.M;
                    q = q < 0 ? q + a.M : q;
                } else {
                    q = slot_exp<g>(myrep, M8);
                }
                const float2 R = __ldg(ph + q);
                const float zr = xr[g], zi = xi[g];
                xr[g] = R.x * zr + R.y * zi;  // conj(R) Z
                xi[g] = R.x * zi - R.y * zr;
            });
        }
        if (free_orbit) {
            static_for<0, 24>([&](auto Gc) {
                constexpr int g = decltype(Gc)::value;
                float ar = 0.f, ai = 0.f;
#pragma unroll
                for (int h = 0; h < 24; ++h) {
                    float2 m;
                    if constexpr (SKEW) m = sc->m[g][h];
                    else m = c_core[MODE][g][h];
                    ar = fmaf(m.x, xr[h], ar);
                    ai = fmaf(m.y, xr[h], ai);
                    if (CIN) {
                        ar = fmaf(-m.y, xi[h], ar);
                        ai = fmaf(m.x, xi[h], ai);
                    }
                }
                if (MODE == MODE_FWD) {
                    int q;
                    if constexpr (SKEW) {
                        q = rep_dot(myrep, sc->u[g][0], sc->u[g][1], sc->u[g][2]) % a.M;
                        q = q < 0 ? q + a.M : q;
                    } else {
                        q = slot_exp<g>(myrep, M8);
                    }
                    const float2 R = __ldg(ph + q);
                    *reinterpret_cast<float2*>(row + 2 * g) =
                        make_float2(a.scale * (R.x * ar - R.y * ai), a.scale * (R.x * ai + R.y * ar));
                } else if (ROUT && !PAIR) {
                    row[2 * g] = a.scale * ar;
                } else {
                    *reinterpret_cast<float2*>(row + 2 * g) = make_float2(a.scale * ar, a.scale * ai);
                }
            });
        } else {
            // orbits on the alcove boundary: the tile's class core (staged in
            // this warp's shared-memory slot above, when the launch provides one)
            const float* M = core_in_smem ? reinterpret_cast<const float*>(smem_raw) + kMixWarps * 32 * kMixRow + warp * 1152
                                          : a.mats + (size_t)mycls * 1152;
#pragma unroll 1
            for (int g = 0; g < 24; ++g) {
                float ar = 0.f, ai = 0.f;
#pragma unroll
                for (int h = 0; h < 24; ++h) {
                    const float2 m = *reinterpret_cast<const float2*>(M + 2 * (g * 24 + h));
                    ar = fmaf(m.x, xr[h], ar);
                    ai = fmaf(m.y, xr[h], ai);
                    if (CIN) {
                        ar = fmaf(-m.y, xi[h], ar);
                        ai = fmaf(m.x, xi[h], ai);
                    }
                }
                if (MODE == MODE_FWD) {
                    int q;
                    if constexpr (SKEW) {
                        q = skew_exp(a, myrep, g);
                    } else {
                        q = (int)(myrep & 1023) * c_u[g][0] + (int)((myrep >> 10) & 1023) * c_u[g][1] +
                            (int)((myrep >> 20) & 1023) * c_u[g][2];
                        q = q < 0 ? q + M8 : q;
                    }
                    const float2 R = __ldg(ph + q);
                    *reinterpret_cast<float2*>(row + 2 * g) =
                        make_float2(a.scale * (R.x * ar - R.y * ai), a.scale * (R.x * ai + R.y * ar));
                } else if (ROUT && !PAIR) {
                    row[2 * g] = a.scale * ar;
                } else {
                    *reinterpret_cast<float2*>(row + 2 * g) = make_float2(a.scale * ar, a.scale * ai);
                }
            }
        }
    }
    __syncwarp();
    // ---- scatter canonical slots
    const uint32_t can_d[3] = {mycanon, __shfl_sync(0xffffffffu, mycanon, rsel[1]),
                               __shfl_sync(0xffffffffu, mycanon, rsel[2])};
    static_for<0, 24>([&](auto Gc) {
        constexpr int g = decltype(Gc)::value;
        constexpr int d = WD<g>::v;
        const int r = rsel[d];
        const int gi = __shfl_sync(0xffffffffu, slot_flat<g>(a, myrep, free_orbit, mycls), r);
        const uint32_t cm = d == 1 ? can_d[1] : d == 2 ? can_d[2] : can_d[0];
        if (act && ((cm >> g) & 1u)) {
            if (PAIR && MODE == MODE_FWD) {
                reinterpret_cast<float2*>(out)[pb + gi] = *reinterpret_cast<const float2*>(rows + r * kMixRow + 2 * g);
            } else if (PAIR) {
                const float2 v = *reinterpret_cast<const float2*>(rows + r * kMixRow + 2 * g);
                out[pb + gi] = v.x;
                out[pb1 + gi] = v.y;
            } else if (COUT) {
                reinterpret_cast<float2*>(out)[base + gi] = *reinterpret_cast<const float2*>(rows + r * kMixRow + 2 * g);
            } else {
                out[base + gi] = rows[r * kMixRow + 2 * g];
            }
        }
    });
}

template <int MODE, bool RIN, bool ROUT, bool PAIR = false>
__global__ void __launch_bounds__(kMixThreads, 3) mix_tiled_kernel(const float* __restrict__ in,
                                                                   float* __restrict__ out, const TiledMixArgs a,
                                                                   int ntiles, int tile0 = 0, int core_in_smem = 0,
                                                                   const int64_t* voff = nullptr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    mix_tiled_body<MODE, RIN, ROUT, PAIR>(in, out, a, ntiles, tile0 + blockIdx.x * kMixWarps + (threadIdx.x >> 5),
                                          blockIdx.y, core_in_smem, voff, smem_raw);
}

inline size_t mix_tiled_smem(int) { return (size_t)kMixWarps * 32 * kMixRow * 4; }
// launches over boundary tiles also stage one class core per warp
inline size_t mix_tiled_smem_core(int n) { return mix_tiled_smem(n) + (size_t)kMixWarps * 1152 * 4; }

// Skew plans (mix_skew.cu): tiles [tile0, ntiles) of `nvol` volumes (the
// free tiles on sc, the boundary tiles on their staged class cores: a launch
// covers one kind), `mode` with real input (forward) or real output (inverse
// / adjoint) as given; volume v of in / out at v n^3 values of the real or
// complex type.
cudaError_t launch_mix_tiled_skew(const TiledMixArgs& a, const SkewCore& sc, int mode, bool real_io, const float* in,
                                  float* out, int tile0, int ntiles, bool boundary, int64_t nvol, cudaStream_t st);

}  // namespace fcc
