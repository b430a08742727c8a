// Measurement aid: the global-memory accesses of the forward tensor-core
// mixing (mix_tc_fwd_pair_kernel) with its arithmetic taken out.
//
// Same grid, block size, dynamic shared memory (so the same resident blocks
// per SM), group order and addresses: per group of 4 plan tiles every
// thread gathers its 12 slots of both volumes of the pair (gather_half) and
// stores 12 complex values where the epilogue stores (canonical slots of a
// boundary class only).  No operand split, no MMA, no tensor memory, no
// barrier.  Its time is the ceiling the mixing's own access pattern puts on
// the mixing kernel; what it writes is meaningless.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mix_tc.cuh"

namespace fcc {

template <int H, bool BND>
__device__ __forceinline__ void replay_store_half(const TiledMixArgs& a, uint32_t rep, const int* off, uint32_t cmask,
                                                  float2* out, int64_t pb, const float* vr, const float* vi) {
    if (rep == 0xffffffffu) return;
    static_for<0, 12>([&](auto Sc) {
        constexpr int g = H + decltype(Sc)::value;
        const int gi = rep_dot(rep, a.lin[g][0], a.lin[g][1], a.lin[g][2]) + (BND ? __ldg(off + g) : a.lin[g][3]);
        if (!BND || ((cmask >> g) & 1u)) out[pb + gi] = make_float2(vr[g - H], vi[g - H]);
    });
}

template <int KIND>
__global__ void __launch_bounds__(kTcThreads, TcLayout<KIND>::blocks_per_sm)
mix_replay_pair_kernel(const float* __restrict__ in, float* __restrict__ out, const TiledMixArgs a, int nfree_tiles,
                       const uint32_t* __restrict__ reps32, const TcBoundary bnd) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int half = tid >> 7, wq = warp & 3;
    const int64_t pb = (int64_t)blockIdx.y * 2 * a.n3;
    const float* __restrict__ in0 = in + pb;
    const float* __restrict__ in1 = in + pb + a.n3;
    float2* o2 = reinterpret_cast<float2*>(out);
    const uint32_t kNone = 0xffffffffu;
    const int ngroups = (nfree_tiles + 3) / 4;
    const int nall = ngroups + bnd.ngroups;
    float vr[12], vi[12];
    for (int grp = blockIdx.x; grp < nall; grp += (int)gridDim.x) {
        if (grp < ngroups) {
            const int tile = grp * 4 + wq;
            const uint32_t rp = tile < nfree_tiles ? __ldg(reps32 + (size_t)tile * 32 + lane) : kNone;
            if (half == 0) {
                gather_half<0, false>(a, in0, in1, rp, nullptr, vr, vi);
                replay_store_half<0, false>(a, rp, nullptr, 0u, o2, pb, vr, vi);
            } else {
                gather_half<12, false>(a, in0, in1, rp, nullptr, vr, vi);
                replay_store_half<12, false>(a, rp, nullptr, 0u, o2, pb, vr, vi);
            }
        } else {
            const int* gr = bnd.group + 8 * (grp - ngroups);
            const int cls = __ldg(gr);
            const int tile = __ldg(gr + 1 + wq);
            const uint32_t rp = tile >= 0 ? __ldg(reps32 + (size_t)tile * 32 + lane) : kNone;
            const int* off = bnd.off + 24 * cls;
            const uint32_t cm = __ldg(bnd.canon_mask + cls);
            if (half == 0) {
                gather_half<0, true>(a, in0, in1, rp, off, vr, vi);
                replay_store_half<0, true>(a, rp, off, cm, o2, pb, vr, vi);
            } else {
                gather_half<12, true>(a, in0, in1, rp, off, vr, vi);
                replay_store_half<12, true>(a, rp, off, cm, o2, pb, vr, vi);
            }
        }
    }
}

}  // namespace fcc
