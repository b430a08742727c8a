// Orbit mixing of shifted plans, DCT_n(r,s,t) of Def. 2: the tiled body of
// mix_tiled.cuh with the plan's free-orbit core and row-phase weights as a
// __grid_constant__ parameter (SKEW), in a translation unit of its own.
#include "fft_fast.cuh"
#include "mix_tiled.cuh"

namespace fcc {

namespace {

template <int MODE, bool RIN, bool ROUT>
__global__ void __launch_bounds__(kMixThreads, 3)
mix_skew_kernel(const float* __restrict__ in, float* __restrict__ out, const __grid_constant__ TiledMixArgs a,
                const __grid_constant__ SkewCore sc, int ntiles, int tile0, int core_in_smem) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    mix_tiled_body<MODE, RIN, ROUT, false, true>(in, out, a, ntiles, tile0 + blockIdx.x * kMixWarps + (threadIdx.x >> 5),
                                                 blockIdx.y, core_in_smem, nullptr, smem_raw, &sc);
}

template <int MODE, bool RIN, bool ROUT>
cudaError_t launch_one(const TiledMixArgs& a, const SkewCore& sc, const float* in, float* out, int tile0, int ntiles,
                       bool boundary, int64_t nvol, cudaStream_t st) {
    static DeviceOnce attr;
    if (!attr.done()) {
        cudaFuncSetAttribute(mix_skew_kernel<MODE, RIN, ROUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mix_tiled_smem_core(a.n));
        attr.mark();
    }
    const size_t smem = boundary ? mix_tiled_smem_core(a.n) : mix_tiled_smem(a.n);
    const int64_t vin = a.n3 * ((MODE == MODE_FWD && RIN) ? 1 : 2);
    const int64_t vout = a.n3 * ((MODE != MODE_FWD && ROUT) ? 1 : 2);
    for (int64_t v0 = 0; v0 < nvol; v0 += 65535) {
        const int64_t nv = nvol - v0 < 65535 ? nvol - v0 : 65535;
        dim3 grid((unsigned)((ntiles - tile0 + kMixWarps - 1) / kMixWarps), (unsigned)nv);
        mix_skew_kernel<MODE, RIN, ROUT><<<grid, kMixThreads, smem, st>>>(in + v0 * vin, out + v0 * vout, a, sc, ntiles,
                                                                          tile0, boundary ? 1 : 0);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mix_tiled_skew(const TiledMixArgs& a, const SkewCore& sc, int mode, bool real_io, const float* in,
                                  float* out, int tile0, int ntiles, bool boundary, int64_t nvol, cudaStream_t st) {
    if (a.ncls > kMaxClasses || ntiles <= tile0) return cudaErrorInvalidValue;
    if (mode == MODE_FWD)
        return real_io ? launch_one<MODE_FWD, true, false>(a, sc, in, out, tile0, ntiles, boundary, nvol, st)
                       : launch_one<MODE_FWD, false, false>(a, sc, in, out, tile0, ntiles, boundary, nvol, st);
    if (mode == MODE_INV)
        return real_io ? launch_one<MODE_INV, false, true>(a, sc, in, out, tile0, ntiles, boundary, nvol, st)
                       : launch_one<MODE_INV, false, false>(a, sc, in, out, tile0, ntiles, boundary, nvol, st);
    return real_io ? launch_one<MODE_ADJ, false, true>(a, sc, in, out, tile0, ntiles, boundary, nvol, st)
                   : launch_one<MODE_ADJ, false, false>(a, sc, in, out, tile0, ntiles, boundary, nvol, st);
}

}  // namespace fcc
