// The persistent ragged-batch kernel (see ragged.cuh), in a translation unit
// of its own: it instantiates the DFT bodies of every register-radix order.
#include <cooperative_groups.h>

#include "fft_fast.cuh"
#include "ragged.cuh"

namespace cg = cooperative_groups;

namespace fcc {

namespace {

// order index of unit u of stage s (orders listed with increasing first unit)
__device__ __forceinline__ int order_of(const RaggedArgs& ra, int s, int64_t u) {
    int o = 0;
    while (o + 1 < ra.norders && ra.o[o + 1].first[s] <= u) ++o;
    return o;
}

template <int N>
__device__ __forceinline__ void slab_unit(const RaggedOrder& A, float* out, int64_t lu, unsigned char* smem) {
    const int64_t vol = lu / N;
    const int64_t base = A.voff[vol] + (lu % N) * (int64_t)N * N;
    fft_slab_body<N, 1, kRaggedThreads / 32>((const float2*)out, (float2*)out, A.tw, base, smem);
}

template <int N>
__device__ __forceinline__ void pencil_unit(const RaggedOrder& A, float* out, int64_t lu, unsigned char* smem) {
    constexpr int CBLK = (N + FastLayout<N>::CPB - 1) / FastLayout<N>::CPB;
    const int64_t vol = lu / (N * CBLK);
    const int rem = (int)(lu - vol * N * CBLK);
    fft_pencil_body<N, 1>((const float2*)out, (float2*)out, A.tw, A.voff[vol], rem / CBLK, rem % CBLK, smem);
}

#define FCC_RAGGED_ORDERS(X) X(128) X(96) X(88) X(80) X(72) X(64) X(56) X(48) X(40) X(32) X(24) X(16) X(8)

__global__ void __launch_bounds__(kRaggedThreads, 1)
ragged_persistent_kernel(const float* __restrict__ in, float* out, const __grid_constant__ RaggedArgs ra) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::grid_group grid = cg::this_grid();
    const int warp = threadIdx.x >> 5;
    // 1. orbit mixing: warps are independent (own shared-memory slots)
    for (int64_t u = blockIdx.x; u < ra.units[0]; u += gridDim.x) {
        const RaggedOrder& A = ra.o[order_of(ra, 0, u)];
        const int64_t lu = u - A.first[0];
        const int upv = (A.ntiles + kMixWarps - 1) / kMixWarps;
        const int64_t vol = lu / upv;
        const int tile = (int)(lu - vol * upv) * kMixWarps + warp;
        if (ra.real_in)
            mix_tiled_body<MODE_FWD, true, false>(in, out, A.mix, A.ntiles, tile, vol, 1, A.voff, smem_raw);
        else
            mix_tiled_body<MODE_FWD, false, false>(in, out, A.mix, A.ntiles, tile, vol, 1, A.voff, smem_raw);
        __syncwarp();
    }
    __threadfence();
    grid.sync();
    // 2. slabs (block-wide: the body synchronises the block)
    for (int64_t u = blockIdx.x; u < ra.units[1]; u += gridDim.x) {
        const RaggedOrder& A = ra.o[order_of(ra, 1, u)];
        const int64_t lu = u - A.first[1];
        switch (A.mix.n) {
#define FCC_CASE(NN) case NN: slab_unit<NN>(A, out, lu, smem_raw); break;
            FCC_RAGGED_ORDERS(FCC_CASE)
#undef FCC_CASE
            default: break;
        }
        __syncthreads();   // shared memory is reused by the next unit
    }
    __threadfence();
    grid.sync();
    // 3. pencils
    for (int64_t u = blockIdx.x; u < ra.units[2]; u += gridDim.x) {
        const RaggedOrder& A = ra.o[order_of(ra, 2, u)];
        const int64_t lu = u - A.first[2];
        switch (A.mix.n) {
#define FCC_CASE(NN) case NN: pencil_unit<NN>(A, out, lu, smem_raw); break;
            FCC_RAGGED_ORDERS(FCC_CASE)
#undef FCC_CASE
            default: break;
        }
        __syncthreads();
    }
}

template <int N>
size_t stage_smem() {
    const size_t slab = slab_smem_for<N>(kRaggedThreads / 32);
    const size_t pencil = FastLayout<N>::pencil_smem;
    return slab > pencil ? slab : pencil;
}

}  // namespace

bool ragged_order_supported(int n) {
    switch (n) {
#define FCC_CASE(NN) case NN:
        FCC_RAGGED_ORDERS(FCC_CASE)
#undef FCC_CASE
        return true;
        default:
            return false;
    }
}

int64_t ragged_units(int n, int ntiles, int nvol, int stage) {
    if (stage == 0) return (int64_t)nvol * ((ntiles + kMixWarps - 1) / kMixWarps);
    if (stage == 1) return (int64_t)nvol * n;
    int cpb = 1;
    switch (n) {
#define FCC_CASE(NN) case NN: cpb = FastLayout<NN>::CPB; break;
        FCC_RAGGED_ORDERS(FCC_CASE)
#undef FCC_CASE
        default: break;
    }
    return (int64_t)nvol * n * ((n + cpb - 1) / cpb);
}

size_t ragged_smem_for(const int* orders, int count) {
    size_t m = mix_tiled_smem_core(0);
    for (int i = 0; i < count; ++i) {
        size_t s = 0;
        switch (orders[i]) {
#define FCC_CASE(NN) case NN: s = stage_smem<NN>(); break;
            FCC_RAGGED_ORDERS(FCC_CASE)
#undef FCC_CASE
            default: break;
        }
        m = s > m ? s : m;
    }
    return m;
}

cudaError_t ragged_upload_constants(const float2* cores, const int* W, const int* u) {
    cudaError_t e = cudaMemcpyToSymbol(c_core, cores, sizeof(float2) * 3 * 576);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_W, W, sizeof(int) * 24 * 9);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_u, u, sizeof(int) * 24 * 3);
    return e;
}

cudaError_t launch_ragged_persistent(const RaggedArgs& args, const float* in, float* out, size_t smem,
                                     int grid_blocks, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(ragged_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ragged_persistent_kernel, kRaggedThreads, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int resident = per_sm * sms;
    const int blocks = grid_blocks > 0 && grid_blocks < resident ? grid_blocks : resident;
    const RaggedArgs* ap = &args;
    void* kargs[] = {(void*)&in, (void*)&out, (void*)ap};
    return cudaLaunchCooperativeKernel((const void*)ragged_persistent_kernel, dim3((unsigned)blocks), dim3(kRaggedThreads),
                                       kargs, smem, st);
}

}  // namespace fcc
