// Instantiations and host launchers of the fast DFT passes (fft_fast.cuh),
// kept in their own translation unit so they compile in parallel with the
// rest of the library.
#include "fft_fast.cuh"
#include "fft_slab128.cuh"

namespace fcc {

namespace {

template <int N>
cudaError_t launch_n(bool slab, int sign, const float2* in, float2* out, int64_t nvol, const float2* tw,
                     int64_t vstride, const int64_t* voff, cudaStream_t st) {
    using L = FastLayout<N>;
    // 16-byte accesses: refuse (without launching) bases that are not aligned
    if (((((uintptr_t)in) | ((uintptr_t)out)) & 15u) != 0 || (!voff && vstride % 2 != 0)) return cudaErrorMisalignedAddress;
    static DeviceOnce attr;
    if (!attr.done()) {
        cudaFuncSetAttribute(fft_slab_kernel<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::slab_smem);
        cudaFuncSetAttribute(fft_slab_kernel<N, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::slab_smem);
        cudaFuncSetAttribute(fft_pencil_kernel<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::pencil_smem);
        cudaFuncSetAttribute(fft_pencil_kernel<N, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::pencil_smem);
        attr.mark();
    }
    if (slab) {
        const int64_t g = nvol * N;
        if (g > 0x7fffffffLL) return cudaErrorInvalidValue;
        if constexpr (N == 128) {   // 16 warps per slab, exchange inside the slab
            static DeviceOnce attr128;
            if (!attr128.done()) {
                cudaFuncSetAttribute(fft_slab128_kernel<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlab128Smem);
                cudaFuncSetAttribute(fft_slab128_kernel<-1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlab128Smem);
                attr128.mark();
            }
            if (sign > 0) fft_slab128_kernel<1, false><<<(unsigned)g, kSlab128Threads, kSlab128Smem, st>>>(in, out, tw, vstride, voff, nullptr);
            else fft_slab128_kernel<-1, false><<<(unsigned)g, kSlab128Threads, kSlab128Smem, st>>>(in, out, tw, vstride, voff, nullptr);
            return cudaGetLastError();
        }
        if (sign > 0) fft_slab_kernel<N, 1><<<(unsigned)g, L::SLAB_THREADS, L::slab_smem, st>>>(in, out, tw, vstride, voff);
        else fft_slab_kernel<N, -1><<<(unsigned)g, L::SLAB_THREADS, L::slab_smem, st>>>(in, out, tw, vstride, voff);
    } else {
        const int64_t g = nvol * N * ((N + L::CPB - 1) / L::CPB);
        if (g > 0x7fffffffLL) return cudaErrorInvalidValue;
        if (sign > 0) fft_pencil_kernel<N, 1><<<(unsigned)g, kFastThreads, L::pencil_smem, st>>>(in, out, tw, vstride, voff);
        else fft_pencil_kernel<N, -1><<<(unsigned)g, kFastThreads, L::pencil_smem, st>>>(in, out, tw, vstride, voff);
    }
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_pair_n(const float2* in, float2* out, int64_t npairs, const float2* tw, int64_t vstride,
                          cudaStream_t st, bool packed, const float2* pre, const int64_t* poff) {
    using L = FastLayout<N>;
    if (poff ? packed : vstride < 2 * (int64_t)N * N * N) return cudaErrorInvalidValue;
    // packed: 4-byte stores to a separate output (the complex input is not overwritten in place)
    if (packed && (((uintptr_t)out & 3u) != 0 || (const void*)in == (const void*)out)) return cudaErrorInvalidValue;
    const size_t sm = L::pencil_smem, smp = L::pencil_smem + N * sizeof(float2);
    static DeviceOnce attr;
    if (!attr.done()) {
        cudaFuncSetAttribute(fft_pencil_pair_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(fft_pencil_pair_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(fft_pencil_pair_kernel<N, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
        cudaFuncSetAttribute(fft_pencil_pair_kernel<N, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
        attr.mark();
    }
    const int64_t g = npairs * (N / 2 + 1) * PairLayout<N>::CBLK;
    if (g > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (packed && pre) fft_pencil_pair_kernel<N, true, true><<<(unsigned)g, kFastThreads, smp, st>>>(in, out, tw, vstride, pre);
    else if (packed) fft_pencil_pair_kernel<N, true><<<(unsigned)g, kFastThreads, sm, st>>>(in, out, tw, vstride);
    else if (pre) fft_pencil_pair_kernel<N, false, true><<<(unsigned)g, kFastThreads, smp, st>>>(in, out, tw, vstride, pre, poff);
    else fft_pencil_pair_kernel<N><<<(unsigned)g, kFastThreads, sm, st>>>(in, out, tw, vstride, nullptr, poff);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_slab_pre_n(const float2* in, float2* out, int64_t nvol, const float2* tw, const float2* pre,
                              int64_t vstride, cudaStream_t st) {
    using L = FastLayout<N>;
    if (((((uintptr_t)in) | ((uintptr_t)out)) & 15u) != 0 || vstride % 2 != 0 || !pre) return cudaErrorInvalidValue;
    const size_t smp = L::slab_smem + N * sizeof(float2);
    static DeviceOnce attr;
    if (!attr.done()) {
        cudaFuncSetAttribute(fft_slab_kernel<N, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
        attr.mark();
    }
    const int64_t g = nvol * N;
    if (g > 0x7fffffffLL) return cudaErrorInvalidValue;
    if constexpr (N == 128) {
        static DeviceOnce attr128;
        if (!attr128.done()) {
            cudaFuncSetAttribute(fft_slab128_kernel<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlab128Smem);
            attr128.mark();
        }
        fft_slab128_kernel<1, true><<<(unsigned)g, kSlab128Threads, kSlab128Smem, st>>>(in, out, tw, vstride, nullptr, pre);
        return cudaGetLastError();
    }
    fft_slab_kernel<N, 1, true><<<(unsigned)g, L::SLAB_THREADS, smp, st>>>(in, out, tw, vstride, nullptr, pre);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_merge_n(const float2* in, float2* out, int64_t npairs, const float2* tw, cudaStream_t st,
                           bool packed, const int64_t* poff) {
    using L = FastLayout<N>;
    if (packed && (((uintptr_t)in & 3u) != 0 || poff)) return cudaErrorInvalidValue;
    static DeviceOnce attr;
    if (!attr.done()) {
        cudaFuncSetAttribute(fft_pencil_merge_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::pencil_smem);
        cudaFuncSetAttribute(fft_pencil_merge_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)L::pencil_smem);
        attr.mark();
    }
    const int64_t n3 = (int64_t)N * N * N;
    const int64_t g = npairs * (N / 2 + 1) * PairLayout<N>::CBLK;
    if (g > 0x7fffffffLL) return cudaErrorInvalidValue;
    // in_vstride 2 n^3: complex values per pair of complex volumes, or floats per pair of packed ones
    if (packed) fft_pencil_merge_kernel<N, true><<<(unsigned)g, kFastThreads, L::pencil_smem, st>>>(in, out, tw, 2 * n3, n3);
    else fft_pencil_merge_kernel<N><<<(unsigned)g, kFastThreads, L::pencil_smem, st>>>(in, out, tw, 2 * n3, n3, poff);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fast_pencil_merge(int n, const float2* in, float2* out, int64_t npairs, const float2* tw,
                                     cudaStream_t st, bool packed, const int64_t* poff) {
    switch (n) {
#define FCC_CASE(NN) case NN: return launch_merge_n<NN>(in, out, npairs, tw, st, packed, poff);
        FCC_CASE(128) FCC_CASE(96) FCC_CASE(88) FCC_CASE(80) FCC_CASE(72) FCC_CASE(64) FCC_CASE(56)
        FCC_CASE(48) FCC_CASE(40) FCC_CASE(32) FCC_CASE(24) FCC_CASE(16) FCC_CASE(8)
#undef FCC_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fast_pencil_pair(int n, const float2* in, float2* out, int64_t npairs, const float2* tw,
                                    int64_t vstride, cudaStream_t st, bool packed, const float2* pre,
                                    const int64_t* poff) {
    switch (n) {
#define FCC_CASE(NN) case NN: return launch_pair_n<NN>(in, out, npairs, tw, vstride, st, packed, pre, poff);
        FCC_CASE(128) FCC_CASE(96) FCC_CASE(88) FCC_CASE(80) FCC_CASE(72) FCC_CASE(64) FCC_CASE(56)
        FCC_CASE(48) FCC_CASE(40) FCC_CASE(32) FCC_CASE(24) FCC_CASE(16) FCC_CASE(8)
#undef FCC_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fast_slab_pre(int n, const float2* in, float2* out, int64_t nvol, const float2* tw,
                                 const float2* pre, int64_t vstride, cudaStream_t st) {
    switch (n) {
#define FCC_CASE(NN) case NN: return launch_slab_pre_n<NN>(in, out, nvol, tw, pre, vstride, st);
        FCC_CASE(128) FCC_CASE(96) FCC_CASE(88) FCC_CASE(80) FCC_CASE(72) FCC_CASE(64) FCC_CASE(56)
        FCC_CASE(48) FCC_CASE(40) FCC_CASE(32) FCC_CASE(24) FCC_CASE(16) FCC_CASE(8)
#undef FCC_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

bool has_fast_fft(int n) {
    switch (n) {
        case 128: case 96: case 88: case 80: case 72: case 64: case 56: case 48: case 40: case 32: case 24:
        case 16: case 8:
            return true;
        default:
            return false;
    }
}

cudaError_t launch_fast_fft(int n, bool slab, int sign, const float2* in, float2* out, int64_t nvol,
                            const float2* tw, int64_t vstride, const int64_t* voff, cudaStream_t st) {
    switch (n) {
#define FCC_CASE(NN) case NN: return launch_n<NN>(slab, sign, in, out, nvol, tw, vstride, voff, st);
        FCC_CASE(128) FCC_CASE(96) FCC_CASE(88) FCC_CASE(80) FCC_CASE(72) FCC_CASE(64) FCC_CASE(56)
        FCC_CASE(48) FCC_CASE(40) FCC_CASE(32) FCC_CASE(24) FCC_CASE(16) FCC_CASE(8)
#undef FCC_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace fcc
