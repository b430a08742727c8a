// Inverse / adjoint orbit mixing of paired real volumes on the tensor cores
// (tcgen05, accumulator in tensor memory): x_h = sum_g M[h][g] conj(R_g) Z_g
// over the canonical slots g, M the class's inverse or adjoint block.
//
// These blocks are not 8th roots of unity, so both operands are split: the
// real-form block C (48 x 48: row 2h + c, column 2g + c') and the gathered
// values conj(R_g) Z_g into three BF16 terms each (24 significant bits), and
// the six products C_j X_i with i + j <= 2 accumulate in FP32 (the dropped
// products are below 2^-24 of the result).  The MMA has one row per orbit:
// D (M = 128 orbits x N = 48) = sum X_i (128 x 48) * C_j^T; both operands
// K-major without swizzle, as in the forward kernel (mix_tc.cuh), whose block
// structure this kernel shares: threads t and t + 128 own orbit t (slots
// 0-11 and 12-23), free groups of 4 tiles first, then boundary groups of one
// class each with that class's images, offsets and canonical slots.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "mix_tc.cuh"

namespace fcc {

struct TcInvLayout {
    static constexpr int KE = 8;                        // BF16 per 16-byte core-matrix row
    static constexpr int KI = 16;                       // K per MMA instruction
    static constexpr int NOUT = 48;                     // 24 slots x (re, im)
    static constexpr uint32_t LBO = 128;
    static constexpr uint32_t SBO = (kTcK / KE) * 128;  // 768
    static constexpr uint32_t XMAT = 16 * SBO;          // 128 x 48 data term
    static constexpr uint32_t CMAT = (NOUT / 8) * SBO;  // 48 x 48 block term
    static constexpr size_t image_bytes = 3 * (size_t)CMAT;   // three terms of one class block
    static constexpr size_t smem = image_bytes + 3 * (size_t)XMAT + 64;
    static constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NOUT >> 3) << 17) | ((128u >> 4) << 24);
    __host__ __device__ static constexpr uint32_t off(int r, int k) {
        return (uint32_t)((r / 8) * SBO + (k / KE) * LBO + (r % 8) * 16 + (k % KE) * 2);
    }
};

// Loads of slots H .. H + 11 of a representative: Z_g from the compact complex
// volume at `in` (zero for the non-canonical slots of a boundary class); they
// stay in flight until conj_phase_half consumes them.
template <int H, bool BND>
__device__ __forceinline__ void gather_inv_half(const TiledMixArgs& a, const float2* in, uint32_t rp, const int* off,
                                                uint32_t cmask, float2* z) {
    const bool act = rp != 0xffffffffu;
    static_for<0, 12>([&](auto Sc) {
        constexpr int g = H + decltype(Sc)::value;
        const int o = BND ? __ldg(off + g) : a.lin[g][3];
        const int gi = act ? rep_dot(rp, a.lin[g][0], a.lin[g][1], a.lin[g][2]) + o : 0;
        const bool use = act && (!BND || ((cmask >> g) & 1u));
        z[g - H] = use ? __ldg(in + gi) : make_float2(0.f, 0.f);
    });
}

// conj(R_g) Z_g for slots H .. H + 11 (the row phase from the L1-resident table)
template <int H>
__device__ __forceinline__ void conj_phase_half(const TiledMixArgs& a, uint32_t rp, int M8, const float2* z, float* vr,
                                                float* vi) {
    static_for<0, 12>([&](auto Sc) {
        constexpr int g = H + decltype(Sc)::value;
        int q = rp != 0xffffffffu ? rep_dot(rp, c_u[g][0], c_u[g][1], c_u[g][2]) : 0;
        q = q < 0 ? q + M8 : q;
        const float2 R = __ldg(a.phase + q);
        vr[g - H] = R.x * z[g - H].x + R.y * z[g - H].y;
        vi[g - H] = R.x * z[g - H].y - R.y * z[g - H].x;
    });
}

// Epilogue for output slots H .. H + 11: TMEM columns 2H .. 2H + 23 of lane
// trow, scaled, real part to volume 2p and imaginary part to volume 2p + 1.
template <int H, bool BND>
__device__ __forceinline__ void epilogue_inv_half(const TiledMixArgs& a, uint32_t trow, uint32_t rep, const int* off,
                                                  uint32_t cmask, float scale, float* out0, float* out1) {
    uint32_t v[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(trow + (uint32_t)(2 * H)));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23])
                 : "r"(trow + (uint32_t)(2 * H + 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (rep == 0xffffffffu) return;
    static_for<0, 12>([&](auto Sc) {
        constexpr int s = decltype(Sc)::value;
        constexpr int h = H + s;
        const int gi = rep_dot(rep, a.lin[h][0], a.lin[h][1], a.lin[h][2]) + (BND ? __ldg(off + h) : a.lin[h][3]);
        if (!BND || ((cmask >> h) & 1u)) {
            out0[gi] = scale * __uint_as_float(v[2 * s]);
            out1[gi] = scale * __uint_as_float(v[2 * s + 1]);
        }
    });
}

// grid.x: blocks looping over the free groups, then the boundary groups;
// grid.y: pairs.  in: compact complex volume p at p n^3 (float2); out: real
// volumes 2p, 2p + 1.  images: three BF16 terms of the free class's block
// (free_image) and of every class (bnd.core_images, image_bytes each).
__global__ void __launch_bounds__(kTcThreads, 3)
mix_tc_inv_pair_kernel(const float2* __restrict__ in, float* __restrict__ out, const TiledMixArgs a, int nfree_tiles,
                       const uint32_t* __restrict__ reps32, const uint4* __restrict__ free_image, float scale,
                       int* status, const TcBoundary bnd, int wait_test) {
    using L = TcInvLayout;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* Cs = smem_raw;                 // 3 terms of the 48 x 48 block
    unsigned char* Xs = Cs + L::image_bytes;      // 3 terms of the 128 x 48 data
    uint64_t* bar = reinterpret_cast<uint64_t*>(Xs + 3 * L::XMAT);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & 127, half = tid >> 7, wq = warp & 3;
    const int M8 = 8 * a.n;
    const float2* __restrict__ inp = in + (int64_t)blockIdx.y * a.n3;
    float* out0 = out + (int64_t)blockIdx.y * 2 * a.n3;
    float* out1 = out0 + a.n3;

    for (int e = tid; e < (int)(L::image_bytes / 16); e += kTcThreads) reinterpret_cast<uint4*>(Cs)[e] = free_image[e];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)), "r"(64));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *s_tmem;
    const uint32_t trow = tmem + ((uint32_t)(wq * 32) << 16);

    const int ngroups = (nfree_tiles + 3) / 4;
    const int nall = ngroups + bnd.ngroups;
    const uint32_t kNone = 0xffffffffu;
    uint32_t phase = 0;
    bool ok = true;
    auto cls_of = [&](int g) -> int { return g < ngroups || g >= nall ? a.free_class : __ldg(bnd.group + 8 * (g - ngroups)); };
    auto rep_of = [&](int g) -> uint32_t {
        if (g < ngroups) {
            const int tile = g * 4 + wq;
            return tile < nfree_tiles ? __ldg(reps32 + (size_t)tile * 32 + lane) : kNone;
        }
        if (g >= nall) return kNone;
        const int tile = __ldg(bnd.group + 8 * (g - ngroups) + 1 + wq);
        return tile >= 0 ? __ldg(reps32 + (size_t)tile * 32 + lane) : kNone;
    };
    float2 zz[12];
    auto gather = [&](uint32_t rp, int c) {   // warp-uniform branches
        if (c == a.free_class) {
            if (half == 0) gather_inv_half<0, false>(a, inp, rp, nullptr, 0u, zz);
            else gather_inv_half<12, false>(a, inp, rp, nullptr, 0u, zz);
        } else {
            const int* off = bnd.off + 24 * c;
            const uint32_t cm = __ldg(bnd.canon_mask + c);
            if (half == 0) gather_inv_half<0, true>(a, inp, rp, off, cm, zz);
            else gather_inv_half<12, true>(a, inp, rp, off, cm, zz);
        }
    };

    const int gstep = (int)gridDim.x;
    int grp = blockIdx.x;
    int core_cls = a.free_class;
    uint32_t rcur = rep_of(grp), rnext = rep_of(grp + gstep);
    int ccur = cls_of(grp), cnext = cls_of(grp + gstep);
    if (grp < nall) gather(rcur, ccur);
    for (; grp < nall && ok; grp += gstep) {
        const uint32_t rep = rcur;
        const int cls = ccur;
        if (cls != core_cls) {   // block-uniform; the previous MMA has completed
            const uint4* src = bnd.core_images + (size_t)cls * (L::image_bytes / 16);
            for (int e = tid; e < (int)(L::image_bytes / 16); e += kTcThreads) reinterpret_cast<uint4*>(Cs)[e] = __ldg(src + e);
            core_cls = cls;
        }
        {
            float vr[12], vi[12];
            if (half == 0) {
                conj_phase_half<0>(a, rep, M8, zz, vr, vi);
                store_half<0, 0>(Xs, row, vr, vi);
            } else {
                conj_phase_half<12>(a, rep, M8, zz, vr, vi);
                store_half<0, 12>(Xs, row, vr, vi);
            }
        }
        rcur = rnext;
        ccur = cnext;
        if (grp + gstep < nall) gather(rcur, ccur);
        rnext = rep_of(grp + 2 * gstep);
        cnext = cls_of(grp + 2 * gstep);
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0 && !wait_test) {
            const uint32_t xb = smem_addr(Xs), cb = smem_addr(Cs);
            // the six products X_i C_j with i + j <= 2 (pair pr: i = PI, j = PJ)
            static_for<0, 6>([&](auto Pc) {
                constexpr int pr = decltype(Pc)::value;
                constexpr int PI = pr == 2 || pr == 4 ? 1 : pr == 5 ? 2 : 0;
                constexpr int PJ = pr == 1 || pr == 4 ? 1 : pr == 3 ? 2 : 0;
#pragma unroll
                for (int ks = 0; ks < kTcK / L::KI; ++ks) {
                    const uint32_t koff = (uint32_t)(ks * L::KI / L::KE) * L::LBO;
                    const uint64_t da = umma_desc(xb + PI * L::XMAT + koff, L::LBO, L::SBO);
                    const uint64_t db = umma_desc(cb + PJ * L::CMAT + koff, L::LBO, L::SBO);
                    const uint32_t acc = (pr > 0 || ks > 0) ? 1u : 0u;
                    asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                                 "l"(da), "l"(db), "r"(L::idesc), "r"(acc));
                }
            });
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar)));
        }
        uint32_t done = 1;
        if (tid == 0) {
            done = 0;
            if (wait_test) {
                for (uint32_t it = 0; it < kTcTestWaitLimit && !done; ++it) {
                    asm volatile("{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                                 : "=r"(done)
                                 : "r"(smem_addr(bar)), "r"(phase));
                }
            } else {
                for (uint32_t it = 0; it < kTcWaitLimit && !done; ++it) {
                    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                                 : "=r"(done)
                                 : "r"(smem_addr(bar)), "r"(phase));
                }
            }
        }
        phase ^= 1u;
        if (!__syncthreads_and((int)done)) {
            if (tid == 0) {
                *(volatile int*)status = 1;
                __threadfence_system();
            }
            ok = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {   // warp-uniform: tcgen05.ld is executed by whole warps
            if (cls == a.free_class) {
                if (half == 0) epilogue_inv_half<0, false>(a, trow, rep, nullptr, 0u, scale, out0, out1);
                else epilogue_inv_half<12, false>(a, trow, rep, nullptr, 0u, scale, out0, out1);
            } else {
                const int* off = bnd.off + 24 * cls;
                const uint32_t cm = __ldg(bnd.canon_mask + cls);
                if (half == 0) epilogue_inv_half<0, true>(a, trow, rep, off, cm, scale, out0, out1);
                else epilogue_inv_half<12, true>(a, trow, rep, off, cm, scale, out0, out1);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64));
}

// Host side: three BF16 terms of the real form of a 24 x 24 complex block M
// (row 2h + c: Re / Im of x_h; column 2g + c': Re / Im of the input of slot g).
inline void build_tc_inv_image(const std::complex<double>* M, std::vector<unsigned char>& img) {
    using L = TcInvLayout;
    img.assign(L::image_bytes, 0);
    auto bf16 = [](double v) -> uint16_t {   // round to nearest even (finite values)
        const float f = (float)v;
        uint32_t u;
        std::memcpy(&u, &f, 4);
        u += 0x7FFFu + ((u >> 16) & 1u);
        return (uint16_t)(u >> 16);
    };
    auto val = [](uint16_t b) -> double {
        const uint32_t u = (uint32_t)b << 16;
        float f;
        std::memcpy(&f, &u, 4);
        return f;
    };
    auto put = [&](int r, int k, double v) {
        double rest = v;
        for (int t = 0; t < 3; ++t) {
            const uint16_t b = bf16(rest);
            std::memcpy(&img[(size_t)t * L::CMAT + L::off(r, k)], &b, 2);
            rest -= val(b);
        }
    };
    for (int h = 0; h < 24; ++h)
        for (int g = 0; g < 24; ++g) {
            const double re = M[h * 24 + g].real(), im = M[h * 24 + g].imag();
            put(2 * h, 2 * g, re);
            put(2 * h, 2 * g + 1, -im);
            put(2 * h + 1, 2 * g, im);
            put(2 * h + 1, 2 * g + 1, re);
        }
}

}  // namespace fcc
