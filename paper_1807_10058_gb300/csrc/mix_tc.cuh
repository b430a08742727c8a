// Forward orbit mixing of paired real volumes with the orbit core on the
// 5th-generation tensor cores (tcgen05, accumulator in tensor memory).
//
// For the free orbits the forward core is E / 24 with E[g][h] an 8th root of
// unity.  In real form, with outputs (Re Z_g, Im Z_g) and inputs
// (Re x_h, Im x_h), the 48 x 48 matrix has entries 0, +-1, +-1/sqrt(2); it is
// split exactly as A1 + A2 / sqrt(2) with A1, A2 in {0, +-1}, both exact in
// BF16 and TF32.  The FP32 inputs are split into three terms of the MMA
// input type (x = x0 + x1 + x2; 24 / 33 significant bits for BF16 / TF32),
// so D = A (x0 + x1 + x2) is accumulated in FP32 on the tensor cores with no
// rounding of the operands.  The epilogue forms A1 x + A2 x / sqrt(2),
// applies the row phase R_g / 24 and scatters as the SIMT kernel does.
//
// Block = 4 warps = 4 tiles of the plan (<= 128 orbits), one MMA tile
// M = 128 (rows 32w + 4s + p: output slot g = 8w + s, part p = A1 re, A1 im,
// A2 re, A2 im; rows 96..127 are zero), N = 128 (orbits), K = 48 per term.
// Operands are K-major, no swizzle: 8-row x 16-byte core matrices, LBO =
// 128 bytes between core matrices along K, SBO between 8-row groups.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "mix_tiled.cuh"

namespace fcc {

constexpr int kTcThreads = 128;
constexpr int kTcK = 48;                       // real inputs per orbit
constexpr uint32_t kTcWaitLimit = 1u << 26;    // bounded mbarrier wait

template <int KIND>  // 0: BF16 terms, 1: TF32 terms
struct TcLayout {
    static constexpr int ES = KIND == 0 ? 2 : 4;          // bytes per element
    static constexpr int KE = 16 / ES;                    // elements per core-matrix row
    static constexpr int KI = KIND == 0 ? 16 : 8;         // K per MMA instruction
    static constexpr uint32_t LBO = 128;                  // K-direction core stride
    static constexpr uint32_t SBO = (kTcK / KE) * 128;    // 8-row group stride
    static constexpr uint32_t MAT = 16 * SBO;             // one 128 x 48 operand
    static constexpr int TERMS = 3;
    static constexpr size_t a_bytes = MAT;
    static constexpr size_t b_bytes = (size_t)TERMS * MAT;
    static constexpr size_t out_stride = 25;              // float2 per orbit row (24 + pad)
    static constexpr size_t out_bytes = 128 * out_stride * 8;
    // the epilogue reuses the consumed B operand: a per-warp transpose of 16
    // orbits x (8 slots x 4 parts + pad), then the staged output rows
    static constexpr size_t xch_floats = 16 * 36;
    static constexpr size_t xch_bytes = 3 * xch_floats * 4;
    static_assert(xch_bytes + out_bytes <= b_bytes, "epilogue staging must fit in the B operand");
    static constexpr size_t smem = a_bytes + b_bytes + 128 * (4 + 1 + 1) + 64;
    static constexpr uint32_t idesc = (1u << 4) | ((KIND == 0 ? 1u : 2u) << 7) | ((KIND == 0 ? 1u : 2u) << 10) |
                                      ((128u >> 3) << 17) | ((128u >> 4) << 24);
    // byte offset of element (row r, k) inside one operand
    __host__ __device__ static constexpr uint32_t off(int r, int k) {
        return (uint32_t)((r / 8) * SBO + (k / KE) * LBO + (r % 8) * 16 + (k % KE) * ES);
    }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture; swizzle none
    return d;
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

// Store the three-term split of (re, im) at column n, rows k = 2g, 2g + 1.
template <int KIND>
__device__ __forceinline__ void store_terms(unsigned char* B, int n, int g, float re, float im) {
    using L = TcLayout<KIND>;
    const uint32_t o = L::off(n, 2 * g);
    if (KIND == 0) {
        float rr = re, ri = im;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const __nv_bfloat16 hr = __float2bfloat16_rn(rr), hi = __float2bfloat16_rn(ri);
            __nv_bfloat162 v;
            v.x = hr;
            v.y = hi;
            *reinterpret_cast<__nv_bfloat162*>(B + t * L::MAT + o) = v;
            rr -= __bfloat162float(hr);
            ri -= __bfloat162float(hi);
        }
    } else {
        float rr = re, ri = im;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const float tr = tf32_round(rr), ti = tf32_round(ri);
            *reinterpret_cast<float2*>(B + t * L::MAT + o) = make_float2(tr, ti);
            rr -= tr;
            ri -= ti;
        }
    }
}

// grid.x: blocks looping over groups of 4 free tiles; grid.y: pairs of real volumes.
// status: set to 1 if a tensor-core completion wait exceeded its bound.
template <int KIND>
__global__ void __launch_bounds__(kTcThreads, KIND == 0 ? 4 : 2) mix_tc_fwd_pair_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                                     const TiledMixArgs a, int nfree_tiles,
                                                                     const uint4* __restrict__ a_image, int* status) {
    using L = TcLayout<KIND>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* As = smem_raw;
    unsigned char* Bs = As + L::a_bytes;
    float2* outs = reinterpret_cast<float2*>(Bs + L::xch_bytes);                // [128][25], inside B
    uint32_t* s_rep = reinterpret_cast<uint32_t*>(Bs + L::b_bytes);
    uint8_t* s_pb = reinterpret_cast<uint8_t*>(s_rep + 128);
    uint8_t* s_pc = s_pb + 128;
    uint64_t* bar = reinterpret_cast<uint64_t*>(s_pc + 128 + 24);              // 8-byte aligned
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, M8 = 8 * n;
    const int64_t pb = (int64_t)blockIdx.y * 2 * a.n3;
    const float2* __restrict__ ph = a.phase;

    // the A operand: one image, loaded once per block
    for (int e = tid; e < (int)(L::a_bytes / 16); e += kTcThreads)
        reinterpret_cast<uint4*>(As)[e] = a_image[e];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)), "r"(128));
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

    const float rs2 = 0.70710678118654752440f;
    const int ngroups = (nfree_tiles + 3) / 4;
    uint32_t phase = 0;
    bool ok = true;

    for (int grp = blockIdx.x; grp < ngroups && ok; grp += gridDim.x) {
        // ---- gather this warp's tile into the B operand (three terms)
        const int tile = grp * 4 + warp;
        const bool have = tile < nfree_tiles;
        int o0 = 0, cnt = 0;
        if (have) {
            o0 = a.tile_off[tile];
            cnt = a.tile_off[tile + 1] - o0;
        }
        const bool act = lane < cnt;
        uint32_t myrep = 0;
        int rsel[4] = {lane, lane, lane, lane};
        if (act) {
            myrep = __ldg(a.reps + o0 + lane);
            rsel[1] = __ldg(a.permb + o0 + lane);
            rsel[2] = __ldg(a.permc + o0 + lane);
        }
        s_rep[warp * 32 + lane] = myrep;
        {
            float vr[24], vi[24];
            static_for<0, 24>([&](auto Gc) {
                constexpr int g = decltype(Gc)::value;
                const int r = rsel[WD<g>::v];
                const int gi = __shfl_sync(0xffffffffu, rep_dot(myrep, a.lin[g][0], a.lin[g][1], a.lin[g][2]) + a.lin[g][3], r);
                vr[g] = 0.f;
                vi[g] = 0.f;
                if (act) {
                    vr[g] = __ldg(in + pb + gi);
                    vi[g] = __ldg(in + pb + a.n3 + gi);
                }
            });
            if (act) {
                static_for<0, 24>([&](auto Gc) {
                    constexpr int g = decltype(Gc)::value;
                    store_terms<KIND>(Bs, warp * 32 + rsel[WD<g>::v], g, vr[g], vi[g]);
                });
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- one thread issues the MMAs and commits to the barrier
        if (tid == 0) {
            const uint32_t ab = smem_addr(As), bb = smem_addr(Bs);
#pragma unroll
            for (int t = 0; t < L::TERMS; ++t) {
#pragma unroll
                for (int ks = 0; ks < kTcK / L::KI; ++ks) {
                    const uint32_t koff = (uint32_t)(ks * L::KI / L::KE) * L::LBO;
                    const uint64_t da = umma_desc(ab + koff, L::LBO, L::SBO);
                    const uint64_t db = umma_desc(bb + t * L::MAT + koff, L::LBO, L::SBO);
                    const uint32_t acc = (t > 0 || ks > 0) ? 1u : 0u;
                    if (KIND == 0)
                        asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                                     "l"(da), "l"(db), "r"(L::idesc), "r"(acc));
                    else
                        asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                                     "l"(da), "l"(db), "r"(L::idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar)));
        }
        uint32_t done = 0;
        for (uint32_t it = 0; it < kTcWaitLimit && !done; ++it) {
            asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                         : "=r"(done)
                         : "r"(smem_addr(bar)), "r"(phase));
        }
        phase ^= 1u;
        // block-uniform decision: every thread must take the same path below
        if (!__syncthreads_and((int)done)) {
            if (tid == 0) atomicExch(status, 1);
            ok = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- epilogue: warp w < 3 holds rows 32w + 4s + p (slot g = 8w + s, part
        // p).  Per chunk of 32 orbits: TMEM -> registers -> a per-warp transpose in
        // shared memory (aliasing the consumed B operand) -> lane = orbit combines
        // A1 + A2 / sqrt 2 for its 8 slots, applies R_g / 24, stages [orbit][slot].
        if (ok && warp < 3) {
            float* xch = reinterpret_cast<float*>(Bs) + warp * L::xch_floats;   // [16 orbits][36]
            const int s_own = lane >> 2, p_own = lane & 3;
            const int half = lane >> 4, ol = lane & 15;    // two lanes per orbit: slots 4 half .. 4 half + 3
#pragma unroll 1
            for (int c0 = 0; c0 < 128; c0 += 16) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
                      "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 16; ++j) xch[j * 36 + s_own * 4 + p_own] = __uint_as_float(v[j]);
                __syncwarp();
                const int col = c0 + ol;
                const uint32_t rp = s_rep[col];
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4) {
                    const int s8 = 4 * half + s4;
                    const float4 q4 = *reinterpret_cast<const float4*>(xch + ol * 36 + s8 * 4);
                    const float re = fmaf(q4.z, rs2, q4.x), im = fmaf(q4.w, rs2, q4.y);
                    const int g = 8 * warp + s8;
                    int q = rep_dot(rp, c_u[g][0], c_u[g][1], c_u[g][2]);
                    q = q < 0 ? q + M8 : q;
                    const float2 R = __ldg(ph + q);
                    const float sc = 1.0f / 24.0f;
                    outs[col * L::out_stride + g] = make_float2(sc * (R.x * re - R.y * im), sc * (R.x * im + R.y * re));
                }
                __syncwarp();
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        // ---- scatter this warp's tile (all slots of a free orbit are canonical)
        if (ok) {
            static_for<0, 24>([&](auto Gc) {
                constexpr int g = decltype(Gc)::value;
                const int r = rsel[WD<g>::v];
                const int gi = __shfl_sync(0xffffffffu, rep_dot(myrep, a.lin[g][0], a.lin[g][1], a.lin[g][2]) + a.lin[g][3], r);
                if (act) reinterpret_cast<float2*>(out)[pb + gi] = outs[(warp * 32 + r) * L::out_stride + g];
            });
        }
        __syncthreads();   // the next gather overwrites B and the staging rows
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

// Host side: the A image (rows 32w + 4s + p, columns 2h + c) in the operand
// layout, from the free-orbit forward core fwd (24 x 24 complex, = E / 24).
template <int KIND>
inline bool build_tc_a_image(const std::complex<double>* fwd, std::vector<unsigned char>& img) {
    using L = TcLayout<KIND>;
    img.assign(L::a_bytes, 0);
    const double h = std::sqrt(0.5);
    auto put = [&](int r, int k, double v) {
        const uint32_t o = L::off(r, k);
        if (KIND == 0) {
            const uint16_t b = v > 0.5 ? 0x3F80 : v < -0.5 ? 0xBF80 : 0x0000;   // +1, -1, 0 in BF16
            std::memcpy(&img[o], &b, 2);
        } else {
            const float f = (float)v;
            std::memcpy(&img[o], &f, 4);
        }
    };
    for (int g = 0; g < 24; ++g) {
        const int w = g / 8, s = g % 8;
        for (int hh = 0; hh < 24; ++hh) {
            const std::complex<double> c = fwd[g * 24 + hh] * 24.0;   // an 8th root of unity
            const double cr = c.real(), ci = c.imag();
            const bool odd = std::fabs(std::fabs(cr) - h) < 1e-9 && std::fabs(std::fabs(ci) - h) < 1e-9;
            const bool even = (std::fabs(std::fabs(cr) - 1) < 1e-9 && std::fabs(ci) < 1e-9) ||
                              (std::fabs(std::fabs(ci) - 1) < 1e-9 && std::fabs(cr) < 1e-9);
            if (!odd && !even) return false;
            const double sr = odd ? cr / h : cr, si = odd ? ci / h : ci;   // +-1 or 0
            const int pre = odd ? 2 : 0;   // A2 rows carry the 1/sqrt(2) entries
            const int rre = 32 * w + 4 * s + pre, rim = rre + 1;
            put(rre, 2 * hh, sr);
            put(rre, 2 * hh + 1, -si);
            put(rim, 2 * hh, si);
            put(rim, 2 * hh + 1, sr);
        }
    }
    return true;
}

}  // namespace fcc
