// Forward orbit mixing of paired real volumes with the orbit core on the
// 5th-generation tensor cores (tcgen05, accumulator in tensor memory).
//
// For the free orbits the forward core is E / 24 with E[g][h] an 8th root of
// unity.  In real form, with outputs (Re Z_g, Im Z_g) and inputs
// (Re x_h, Im x_h), the 48 x 48 matrix has entries 0, +-1, +-1/sqrt(2); it is
// split exactly as A1 + A2 / sqrt(2) with A1, A2 in {0, +-1}, both exact in
// BF16 and TF32.  The FP32 inputs are split into terms of the MMA input type
// (BF16: x = x0 + x1 + x2, 24 significant bits; TF32: x = x0 + x1, the
// second term rounded again, 22 bits), so the products with the exact core
// lose nothing but the last bits of x and accumulate in FP32 on the tensor
// cores.  With the core exact, the TF32 form's third product of a 2-way split
// (low part of the matrix times high part of x) is identically zero.
//
// MMA orientation: one row per orbit.  D (M = 128 orbits x N = 96) =
// X (128 x K) * C^T, K = 48 real inputs per term (column 2h + c: slot h, real
// or imaginary part), C (96 x K) the core image with row 4g + p: output slot
// g, part p = A1 re, A1 im, A2 re, A2 im.  Both operands are K-major without
// swizzle: 8-row x 16-byte core matrices, LBO = 128 bytes between core
// matrices along K, SBO between 8-row groups.  Thread t owns orbit t of the
// block's tile: it writes row t of X and reads TMEM lane t in the epilogue,
// so no transpose is needed anywhere.
//
// Pipeline per block (4 warps = 4 tiles of the plan, <= 128 orbits): the
// gather loads of the next tile are issued right after the MMAs of the
// current one and are in flight during its completion wait and epilogue.
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
    static constexpr int TERMS = KIND == 0 ? 3 : 2;
    static constexpr int NOUT = 96;                       // 24 slots x 4 parts
    static constexpr uint32_t LBO = 128;                  // K-direction core stride
    static constexpr uint32_t SBO = (kTcK / KE) * 128;    // 8-row group stride
    static constexpr uint32_t XMAT = 16 * SBO;            // one 128 x 48 data term
    static constexpr uint32_t CMAT = (NOUT / 8) * SBO;    // the 96 x 48 core
    static constexpr size_t core_bytes = CMAT;
    static constexpr size_t smem = CMAT + (size_t)TERMS * XMAT + 64;
    static constexpr uint32_t idesc = (1u << 4) | ((KIND == 0 ? 1u : 2u) << 7) | ((KIND == 0 ? 1u : 2u) << 10) |
                                      ((uint32_t)(NOUT >> 3) << 17) | ((128u >> 4) << 24);
    static constexpr int blocks_per_sm = KIND == 0 ? 4 : 3;   // shared memory; TMEM allows 4
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

// Row `row` of the data operand: the split of the 48 inputs of one orbit,
// 16 bytes (one core-matrix row) per store.
template <int KIND>
__device__ __forceinline__ void store_row(unsigned char* X, int row, const float* vr, const float* vi) {
    using L = TcLayout<KIND>;
    if (KIND == 0) {
#pragma unroll
        for (int c = 0; c < kTcK / 8; ++c) {   // slots 4c .. 4c + 3
            float r[8];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                r[2 * e] = vr[4 * c + e];
                r[2 * e + 1] = vi[4 * c + e];
            }
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(r[2 * e], r[2 * e + 1]);
                    w[e] = *reinterpret_cast<const uint32_t*>(&h);
                    if (t < 2) {
                        r[2 * e] -= __low2float(h);
                        r[2 * e + 1] -= __high2float(h);
                    }
                }
                *reinterpret_cast<uint4*>(X + t * L::XMAT + L::off(row, 8 * c)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < kTcK / 4; ++c) {   // slots 2c, 2c + 1
            const float r0 = vr[2 * c], i0 = vi[2 * c], r1 = vr[2 * c + 1], i1 = vi[2 * c + 1];
            const float hr0 = tf32_round(r0), hi0 = tf32_round(i0), hr1 = tf32_round(r1), hi1 = tf32_round(i1);
            *reinterpret_cast<float4*>(X + L::off(row, 4 * c)) = make_float4(hr0, hi0, hr1, hi1);
            *reinterpret_cast<float4*>(X + L::XMAT + L::off(row, 4 * c)) =
                make_float4(tf32_round(r0 - hr0), tf32_round(i0 - hi0), tf32_round(r1 - hr1), tf32_round(i1 - hi1));
        }
    }
}

// grid.x: blocks looping over groups of 4 free tiles; grid.y: pairs of real volumes.
// status: set to 1 if a tensor-core completion wait exceeded its bound.
template <int KIND>
__global__ void __launch_bounds__(kTcThreads, TcLayout<KIND>::blocks_per_sm)
mix_tc_fwd_pair_kernel(const float* __restrict__ in, float* __restrict__ out, const TiledMixArgs a, int nfree_tiles,
                       const uint4* __restrict__ core_image, int* status) {
    using L = TcLayout<KIND>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* Cs = smem_raw;                 // core, 96 x 48
    unsigned char* Xs = Cs + L::CMAT;             // data terms, 128 x 48 each
    uint64_t* bar = reinterpret_cast<uint64_t*>(Xs + L::TERMS * L::XMAT);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, M8 = 8 * n;
    const int64_t pb = (int64_t)blockIdx.y * 2 * a.n3;
    const float2* __restrict__ ph = a.phase;

    for (int e = tid; e < (int)(L::core_bytes / 16); e += kTcThreads)
        reinterpret_cast<uint4*>(Cs)[e] = core_image[e];
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
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's TMEM lanes

    const float rs2 = 0.70710678118654752440f;
    const float sc = 1.0f / 24.0f;
    const int ngroups = (nfree_tiles + 3) / 4;
    uint32_t phase = 0;
    bool ok = true;

    // gather of one tile into registers: thread = orbit, all 48 loads in flight
    float vr[24], vi[24];
    uint32_t nrep = 0;
    bool nact = false;
    auto gather = [&](int grp) {
        const int tile = grp * 4 + warp;
        int o0 = 0, cnt = 0;
        if (tile < nfree_tiles) {
            o0 = __ldg(a.tile_off + tile);
            cnt = __ldg(a.tile_off + tile + 1) - o0;
        }
        nact = lane < cnt;
        nrep = nact ? __ldg(a.reps + o0 + lane) : 0u;
        static_for<0, 24>([&](auto Gc) {
            constexpr int g = decltype(Gc)::value;
            const int gi = rep_dot(nrep, a.lin[g][0], a.lin[g][1], a.lin[g][2]) + a.lin[g][3];
            vr[g] = nact ? __ldg(in + pb + gi) : 0.f;
            vi[g] = nact ? __ldg(in + pb + a.n3 + gi) : 0.f;
        });
    };

    int grp = blockIdx.x;
    if (grp < ngroups) gather(grp);
    for (; grp < ngroups && ok; grp += gridDim.x) {
        const uint32_t rep = nrep;
        const bool act = nact;
        store_row<KIND>(Xs, tid, vr, vi);
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t xb = smem_addr(Xs), cb = smem_addr(Cs);
#pragma unroll
            for (int t = 0; t < L::TERMS; ++t) {
#pragma unroll
                for (int ks = 0; ks < kTcK / L::KI; ++ks) {
                    const uint32_t koff = (uint32_t)(ks * L::KI / L::KE) * L::LBO;
                    const uint64_t da = umma_desc(xb + t * L::XMAT + koff, L::LBO, L::SBO);
                    const uint64_t db = umma_desc(cb + koff, L::LBO, L::SBO);
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
        // the next tile's loads overlap the MMAs, the wait and this epilogue
        const int nxt = grp + (int)gridDim.x;
        if (nxt < ngroups) gather(nxt);
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
        if (ok) {
            // epilogue: TMEM lane = this thread's orbit; 32 columns = 8 slots per load
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uint32_t v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                      "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                      "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(trow + (uint32_t)(32 * c)));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                static_for<0, 8>([&](auto Sc) {
                    constexpr int s8 = decltype(Sc)::value;
                    const int g = 8 * c + s8;
                    const float re = fmaf(__uint_as_float(v[4 * s8 + 2]), rs2, __uint_as_float(v[4 * s8]));
                    const float im = fmaf(__uint_as_float(v[4 * s8 + 3]), rs2, __uint_as_float(v[4 * s8 + 1]));
                    int q = rep_dot(rep, c_u[g][0], c_u[g][1], c_u[g][2]);
                    q = q < 0 ? q + M8 : q;
                    const int gi = rep_dot(rep, a.lin[g][0], a.lin[g][1], a.lin[g][2]) + a.lin[g][3];
                    if (act) {
                        const float2 R = __ldg(ph + q);
                        reinterpret_cast<float2*>(out)[pb + gi] =
                            make_float2(sc * (R.x * re - R.y * im), sc * (R.x * im + R.y * re));
                    }
                });
            }
        }
        // TMEM reads complete before the next tile's MMAs (issued after the next barrier)
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

// Host side: the core image (row 4g + p, column 2h + c) in the operand
// layout, from the free-orbit forward core fwd (24 x 24 complex, = E / 24).
template <int KIND>
inline bool build_tc_core_image(const std::complex<double>* fwd, std::vector<unsigned char>& img) {
    using L = TcLayout<KIND>;
    img.assign(L::core_bytes, 0);
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
        for (int hh = 0; hh < 24; ++hh) {
            const std::complex<double> c = fwd[g * 24 + hh] * 24.0;   // an 8th root of unity
            const double cr = c.real(), ci = c.imag();
            const bool odd = std::fabs(std::fabs(cr) - h) < 1e-9 && std::fabs(std::fabs(ci) - h) < 1e-9;
            const bool even = (std::fabs(std::fabs(cr) - 1) < 1e-9 && std::fabs(ci) < 1e-9) ||
                              (std::fabs(std::fabs(ci) - 1) < 1e-9 && std::fabs(cr) < 1e-9);
            if (!odd && !even) return false;
            const double sr = odd ? cr / h : cr, si = odd ? ci / h : ci;   // +-1 or 0
            const int pre = odd ? 2 : 0;   // A2 rows carry the 1/sqrt(2) entries
            const int rre = 4 * g + pre, rim = rre + 1;
            put(rre, 2 * hh, sr);
            put(rre, 2 * hh + 1, -si);
            put(rim, 2 * hh, si);
            put(rim, 2 * hh + 1, sr);
        }
    }
    return true;
}

}  // namespace fcc
