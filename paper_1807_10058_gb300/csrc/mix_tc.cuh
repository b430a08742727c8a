// Forward orbit mixing of paired real volumes with the orbit core on the
// 5th-generation tensor cores (tcgen05, accumulator in tensor memory).
//
// For every orbit class the forward core is E / 24 with E[g][h] an 8th root
// of unity.  In real form, with outputs (Re Z_g, Im Z_g) and inputs
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
// matrices along K, SBO between 8-row groups.  Threads t and t + 128 own
// orbit t of the block's tile, slots 0-11 and 12-23: each writes its half of
// row t of X and reads its half of TMEM lane t in the epilogue, so no
// transpose is needed anywhere.
//
// Pipeline per block (8 warps; a block tile = 4 tiles of the plan, <= 128
// orbits): the gather loads of the next block tile are issued as soon as the
// current one's data operand is stored, so they are in flight during the
// barrier, the MMAs, the completion wait and the epilogue.  Representatives
// come from a table padded to 32 per plan tile (all ones = no orbit), read a
// tile ahead, so no chain of dependent table loads precedes the gather.  The
// free tiles come first, then the boundary tiles in groups of one class with
// that class's core image, wrap offsets and canonical-slot mask.
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

constexpr int kTcThreads = 256;   // two threads per orbit: slots 0-11 and 12-23
constexpr int kTcK = 48;                       // real inputs per orbit
constexpr uint32_t kTcWaitLimit = 1u << 26;    // bounded mbarrier wait
constexpr uint32_t kTcTestWaitLimit = 1u << 16;   // non-blocking polls of the timeout test

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
    static constexpr int blocks_per_sm = KIND == 0 ? 4 : 3;   // TMEM allows 4; TF32: shared memory
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

// Slots H .. H + 11 of row `row` of the data operand: the split of 24 inputs
// of one orbit, 16 bytes (one core-matrix row) per store.
template <int KIND, int H>
__device__ __forceinline__ void store_half(unsigned char* X, int row, const float* vr, const float* vi) {
    using L = TcLayout<KIND>;
    if (KIND == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {   // slots H + 4c .. H + 4c + 3
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
                *reinterpret_cast<uint4*>(X + t * L::XMAT + L::off(row, 2 * H + 8 * c)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) {   // slots H + 2c, H + 2c + 1
            const float r0 = vr[2 * c], i0 = vi[2 * c], r1 = vr[2 * c + 1], i1 = vi[2 * c + 1];
            const float hr0 = tf32_round(r0), hi0 = tf32_round(i0), hr1 = tf32_round(r1), hi1 = tf32_round(i1);
            *reinterpret_cast<float4*>(X + L::off(row, 2 * H + 4 * c)) = make_float4(hr0, hi0, hr1, hi1);
            *reinterpret_cast<float4*>(X + L::XMAT + L::off(row, 2 * H + 4 * c)) =
                make_float4(tf32_round(r0 - hr0), tf32_round(i0 - hi0), tf32_round(r1 - hr1), tf32_round(i1 - hi1));
        }
    }
}

// Loads of slots H .. H + 11 of representative rp (both volumes of the pair).
// off: per-slot wrap offsets of a boundary class (nullptr: the free class's,
// a.lin[g][3]).
template <int H, bool BND>
__device__ __forceinline__ void gather_half(const TiledMixArgs& a, const float* in0, const float* in1, uint32_t rp,
                                            const int* off, float* vr, float* vi) {
    const bool act = rp != 0xffffffffu;
    static_for<0, 12>([&](auto Sc) {
        constexpr int g = H + decltype(Sc)::value;
        const int o = BND ? __ldg(off + g) : a.lin[g][3];
        const int gi = act ? rep_dot(rp, a.lin[g][0], a.lin[g][1], a.lin[g][2]) + o : 0;
        vr[g - H] = act ? __ldg(in0 + gi) : 0.f;
        vi[g - H] = act ? __ldg(in1 + gi) : 0.f;
    });
}

// Epilogue for slots H .. H + 11 of this thread's orbit: TMEM columns 4H ..
// 4H + 47 of lane trow, A1 + A2 / sqrt 2, row phase R_g / 24, scatter.
// off, cmask: wrap offsets and canonical slots of the tile's class (a
// boundary class writes each of its distinct points once).
// PH = false: no row phase and no 1/24 (the caller's core image carries the
// wrap factor of R_g and the DFT passes apply the rest, see
// mix_tc_fwd_pair_kernel).
template <int H, bool BND, bool PH = true>
__device__ __forceinline__ void epilogue_half(const TiledMixArgs& a, uint32_t trow, uint32_t rep, const int* off,
                                              uint32_t cmask, float2* out, int64_t pb, int M8) {
    const float rs2 = 0.70710678118654752440f;
    const float sc = 1.0f / 24.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
              "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(trow + (uint32_t)(4 * H + 16 * c)));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (rep != 0xffffffffu) {
            static_for<0, 4>([&](auto Sc) {
                constexpr int s4 = decltype(Sc)::value;
                const int g = H + 4 * c + s4;
                const float re = fmaf(__uint_as_float(v[4 * s4 + 2]), rs2, __uint_as_float(v[4 * s4]));
                const float im = fmaf(__uint_as_float(v[4 * s4 + 3]), rs2, __uint_as_float(v[4 * s4 + 1]));
                const int gi = rep_dot(rep, a.lin[g][0], a.lin[g][1], a.lin[g][2]) + (BND ? __ldg(off + g) : a.lin[g][3]);
                if (PH && (!BND || ((cmask >> g) & 1u))) {
                    int q = rep_dot(rep, c_u[g][0], c_u[g][1], c_u[g][2]);
                    q = q < 0 ? q + M8 : q;
                    const float2 R = __ldg(a.phase + q);
                    out[pb + gi] = make_float2(sc * (R.x * re - R.y * im), sc * (R.x * im + R.y * re));
                } else if (!PH && (!BND || ((cmask >> g) & 1u))) {
                    out[pb + gi] = make_float2(re, im);
                }
            });
        }
    }
}

// Boundary (non-free) tiles on the tensor cores: groups of up to 4 tiles of
// one class, after the free groups.  group[8 g] = class, group[8 g + 1 + w] =
// tile of warp w (-1: none); per class: its core image (the free core's
// layout), wrap offsets off[24 c + g] and canonical-slot mask.
struct TcBoundary {
    const int* group;
    int ngroups;
    const uint4* core_images;   // [class][core_bytes / 16]
    const int* off;
    const uint32_t* canon_mask;
};

// grid.x: blocks looping over groups of 4 free tiles, then the boundary
// groups; grid.y: pairs of real volumes.
// reps32: representatives of every tile, 32 per tile, 0xffffffff = none.
// status: set to 1 if a tensor-core completion wait exceeded its bound.
// wait_test: issue no MMA and no completion signal, so that the (shortened)
// wait runs out -- the test of the timeout path; nothing is written then.
//
// PH = false (canonical shift, orders with register DFT passes): with
// W_g kO = kappa_g + n m_g the row phase factors as
// R_g = w_{8n}^{kappa_g . v} w_8^{m_g . v}.  The second factor depends only on
// the slot and the class's wrap vectors: the core images passed in carry it
// in their rows (still 8th roots of unity, so the split stays exact).  The
// first factor and the 1/24 are a separable modulation of Z that the DFT
// passes apply to their inputs (fft_slab_kernel / fft_pencil_pair_kernel with
// PRE), so the kernel writes sum_h w_8^{m_g . v} E[g][h] x[kappa_h] as is.
template <int KIND, bool PH = true, bool RG = false>
__global__ void __launch_bounds__(kTcThreads, TcLayout<KIND>::blocks_per_sm)
mix_tc_fwd_pair_kernel(const float* __restrict__ in, float* __restrict__ out, const TiledMixArgs a, int nfree_tiles,
                       const uint32_t* __restrict__ reps32, const uint4* __restrict__ core_image, int* status,
                       const TcBoundary bnd, int wait_test, const int64_t* __restrict__ poff = nullptr) {
    using L = TcLayout<KIND>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* Cs = smem_raw;                 // core, 96 x 48
    unsigned char* Xs = Cs + L::CMAT;             // data terms, 128 x 48 each
    uint64_t* bar = reinterpret_cast<uint64_t*>(Xs + L::TERMS * L::XMAT);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & 127, half = tid >> 7, wq = warp & 3;   // orbit row; slot half; TMEM lane quarter
    const int n = a.n, M8 = 8 * n;
    // pair blockIdx.y: volumes 2p, 2p + 1 (RG, ragged batches: poff's two
    // point offsets of the pair); Z goes to the first volume's complex region
    const int64_t pb = RG ? __ldg(poff + 2 * blockIdx.y) : (int64_t)blockIdx.y * 2 * a.n3;

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
    const uint32_t trow = tmem + ((uint32_t)(wq * 32) << 16);   // this warp's TMEM lanes

    const int ngroups = (nfree_tiles + 3) / 4;
    uint32_t phase = 0;
    bool ok = true;

    // gather of one tile into registers: two threads per orbit, 24 loads each in flight
    const uint32_t kNone = 0xffffffffu;
    const float* __restrict__ in0 = in + pb;
    const float* __restrict__ in1 = RG ? in + __ldg(poff + 2 * blockIdx.y + 1) : in + pb + a.n3;
    const int nall = ngroups + bnd.ngroups;
    // class of group g (block-uniform; free class for the free groups)
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
    float vr[12], vi[12];
    auto gather = [&](uint32_t rp, int c) {   // warp-uniform branches: slot half, free or boundary class
        if (c == a.free_class) {
            if (half == 0) gather_half<0, false>(a, in0, in1, rp, nullptr, vr, vi);
            else gather_half<12, false>(a, in0, in1, rp, nullptr, vr, vi);
        } else {
            const int* off = bnd.off + 24 * c;
            if (half == 0) gather_half<0, true>(a, in0, in1, rp, off, vr, vi);
            else gather_half<12, true>(a, in0, in1, rp, off, vr, vi);
        }
    };

    const int gstep = (int)gridDim.x;
    int grp = blockIdx.x;
    int core_cls = a.free_class;   // class whose core image is in Cs
    uint32_t rcur = rep_of(grp), rnext = rep_of(grp + gstep);
    int ccur = cls_of(grp), cnext = cls_of(grp + gstep);
    if (grp < nall) gather(rcur, ccur);
    for (; grp < nall && ok; grp += gstep) {
        const uint32_t rep = rcur;
        const int cls = ccur;
        if (cls != core_cls) {   // block-uniform; the previous MMA has completed
            const uint4* src = bnd.core_images + (size_t)cls * (L::core_bytes / 16);
            for (int e = tid; e < (int)(L::core_bytes / 16); e += kTcThreads) reinterpret_cast<uint4*>(Cs)[e] = __ldg(src + e);
            core_cls = cls;
        }
        if (half == 0) store_half<KIND, 0>(Xs, row, vr, vi);
        else store_half<KIND, 12>(Xs, row, vr, vi);
        // the next tile's loads overlap the barrier, the MMAs, the wait and the epilogue
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
        // thread 0 waits for the MMAs; the block barrier below passes the
        // completion on to the other threads
        uint32_t done = 1;
        if (tid == 0) {
            done = 0;
            if (wait_test) {   // non-blocking polls: the test's wait ends after kTcTestWaitLimit of them
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
        // block-uniform decision: every thread must take the same path below
        if (!__syncthreads_and((int)done)) {
            if (tid == 0) {   // host-mapped word: a plain store made visible system-wide
                *(volatile int*)status = 1;
                __threadfence_system();
            }
            ok = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {   // warp-uniform: tcgen05.ld is executed by whole warps
            float2* o2 = reinterpret_cast<float2*>(out);
            if (cls == a.free_class) {
                if (half == 0) epilogue_half<0, false, PH>(a, trow, rep, nullptr, 0u, o2, pb, M8);
                else epilogue_half<12, false, PH>(a, trow, rep, nullptr, 0u, o2, pb, M8);
            } else {
                const int* off = bnd.off + 24 * cls;
                const uint32_t cm = __ldg(bnd.canon_mask + cls);
                if (half == 0) epilogue_half<0, true, PH>(a, trow, rep, off, cm, o2, pb, M8);
                else epilogue_half<12, true, PH>(a, trow, rep, off, cm, o2, pb, M8);
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
