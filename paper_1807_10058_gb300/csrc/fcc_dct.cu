// C ABI of libfccdct (declared in include/fcc_dct.h): plans, schedules,
// launches, error handling.  All compute runs in the kernels of the headers
// included below (generic: kernels.cuh; tiled FP32 mixing: mix_tiled.cuh;
// tensor-core mixing: mix_tc.cuh, mix_tc_inv.cuh; register-radix DFT passes:
// fft_fast.cuh; pairing: pair.cuh; persistent ragged launch: ragged.cu).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <numeric>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "fcc_dct.h"
#include "fft_fast.cuh"
#include "kernels.cuh"
#include "mix_tc.cuh"
#include "mix_tc_inv.cuh"
#include "mix_replay.cuh"
#include "ragged.cuh"
#include "mix_tiled.cuh"
#include "pair.cuh"
#include "plan.h"
#include "radix2.h"

using namespace fcc;

namespace {

thread_local fcc_status g_last = FCC_OK;

fcc_status fail(fcc_status s) {
    g_last = s;
    return s;
}

bool is_double(int dtype) { return dtype == FCC_R64 || dtype == FCC_C64; }
bool is_tc(int dtype) { return dtype == FCC_R32_TF32X3 || dtype == FCC_R32_BF16X3 || dtype == FCC_R32_BF16X6; }
// BF16 terms (the 6-product form of a 3-way split of both operands reduces to
// the 3 products of BF16X3: the core's low parts are zero)
bool is_bf16(int dtype) { return dtype == FCC_R32_BF16X3 || dtype == FCC_R32_BF16X6; }
bool is_real_in(int dtype) { return dtype != FCC_C64 && dtype != FCC_C32; }

// Device copy of one order's tables.
struct OrderTables {
    int n = 0;
    int64_t n_orbits = 0;
    int n_classes = 0;
    std::vector<int> radices;
    uint32_t* reps = nullptr;
    uint8_t* cls = nullptr;
    int8_t* wrap = nullptr;
    uint32_t* canon_mask = nullptr;
    void* mat[3] = {nullptr, nullptr, nullptr};  // fwd, inv, adj
    void* phase = nullptr;                        // [M] complex, exp(2 pi i e / M), M = d n
    int u[24][3] = {};                            // W_h^T v for the shift c = v / d
    int* u_dev = nullptr;                         // the same on the device
    int M = 0;
    std::vector<SkewCore> skew_core;              // skew FP32 plans: free-orbit core per mode + weights
    void* tw = nullptr;                           // [n] complex, exp(+2 pi i j / n)
    // tiled mixing (FP32 plans)
    int free_class = -1;
    int ntiles = 0;
    int32_t* tile_off = nullptr;
    uint32_t* tile_reps = nullptr;
    uint8_t* tile_cls = nullptr;
    uint8_t* tile_pb = nullptr;
    uint8_t* tile_pc = nullptr;
    int free_tiles = 0;
    // tensor-core dtypes: the operand image of the free-orbit forward core and
    // the free tiles' representatives padded to 32 per tile (0xffffffff = none)
    void* tc_core_image = nullptr;
    uint32_t* tc_reps32 = nullptr;
    // ... and the boundary tiles: per-class core images, wrap offsets, and
    // groups of up to 4 tiles of one class (see TcBoundary)
    void* tc_core_images = nullptr;
    int* tc_off = nullptr;
    int* tc_bgroups = nullptr;
    int tc_nbgroups = 0;
    // inverse / adjoint blocks of every class, three BF16 terms each (six-product form)
    void* tc_inv_images[2] = {nullptr, nullptr};
    // phase-free forward (canonical shift): core images with the wrap factor
    // w_8^{m_g.v} in row g (free class, then every class), and the input
    // modulations of the slab pass (w_{8n}^{v3 c}) and of the pencil pass
    // (w_{8n}^{v1 k} / 24); null where the row phase stays in the mixing
    void* tc_core_image_f = nullptr;
    void* tc_core_images_f = nullptr;
    void* pre_slab = nullptr;
    void* pre_pencil = nullptr;
    // ragged plans: point offsets of this order's volumes (device), when all even
    int64_t* voff = nullptr;
    int nvoff = 0;
    // ragged plans of real volumes: this order's volumes paired in their order
    // of appearance, two point offsets per pair (pvoff) and the first of each
    // pair (pzoff, where the pair's complex transform runs); the last volume of
    // an odd count stays single (voff[nvoff - 1])
    int64_t* pvoff = nullptr;
    int64_t* pzoff = nullptr;
    int npairs_r = 0;
    int64_t single_off = -1;         // host copy of that last volume's point offset
};

constexpr int kMaxStreams = 4;
constexpr double kPi = 3.14159265358979323846;

}  // namespace

struct fcc_plan {
    int device = 0;
    int dtype = 0;
    int batch = 0;
    bool uniform = true;
    // shift c = v / d of DCT_n(r,s,t); skew: any shift other than (1/8, 0, 3/8)
    int shift_v[3] = {1, 0, 3};
    int shift_d = 8;
    bool skew = false;
    bool invertible = true;          // every class block of every order invertible
    std::vector<int> orders;         // per volume
    std::vector<int64_t> offset;     // point offset of each volume
    int64_t points = 0;
    std::map<int, OrderTables> tabs;
    void* scratch = nullptr;         // complex workspace for inverse / adjoint
    int64_t scratch_points = 0;
    void* packed_ws = nullptr;       // complex workspace of the packed forward / inverse (first call)
    int64_t packed_slot = 0;         // its complex values per internal stream
    int packed_streams = 0;
    void* host_in_dev = nullptr;     // device staging for the *_host entry points
    void* host_out_dev = nullptr;
    cudaStream_t copy_in = nullptr, copy_out = nullptr;   // *_host: copies overlapping the transform
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_host = nullptr;
    std::vector<void*> allocs;
    std::vector<int64_t> alloc_bytes;   // sizes of allocs (live-byte bookkeeping)
    R2Plan* r2 = nullptr;               // set: the forward runs the radix-2 recursion (fcc_dct_plan_radix2)
    // chunked schedule: volumes per chunk and internal streams (fork / join
    // with the caller's stream through events)
    int64_t chunk_bytes = 32ll << 20;
    int nstreams = 2;
    bool pairing = true;             // real dtypes: two volumes per complex transform
    bool ragged_fast = true;         // ragged FP32 forward: per-order launches over offset tables
    int ragged_mode = 0;             // FCC_SCHED_RAGGED: 0 per-order launches, 1 one persistent launch, 2 per run of volumes
    int tc_blocks = 0;               // FCC_SCHED_TC_BLOCKS: tensor-core mixing blocks per SM in the grid (0 = resident maximum)
    int tc_fold = 1;                 // FCC_SCHED_TC_FOLD: 1 = row phase applied by the DFT passes (phase-free mixing)
    int wait_test = 0;               // fcc_dct_test_wait_timeout
    int scratch_streams = 1;         // internal streams the inverse / adjoint workspace was sized for
    int num_sms = 1;
    // device-side wait timeouts of the tensor-core kernels: a word of pinned,
    // mapped host memory, so that the host reads it without a device sync
    int* h_status = nullptr;
    int* d_status = nullptr;         // its device address
    cudaStream_t streams[kMaxStreams] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t bnd_ev = nullptr;    // boundary tiles done (forward)
    cudaStream_t bnd_stream = nullptr;   // boundary tiles, concurrent with the chunks' free mixing
    cudaEvent_t bnd_join = nullptr;
    cudaEvent_t join_ev[kMaxStreams] = {};
    // per-kernel timing (fcc_dct_profile_enable)
    bool profiling = false;
    struct Rec { const char* name; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

size_t real_size(int dtype) { return is_double(dtype) ? 8 : 4; }

template <typename T>
std::vector<T> to_pairs(const std::vector<cd>& v) {
    std::vector<T> out(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        out[2 * i] = (T)v[i].real();
        out[2 * i + 1] = (T)v[i].imag();
    }
    return out;
}

// Allocation bookkeeping and the one-shot failure of fcc_dct_test_fail_alloc.
std::atomic<int64_t> g_alloc_seq{0};       // allocations made so far
std::atomic<int64_t> g_fail_at{0};         // sequence number that fails (0: none)
std::atomic<int64_t> g_live_plans{0};
std::atomic<int64_t> g_live_dev_bytes{0};

// true if this allocation is the armed one (the hook disarms itself)
bool injected_failure() {
    const int64_t seq = ++g_alloc_seq;
    int64_t want = g_fail_at.load();
    return want != 0 && seq == want && g_fail_at.compare_exchange_strong(want, 0);
}

fcc_status dev_alloc(fcc_plan* p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return FCC_OK;
    if (injected_failure() || cudaMalloc(ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return FCC_ERR_ALLOC;
    }
    p->allocs.push_back(*ptr);
    p->alloc_bytes.push_back((int64_t)bytes);
    g_live_dev_bytes += (int64_t)bytes;
    return FCC_OK;
}

fcc_status upload(fcc_plan* p, void** ptr, const void* src, size_t bytes) {
    fcc_status s = dev_alloc(p, ptr, bytes);
    if (s != FCC_OK) return s;
    if (bytes && cudaMemcpy(*ptr, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return FCC_ERR_CUDA;
    return FCC_OK;
}

template <typename T>
fcc_status build_tables(fcc_plan* p, int n, OrderTables& t) {
    HostPlan hp;
    const int rc = build_host_plan(n, hp, p->shift_v, p->shift_d);
    if (rc == -1) return FCC_ERR_INVALID_ARG;
    if (rc != 0) return FCC_ERR_UNSUPPORTED;
    if (!hp.invertible) {
        if (!p->skew) return FCC_ERR_UNSUPPORTED;   // the canonical blocks are never singular
        p->invertible = false;
    }
    t.n = n;
    t.M = hp.d * n;
    std::memcpy(t.u, hp.u, sizeof(t.u));
    t.n_orbits = (int64_t)hp.reps.size();
    t.n_classes = (int)hp.classes.size();
    t.radices = fft_radices(n);
    if ((int)t.radices.size() > kMaxStages) return FCC_ERR_UNSUPPORTED;
    for (int r : t.radices)
        if (r > 31) return FCC_ERR_UNSUPPORTED;
    std::vector<int8_t> wrap(72 * t.n_classes);
    std::vector<uint32_t> cm(t.n_classes);
    std::vector<cd> mats[3];
    for (int c = 0; c < t.n_classes; ++c) {
        const OrbitClass& oc = hp.classes[c];
        std::memcpy(&wrap[72 * c], oc.wrap, 72);
        cm[c] = oc.canon_mask;
        mats[0].insert(mats[0].end(), oc.fwd.begin(), oc.fwd.end());
        mats[1].insert(mats[1].end(), oc.inv.begin(), oc.inv.end());
        mats[2].insert(mats[2].end(), oc.adj.begin(), oc.adj.end());
    }
    std::vector<cd> phase(t.M), tw(n);
    for (int e = 0; e < t.M; ++e) phase[e] = std::polar(1.0, 2.0 * M_PI * e / (double)t.M);
    for (int j = 0; j < n; ++j) tw[j] = std::polar(1.0, 2.0 * M_PI * j / (double)n);
    fcc_status s;
    if ((s = upload(p, (void**)&t.reps, hp.reps.data(), hp.reps.size() * 4))) return s;
    if ((s = upload(p, (void**)&t.cls, hp.cls.data(), hp.cls.size()))) return s;
    if ((s = upload(p, (void**)&t.wrap, wrap.data(), wrap.size()))) return s;
    if ((s = upload(p, (void**)&t.canon_mask, cm.data(), cm.size() * 4))) return s;
    for (int m = 0; m < 3; ++m) {
        auto v = to_pairs<T>(mats[m]);
        if ((s = upload(p, &t.mat[m], v.data(), v.size() * sizeof(T)))) return s;
    }
    auto ph = to_pairs<T>(phase);
    if ((s = upload(p, &t.phase, ph.data(), ph.size() * sizeof(T)))) return s;
    if ((s = upload(p, (void**)&t.u_dev, &t.u[0][0], sizeof(t.u)))) return s;
    auto twv = to_pairs<T>(tw);
    if ((s = upload(p, &t.tw, twv.data(), twv.size() * sizeof(T)))) return s;
    t.free_class = hp.free_class;
    t.ntiles = (int)hp.tile_off.size() - 1;
    t.free_tiles = hp.free_tiles;
    if (is_tc(p->dtype) && hp.free_class >= 0) {
        std::vector<unsigned char> img;
        const bool ok = is_bf16(p->dtype) ? build_tc_core_image<0>(hp.classes[hp.free_class].fwd.data(), img)
                                                   : build_tc_core_image<1>(hp.classes[hp.free_class].fwd.data(), img);
        if (!ok) return FCC_ERR_UNSUPPORTED;
        if ((s = upload(p, &t.tc_core_image, img.data(), img.size()))) return s;
        // phase-free form: R_g = w_{dn}^{kappa_g.v} w_d^{m_g.v}; the class's
        // wrap factor goes into row g of its core, the rest into the DFT passes
        const bool fold = sizeof(T) == 4 && hp.d == 8 && hp.v[1] == 0;
        auto folded = [&](const OrbitClass& oc, std::vector<unsigned char>& out) -> bool {
            std::vector<cd> f(oc.fwd);
            for (int g = 0; g < 24; ++g) {
                const int e = oc.wrap[g][0] * hp.v[0] + oc.wrap[g][1] * hp.v[1] + oc.wrap[g][2] * hp.v[2];
                const cd w = std::polar(1.0, 2.0 * kPi * (double)(((e % hp.d) + hp.d) % hp.d) / hp.d);
                for (int h = 0; h < 24; ++h) f[g * 24 + h] *= w;
            }
            return is_bf16(p->dtype) ? build_tc_core_image<0>(f.data(), out) : build_tc_core_image<1>(f.data(), out);
        };
        if (fold) {
            std::vector<unsigned char> fimg, fall, one;
            if (!folded(hp.classes[hp.free_class], fimg)) return FCC_ERR_UNSUPPORTED;
            for (size_t c = 0; c < hp.classes.size(); ++c) {
                if (!folded(hp.classes[c], one)) return FCC_ERR_UNSUPPORTED;
                fall.insert(fall.end(), one.begin(), one.end());
            }
            std::vector<cd> ps(n), pp(n);
            const int M = hp.d * n;
            for (int c = 0; c < n; ++c) {
                ps[c] = std::polar(1.0, 2.0 * kPi * (double)(((int64_t)hp.v[2] * c) % M) / M);
                pp[c] = std::polar(1.0 / 24.0, 2.0 * kPi * (double)(((int64_t)hp.v[0] * c) % M) / M);
            }
            auto psv = to_pairs<float>(ps), ppv = to_pairs<float>(pp);
            if ((s = upload(p, &t.tc_core_image_f, fimg.data(), fimg.size()))) return s;
            if ((s = upload(p, &t.tc_core_images_f, fall.data(), fall.size()))) return s;
            if ((s = upload(p, &t.pre_slab, psv.data(), psv.size() * 4))) return s;
            if ((s = upload(p, &t.pre_pencil, ppv.data(), ppv.size() * 4))) return s;
        }
        const int ntl = (int)hp.tile_off.size() - 1;
        std::vector<uint32_t> r32((size_t)std::max(1, ntl) * 32, 0xffffffffu);
        for (int tl = 0; tl < ntl; ++tl)
            for (int o = hp.tile_off[tl]; o < hp.tile_off[tl + 1]; ++o) r32[(size_t)tl * 32 + (o - hp.tile_off[tl])] = hp.tile_reps[o];
        if ((s = upload(p, (void**)&t.tc_reps32, r32.data(), r32.size() * 4))) return s;
        // boundary classes: core images, wrap offsets, groups of <= 4 tiles
        std::vector<unsigned char> imgs, one;
        std::vector<int> off(hp.classes.size() * 24);
        for (size_t c = 0; c < hp.classes.size(); ++c) {
            const bool okc = is_bf16(p->dtype) ? build_tc_core_image<0>(hp.classes[c].fwd.data(), one)
                                                        : build_tc_core_image<1>(hp.classes[c].fwd.data(), one);
            if (!okc) return FCC_ERR_UNSUPPORTED;
            imgs.insert(imgs.end(), one.begin(), one.end());
            for (int g = 0; g < 24; ++g)
                off[c * 24 + g] = -n * (hp.classes[c].wrap[g][0] * n * n + hp.classes[c].wrap[g][1] * n + hp.classes[c].wrap[g][2]);
        }
        std::vector<int> groups;
        for (int tl = hp.free_tiles; tl < ntl;) {
            const int c = hp.tile_cls[hp.tile_off[tl]];
            int grp[8] = {c, -1, -1, -1, -1, 0, 0, 0};
            for (int w = 0; w < 4 && tl < ntl && hp.tile_cls[hp.tile_off[tl]] == c; ++w, ++tl) grp[1 + w] = tl;
            groups.insert(groups.end(), grp, grp + 8);
        }
        t.tc_nbgroups = (int)(groups.size() / 8);
        for (int md = 0; md < 2; ++md) {
            std::vector<unsigned char> all;
            for (size_t c = 0; c < hp.classes.size(); ++c) {
                build_tc_inv_image(md == 0 ? hp.classes[c].inv.data() : hp.classes[c].adj.data(), one);
                all.insert(all.end(), one.begin(), one.end());
            }
            if ((s = upload(p, &t.tc_inv_images[md], all.data(), all.size()))) return s;
        }
        if ((s = upload(p, &t.tc_core_images, imgs.data(), imgs.size()))) return s;
        if ((s = upload(p, (void**)&t.tc_off, off.data(), off.size() * 4))) return s;
        if (!groups.empty() && (s = upload(p, (void**)&t.tc_bgroups, groups.data(), groups.size() * 4))) return s;
    }
    if ((s = upload(p, (void**)&t.tile_off, hp.tile_off.data(), hp.tile_off.size() * 4))) return s;
    if ((s = upload(p, (void**)&t.tile_reps, hp.tile_reps.data(), hp.tile_reps.size() * 4))) return s;
    if ((s = upload(p, (void**)&t.tile_cls, hp.tile_cls.data(), hp.tile_cls.size()))) return s;
    if ((s = upload(p, (void**)&t.tile_pb, hp.tile_perm_b.data(), hp.tile_perm_b.size()))) return s;
    if ((s = upload(p, (void**)&t.tile_pc, hp.tile_perm_c.data(), hp.tile_perm_c.size()))) return s;
    if (hp.free_class >= 0) {
        // the kernels hard-wire the free-orbit wrap vectors
        for (int g = 0; g < 24; ++g)
            for (int i = 0; i < 3; ++i)
                if (hp.classes[hp.free_class].wrap[g][i] != wc::K::t.fw[g][i]) return FCC_ERR_UNSUPPORTED;
    }
    if (sizeof(T) == 4 && p->skew) {
        // the row-phase weights serve every orbit (the inverse / adjoint
        // apply conj(R) to all slots); the core only the free orbits
        t.skew_core.assign(3, SkewCore{});
        for (int md = 0; md < 3; ++md) {
            std::memcpy(t.skew_core[md].u, hp.u, sizeof(hp.u));
            if (hp.free_class < 0) continue;
            const OrbitClass& oc = hp.classes[hp.free_class];
            const std::vector<cd>& m = md == 0 ? oc.fwd : md == 1 ? oc.inv : oc.adj;
            for (int e = 0; e < 576; ++e)
                t.skew_core[md].m[e / 24][e % 24] = make_float2((float)m[e].real(), (float)m[e].imag());
        }
    }
    if (sizeof(T) == 4 && hp.free_class >= 0 && !p->skew) {
        // the free-orbit cores do not depend on n: one constant copy per device
        // (for the canonical shift; skew plans mix with the generic kernel)
        std::vector<float2> core(3 * 576);
        const OrbitClass& oc = hp.classes[hp.free_class];
        for (int e = 0; e < 576; ++e) {
            core[e] = make_float2((float)oc.fwd[e].real(), (float)oc.fwd[e].imag());
            core[576 + e] = make_float2((float)oc.inv[e].real(), (float)oc.inv[e].imag());
            core[1152 + e] = make_float2((float)oc.adj[e].real(), (float)oc.adj[e].imag());
        }
        if (cudaMemcpyToSymbol(c_core, core.data(), core.size() * sizeof(float2)) != cudaSuccess) return FCC_ERR_CUDA;
        // the persistent ragged kernel's translation unit holds its own copies
        const WeylGroup& G = weyl();
        if (ragged_upload_constants(core.data(), &G.m[0][0], &G.u[0][0]) != cudaSuccess) return FCC_ERR_CUDA;
    }
    return FCC_OK;
}

fcc_status upload_group() {
    const WeylGroup& G = weyl();
    // the kernels' compile-time copy of W must match the plan builder's
    for (int g = 0; g < 24; ++g)
        for (int i = 0; i < 9; ++i)
            if (wc::K::t.m[g][i] != G.m[g][i]) return FCC_ERR_UNSUPPORTED;
    if (cudaMemcpyToSymbol(c_W, G.m, sizeof(G.m)) != cudaSuccess) return FCC_ERR_CUDA;
    if (cudaMemcpyToSymbol(c_u, G.u, sizeof(G.u)) != cudaSuccess) return FCC_ERR_CUDA;
    int dir[24];
    slot_directions(dir);
    for (int g = 0; g < 24; ++g)
        if (dir[g] != wc::K::t.dir[g]) return FCC_ERR_UNSUPPORTED;
    return FCC_OK;
}

void release(fcc_plan* p) {
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    if (p->r2) r2_destroy(p->r2);
    for (void* a : p->allocs) cudaFree(a);
    for (int64_t b : p->alloc_bytes) g_live_dev_bytes -= b;
    --g_live_plans;
    for (auto& r : p->recs) { if (r.a) cudaEventDestroy(r.a); if (r.b) cudaEventDestroy(r.b); }
    for (int i = 0; i < kMaxStreams; ++i) {
        if (p->streams[i]) cudaStreamDestroy(p->streams[i]);
        if (p->join_ev[i]) cudaEventDestroy(p->join_ev[i]);
    }
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->bnd_ev) cudaEventDestroy(p->bnd_ev);
    if (p->bnd_join) cudaEventDestroy(p->bnd_join);
    if (p->h_status) cudaFreeHost(p->h_status);
    for (cudaEvent_t e : {p->ev_in, p->ev_out, p->ev_host})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t q : {p->copy_in, p->copy_out})
        if (q) cudaStreamDestroy(q);
    if (p->bnd_stream) cudaStreamDestroy(p->bnd_stream);
    for (auto e : p->event_pool) cudaEventDestroy(e);
    cudaSetDevice(cur);
    delete p;
}

// c = v / d in lowest terms is (1/8, 0, 3/8): the canonical kernels apply
bool canonical_shift(const int* v, int d) {
    int g = d;
    for (int i = 0; i < 3; ++i) g = std::gcd(g, std::abs(v[i]));
    return v[0] / g == 1 && v[1] == 0 && v[2] / g == 3 && d / g == 8;
}

// v, d: the shift c = v / d (v = nullptr: (1/8, 0, 3/8)).
fcc_plan* make_plan(const std::vector<int>& orders, int dtype, const int* v = nullptr, int d = 8) {
    if (dtype < FCC_R64 || dtype > FCC_R32_BF16X6) { fail(FCC_ERR_INVALID_ARG); return nullptr; }
    if (orders.empty()) { fail(FCC_ERR_INVALID_ARG); return nullptr; }
    for (int n : orders)
        if (n < 1 || n > FCC_MAX_ORDER) { fail(FCC_ERR_INVALID_ARG); return nullptr; }
    fcc_plan* p = injected_failure() ? nullptr : new (std::nothrow) fcc_plan();
    if (!p) { fail(FCC_ERR_ALLOC); return nullptr; }
    ++g_live_plans;
    if (cudaGetDevice(&p->device) != cudaSuccess) { cudaGetLastError(); --g_live_plans; delete p; fail(FCC_ERR_CUDA); return nullptr; }
    p->dtype = dtype;
    if (v && !canonical_shift(v, d)) {   // (1/8, 0, 3/8) in other terms keeps the canonical tables
        for (int i = 0; i < 3; ++i) p->shift_v[i] = v[i];
        p->shift_d = d;
        p->skew = true;
    }
    p->batch = (int)orders.size();
    p->orders = orders;
    p->uniform = std::all_of(orders.begin(), orders.end(), [&](int n) { return n == orders[0]; });
    int64_t off = 0;
    int64_t maxpts = 0;
    for (int n : orders) {
        p->offset.push_back(off);
        const int64_t n3 = (int64_t)n * n * n;
        off += n3;
        maxpts = std::max(maxpts, n3);
    }
    p->points = off;
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (p->num_sms < 1) p->num_sms = 1;
    fcc_status s = upload_group();
    if (s == FCC_OK) {
        if (injected_failure() || cudaHostAlloc((void**)&p->h_status, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            p->h_status = nullptr;
            s = FCC_ERR_ALLOC;
        } else {
            *(volatile int*)p->h_status = 0;
            if (cudaHostGetDevicePointer((void**)&p->d_status, p->h_status, 0) != cudaSuccess) s = FCC_ERR_CUDA;
        }
    }
    for (int n : orders) {
        if (s != FCC_OK) break;
        if (p->tabs.count(n)) continue;
        OrderTables t;
        s = is_double(dtype) ? build_tables<double>(p, n, t) : build_tables<float>(p, n, t);
        p->tabs[n] = t;
    }
    if (s == FCC_OK && !p->uniform && !is_double(dtype)) {
        // ragged: per order, the point offsets of its volumes (all even, so that
        // 16-byte accesses of the DFT passes stay aligned)
        std::map<int, std::vector<int64_t>> offs;
        bool even = true;
        for (size_t v = 0; v < orders.size(); ++v) {
            offs[orders[v]].push_back(p->offset[v]);
            even = even && (p->offset[v] % 2 == 0);
        }
        if (even)
            for (auto& kv : offs) {
                OrderTables& t = p->tabs[kv.first];
                t.nvoff = (int)kv.second.size();
                if ((s = upload(p, (void**)&t.voff, kv.second.data(), kv.second.size() * sizeof(int64_t)))) break;
                if (is_real_in(dtype) && t.nvoff % 2 == 1) t.single_off = kv.second.back();
                if (is_real_in(dtype) && t.nvoff >= 2) {
                    t.npairs_r = t.nvoff / 2;
                    std::vector<int64_t> first((size_t)t.npairs_r);
                    for (int q = 0; q < t.npairs_r; ++q) first[q] = kv.second[2 * q];
                    if ((s = upload(p, (void**)&t.pvoff, kv.second.data(), 2 * (size_t)t.npairs_r * sizeof(int64_t)))) break;
                    if ((s = upload(p, (void**)&t.pzoff, first.data(), first.size() * sizeof(int64_t)))) break;
                }
            }
    }
    if (s == FCC_OK) {
        if (const char* e = std::getenv("FCC_CHUNK_MB")) p->chunk_bytes = std::max(1, std::atoi(e)) * (1ll << 20);
        if (const char* e = std::getenv("FCC_STREAMS")) p->nstreams = std::min(kMaxStreams, std::max(1, std::atoi(e)));
        if (const char* e = std::getenv("FCC_PAIRING")) p->pairing = std::atoi(e) != 0;
        if (const char* e = std::getenv("FCC_RAGGED_GROUPED")) p->ragged_fast = std::atoi(e) != 0;
        for (int i = 0; i < kMaxStreams && s == FCC_OK; ++i) {
            if (cudaStreamCreateWithFlags(&p->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->join_ev[i], cudaEventDisableTiming) != cudaSuccess)
                s = FCC_ERR_CUDA;
        }
        if (s == FCC_OK && cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming) != cudaSuccess) s = FCC_ERR_CUDA;
        if (s == FCC_OK && cudaEventCreateWithFlags(&p->bnd_ev, cudaEventDisableTiming) != cudaSuccess) s = FCC_ERR_CUDA;
        if (s == FCC_OK && cudaEventCreateWithFlags(&p->bnd_join, cudaEventDisableTiming) != cudaSuccess) s = FCC_ERR_CUDA;
        if (s == FCC_OK && cudaStreamCreateWithFlags(&p->bnd_stream, cudaStreamNonBlocking) != cudaSuccess) s = FCC_ERR_CUDA;
        for (cudaStream_t* q : {&p->copy_in, &p->copy_out})
            if (s == FCC_OK && cudaStreamCreateWithFlags(q, cudaStreamNonBlocking) != cudaSuccess) s = FCC_ERR_CUDA;
        for (cudaEvent_t* e : {&p->ev_in, &p->ev_out, &p->ev_host})
            if (s == FCC_OK && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) s = FCC_ERR_CUDA;
    }
    if (s == FCC_OK) {
        // workspace for inverse / adjoint: one chunk per internal stream
        const int64_t bytes_per_pt = 2 * real_size(dtype);
        int64_t chunk_pts = std::max<int64_t>(maxpts, p->chunk_bytes / bytes_per_pt);
        chunk_pts = std::min<int64_t>(chunk_pts, p->points);
        p->scratch_points = chunk_pts;
        p->scratch_streams = p->nstreams;
        s = dev_alloc(p, &p->scratch, chunk_pts * bytes_per_pt * p->nstreams);
    }
    if (s != FCC_OK) {
        release(p);
        fail(s);
        return nullptr;
    }
    return p;
}

// --- optional per-kernel events ------------------------------------------

thread_local fcc_plan* g_prof_plan = nullptr;  // plan whose launches are being recorded

cudaEvent_t take_event(fcc_plan* p) {
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

// Every launch site opens one: an NVTX range named after the kernel (host
// side, for timeline tools; free without one attached) and, while the plan's
// profiling is on, a pair of events around the launch.
struct ProfScope {
    fcc_plan* p;
    fcc_plan::Rec r{nullptr, nullptr, nullptr};
    cudaStream_t st;
    ProfScope(const char* name, cudaStream_t s) : p(g_prof_plan), st(s) {
        nvtxRangePushA(name);
        if (!p || !p->profiling) { p = nullptr; return; }
        r.name = name;
        r.a = take_event(p);
        r.b = take_event(p);
        if (r.a) cudaEventRecord(r.a, st);
    }
    ~ProfScope() {
        nvtxRangePop();
        if (!p) return;
        if (r.b) cudaEventRecord(r.b, st);
        p->recs.push_back(r);
    }
};

// NVTX range around one entry-point call (the transform's stages nest inside).
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
};

// --- launches -------------------------------------------------------------

template <typename T>
fcc_status launch_fft(const OrderTables& t, const T* in, T* out, int64_t nvol, int axis, int sign,
                      cudaStream_t st, int64_t vstride = 0) {
    const int n = t.n;
    if (n == 1) {   // the identity
        const size_t pitch = (size_t)(vstride > 1 ? vstride : 1) * 2 * sizeof(T);
        if (in != out) cudaMemcpy2DAsync(out, pitch, in, pitch, 2 * sizeof(T), (size_t)nvol, cudaMemcpyDeviceToDevice, st);
        return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
    }
    FftArgs a{};
    a.n = n;
    a.nstages = (int)t.radices.size();
    for (int s = 0; s < a.nstages; ++s) a.radix[s] = t.radices[s];
    a.axis = axis;
    const int budget = (int)((sizeof(T) == 4 ? 4096 : 2048));
    a.P = std::max(1, budget / n);
    if (axis != 2) a.P = std::min(a.P, n);
    a.nvol = nvol;
    a.vstride = vstride > 0 ? vstride : (int64_t)n * n * n;
    a.sign = sign;
    int64_t tiles;
    if (axis == 2) tiles = (nvol * n * n + a.P - 1) / a.P;
    else tiles = nvol * n * ((n + a.P - 1) / a.P);
    const size_t smem = (size_t)(4 * a.P * (n + 1) + 2 * n) * sizeof(T);
    static DeviceOnce attr;   // one per instantiation of this function template
    if (!attr.done()) {
        cudaFuncSetAttribute(fft_axis_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr.mark();
    }
    if (tiles > 0x7fffffffLL) return FCC_ERR_UNSUPPORTED;
    static const char* names[3] = {"fft_axis0", "fft_axis1", "fft_axis2"};
    ProfScope ps(names[axis], st);
    fft_axis_kernel<T><<<(unsigned)tiles, 256, smem, st>>>(in, out, (const T*)t.tw, a);
    return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}

template <typename T>
fcc_status launch_mix(const OrderTables& t, int mode, bool real_in, bool real_out, const T* in, T* out,
                      int64_t nvol, T scale, cudaStream_t st) {
    MixArgs<T> a;
    a.reps = t.reps;
    a.cls = t.cls;
    a.mats = (const T*)t.mat[mode];
    a.wrap = t.wrap;
    a.canon_mask = t.canon_mask;
    a.phase = (const T*)t.phase;
    std::memcpy(a.u, t.u, sizeof(a.u));
    a.M = t.M;
    a.n = t.n;
    a.n_orbits = t.n_orbits;
    a.n3 = (int64_t)t.n * t.n * t.n;
    a.scale = scale;
    const unsigned bx = (unsigned)((t.n_orbits + 127) / 128);
    for (int64_t v0 = 0; v0 < nvol; v0 += 65535) {
        const int64_t nv = std::min<int64_t>(65535, nvol - v0);
        dim3 grid(bx, (unsigned)nv);
        static const char* names[3] = {"orbit_mix_fwd", "orbit_mix_inv", "orbit_mix_adj"};
        ProfScope ps(names[mode], st);
        const T* src = in + v0 * a.n3 * ((mode == MODE_FWD && real_in) ? 1 : 2);
        T* dst = out + v0 * a.n3 * ((mode != MODE_FWD && real_out) ? 1 : 2);
        if (mode == MODE_FWD) {
            if (real_in) orbit_mix_kernel<T, MODE_FWD, true, false><<<grid, 128, 0, st>>>(src, dst, a);
            else orbit_mix_kernel<T, MODE_FWD, false, false><<<grid, 128, 0, st>>>(src, dst, a);
        } else if (mode == MODE_INV) {
            if (real_out) orbit_mix_kernel<T, MODE_INV, false, true><<<grid, 128, 0, st>>>(src, dst, a);
            else orbit_mix_kernel<T, MODE_INV, false, false><<<grid, 128, 0, st>>>(src, dst, a);
        } else {
            if (real_out) orbit_mix_kernel<T, MODE_ADJ, false, true><<<grid, 128, 0, st>>>(src, dst, a);
            else orbit_mix_kernel<T, MODE_ADJ, false, false><<<grid, 128, 0, st>>>(src, dst, a);
        }
    }
    return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}

// --- FP32 fast path -------------------------------------------------------

// fast DFT passes (fft_fast.cu), wrapped with the per-kernel timing scope
fcc_status fast_fft(int n, bool slab, int sign, const float2* in, float2* out, int64_t nvol, const float2* tw,
                    int64_t vstride, cudaStream_t st, const int64_t* voff = nullptr) {
    ProfScope ps(slab ? "fft_slab" : "fft_pencil", st);
    return launch_fast_fft(n, slab, sign, in, out, nvol, tw, vstride, voff, st) == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}

// Dynamic shared memory limits of every instantiation of mix_tiled_kernel
// (set once per device, before the first launch of any of them).
void set_mix_tiled_attributes() {
    static DeviceOnce attr;
    if (attr.done()) return;
    const int lim = 200 * 1024;
    cudaFuncSetAttribute(mix_tiled_kernel<MODE_FWD, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(mix_tiled_kernel<MODE_FWD, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(mix_tiled_kernel<MODE_INV, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(mix_tiled_kernel<MODE_INV, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(mix_tiled_kernel<MODE_ADJ, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(mix_tiled_kernel<MODE_ADJ, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(mix_tiled_kernel<MODE_FWD, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(mix_tiled_kernel<MODE_INV, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(mix_tiled_kernel<MODE_ADJ, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    attr.mark();
}

// which: 0 = every tile, 1 = free tiles only, 2 = boundary tiles only
TiledMixArgs make_mix_args(const OrderTables& t, int mode, float scale) {
    TiledMixArgs a;
    a.tile_off = t.tile_off;
    a.reps = t.tile_reps;
    a.cls = t.tile_cls;
    a.permb = t.tile_pb;
    a.permc = t.tile_pc;
    a.mats = (const float*)t.mat[mode];
    a.wrap = t.wrap;
    a.canon_mask = t.canon_mask;
    a.phase = (const float2*)t.phase;
    a.uv = t.u_dev;
    a.M = t.M;
    a.n = t.n;
    const int n = t.n;
    for (int g = 0; g < 24; ++g) {
        for (int j = 0; j < 3; ++j)
            a.lin[g][j] = wc::K::t.m[g][j] * n * n + wc::K::t.m[g][3 + j] * n + wc::K::t.m[g][6 + j];
        a.lin[g][3] = -n * (wc::K::t.fw[g][0] * n * n + wc::K::t.fw[g][1] * n + wc::K::t.fw[g][2]);
    }
    a.ncls = t.n_classes;
    a.free_class = t.free_class;
    a.n3 = (int64_t)t.n * t.n * t.n;
    a.scale = scale;
    return a;
}

fcc_status launch_mix_tiled(const OrderTables& t, int mode, bool real_in, bool real_out, const float* in,
                            float* out, int64_t nvol, float scale, cudaStream_t st, bool pair = false, int which = 0,
                            const int64_t* voff = nullptr) {
    TiledMixArgs a = make_mix_args(t, mode, scale);
    if (t.n_classes > kMaxClasses) return FCC_ERR_UNSUPPORTED;
    const size_t smem = mix_tiled_smem(t.n);
    set_mix_tiled_attributes();
    static const char* names[3] = {"mix_tiled_fwd", "mix_tiled_inv", "mix_tiled_adj"};
    // two launches: free tiles (cores in constant memory) and boundary tiles
    // (one class core per warp staged in shared memory)
    const int ranges[2][2] = {{0, t.free_tiles}, {t.free_tiles, t.ntiles}};
    for (int rg = 0; rg < 2; ++rg) {
        const int tile0 = ranges[rg][0], tile1 = ranges[rg][1];
        if (tile1 <= tile0 || (which == 1 && rg == 1) || (which == 2 && rg == 0)) continue;
        const size_t sm = rg == 0 ? smem : mix_tiled_smem_core(t.n);
        const int core = rg == 1;
        for (int64_t v0 = 0; v0 < nvol; v0 += 65535) {
            const int64_t nv = std::min<int64_t>(65535, nvol - v0);
            dim3 grid((unsigned)((tile1 - tile0 + kMixWarps - 1) / kMixWarps), (unsigned)nv);
            const int nt = tile1;
            if (pair) {
                // nvol counts pairs; forward: real x (2 volumes per pair) -> complex Z at even volumes;
                // inverse / adjoint: compact complex -> real volumes 2p, 2p+1.  Ragged (voff: two
                // point offsets per pair): the real volumes at the listed offsets, Z at the first
                const int64_t* po = voff ? voff + 2 * v0 : nullptr;
                const float* src = voff && mode == MODE_FWD ? in : in + v0 * a.n3 * 2;
                float* dst = voff ? out : out + v0 * a.n3 * (mode == MODE_FWD ? 4 : 2);
                ProfScope ps(names[mode], st);
                if (mode == MODE_FWD) mix_tiled_kernel<MODE_FWD, true, false, true><<<grid, kMixThreads, sm, st>>>(src, dst, a, nt, tile0, core, po);
                else if (mode == MODE_INV) mix_tiled_kernel<MODE_INV, false, true, true><<<grid, kMixThreads, sm, st>>>(src, dst, a, nt, tile0, core, po);
                else mix_tiled_kernel<MODE_ADJ, false, true, true><<<grid, kMixThreads, sm, st>>>(src, dst, a, nt, tile0, core, po);
                continue;
            }
            const float* src = in + v0 * a.n3 * ((mode == MODE_FWD && real_in) ? 1 : 2);
            float* dst = out + v0 * a.n3 * ((mode != MODE_FWD && real_out) ? 1 : 2);
            ProfScope ps(names[mode], st);
            if (voff) {   // ragged: volumes at the listed point offsets (forward only)
                if (real_in) mix_tiled_kernel<MODE_FWD, true, false><<<grid, kMixThreads, sm, st>>>(in, out, a, nt, tile0, core, voff + v0);
                else mix_tiled_kernel<MODE_FWD, false, false><<<grid, kMixThreads, sm, st>>>(in, out, a, nt, tile0, core, voff + v0);
            } else if (mode == MODE_FWD) {
                if (real_in) mix_tiled_kernel<MODE_FWD, true, false><<<grid, kMixThreads, sm, st>>>(src, dst, a, nt, tile0, core);
                else mix_tiled_kernel<MODE_FWD, false, false><<<grid, kMixThreads, sm, st>>>(src, dst, a, nt, tile0, core);
            } else if (mode == MODE_INV) {
                if (real_out) mix_tiled_kernel<MODE_INV, false, true><<<grid, kMixThreads, sm, st>>>(src, dst, a, nt, tile0, core);
                else mix_tiled_kernel<MODE_INV, false, false><<<grid, kMixThreads, sm, st>>>(src, dst, a, nt, tile0, core);
            } else {
                if (real_out) mix_tiled_kernel<MODE_ADJ, false, true><<<grid, kMixThreads, sm, st>>>(src, dst, a, nt, tile0, core);
                else mix_tiled_kernel<MODE_ADJ, false, false><<<grid, kMixThreads, sm, st>>>(src, dst, a, nt, tile0, core);
            }
        }
    }
    return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}

// 3-D DFT of nvol complex volumes: fast slab + pencil passes when the order
// has a register factorisation, else the generic pass per axis.
// volume v of in and out starts at v * vstride complex values.
fcc_status launch_dft3(const OrderTables& t, int sign, const float* in, float* out, int64_t nvol, cudaStream_t st,
                       int64_t vstride = 0) {
    const int64_t n3 = (int64_t)t.n * t.n * t.n;
    if (vstride == 0) vstride = n3;
    // the fast passes move 16-byte pairs of complex values: they need 16-byte
    // aligned volume bases (ragged batches can place a volume at an odd offset)
    const bool aligned = ((((uintptr_t)in) | ((uintptr_t)out)) & 15u) == 0 && vstride % 2 == 0;
    if (has_fast_fft(t.n) && aligned) {
        const float2* tw = (const float2*)t.tw;
        fcc_status s;
        if (sign > 0) {
            if ((s = fast_fft(t.n, true, sign, (const float2*)in, (float2*)out, nvol, tw, vstride, st))) return s;
            return fast_fft(t.n, false, sign, (const float2*)out, (float2*)out, nvol, tw, vstride, st);
        }
        if ((s = fast_fft(t.n, false, sign, (const float2*)in, (float2*)out, nvol, tw, vstride, st))) return s;
        return fast_fft(t.n, true, sign, (const float2*)out, (float2*)out, nvol, tw, vstride, st);
    }
    // generic passes: one launch per axis over every (possibly strided) volume
    fcc_status s = launch_fft<float>(t, in, out, nvol, 0, sign, st, vstride);
    if (!s) s = launch_fft<float>(t, out, out, nvol, 1, sign, st, vstride);
    if (!s) s = launch_fft<float>(t, out, out, nvol, 2, sign, st, vstride);
    return s;
}

fcc_status launch_pair(bool split, int n, const float* in, float* out, int64_t npairs, cudaStream_t st) {
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t per_pair = (int64_t)n * n * (n / 2 + 1);
    for (int64_t p0 = 0; p0 < npairs; p0 += 65535) {
        const int64_t np = std::min<int64_t>(65535, npairs - p0);
        dim3 grid((unsigned)((per_pair + 255) / 256), (unsigned)np);
        if (split) {
            ProfScope ps("pair_split", st);
            pair_split_kernel<<<grid, 256, 0, st>>>((float2*)out + p0 * 2 * n3, n, n3, per_pair);
        } else {
            ProfScope ps("pair_merge", st);
            pair_merge_kernel<<<grid, 256, 0, st>>>((const float2*)in + p0 * 2 * n3, (float2*)out + p0 * n3, n, n3,
                                                    per_pair);
        }
    }
    return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}

// Forward 3-D DFT of `np` paired chunks (Y of pair p at volume 2p of y) and
// the split into D x1, D x2: the fast path fuses the split into the last
// (pencil) pass; otherwise DFT passes then the split kernel.
// fold: the inputs are the phase-free sums of launch_mix_tc_pairs(..., fold);
// the slab and pencil passes apply the row phase's grid factor and 1/24.
bool fold_ok(const OrderTables& t, const float* y) {
    return t.tc_core_image_f && t.pre_slab && has_fast_fft(t.n) && ((uintptr_t)y & 15u) == 0;
}

fcc_status dft3_split_pairs(const OrderTables& t, float* y, int64_t np, cudaStream_t st, bool fold = false) {
    const int64_t n3 = (int64_t)t.n * t.n * t.n;
    if (fold) {
        if (!fold_ok(t, y)) return FCC_ERR_UNSUPPORTED;
        const float2* tw = (const float2*)t.tw;
        {
            ProfScope ps("fft_slab", st);
            if (launch_fast_slab_pre(t.n, (const float2*)y, (float2*)y, np, tw, (const float2*)t.pre_slab, 2 * n3, st) !=
                cudaSuccess)
                return FCC_ERR_CUDA;
        }
        ProfScope ps("fft_pencil_pair", st);
        return launch_fast_pencil_pair(t.n, (const float2*)y, (float2*)y, np, tw, 2 * n3, st, false,
                                       (const float2*)t.pre_pencil) == cudaSuccess
                   ? FCC_OK
                   : FCC_ERR_CUDA;
    }
    if (has_fast_fft(t.n) && ((uintptr_t)y & 15u) == 0) {
        const float2* tw = (const float2*)t.tw;
        fcc_status s = fast_fft(t.n, true, +1, (const float2*)y, (float2*)y, np, tw, 2 * n3, st);
        if (s) return s;
        ProfScope ps("fft_pencil_pair", st);
        return launch_fast_pencil_pair(t.n, (const float2*)y, (float2*)y, np, tw, 2 * n3, st) == cudaSuccess
                   ? FCC_OK
                   : FCC_ERR_CUDA;
    }
    fcc_status s = launch_dft3(t, +1, y, y, np, st, 2 * n3);
    return s ? s : launch_pair(true, t.n, nullptr, y, np, st);
}

// Inverse / adjoint of `np` paired chunks: W = P(v1) + i P(v2) into the compact
// workspace and its - sign 3-D DFT; the fast path fuses the merge into the
// first (pencil) pass.
fcc_status merge_dft3_pairs(const OrderTables& t, const float* y, float* ws, int64_t np, cudaStream_t st) {
    if (has_fast_fft(t.n) && ((((uintptr_t)y) | ((uintptr_t)ws)) & 15u) == 0) {
        const float2* tw = (const float2*)t.tw;
        {
            ProfScope ps("fft_pencil_merge", st);
            if (launch_fast_pencil_merge(t.n, (const float2*)y, (float2*)ws, np, tw, st) != cudaSuccess) return FCC_ERR_CUDA;
        }
        const int64_t n3 = (int64_t)t.n * t.n * t.n;
        return fast_fft(t.n, true, -1, (const float2*)ws, (float2*)ws, np, tw, n3, st);
    }
    fcc_status s = launch_pair(false, t.n, y, ws, np, st);
    return s ? s : launch_dft3(t, -1, ws, ws, np, st);
}

// Forward mixing of `np` pairs of real volumes with the orbit core on the
// tensor cores for the free tiles, the SIMT kernel for the boundary tiles.
// fold: the phase-free form (pair with dft3_split_pairs(..., fold)): the
// mixing writes the sums without row phase and 1/24, the DFT passes modulate.
fcc_status launch_mix_tc_pairs(const fcc_plan* p, const OrderTables& t, const float* in, float* out, int64_t np,
                               cudaStream_t st, bool fold = false, const int64_t* poff = nullptr) {
    TiledMixArgs a = make_mix_args(t, MODE_FWD, 1.f);
    const bool bf16 = is_bf16(p->dtype);
    const size_t smem = bf16 ? TcLayout<0>::smem : TcLayout<1>::smem;
    set_mix_tiled_attributes();
    static DeviceOnce attr;
    if (!attr.done()) {
        cudaFuncSetAttribute(mix_tc_fwd_pair_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcLayout<0>::smem);
        cudaFuncSetAttribute(mix_tc_fwd_pair_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcLayout<1>::smem);
        cudaFuncSetAttribute(mix_tc_fwd_pair_kernel<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcLayout<0>::smem);
        cudaFuncSetAttribute(mix_tc_fwd_pair_kernel<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcLayout<1>::smem);
        cudaFuncSetAttribute(mix_tc_fwd_pair_kernel<0, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcLayout<0>::smem);
        cudaFuncSetAttribute(mix_tc_fwd_pair_kernel<1, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcLayout<1>::smem);
        attr.mark();
    }
    if (fold && !(t.tc_core_image_f && t.tc_core_image)) return FCC_ERR_UNSUPPORTED;
    if (fold && poff) return FCC_ERR_UNSUPPORTED;   // the modulated DFT passes take consecutive pairs
    for (int64_t v0 = 0; v0 < np; v0 += 65535) {
        const int64_t nv = std::min<int64_t>(65535, np - v0);
        // ragged pairs (poff: two point offsets per pair): the kernel reads its table
        const float* src = poff ? in : in + v0 * a.n3 * 2;
        float* dst = poff ? out : out + v0 * a.n3 * 4;
        const int64_t* po = poff ? poff + 2 * v0 : nullptr;
        if (t.free_tiles > 0 && t.tc_core_image) {
            const int ngroups = (t.free_tiles + 3) / 4 + t.tc_nbgroups;
            const TcBoundary bnd = {t.tc_bgroups, t.tc_nbgroups,
                                    (const uint4*)(fold ? t.tc_core_images_f : t.tc_core_images), t.tc_off, t.canon_mask};
            const int lim = bf16 ? TcLayout<0>::blocks_per_sm : TcLayout<1>::blocks_per_sm;
            const int per_sm = p->tc_blocks > 0 ? std::min(p->tc_blocks, lim) : lim;
            const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(ngroups, (int64_t)per_sm * p->num_sms / nv + 1));
            dim3 grid((unsigned)gx, (unsigned)nv);
            ProfScope ps("mix_tc_fwd", st);
            const uint4* ci = (const uint4*)(fold ? t.tc_core_image_f : t.tc_core_image);
            if (po && bf16)   // ragged pairs: the table-reading instantiation (row phase in the epilogue)
                mix_tc_fwd_pair_kernel<0, true, true><<<grid, kTcThreads, smem, st>>>(src, dst, a, t.free_tiles, t.tc_reps32, ci,
                                                                                p->d_status, bnd, p->wait_test, po);
            else if (po)
                mix_tc_fwd_pair_kernel<1, true, true><<<grid, kTcThreads, smem, st>>>(src, dst, a, t.free_tiles, t.tc_reps32, ci,
                                                                                p->d_status, bnd, p->wait_test, po);
            else if (bf16 && fold)
                mix_tc_fwd_pair_kernel<0, false><<<grid, kTcThreads, smem, st>>>(src, dst, a, t.free_tiles, t.tc_reps32, ci,
                                                                                 p->d_status, bnd, p->wait_test);
            else if (bf16)
                mix_tc_fwd_pair_kernel<0><<<grid, kTcThreads, smem, st>>>(src, dst, a, t.free_tiles, t.tc_reps32, ci,
                                                                          p->d_status, bnd, p->wait_test);
            else if (fold)
                mix_tc_fwd_pair_kernel<1, false><<<grid, kTcThreads, smem, st>>>(src, dst, a, t.free_tiles, t.tc_reps32, ci,
                                                                                 p->d_status, bnd, p->wait_test);
            else
                mix_tc_fwd_pair_kernel<1><<<grid, kTcThreads, smem, st>>>(src, dst, a, t.free_tiles, t.tc_reps32, ci,
                                                                          p->d_status, bnd, p->wait_test);
        }
        if (!t.tc_core_image) {   // no free orbits at this order: every tile is a boundary tile
            dim3 grid((unsigned)((t.ntiles + kMixWarps - 1) / kMixWarps), (unsigned)nv);
            ProfScope ps("mix_tiled_fwd", st);
            mix_tiled_kernel<MODE_FWD, true, false, true><<<grid, kMixThreads, mix_tiled_smem_core(t.n), st>>>(
                src, dst, a, t.ntiles, 0, 1, po);
        }
    }
    return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}

// Inverse / adjoint mixing of `np` pairs on the tensor cores: compact complex
// W (pair p at p n^3 of in) -> real volumes 2p, 2p + 1 of out.
fcc_status launch_mix_tc_inv_pairs(const fcc_plan* p, const OrderTables& t, int mode, const float* in, float* out,
                                   int64_t np, float scale, cudaStream_t st) {
    TiledMixArgs a = make_mix_args(t, mode, scale);
    const int md = mode == MODE_INV ? 0 : 1;
    static DeviceOnce attr;
    if (!attr.done()) {
        cudaFuncSetAttribute(mix_tc_inv_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcInvLayout::smem);
        attr.mark();
    }
    const TcBoundary bnd = {t.tc_bgroups, t.tc_nbgroups, (const uint4*)t.tc_inv_images[md], t.tc_off, t.canon_mask};
    const uint4* free_image = (const uint4*)((const unsigned char*)t.tc_inv_images[md] + (size_t)t.free_class * TcInvLayout::image_bytes);
    for (int64_t v0 = 0; v0 < np; v0 += 65535) {
        const int64_t nv = std::min<int64_t>(65535, np - v0);
        const int ngroups = (t.free_tiles + 3) / 4 + t.tc_nbgroups;
        const int per_sm = p->tc_blocks > 0 ? std::min(p->tc_blocks, 3) : 3;   // 80 registers: 3 blocks per SM
        const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(ngroups, (int64_t)per_sm * p->num_sms / nv + 1));
        ProfScope ps(mode == MODE_INV ? "mix_tc_inv" : "mix_tc_adj", st);
        mix_tc_inv_pair_kernel<<<dim3((unsigned)gx, (unsigned)nv), kTcThreads, TcInvLayout::smem, st>>>(
            (const float2*)in + v0 * a.n3, out + v0 * a.n3 * 2, a, t.free_tiles, t.tc_reps32, free_image, scale,
            p->d_status, bnd, p->wait_test);
    }
    return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}

int64_t chunk_vols(const fcc_plan* p, int n) {
    const int64_t n3 = (int64_t)n * n * n;
    return std::max<int64_t>(1, p->chunk_bytes / (n3 * 8));
}

// FP32: chunks of volumes round-robin over the internal streams so that each
// chunk's complex intermediate stays in L2 between its passes.
fcc_status run_group_fast(fcc_plan* p, int which, const OrderTables& t, const float* in, float* out, int64_t nvol,
                          cudaStream_t st) {
    const bool rin = is_real_in(p->dtype);
    const int64_t n3 = (int64_t)t.n * t.n * t.n;
    const int64_t cv = std::min<int64_t>(chunk_vols(p, t.n), std::max<int64_t>(1, p->scratch_points / n3));
    // inverse / adjoint give each stream a slice of the workspace
    const int ns = which == 0 ? p->nstreams : std::min(p->nstreams, p->scratch_streams);
    // real dtypes: two real volumes per complex transform (see pair_split_kernel)
    const bool pairing = rin && p->pairing && nvol >= 2;
    const int64_t npairs = pairing ? nvol / 2 : 0;
    const int64_t cp = cv;   // pairs per chunk: one complex volume of intermediate per pair
    // forward: the boundary (non-free) tiles of every pair in one launch on a
    // stream of their own, concurrent with the chunks' free mixing; each
    // chunk's DFT passes wait for it
    // (the tensor-core kernel takes the boundary tiles itself)
    const bool tc_all = is_tc(p->dtype) && t.tc_core_image;
    const bool split_boundary = which == 0 && npairs > 0 && t.free_tiles > 0 && t.ntiles > t.free_tiles && !tc_all;
    // one chunk, or one internal stream, and no concurrent boundary launch:
    // everything on the caller's stream, in order, with no fork / join events
    // (a small call's cost is mostly the enqueueing; with the boundary tiles
    // on a stream of their own the dependent chain stays one launch shorter)
    const int64_t nchunks = (npairs + cp - 1) / cp + (nvol - 2 * npairs + cv - 1) / cv;
    const bool direct = (ns == 1 || nchunks <= 1) && !split_boundary;
    if (!direct) {
        if (cudaEventRecord(p->fork_ev, st) != cudaSuccess) return FCC_ERR_CUDA;
        for (int i = 0; i < ns; ++i)
            if (cudaStreamWaitEvent(p->streams[i], p->fork_ev, 0) != cudaSuccess) return FCC_ERR_CUDA;
    }
    auto stream_of = [&](int c) { return direct ? st : p->streams[c % ns]; };
    auto slice_of = [&](int c) { return direct ? 0 : c % ns; };
    fcc_status s = FCC_OK;
    int c = 0;
    if (split_boundary) {
        if (cudaStreamWaitEvent(p->bnd_stream, p->fork_ev, 0) != cudaSuccess) return FCC_ERR_CUDA;
        s = launch_mix_tiled(t, MODE_FWD, true, false, in, out, npairs, 1.f, p->bnd_stream, true, 2);
        if (!s && cudaEventRecord(p->bnd_ev, p->bnd_stream) != cudaSuccess) s = FCC_ERR_CUDA;
    }
    for (int64_t p0 = 0; p0 < npairs && !s; p0 += cp, ++c) {
        const int64_t np = std::min(cp, npairs - p0);
        cudaStream_t ss = stream_of(c);
        if (which == 0) {
            const float* x = in + 2 * p0 * n3;
            float* y = out + 2 * p0 * n3 * 2;
            const int part = split_boundary ? 1 : 0;
            const bool fold = tc_all && p->tc_fold && fold_ok(t, y);
            if (is_tc(p->dtype)) {
                s = launch_mix_tc_pairs(p, t, x, y, np, ss, fold);
            } else {
                s = launch_mix_tiled(t, MODE_FWD, true, false, x, y, np, 1.f, ss, true, part);
            }
            if (!s && split_boundary && cudaStreamWaitEvent(ss, p->bnd_ev, 0) != cudaSuccess) s = FCC_ERR_CUDA;
            if (!s) s = dft3_split_pairs(t, y, np, ss, fold);
        } else {
            float* ws = (float*)p->scratch + (size_t)slice_of(c) * p->scratch_points * 2;
            const float* y = in + 2 * p0 * n3 * 2;
            float* x = out + 2 * p0 * n3;
            s = merge_dft3_pairs(t, y, ws, np, ss);
            const float scale = which == 1 ? (float)(1.0 / (double)n3) : 1.f;
            if (!s && tc_all) s = launch_mix_tc_inv_pairs(p, t, which == 1 ? MODE_INV : MODE_ADJ, ws, x, np, scale, ss);
            else if (!s) s = launch_mix_tiled(t, which == 1 ? MODE_INV : MODE_ADJ, false, true, ws, x, np, scale, ss, true);
        }
    }
    for (int64_t v0 = 2 * npairs; v0 < nvol && !s; v0 += cv, ++c) {
        const int64_t nv = std::min(cv, nvol - v0);
        cudaStream_t ss = stream_of(c);
        if (which == 0) {
            const float* x = in + v0 * n3 * (rin ? 1 : 2);
            float* y = out + v0 * n3 * 2;
            s = launch_mix_tiled(t, MODE_FWD, rin, false, x, y, nv, 1.f, ss);
            if (!s) s = launch_dft3(t, +1, y, y, nv, ss);
        } else {
            float* ws = (float*)p->scratch + (size_t)slice_of(c) * p->scratch_points * 2;
            const float* y = in + v0 * n3 * 2;
            float* x = out + v0 * n3 * (rin ? 1 : 2);
            s = launch_dft3(t, -1, y, ws, nv, ss);
            const float scale = which == 1 ? (float)(1.0 / (double)n3) : 1.f;
            if (!s) s = launch_mix_tiled(t, which == 1 ? MODE_INV : MODE_ADJ, false, rin, ws, x, nv, scale, ss);
        }
    }
    if (direct) return s;
    for (int i = 0; i < ns; ++i) {
        if (cudaEventRecord(p->join_ev[i], p->streams[i]) != cudaSuccess) return FCC_ERR_CUDA;
        if (cudaStreamWaitEvent(st, p->join_ev[i], 0) != cudaSuccess) return FCC_ERR_CUDA;
    }
    if (split_boundary) {
        if (cudaEventRecord(p->bnd_join, p->bnd_stream) != cudaSuccess) return FCC_ERR_CUDA;
        if (cudaStreamWaitEvent(st, p->bnd_join, 0) != cudaSuccess) return FCC_ERR_CUDA;
    }
    return s;
}

// Ragged FP32 forward in one cooperative launch (ragged.cuh): every order has
// a register-radix DFT and even volume offsets; at most kRaggedMaxOrders orders.
bool ragged_persistent_ok(const fcc_plan* p) {
    if (p->tabs.size() > (size_t)kRaggedMaxOrders) return false;
    for (const auto& kv : p->tabs)
        if (!ragged_order_supported(kv.first) || kv.second.free_class < 0) return false;
    return true;
}

fcc_status run_ragged_persistent(fcc_plan* p, const float* in, float* out, cudaStream_t st) {
    RaggedArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.real_in = is_real_in(p->dtype) ? 1 : 0;
    std::vector<int> ords;
    int64_t first[3] = {0, 0, 0};
    for (const auto& kv : p->tabs) {
        const OrderTables& t = kv.second;
        RaggedOrder& o = ra.o[ra.norders++];
        o.mix = make_mix_args(t, MODE_FWD, 1.f);
        o.ntiles = t.ntiles;
        o.nvol = t.nvoff;
        o.tw = (const float2*)t.tw;
        o.voff = t.voff;
        for (int k = 0; k < 3; ++k) {
            o.first[k] = first[k];
            first[k] += ragged_units(t.n, t.ntiles, t.nvoff, k);
        }
        ords.push_back(t.n);
    }
    for (int k = 0; k < 3; ++k) ra.units[k] = first[k];
    const size_t smem = ragged_smem_for(ords.data(), (int)ords.size());
    ProfScope ps("ragged_persistent", st);
    const cudaError_t e = launch_ragged_persistent(ra, in, out, smem, 0, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FCC_ERR_CUDA;
    }
    return FCC_OK;
}

// Ragged FP32 forward: per distinct order, one mixing launch and one slab and
// one pencil launch over that order's volumes (device table of point
// offsets), the orders spread over the internal streams.
bool ragged_fast_ok(const fcc_plan* p, int which) {
    if (p->uniform || which != 0 || is_double(p->dtype)) return false;
    for (const auto& kv : p->tabs)
        if (!kv.second.voff || !has_fast_fft(kv.first)) return false;
    return true;
}

// Ragged inverse / adjoint of real volumes, per order: the pairs (merge fused
// into the first pencil pass, reading each pair at its two offsets), the slab
// pass and the inverse mixing writing both volumes back to their offsets, in
// chunks of the workspace; an odd leftover volume alone.
bool ragged_fast_inv_ok(const fcc_plan* p) {
    if (p->uniform || is_double(p->dtype) || !is_real_in(p->dtype) || !p->pairing) return false;
    for (const auto& kv : p->tabs)
        if (!kv.second.voff || !has_fast_fft(kv.first)) return false;
    return true;
}

fcc_status run_ragged_fast_inv(fcc_plan* p, int which, const float* in, float* out, cudaStream_t st) {
    const int ns = std::min(p->nstreams, p->scratch_streams);
    if (cudaEventRecord(p->fork_ev, st) != cudaSuccess) return FCC_ERR_CUDA;
    for (int i = 0; i < ns; ++i)
        if (cudaStreamWaitEvent(p->streams[i], p->fork_ev, 0) != cudaSuccess) return FCC_ERR_CUDA;
    const int mode = which == 1 ? MODE_INV : MODE_ADJ;
    fcc_status s = FCC_OK;
    int c = 0;
    for (auto it = p->tabs.begin(); it != p->tabs.end() && !s; ++it) {
        const OrderTables& t = it->second;
        const int64_t n3 = (int64_t)t.n * t.n * t.n;
        const float2* tw = (const float2*)t.tw;
        const float scale = which == 1 ? (float)(1.0 / (double)n3) : 1.f;
        const int64_t cp = std::max<int64_t>(1, p->scratch_points / n3);   // pairs per workspace slice
        for (int64_t p0 = 0; p0 < t.npairs_r && !s; p0 += cp, ++c) {
            const int64_t np = std::min<int64_t>(cp, t.npairs_r - p0);
            cudaStream_t ss = p->streams[c % ns];
            float* ws = (float*)p->scratch + (size_t)(c % ns) * p->scratch_points * 2;
            {
                ProfScope ps("fft_pencil_merge", ss);
                if (launch_fast_pencil_merge(t.n, (const float2*)in, (float2*)ws, np, tw, ss, false, t.pvoff + 2 * p0) !=
                    cudaSuccess)
                    s = FCC_ERR_CUDA;
            }
            if (!s) s = fast_fft(t.n, true, -1, (const float2*)ws, (float2*)ws, np, tw, n3, ss);
            if (!s) s = launch_mix_tiled(t, mode, false, true, ws, out, np, scale, ss, true, 0, t.pvoff + 2 * p0);
        }
        if (t.single_off >= 0 && !s) {
            cudaStream_t ss = p->streams[c % ns];
            float* ws = (float*)p->scratch + (size_t)(c % ns) * p->scratch_points * 2;
            ++c;
            s = launch_dft3(t, -1, in + 2 * t.single_off, ws, 1, ss);
            if (!s) s = launch_mix_tiled(t, mode, false, true, ws, out + t.single_off, 1, scale, ss);
        }
    }
    for (int i = 0; i < ns; ++i) {
        if (cudaEventRecord(p->join_ev[i], p->streams[i]) != cudaSuccess) return FCC_ERR_CUDA;
        if (cudaStreamWaitEvent(st, p->join_ev[i], 0) != cudaSuccess) return FCC_ERR_CUDA;
    }
    return s;
}

// Pairs of real volumes the ragged forward transforms together at order t.n.
int ragged_pairs(const fcc_plan* p, const OrderTables& t) {
    return is_real_in(p->dtype) && p->pairing && t.pvoff ? t.npairs_r : 0;
}

fcc_status run_ragged_fast(fcc_plan* p, const float* in, float* out, cudaStream_t st) {
    const bool rin = is_real_in(p->dtype);
    const int ns = p->nstreams;
    if (cudaEventRecord(p->fork_ev, st) != cudaSuccess) return FCC_ERR_CUDA;
    for (int i = 0; i < ns; ++i)
        if (cudaStreamWaitEvent(p->streams[i], p->fork_ev, 0) != cudaSuccess) return FCC_ERR_CUDA;
    fcc_status s = FCC_OK;
    int c = 0;
    for (auto it = p->tabs.begin(); it != p->tabs.end() && !s; ++it, ++c) {
        const OrderTables& t = it->second;
        cudaStream_t ss = p->streams[c % ns];
        const float2* tw = (const float2*)t.tw;
        // real volumes: pairs of this order's volumes as one complex transform
        // each (Z and Y in the first volume's output, the split writes both)
        const int np = ragged_pairs(p, t);
        if (np > 0) {
            // tensor-core dtypes mix on the tensor cores (row phase in the epilogue)
            if (is_tc(p->dtype)) s = launch_mix_tc_pairs(p, t, in, out, np, ss, false, t.pvoff);
            else s = launch_mix_tiled(t, MODE_FWD, true, false, in, out, np, 1.f, ss, true, 0, t.pvoff);
            if (!s) s = fast_fft(t.n, true, +1, (const float2*)out, (float2*)out, np, tw, 0, ss, t.pzoff);
            if (!s) {
                ProfScope ps("fft_pencil_pair", ss);
                if (launch_fast_pencil_pair(t.n, (const float2*)out, (float2*)out, np, tw, 0, ss, false, nullptr,
                                            t.pvoff) != cudaSuccess)
                    s = FCC_ERR_CUDA;
            }
        }
        const int single = t.nvoff - 2 * np;   // volumes transformed one by one
        if (single > 0 && !s) {
            const int64_t* vo = t.voff + 2 * np;
            s = launch_mix_tiled(t, MODE_FWD, rin, false, in, out, single, 1.f, ss, false, 0, vo);
            if (!s) s = fast_fft(t.n, true, +1, (const float2*)out, (float2*)out, single, tw, 0, ss, vo);
            if (!s) s = fast_fft(t.n, false, +1, (const float2*)out, (float2*)out, single, tw, 0, ss, vo);
        }
    }
    for (int i = 0; i < ns; ++i) {
        if (cudaEventRecord(p->join_ev[i], p->streams[i]) != cudaSuccess) return FCC_ERR_CUDA;
        if (cudaStreamWaitEvent(st, p->join_ev[i], 0) != cudaSuccess) return FCC_ERR_CUDA;
    }
    return s;
}

// Orbit mixing of a skew plan: the tiled kernels (free tiles on the plan's
// free core, boundary tiles on their staged class cores, the plan's row
// phases), else the generic per-orbit kernel.
bool skew_tiled(const OrderTables& t) { return t.n_classes <= kMaxClasses; }

// part: 0 every tile, 1 free tiles only, 2 boundary tiles only (tiled form)
fcc_status launch_mix_skew(const OrderTables& t, int mode, bool real_io, const float* in, float* out, int64_t nvol,
                           float scale, cudaStream_t st, int part = 0) {
    if (!skew_tiled(t))
        return launch_mix<float>(t, mode, mode == MODE_FWD && real_io, mode != MODE_FWD && real_io, in, out, nvol, scale,
                                 st);
    static const char* names[2][3] = {{"mix_skew_fwd", "mix_skew_inv", "mix_skew_adj"},
                                      {"mix_skew_bnd_fwd", "mix_skew_bnd_inv", "mix_skew_bnd_adj"}};
    const TiledMixArgs a = make_mix_args(t, mode, scale);
    if (t.skew_core.size() != 3) return FCC_ERR_UNSUPPORTED;   // built for every FP32 skew order
    const SkewCore& sc = t.skew_core[mode];
    const int ranges[2][2] = {{0, t.free_tiles}, {t.free_tiles, t.ntiles}};
    for (int rg = 0; rg < 2; ++rg) {
        if (ranges[rg][1] <= ranges[rg][0] || (part == 1 && rg == 1) || (part == 2 && rg == 0)) continue;
        ProfScope ps(names[rg][mode], st);
        if (launch_mix_tiled_skew(a, sc, mode, real_io, in, out, ranges[rg][0], ranges[rg][1], rg == 1, nvol, st) !=
            cudaSuccess)
            return FCC_ERR_CUDA;
    }
    return FCC_OK;
}

// Skew plans, FP32: the orbit mixing of launch_mix_skew and the
// register-radix DFT passes where the order has them, chunks of volumes
// round-robin over the internal streams (each chunk's intermediate stays in
// L2 between its passes).  The forward mixes the boundary tiles of every
// volume in one launch on a stream of its own, concurrent with the chunks'
// free mixing; each chunk's DFT passes wait for it.  Real volumes are not
// paired: the conjugate-point involution the pairing relies on belongs to
// the shift (1/8, 0, 3/8).
fcc_status run_group_skew(fcc_plan* p, int which, const OrderTables& t, const float* in, float* out, int64_t nvol,
                          cudaStream_t st) {
    const bool rin = is_real_in(p->dtype);
    const int64_t n3 = (int64_t)t.n * t.n * t.n;
    const int ns = which == 0 ? p->nstreams : std::min(p->nstreams, p->scratch_streams);
    if (cudaEventRecord(p->fork_ev, st) != cudaSuccess) return FCC_ERR_CUDA;
    for (int i = 0; i < ns; ++i)
        if (cudaStreamWaitEvent(p->streams[i], p->fork_ev, 0) != cudaSuccess) return FCC_ERR_CUDA;
    fcc_status s = FCC_OK;
    const bool split_boundary = which == 0 && skew_tiled(t) && t.free_tiles > 0 && t.ntiles > t.free_tiles;
    if (split_boundary) {
        if (cudaStreamWaitEvent(p->bnd_stream, p->fork_ev, 0) != cudaSuccess) return FCC_ERR_CUDA;
        s = launch_mix_skew(t, MODE_FWD, rin, in, out, nvol, 1.f, p->bnd_stream, 2);
        if (!s && cudaEventRecord(p->bnd_ev, p->bnd_stream) != cudaSuccess) s = FCC_ERR_CUDA;
    }
    int c = 0;
    if (which == 0) {
        const int64_t cv = chunk_vols(p, t.n);
        const int64_t in_stride = (rin ? 1 : 2) * n3;
        for (int64_t v0 = 0; v0 < nvol && !s; v0 += cv, ++c) {
            const int64_t nv = std::min(cv, nvol - v0);
            cudaStream_t ss = p->streams[c % ns];
            float* y = out + v0 * 2 * n3;
            s = launch_mix_skew(t, MODE_FWD, rin, in + v0 * in_stride, y, nv, 1.f, ss, split_boundary ? 1 : 0);
            if (!s && split_boundary && cudaStreamWaitEvent(ss, p->bnd_ev, 0) != cudaSuccess) s = FCC_ERR_CUDA;
            if (!s) s = launch_dft3(t, +1, y, y, nv, ss);
        }
    } else {
        // each stream its slice of the workspace
        const int64_t chunk = std::max<int64_t>(1, p->scratch_points / n3);
        const float scale = which == 1 ? (float)(1.0 / (double)n3) : 1.f;
        const int64_t out_stride = (rin ? 1 : 2) * n3;
        for (int64_t v0 = 0; v0 < nvol && !s; v0 += chunk, ++c) {
            const int64_t nv = std::min(chunk, nvol - v0);
            cudaStream_t ss = p->streams[c % ns];
            float* ws = (float*)p->scratch + (size_t)(c % ns) * p->scratch_points * 2;
            s = launch_dft3(t, -1, in + v0 * 2 * n3, ws, nv, ss);
            if (!s) s = launch_mix_skew(t, which == 1 ? MODE_INV : MODE_ADJ, rin, ws, out + v0 * out_stride, nv, scale, ss);
        }
    }
    for (int i = 0; i < ns; ++i) {
        if (cudaEventRecord(p->join_ev[i], p->streams[i]) != cudaSuccess) return FCC_ERR_CUDA;
        if (cudaStreamWaitEvent(st, p->join_ev[i], 0) != cudaSuccess) return FCC_ERR_CUDA;
    }
    if (split_boundary) {
        if (cudaEventRecord(p->bnd_join, p->bnd_stream) != cudaSuccess) return FCC_ERR_CUDA;
        if (cudaStreamWaitEvent(st, p->bnd_join, 0) != cudaSuccess) return FCC_ERR_CUDA;
    }
    return s;
}

// Run a group of `nvol` consecutive volumes of the same order.
template <typename T>
fcc_status run_group(fcc_plan* p, int which, const OrderTables& t, const T* in, T* out, int64_t nvol,
                     cudaStream_t st) {
    if (sizeof(T) == 4 && t.n > 1 && p->skew)
        return run_group_skew(p, which, t, (const float*)in, (float*)out, nvol, st);
    if (sizeof(T) == 4 && t.n > 1)
        return run_group_fast(p, which, t, (const float*)in, (float*)out, nvol, st);
    const bool rin = is_real_in(p->dtype);
    const int64_t n3 = (int64_t)t.n * t.n * t.n;
    fcc_status s = FCC_OK;
    if (which == 0) {
        // Z = S x into out, then F along the three axes in place.
        if ((s = launch_mix<T>(t, MODE_FWD, rin, false, in, out, nvol, T(1), st))) return s;
        for (int ax = 2; ax >= 0 && !s; --ax) s = launch_fft<T>(t, out, out, nvol, ax, +1, st);
        return s;
    }
    // inverse / adjoint: conj-sign DFT into the workspace, then the orbit map
    const int64_t chunk = std::max<int64_t>(1, p->scratch_points / n3);
    const T scale = which == 1 ? T(1.0 / (double)n3) : T(1);
    const int64_t in_stride = 2 * n3;
    const int64_t out_stride = (rin ? 1 : 2) * n3;
    T* ws = (T*)p->scratch;
    for (int64_t v0 = 0; v0 < nvol && !s; v0 += chunk) {
        const int64_t nv = std::min(chunk, nvol - v0);
        const T* src = in + v0 * in_stride;
        s = launch_fft<T>(t, src, ws, nv, 0, -1, st);
        if (!s) s = launch_fft<T>(t, ws, ws, nv, 1, -1, st);
        if (!s) s = launch_fft<T>(t, ws, ws, nv, 2, -1, st);
        if (!s) s = launch_mix<T>(t, which == 1 ? MODE_INV : MODE_ADJ, false, rin, ws, out + v0 * out_stride, nv, scale, st);
    }
    return s;
}

// --- Hermitian-packed forward / inverse of real volumes ----------------------
// (layout: pair.cuh)

template <typename T>
fcc_status launch_pack(bool pack, int n, const T* src, T* dst, int64_t nvol, cudaStream_t st) {
    const int64_t total = nvol * (int64_t)n * n * n;
    if (total <= 0) return FCC_OK;
    const int64_t blocks = (total + 255) / 256;
    if (blocks > 0x7fffffffLL) return FCC_ERR_UNSUPPORTED;
    ProfScope ps(pack ? "pack_hermitian" : "unpack_hermitian", st);
    if (pack) pack_hermitian_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(src, dst, n, total);
    else unpack_hermitian_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(src, dst, n, total);
    return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}

// Workspace of the packed calls, allocated by the first one: per internal
// stream a slot of 2 * scratch_points complex values, i.e. a chunk of pairs at
// the paired forward's stride of 2 n^3 complex values per pair.
fcc_status ensure_packed_ws(fcc_plan* p) {
    if (p->packed_ws) return FCC_OK;
    const int64_t slot = 2 * p->scratch_points;
    const int streams = std::max(1, p->scratch_streams);
    fcc_status s = dev_alloc(p, &p->packed_ws, (size_t)slot * 2 * real_size(p->dtype) * streams);
    if (s == FCC_OK) {
        p->packed_slot = slot;
        p->packed_streams = streams;
    }
    return s;
}

// (the sizes the first packed call allocates, before it has run)
int64_t packed_slot_of(const fcc_plan* p) { return p->packed_ws ? p->packed_slot : 2 * p->scratch_points; }
int packed_streams_of(const fcc_plan* p) { return p->packed_ws ? p->packed_streams : std::max(1, p->scratch_streams); }

int64_t packed_pairs_per_chunk(const fcc_plan* p, int n) {
    const int64_t n3 = (int64_t)n * n * n;
    return std::max<int64_t>(1, std::min<int64_t>(chunk_vols(p, n), packed_slot_of(p) / (2 * n3)));
}

// Paired fast path (orders with register DFT passes), chunks of pairs
// round-robin over the internal streams.  Forward: the mixing writes Y of each
// pair into the stream's slot, the slab pass transforms it there and the
// pencil pass, fused with the split, writes the packed volumes 2p, 2p + 1.
// Inverse: the pencil pass reads the packed pairs (fused with the merge into
// W = v1 + i v2) into the slot, then the slab pass and the inverse mixing.
fcc_status run_pairs_packed(fcc_plan* p, int which, const OrderTables& t, const float* in, float* out,
                            int64_t npairs, cudaStream_t st) {
    const int64_t n3 = (int64_t)t.n * t.n * t.n;
    const int ns = std::min(p->nstreams, packed_streams_of(p));
    const int64_t cp = packed_pairs_per_chunk(p, t.n);
    const float2* tw = (const float2*)t.tw;
    const bool tc = is_tc(p->dtype);
    const bool tc_all = tc && t.tc_core_image;
    // one chunk, or one internal stream: on the caller's stream, no fork / join
    const bool direct = ns == 1 || npairs <= cp;
    if (!direct) {
        if (cudaEventRecord(p->fork_ev, st) != cudaSuccess) return FCC_ERR_CUDA;
        for (int i = 0; i < ns; ++i)
            if (cudaStreamWaitEvent(p->streams[i], p->fork_ev, 0) != cudaSuccess) return FCC_ERR_CUDA;
    }
    fcc_status s = FCC_OK;
    int c = 0;
    for (int64_t p0 = 0; p0 < npairs && !s; p0 += cp, ++c) {
        const int64_t np = std::min(cp, npairs - p0);
        cudaStream_t ss = direct ? st : p->streams[c % ns];
        float* ws = (float*)p->packed_ws + (size_t)(direct ? 0 : c % ns) * p->packed_slot * 2;
        const float* src = in + 2 * p0 * n3;
        float* dst = out + 2 * p0 * n3;
        if (which == 0) {
            const bool fold = tc_all && p->tc_fold && fold_ok(t, ws);
            s = tc ? launch_mix_tc_pairs(p, t, src, ws, np, ss, fold)
                   : launch_mix_tiled(t, MODE_FWD, true, false, src, ws, np, 1.f, ss, true);
            if (!s && fold) {
                ProfScope ps("fft_slab", ss);
                if (launch_fast_slab_pre(t.n, (const float2*)ws, (float2*)ws, np, tw, (const float2*)t.pre_slab, 2 * n3, ss) !=
                    cudaSuccess)
                    s = FCC_ERR_CUDA;
            } else if (!s) {
                s = fast_fft(t.n, true, +1, (const float2*)ws, (float2*)ws, np, tw, 2 * n3, ss);
            }
            if (!s) {
                ProfScope ps("fft_pencil_pair_packed", ss);
                if (launch_fast_pencil_pair(t.n, (const float2*)ws, (float2*)dst, np, tw, 2 * n3, ss, true,
                                            fold ? (const float2*)t.pre_pencil : nullptr) != cudaSuccess)
                    s = FCC_ERR_CUDA;
            }
        } else {
            {
                ProfScope ps("fft_pencil_merge_packed", ss);
                if (launch_fast_pencil_merge(t.n, (const float2*)src, (float2*)ws, np, tw, ss, true) != cudaSuccess)
                    s = FCC_ERR_CUDA;
            }
            if (!s) s = fast_fft(t.n, true, -1, (const float2*)ws, (float2*)ws, np, tw, n3, ss);
            const float scale = (float)(1.0 / (double)n3);
            if (!s && tc_all) s = launch_mix_tc_inv_pairs(p, t, MODE_INV, ws, dst, np, scale, ss);
            else if (!s) s = launch_mix_tiled(t, MODE_INV, false, true, ws, dst, np, scale, ss, true);
        }
    }
    if (direct) return s;
    for (int i = 0; i < ns; ++i) {
        if (cudaEventRecord(p->join_ev[i], p->streams[i]) != cudaSuccess) return FCC_ERR_CUDA;
        if (cudaStreamWaitEvent(st, p->join_ev[i], 0) != cudaSuccess) return FCC_ERR_CUDA;
    }
    return s;
}

bool packed_fast(const fcc_plan* p, int n, int64_t nvol) {
    return !is_double(p->dtype) && has_fast_fft(n) && p->pairing && nvol >= 2;
}

// One run of volumes of equal order: the paired fast path where it applies;
// every other volume (an unpaired last one, orders without register DFT
// passes, FP64) goes through the complex transform in the packed workspace
// and the (un)packing kernel on the caller's stream.
template <typename T>
fcc_status run_group_packed(fcc_plan* p, int which, const OrderTables& t, const T* in, T* out, int64_t nvol,
                            cudaStream_t st) {
    const int64_t n3 = (int64_t)t.n * t.n * t.n;
    fcc_status s = FCC_OK;
    int64_t v0 = 0;
    if (packed_fast(p, t.n, nvol)) {
        s = run_pairs_packed(p, which, t, (const float*)in, (float*)out, nvol / 2, st);
        v0 = 2 * (nvol / 2);
    }
    T* ws = (T*)p->packed_ws;
    const int64_t cv = std::max<int64_t>(1, packed_slot_of(p) * packed_streams_of(p) / n3);
    for (; v0 < nvol && !s; v0 += cv) {
        const int64_t nv = std::min(cv, nvol - v0);
        if (which == 0) {
            s = run_group<T>(p, 0, t, in + v0 * n3, ws, nv, st);
            if (!s) s = launch_pack<T>(true, t.n, ws, out + v0 * n3, nv, st);
        } else {
            s = launch_pack<T>(false, t.n, in + v0 * n3, ws, nv, st);
            if (!s) s = run_group<T>(p, 1, t, ws, out + v0 * n3, nv, st);
        }
    }
    return s;
}

template <typename T>
fcc_status run_packed(fcc_plan* p, int which, const void* vin, void* vout, cudaStream_t st) {
    const T* in = (const T*)vin;
    T* out = (T*)vout;
    fcc_status s = FCC_OK;
    int v = 0;
    while (v < p->batch && !s) {
        int e = v + 1;
        while (e < p->batch && p->orders[e] == p->orders[v]) ++e;
        const OrderTables& t = p->tabs.at(p->orders[v]);
        s = run_group_packed<T>(p, which, t, in + p->offset[v], out + p->offset[v], e - v, st);
        v = e;
    }
    return s;
}

// The packed layout exists for real dtypes at the canonical shift (the
// involution pi is a property of (1/8, 0, 3/8)).
fcc_status packed_ok(const fcc_plan* p, int which) {
    if (!is_real_in(p->dtype) || p->skew) return FCC_ERR_UNSUPPORTED;
    if (which == 1 && !p->invertible) return FCC_ERR_UNSUPPORTED;
    return FCC_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int64_t in_bytes(const fcc_plan* p, int which) {
    const int64_t rs = real_size(p->dtype);
    if (which == 0) return p->points * rs * (is_real_in(p->dtype) ? 1 : 2);
    return p->points * rs * 2;
}
int64_t out_bytes(const fcc_plan* p, int which) {
    const int64_t rs = real_size(p->dtype);
    if (which == 0) return p->points * rs * 2;
    return p->points * rs * (is_real_in(p->dtype) ? 1 : 2);
}

template <typename T>
fcc_status run(fcc_plan* p, int which, const void* vin, void* vout, cudaStream_t st) {
    const T* in = (const T*)vin;
    T* out = (T*)vout;
    if (sizeof(T) == 4 && p->ragged_fast && p->ragged_mode != 2 && ragged_fast_ok(p, which)) {
        if (p->ragged_mode == 1 && ragged_persistent_ok(p))
            return run_ragged_persistent(p, (const float*)vin, (float*)vout, st);
        return run_ragged_fast(p, (const float*)vin, (float*)vout, st);
    }
    if (sizeof(T) == 4 && which != 0 && p->ragged_fast && p->ragged_mode != 2 && ragged_fast_inv_ok(p))
        return run_ragged_fast_inv(p, which, (const float*)vin, (float*)vout, st);
    const int64_t rs_in = (which == 0 && is_real_in(p->dtype)) ? 1 : 2;
    const int64_t rs_out = (which != 0 && is_real_in(p->dtype)) ? 1 : 2;
    fcc_status s = FCC_OK;
    int v = 0;
    while (v < p->batch && !s) {
        int e = v + 1;
        while (e < p->batch && p->orders[e] == p->orders[v]) ++e;
        const OrderTables& t = p->tabs.at(p->orders[v]);
        s = run_group<T>(p, which, t, in + p->offset[v] * rs_in, out + p->offset[v] * rs_out, e - v, st);
        v = e;
    }
    return s;
}

fcc_status dispatch(fcc_plan* p, int which, const void* in, void* out, void* stream) {
    static const char* names[3] = {"fcc_dct_forward", "fcc_dct_inverse", "fcc_dct_adjoint"};
    CallRange range(names[which < 0 || which > 2 ? 0 : which]);
    if (!p || !in || !out) return fail(FCC_ERR_INVALID_ARG);
    // a device-side timeout of an earlier call surfaces here (the word is
    // host memory; a call still running may set it later)
    if (*(volatile int*)p->h_status != 0) {
        *(volatile int*)p->h_status = 0;
        return fail(FCC_ERR_TIMEOUT);
    }
    if (which == 1 && !p->invertible) return fail(FCC_ERR_UNSUPPORTED);
    if (!aligned16(in) || !aligned16(out)) return fail(FCC_ERR_INVALID_ARG);
    const uintptr_t a0 = (uintptr_t)in, a1 = a0 + in_bytes(p, which);
    const uintptr_t b0 = (uintptr_t)out, b1 = b0 + out_bytes(p, which);
    if (p->r2) {   // the radix-2 recursion: forward only
        if (which != 0) return fail(FCC_ERR_UNSUPPORTED);
        if (a0 < b1 && b0 < a1) return fail(FCC_ERR_INVALID_ARG);
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != p->device) cudaSetDevice(p->device);
        const fcc_status s = r2_forward(p->r2, in, out, (cudaStream_t)stream);
        if (cur != p->device) cudaSetDevice(cur);
        return s == FCC_OK ? FCC_OK : fail(s);
    }
    if (a0 < b1 && b0 < a1) return fail(FCC_ERR_INVALID_ARG);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return fail(FCC_ERR_CUDA); }
    if (cur != p->device) cudaSetDevice(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    g_prof_plan = p;
    fcc_status s = is_double(p->dtype) ? run<double>(p, which, in, out, st) : run<float>(p, which, in, out, st);
    g_prof_plan = nullptr;
    if (cur != p->device) cudaSetDevice(cur);
    return s == FCC_OK ? FCC_OK : fail(s);
}

fcc_status dispatch_packed(fcc_plan* p, int which, const void* in, void* out, void* stream) {
    CallRange range(which == 0 ? "fcc_dct_forward_packed" : "fcc_dct_inverse_packed");
    if (!p || !in || !out) return fail(FCC_ERR_INVALID_ARG);
    if (p->r2) return fail(FCC_ERR_UNSUPPORTED);
    if (*(volatile int*)p->h_status != 0) {   // as in dispatch
        *(volatile int*)p->h_status = 0;
        return fail(FCC_ERR_TIMEOUT);
    }
    fcc_status s = packed_ok(p, which);
    if (s) return fail(s);
    if (!aligned16(in) || !aligned16(out)) return fail(FCC_ERR_INVALID_ARG);
    const int64_t bytes = p->points * (int64_t)real_size(p->dtype);
    const uintptr_t a0 = (uintptr_t)in, a1 = a0 + bytes, b0 = (uintptr_t)out, b1 = b0 + bytes;
    if (a0 < b1 && b0 < a1) return fail(FCC_ERR_INVALID_ARG);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return fail(FCC_ERR_CUDA); }
    if (cur != p->device) cudaSetDevice(p->device);
    s = ensure_packed_ws(p);
    if (s == FCC_OK) {
        g_prof_plan = p;
        s = is_double(p->dtype) ? run_packed<double>(p, which, in, out, (cudaStream_t)stream)
                                : run_packed<float>(p, which, in, out, (cudaStream_t)stream);
        g_prof_plan = nullptr;
    }
    if (cur != p->device) cudaSetDevice(cur);
    return s == FCC_OK ? FCC_OK : fail(s);
}

// Uniform plans: chunks of ~32 MB of volumes go through three streams -- the
// copy in (copy_in), the transform (the caller's stream, forking as usual)
// and the copy out (copy_out) -- so chunk c + 1 arrives and chunk c - 1
// leaves while chunk c is transformed.  Each event is waited on right after
// it is recorded, so one event per direction serves every chunk.
template <typename T>
fcc_status run_host_pipelined(fcc_plan* p, int which, const char* hin, char* hout, cudaStream_t st, bool packed) {
    const int n = p->orders[0];
    const OrderTables& t = p->tabs.at(n);
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t rs_in = packed || (which == 0 && is_real_in(p->dtype)) ? 1 : 2;
    const int64_t rs_out = packed || (which != 0 && is_real_in(p->dtype)) ? 1 : 2;
    const int64_t vin = n3 * rs_in * (int64_t)sizeof(T), vout = n3 * rs_out * (int64_t)sizeof(T);
    int64_t cv = std::max<int64_t>(2, (32ll << 20) / std::max(vin, vout));
    cv += cv % 2;   // whole pairs of real volumes
    char* din = (char*)p->host_in_dev;
    char* dout = (char*)p->host_out_dev;
    if (cudaEventRecord(p->ev_host, st) != cudaSuccess || cudaStreamWaitEvent(p->copy_in, p->ev_host, 0) != cudaSuccess ||
        cudaStreamWaitEvent(p->copy_out, p->ev_host, 0) != cudaSuccess)
        return FCC_ERR_CUDA;
    fcc_status s = FCC_OK;
    for (int64_t v0 = 0; v0 < p->batch && !s; v0 += cv) {
        const int64_t nv = std::min<int64_t>(cv, p->batch - v0);
        if (cudaMemcpyAsync(din + v0 * vin, hin + v0 * vin, nv * vin, cudaMemcpyHostToDevice, p->copy_in) != cudaSuccess ||
            cudaEventRecord(p->ev_in, p->copy_in) != cudaSuccess || cudaStreamWaitEvent(st, p->ev_in, 0) != cudaSuccess) {
            s = FCC_ERR_CUDA;
            break;
        }
        s = packed ? run_group_packed<T>(p, which, t, (const T*)(din + v0 * vin), (T*)(dout + v0 * vout), nv, st)
                   : run_group<T>(p, which, t, (const T*)(din + v0 * vin), (T*)(dout + v0 * vout), nv, st);
        if (s) break;
        if (cudaEventRecord(p->ev_out, st) != cudaSuccess || cudaStreamWaitEvent(p->copy_out, p->ev_out, 0) != cudaSuccess ||
            cudaMemcpyAsync(hout + v0 * vout, dout + v0 * vout, nv * vout, cudaMemcpyDeviceToHost, p->copy_out) != cudaSuccess)
            s = FCC_ERR_CUDA;
    }
    // the caller's stream completes after the last copy out
    if (cudaEventRecord(p->ev_host, p->copy_out) != cudaSuccess || cudaStreamWaitEvent(st, p->ev_host, 0) != cudaSuccess)
        return FCC_ERR_CUDA;
    return s;
}

fcc_status dispatch_host(fcc_plan* p, int which, const void* hin, void* hout, void* stream, bool packed = false) {
    CallRange range(packed ? "fcc_dct_packed_host" : "fcc_dct_host");
    if (!p || !hin || !hout) return fail(FCC_ERR_INVALID_ARG);
    if (p->r2) return fail(FCC_ERR_UNSUPPORTED);
    if (which == 1 && !p->invertible) return fail(FCC_ERR_UNSUPPORTED);
    if (packed && packed_ok(p, which)) return fail(packed_ok(p, which));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t pk = p->points * (int64_t)real_size(p->dtype);   // a packed (or real) batch
    const int64_t ib = packed ? pk : in_bytes(p, which), ob = packed ? pk : out_bytes(p, which);
    const int64_t cap = std::max(in_bytes(p, 0), in_bytes(p, 1));
    const int64_t capo = std::max(out_bytes(p, 0), out_bytes(p, 1));
    fcc_status s;
    if (!p->host_in_dev && (s = dev_alloc(p, &p->host_in_dev, cap))) return fail(s);
    if (!p->host_out_dev && (s = dev_alloc(p, &p->host_out_dev, capo))) return fail(s);
    if (p->uniform && p->batch >= 4) {
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return fail(FCC_ERR_CUDA); }
        if (cur != p->device) cudaSetDevice(p->device);
        s = packed ? ensure_packed_ws(p) : FCC_OK;
        g_prof_plan = p;
        if (s == FCC_OK)
            s = is_double(p->dtype) ? run_host_pipelined<double>(p, which, (const char*)hin, (char*)hout, st, packed)
                                    : run_host_pipelined<float>(p, which, (const char*)hin, (char*)hout, st, packed);
        g_prof_plan = nullptr;
        if (cur != p->device) cudaSetDevice(cur);
        return s == FCC_OK ? FCC_OK : fail(s);
    }
    if (cudaMemcpyAsync(p->host_in_dev, hin, ib, cudaMemcpyHostToDevice, st) != cudaSuccess) return fail(FCC_ERR_CUDA);
    if ((s = packed ? dispatch_packed(p, which, p->host_in_dev, p->host_out_dev, stream)
                    : dispatch(p, which, p->host_in_dev, p->host_out_dev, stream)))
        return s;
    if (cudaMemcpyAsync(hout, p->host_out_dev, ob, cudaMemcpyDeviceToHost, st) != cudaSuccess) return fail(FCC_ERR_CUDA);
    return FCC_OK;
}

// Launches of one run of `nv` volumes of order n (run_group, excluding the
// ragged fast paths).  Every grid with one row per volume (or pair) is split
// into launches of at most 65,535 rows.
int64_t grid_rows(int64_t rows) { return (rows + 65534) / 65535; }

int group_launches(const fcc_plan* p, int which, int n, int64_t nv) {
    int64_t total = 0;
    const int64_t n3 = (int64_t)n * n * n;
    const int fft = n > 1 ? 3 : 0;   // order 1: the DFT is a copy, no kernel
    if (!is_double(p->dtype) && n > 1 && p->skew) {
        // run_group_skew: per chunk the mixing launches (free and boundary
        // tiles, or the generic kernel) and the DFT passes; the forward
        // mixes the boundary tiles of every volume in one launch set
        const OrderTables& tb = p->tabs.at(n);
        const int dft = has_fast_fft(n) ? 2 : 3;
        const bool tiled = skew_tiled(tb);
        const bool split_b = which == 0 && tiled && tb.free_tiles > 0 && tb.ntiles > tb.free_tiles;
        const int kinds = !tiled ? 1 : split_b ? 1 : (tb.free_tiles > 0 ? 1 : 0) + (tb.ntiles > tb.free_tiles ? 1 : 0);
        if (split_b) total += grid_rows(nv);
        const int64_t cv = which == 0 ? chunk_vols(p, n) : std::max<int64_t>(1, p->scratch_points / n3);
        for (int64_t v0 = 0; v0 < nv; v0 += cv) total += kinds * grid_rows(std::min(cv, nv - v0)) + dft;
    } else if (!is_double(p->dtype) && n > 1) {
        // run_group_fast
        const int64_t cv = std::min<int64_t>(chunk_vols(p, n), std::max<int64_t>(1, p->scratch_points / n3));
        const bool fast = has_fast_fft(n);
        const OrderTables& tb = p->tabs.at(n);
        const int mixl = (tb.free_tiles > 0 ? 1 : 0) + (tb.ntiles > tb.free_tiles ? 1 : 0);
        const bool pairing = is_real_in(p->dtype) && p->pairing && nv >= 2;
        const bool tc = is_tc(p->dtype), tc_all = tc && tb.tc_core_image;   // one launch mixes every tile
        const int64_t npairs = pairing ? nv / 2 : 0;
        const bool split_b = which == 0 && npairs > 0 && tb.free_tiles > 0 && tb.ntiles > tb.free_tiles && !tc_all;
        if (split_b) total += grid_rows(npairs);   // the boundary tiles of every pair
        for (int64_t p0 = 0; p0 < npairs; p0 += cv) {
            const int64_t np = std::min(cv, npairs - p0), rows = grid_rows(np);
            if (which == 0) {
                // mixing (tensor cores: one kernel; else free (+ boundary) tiles),
                // then slab + pencil-with-split, or three passes + the split kernel
                total += (tc ? 1 : split_b ? 1 : mixl) * rows;
                total += fast ? 2 : 3 + rows;
            } else {
                // merge fused into the pencil pass + slab, or merge + three passes;
                // then the mixing
                total += fast ? 2 : rows + 3;
                total += (tc_all ? 1 : mixl) * rows;
            }
        }
        const int64_t rest = nv - 2 * npairs;
        for (int64_t v0 = 0; v0 < rest; v0 += cv) total += mixl * grid_rows(std::min(cv, rest - v0)) + (fast ? 2 : 3);
    } else if (which == 0) {
        total += grid_rows(nv) + fft;
    } else {
        const int64_t chunk = std::max<int64_t>(1, p->scratch_points / n3);
        for (int64_t v0 = 0; v0 < nv; v0 += chunk) total += fft + grid_rows(std::min(chunk, nv - v0));
    }
    return (int)std::min<int64_t>(total, 0x7fffffff);
}

// Launches of the packed forward (which 0) / inverse (1): run_group_packed.
int packed_launches(const fcc_plan* p, int which) {
    if (packed_ok(p, which)) return 0;
    int total = 0;
    int v = 0;
    while (v < p->batch) {
        int e = v + 1;
        while (e < p->batch && p->orders[e] == p->orders[v]) ++e;
        const int n = p->orders[v];
        const int64_t n3 = (int64_t)n * n * n;
        const int64_t nv = e - v;
        int64_t v0 = 0;
        if (packed_fast(p, n, nv)) {
            const OrderTables& tb = p->tabs.at(n);
            const int mixl = (tb.free_tiles > 0 ? 1 : 0) + (tb.ntiles > tb.free_tiles ? 1 : 0);
            const bool tc = is_tc(p->dtype), tc_all = tc && tb.tc_core_image;
            const int mix = which == 0 ? (tc ? 1 : mixl) : (tc_all ? 1 : mixl);
            const int64_t npairs = nv / 2, cp = packed_pairs_per_chunk(p, n);
            for (int64_t p0 = 0; p0 < npairs; p0 += cp) total += mix * (int)grid_rows(std::min(cp, npairs - p0)) + 2;
            v0 = 2 * npairs;
        }
        const int64_t cv = std::max<int64_t>(1, packed_slot_of(p) * packed_streams_of(p) / n3);
        for (; v0 < nv; v0 += cv) total += 1 + group_launches(p, which, n, std::min(cv, nv - v0));
        v = e;
    }
    return total;
}

}  // namespace

extern "C" {

fcc_plan* fcc_dct_plan(int order, int batch, int dtype) {
    if (batch < 1 || order < 1 || order > FCC_MAX_ORDER) { fail(FCC_ERR_INVALID_ARG); return nullptr; }
    return make_plan(std::vector<int>((size_t)batch, order), dtype);
}

static_assert(FCC_MAX_SHIFT_DEN == kMaxShiftDen && FCC_MAX_SHIFT_NUM == kMaxShiftNum, "shift limits");

fcc_plan* fcc_dct_plan_skew(int order, int batch, int dtype, const int* v, int d) {
    if (batch < 1 || order < 1 || order > FCC_MAX_ORDER || !v || d < 1 || d > FCC_MAX_SHIFT_DEN) {
        fail(FCC_ERR_INVALID_ARG);
        return nullptr;
    }
    for (int i = 0; i < 3; ++i)
        if (v[i] < -FCC_MAX_SHIFT_NUM || v[i] > FCC_MAX_SHIFT_NUM) { fail(FCC_ERR_INVALID_ARG); return nullptr; }
    if (dtype < FCC_R64 || dtype > FCC_R32_BF16X6) { fail(FCC_ERR_INVALID_ARG); return nullptr; }
    // the tensor-core forms rely on the exact split of 8th-root cores and on
    // the canonical row phases
    if (is_tc(dtype) && !canonical_shift(v, d)) { fail(FCC_ERR_UNSUPPORTED); return nullptr; }
    return make_plan(std::vector<int>((size_t)batch, order), dtype, v, d);
}

fcc_plan* fcc_dct_plan_radix2(int order, int batch, int dtype, const int* v, int d) {
    if ((dtype != FCC_C64 && dtype != FCC_C32) || !(order == 2 || order == 4 || order == 8 || order == 16) ||
        batch < 1 || batch > 65535) {
        fail(FCC_ERR_INVALID_ARG);
        return nullptr;
    }
    const int canon[3] = {1, 0, 3};
    if (!v) { v = canon; d = 8; }
    if (d < 1 || d > kMaxShiftDen) { fail(FCC_ERR_INVALID_ARG); return nullptr; }
    for (int i = 0; i < 3; ++i)
        if (std::abs(v[i]) > kMaxShiftNum) { fail(FCC_ERR_INVALID_ARG); return nullptr; }
    fcc_plan* p = make_plan(std::vector<int>((size_t)batch, order), dtype, v, d);
    if (!p) return nullptr;
    fcc_status s = FCC_OK;
    auto alloc = [](void* ctx, void** ptr, size_t bytes) -> fcc_status { return dev_alloc((fcc_plan*)ctx, ptr, bytes); };
    p->r2 = r2_build(order, batch, dtype == FCC_C64, v, d, alloc, p, &s);
    if (!p->r2) {
        release(p);
        fail(s);
        return nullptr;
    }
    return p;
}

int fcc_dct_radix2_stats(const fcc_plan* p, int level, double* nnz_per_row, double* max_abs, double* macs_per_point) {
    if (!p || !p->r2) { fail(FCC_ERR_INVALID_ARG); return -1; }
    const int r = r2_stats(p->r2, level, nnz_per_row, max_abs, macs_per_point);
    if (r < 0) fail(FCC_ERR_INVALID_ARG);
    return r;
}

fcc_plan* fcc_dct_plan_ragged(const int* orders, int count, int dtype) {
    if (!orders || count < 1) { fail(FCC_ERR_INVALID_ARG); return nullptr; }
    return make_plan(std::vector<int>(orders, orders + count), dtype);
}

fcc_status fcc_dct_set_schedule(fcc_plan* p, int key, int value) {
    if (!p) return fail(FCC_ERR_INVALID_ARG);
    switch (key) {
        case FCC_SCHED_CHUNK_MB:
            if (value < 1 || value > 1024) return fail(FCC_ERR_INVALID_ARG);
            p->chunk_bytes = (int64_t)value << 20;
            return FCC_OK;
        case FCC_SCHED_STREAMS:
            if (value < 1 || value > kMaxStreams) return fail(FCC_ERR_INVALID_ARG);
            p->nstreams = value;
            return FCC_OK;
        case FCC_SCHED_RAGGED:
            if (value < 0 || value > 2) return fail(FCC_ERR_INVALID_ARG);
            if (value == 1 && (p->uniform || !ragged_fast_ok(p, 0) || !ragged_persistent_ok(p))) return fail(FCC_ERR_UNSUPPORTED);
            p->ragged_mode = value;
            return FCC_OK;
        case FCC_SCHED_TC_BLOCKS:
            if (value < 0 || value > 4) return fail(FCC_ERR_INVALID_ARG);
            p->tc_blocks = value;
            return FCC_OK;
        case FCC_SCHED_TC_FOLD:
            if (value < 0 || value > 1) return fail(FCC_ERR_INVALID_ARG);
            p->tc_fold = value;
            return FCC_OK;
        default:
            return fail(FCC_ERR_INVALID_ARG);
    }
}

int fcc_dct_get_schedule(const fcc_plan* p, int key) {
    if (!p) return -1;
    switch (key) {
        case FCC_SCHED_CHUNK_MB: return (int)(p->chunk_bytes >> 20);
        case FCC_SCHED_STREAMS: return p->nstreams;
        case FCC_SCHED_RAGGED: return p->ragged_mode;
        case FCC_SCHED_TC_BLOCKS: return p->tc_blocks;
        case FCC_SCHED_TC_FOLD: return p->tc_fold;
        default: return -1;
    }
}

namespace {

// The autotuner's cache: one JSON object per line in the file named by
// FCC_AUTOTUNE_CACHE, keyed by the plan's shape, dtype, shift and GPU name;
// a later line for the same key overrides an earlier one.  Reading and
// writing it are advisory: a missing, unreadable or malformed file only
// means that the search runs.
std::string autotune_key(const fcc_plan* p) {
    char gpu[256] = "unknown";
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) {
        std::snprintf(gpu, sizeof gpu, "%s", prop.name);
        for (char* c = gpu; *c; ++c)
            if (*c == '"' || *c == '\\') *c = '_';
    } else {
        cudaGetLastError();
    }
    std::string shape;
    if (p->uniform) {
        shape = "order=" + std::to_string(p->orders[0]);
    } else {   // ragged: the order list, hashed (FNV-1a)
        uint64_t h = 1469598103934665603ull;
        for (int o : p->orders) {
            h ^= (uint64_t)o;
            h *= 1099511628211ull;
        }
        char buf[64];
        std::snprintf(buf, sizeof buf, "ragged=%016llx", (unsigned long long)h);
        shape = buf;
    }
    char key[512];
    std::snprintf(key, sizeof key, "%s batch=%d dtype=%d shift=%d,%d,%d/%d gpu=%s", shape.c_str(), p->batch, p->dtype,
                  p->shift_v[0], p->shift_v[1], p->shift_v[2], p->shift_d, gpu);
    return key;
}

int json_int(const char* line, const char* name, bool& ok) {
    const std::string pat = std::string("\"") + name + "\": ";
    const char* at = std::strstr(line, pat.c_str());
    int v = 0;
    if (!at || std::sscanf(at + pat.size(), "%d", &v) != 1) ok = false;
    return v;
}

// The cached schedule {chunk_mb, streams, ragged, tc_blocks, tc_fold} of `key`.
bool autotune_cache_read(const char* path, const std::string& key, int sched[5]) {
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    const std::string pat = "\"key\": \"" + key + "\"";
    bool found = false;
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
        if (!std::strstr(line, pat.c_str())) continue;
        bool ok = true;
        int s[5] = {json_int(line, "chunk_mb", ok), json_int(line, "streams", ok), json_int(line, "ragged", ok),
                    json_int(line, "tc_blocks", ok), json_int(line, "tc_fold", ok)};
        if (ok && s[0] >= 1 && s[0] <= 4096 && s[1] >= 1 && s[1] <= kMaxStreams && s[2] >= 0 && s[2] <= 2 &&
            s[3] >= 0 && s[3] <= 8 && (s[4] == 0 || s[4] == 1)) {
            std::memcpy(sched, s, sizeof s);
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void autotune_cache_write(const char* path, const std::string& key, const int sched[5], float ms) {
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"chunk_mb\": %d, \"streams\": %d, \"ragged\": %d, \"tc_blocks\": %d, "
                 "\"tc_fold\": %d, \"ms\": %.4f}\n",
                 key.c_str(), sched[0], sched[1], sched[2], sched[3], sched[4], (double)ms);
    std::fclose(f);
}

}  // namespace

fcc_status fcc_dct_autotune(fcc_plan* p, const void* in, void* out, void* stream, int reps, float* best_ms) {
    if (!p || !in || !out || reps < 1 || reps > 100) return fail(FCC_ERR_INVALID_ARG);
    if (p->r2) return fail(FCC_ERR_UNSUPPORTED);
    CallRange range("fcc_dct_autotune");
    cudaStream_t st = (cudaStream_t)stream;
    const char* cache = std::getenv("FCC_AUTOTUNE_CACHE");
    const std::string key = cache && *cache ? autotune_key(p) : std::string();
    int cached[5];
    const bool hit = !key.empty() && autotune_cache_read(cache, key, cached);
    struct Cand { int chunk_mb, streams, ragged, tc, fold; };
    std::vector<Cand> cands;
    const int tc0 = p->tc_blocks, f0 = p->tc_fold;
    if (!p->uniform) {
        const bool fast = !is_double(p->dtype) && ragged_fast_ok(p, 0);
        for (int ns = 1; ns <= kMaxStreams && fast; ++ns) cands.push_back({32, ns, 0, tc0, f0});
        if (fast && ragged_persistent_ok(p)) cands.push_back({32, 2, 1, tc0, f0});
        cands.push_back({32, 2, 2, tc0, f0});
    } else {
        for (int mb : {8, 16, 32, 64})
            for (int ns = 1; ns <= kMaxStreams; ++ns) cands.push_back({mb, ns, 0, tc0, f0});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return fail(FCC_ERR_CUDA);
    }
    const Cand saved = {(int)(p->chunk_bytes >> 20), p->nstreams, p->ragged_mode, p->tc_blocks, p->tc_fold};
    auto apply = [&](const Cand& c) {
        p->chunk_bytes = (int64_t)c.chunk_mb << 20;
        p->nstreams = c.streams;
        p->ragged_mode = c.ragged;
        p->tc_blocks = c.tc;
        p->tc_fold = c.fold;
    };
    auto time_it = [&](const Cand& c, float& ms) -> bool {
        apply(c);
        if (dispatch(p, 0, in, out, stream) != FCC_OK || cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r)
            if (dispatch(p, 0, in, out, stream) != FCC_OK) {
                cudaStreamSynchronize(st);
                cudaGetLastError();
                return false;
            }
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        ms /= (float)reps;
        return true;
    };
    Cand best = saved;
    float best_t = -1.f;
    if (hit) {   // the cached schedule, timed once so that *best_ms is this call's
        const Cand c = {cached[0], cached[1], cached[2], cached[3], cached[4]};
        float ms = 0.f;
        if (time_it(c, ms)) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            apply(c);
            if (best_ms) *best_ms = ms;
            return FCC_OK;
        }
        cands.insert(cands.begin(), c);   // refused here: search as if not cached
    }
    for (const Cand& c : cands) {
        float ms = 0.f;
        if (time_it(c, ms) && (best_t < 0.f || ms < best_t)) {
            best_t = ms;
            best = c;
        }
    }
    // tensor-core forms: then where the row phase is applied, and the grid of
    // the mixing kernel
    if (p->uniform && is_tc(p->dtype) && best_t >= 0.f) {
        {
            Cand c = best;
            c.fold = 1 - c.fold;
            float ms = 0.f;
            if (time_it(c, ms) && ms < best_t) {
                best_t = ms;
                best = c;
            }
        }
        for (int tcb : {2, 3, 4}) {
            Cand c = best;
            c.tc = tcb;
            float ms = 0.f;
            if (time_it(c, ms) && ms < best_t) {
                best_t = ms;
                best = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_t < 0.f) {
        apply(saved);
        return fail(FCC_ERR_CUDA);
    }
    apply(best);
    if (best_ms) *best_ms = best_t;
    if (!key.empty()) {
        const int sched[5] = {best.chunk_mb, best.streams, best.ragged, best.tc, best.fold};
        autotune_cache_write(cache, key, sched, best_t);
    }
    return FCC_OK;
}

fcc_status fcc_dct_diag_mixing_replay(fcc_plan* p, const void* in, void* out, void* stream) {
    CallRange range("fcc_dct_diag_mixing_replay");
    if (!p || !in || !out) return fail(FCC_ERR_INVALID_ARG);
    if (!p->uniform || !is_tc(p->dtype) || p->skew || p->r2 || !p->pairing || p->batch < 2)
        return fail(FCC_ERR_UNSUPPORTED);
    const OrderTables& t = p->tabs.at(p->orders[0]);
    if (t.free_tiles <= 0 || !t.tc_core_image) return fail(FCC_ERR_UNSUPPORTED);
    if (!aligned16(in) || !aligned16(out)) return fail(FCC_ERR_INVALID_ARG);
    const uintptr_t a0 = (uintptr_t)in, a1 = a0 + in_bytes(p, 0);
    const uintptr_t b0 = (uintptr_t)out, b1 = b0 + out_bytes(p, 0);
    if (a0 < b1 && b0 < a1) return fail(FCC_ERR_INVALID_ARG);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return fail(FCC_ERR_CUDA); }
    if (cur != p->device) cudaSetDevice(p->device);
    const cudaStream_t st = (cudaStream_t)stream;
    const bool bf16 = is_bf16(p->dtype);
    const size_t smem = bf16 ? TcLayout<0>::smem : TcLayout<1>::smem;
    static DeviceOnce attr;
    if (!attr.done()) {
        cudaFuncSetAttribute(mix_replay_pair_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcLayout<0>::smem);
        cudaFuncSetAttribute(mix_replay_pair_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcLayout<1>::smem);
        attr.mark();
    }
    // the forward's chunks of pairs (run_group_fast), each chunk's mixing
    // launch replayed on the caller's stream
    const int64_t n3 = (int64_t)t.n * t.n * t.n;
    const int64_t cp = std::min<int64_t>(chunk_vols(p, t.n), std::max<int64_t>(1, p->scratch_points / n3));
    const int64_t npairs = p->batch / 2;
    const TiledMixArgs a = make_mix_args(t, MODE_FWD, 1.f);
    const TcBoundary bnd = {t.tc_bgroups, t.tc_nbgroups, (const uint4*)t.tc_core_images, t.tc_off, t.canon_mask};
    const int ngroups = (t.free_tiles + 3) / 4 + t.tc_nbgroups;
    const int lim = bf16 ? TcLayout<0>::blocks_per_sm : TcLayout<1>::blocks_per_sm;
    const int per_sm = p->tc_blocks > 0 ? std::min(p->tc_blocks, lim) : lim;
    g_prof_plan = p;
    for (int64_t p0 = 0; p0 < npairs; p0 += cp) {
        const int64_t np = std::min(cp, npairs - p0);
        for (int64_t v0 = 0; v0 < np; v0 += 65535) {
            const int64_t nv = std::min<int64_t>(65535, np - v0);
            const float* src = (const float*)in + (p0 + v0) * 2 * n3;
            float* dst = (float*)out + (p0 + v0) * 4 * n3;
            const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(ngroups, (int64_t)per_sm * p->num_sms / nv + 1));
            dim3 grid((unsigned)gx, (unsigned)nv);
            ProfScope ps("mix_replay", st);
            if (bf16) mix_replay_pair_kernel<0><<<grid, kTcThreads, smem, st>>>(src, dst, a, t.free_tiles, t.tc_reps32, bnd);
            else mix_replay_pair_kernel<1><<<grid, kTcThreads, smem, st>>>(src, dst, a, t.free_tiles, t.tc_reps32, bnd);
        }
    }
    g_prof_plan = nullptr;
    if (cur != p->device) cudaSetDevice(cur);
    return cudaGetLastError() == cudaSuccess ? FCC_OK : fail(FCC_ERR_CUDA);
}

fcc_status fcc_dct_forward(fcc_plan* p, const void* in, void* out, void* stream) { return dispatch(p, 0, in, out, stream); }
fcc_status fcc_dct_inverse(fcc_plan* p, const void* in, void* out, void* stream) { return dispatch(p, 1, in, out, stream); }
fcc_status fcc_dct_adjoint(fcc_plan* p, const void* in, void* out, void* stream) { return dispatch(p, 2, in, out, stream); }
fcc_status fcc_dct_forward_host(fcc_plan* p, const void* in, void* out, void* stream) { return dispatch_host(p, 0, in, out, stream); }
fcc_status fcc_dct_inverse_host(fcc_plan* p, const void* in, void* out, void* stream) { return dispatch_host(p, 1, in, out, stream); }
fcc_status fcc_dct_forward_packed(fcc_plan* p, const void* in, void* out, void* stream) { return dispatch_packed(p, 0, in, out, stream); }
fcc_status fcc_dct_inverse_packed(fcc_plan* p, const void* in, void* out, void* stream) { return dispatch_packed(p, 1, in, out, stream); }
fcc_status fcc_dct_forward_packed_host(fcc_plan* p, const void* in, void* out, void* stream) {
    return dispatch_host(p, 0, in, out, stream, true);
}
fcc_status fcc_dct_inverse_packed_host(fcc_plan* p, const void* in, void* out, void* stream) {
    return dispatch_host(p, 1, in, out, stream, true);
}

int fcc_dct_batch(const fcc_plan* p) { return p ? p->batch : 0; }
int64_t fcc_dct_points(const fcc_plan* p) { return p ? p->points : 0; }
int64_t fcc_dct_in_bytes(const fcc_plan* p) { return p ? in_bytes(p, 0) : 0; }
int64_t fcc_dct_out_bytes(const fcc_plan* p) { return p ? out_bytes(p, 0) : 0; }

int fcc_dct_launches(const fcc_plan* p, int which) {
    if (!p) return 0;
    if (p->r2) return which == 0 ? r2_launches(p->r2) : 0;
    if (which == 3 || which == 4) return packed_launches(p, which - 3);
    int total = 0;
    if (!is_double(p->dtype) && p->ragged_fast && p->ragged_mode != 2 && ragged_fast_ok(p, which)) {
        if (p->ragged_mode == 1 && ragged_persistent_ok(p)) return 1;
        for (const auto& kv : p->tabs) {
            const OrderTables& t = kv.second;
            const int mixl = (t.free_tiles > 0 ? 1 : 0) + (t.ntiles > t.free_tiles ? 1 : 0);
            const int np = ragged_pairs(p, t), single = t.nvoff - 2 * np;
            if (np > 0) total += (is_tc(p->dtype) ? 1 : mixl) * (int)grid_rows(np) + 2;
            if (single > 0) total += mixl * (int)grid_rows(single) + 2;
        }
        return total;
    }
    if (!is_double(p->dtype) && which != 0 && p->ragged_fast && p->ragged_mode != 2 && ragged_fast_inv_ok(p)) {
        for (const auto& kv : p->tabs) {   // run_ragged_fast_inv
            const OrderTables& t = kv.second;
            const int mixl = (t.free_tiles > 0 ? 1 : 0) + (t.ntiles > t.free_tiles ? 1 : 0);
            const int64_t n3 = (int64_t)t.n * t.n * t.n, cp = std::max<int64_t>(1, p->scratch_points / n3);
            for (int64_t p0 = 0; p0 < t.npairs_r; p0 += cp) total += 2 + mixl * (int)grid_rows(std::min(cp, t.npairs_r - p0));
            if (t.single_off >= 0) total += 2 + mixl;
        }
        return total;
    }
    int v = 0;
    while (v < p->batch) {
        int e = v + 1;
        while (e < p->batch && p->orders[e] == p->orders[v]) ++e;
        total += group_launches(p, which, p->orders[v], e - v);
        v = e;
    }
    return total;
}

fcc_status fcc_dct_profile_enable(fcc_plan* p, int enable) {
    if (!p) return fail(FCC_ERR_INVALID_ARG);
    p->profiling = enable != 0;
    return FCC_OK;
}

int fcc_dct_profile_read(fcc_plan* p, char* names, double* ms, int* launches, int cap) {
    if (!p || cap < 0) { fail(FCC_ERR_INVALID_ARG); return -1; }
    std::vector<std::string> kinds;
    std::vector<double> tot;
    std::vector<int> cnt;
    for (auto& r : p->recs) {
        float t = 0.f;
        if (r.a && r.b) {
            if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
                cudaGetLastError();
                t = 0.f;
            }
        }
        size_t k = 0;
        while (k < kinds.size() && kinds[k] != r.name) ++k;
        if (k == kinds.size()) { kinds.push_back(r.name); tot.push_back(0); cnt.push_back(0); }
        tot[k] += t;
        cnt[k] += 1;
        if (r.a) p->event_pool.push_back(r.a);
        if (r.b) p->event_pool.push_back(r.b);
    }
    p->recs.clear();
    for (size_t k = 0; k < kinds.size() && (int)k < cap; ++k) {
        if (names) { std::strncpy(names + 48 * k, kinds[k].c_str(), 47); names[48 * k + 47] = 0; }
        if (ms) ms[k] = tot[k];
        if (launches) launches[k] = cnt[k];
    }
    return (int)kinds.size();
}

fcc_status fcc_dct_test_wait_timeout(fcc_plan* p, int enable) {
    if (!p) return fail(FCC_ERR_INVALID_ARG);
    if (!is_tc(p->dtype)) return fail(FCC_ERR_UNSUPPORTED);
    p->wait_test = enable != 0;
    return FCC_OK;
}

fcc_status fcc_dct_check(fcc_plan* p) {
    if (!p) return fail(FCC_ERR_INVALID_ARG);
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    fcc_status s = FCC_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        s = FCC_ERR_CUDA;
    } else if (*(volatile int*)p->h_status != 0) {
        *(volatile int*)p->h_status = 0;
        s = FCC_ERR_TIMEOUT;
    }
    if (cur != p->device) cudaSetDevice(cur);
    return s == FCC_OK ? FCC_OK : fail(s);
}

fcc_status fcc_dct_test_fail_alloc(int nth) {
    if (nth < 0) return fail(FCC_ERR_INVALID_ARG);
    g_fail_at = nth == 0 ? 0 : g_alloc_seq.load() + nth;
    return FCC_OK;
}

int64_t fcc_dct_test_allocations(int64_t* plans, int64_t* device_bytes) {
    if (plans) *plans = g_live_plans.load();
    if (device_bytes) *device_bytes = g_live_dev_bytes.load();
    return g_alloc_seq.load();
}

fcc_status fcc_dct_last_error(void) { return g_last; }

const char* fcc_status_string(fcc_status s) {
    switch (s) {
        case FCC_OK: return "ok";
        case FCC_ERR_INVALID_ARG: return "invalid argument";
        case FCC_ERR_UNSUPPORTED: return "unsupported";
        case FCC_ERR_ALLOC: return "allocation failed";
        case FCC_ERR_CUDA: return "CUDA error";
        case FCC_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

void fcc_dct_destroy(fcc_plan* p) { release(p); }

fcc_status fcc_dct_describe(int order, int64_t* n_orbits, int* n_classes, int* free_class, uint32_t* reps,
                            int32_t* cls, int32_t* wrap, int32_t* canon, double* fwd, double* inv,
                            double* adj) {
    static const int v0[3] = {1, 0, 3};
    return fcc_dct_describe_skew(order, v0, 8, nullptr, n_orbits, n_classes, free_class, reps, cls, wrap, canon, fwd,
                                 inv, adj);
}

fcc_status fcc_dct_describe_tiles(int order, int32_t* ntiles, int32_t* free_tiles, int32_t* tile_off,
                                  uint32_t* tile_reps) {
    static const int v0[3] = {1, 0, 3};
    HostPlan hp;
    const int rc = build_host_plan(order, hp, v0, 8);
    if (rc == -1) return fail(FCC_ERR_INVALID_ARG);
    if (rc != 0) return fail(FCC_ERR_UNSUPPORTED);
    const int nt = (int)hp.tile_off.size() - 1;
    if (ntiles) *ntiles = nt;
    if (free_tiles) *free_tiles = hp.free_tiles;
    if (tile_off)
        for (int t = 0; t <= nt; ++t) tile_off[t] = hp.tile_off[t];
    if (tile_reps)
        for (size_t o = 0; o < hp.tile_reps.size(); ++o) tile_reps[o] = hp.tile_reps[o];
    return FCC_OK;
}

fcc_status fcc_dct_describe_skew(int order, const int* v, int d, int* invertible, int64_t* n_orbits, int* n_classes,
                                 int* free_class, uint32_t* reps, int32_t* cls, int32_t* wrap, int32_t* canon,
                                 double* fwd, double* inv, double* adj) {
    if (!v) return fail(FCC_ERR_INVALID_ARG);
    HostPlan hp;
    const int rc = build_host_plan(order, hp, v, d);
    if (rc == -1) return fail(FCC_ERR_INVALID_ARG);
    if (rc != 0) return fail(FCC_ERR_UNSUPPORTED);
    if (invertible) *invertible = hp.invertible ? 1 : 0;
    if (n_orbits) *n_orbits = (int64_t)hp.reps.size();
    if (n_classes) *n_classes = (int)hp.classes.size();
    if (free_class) *free_class = hp.free_class;
    for (size_t o = 0; o < hp.reps.size(); ++o) {
        if (reps) reps[o] = hp.reps[o];
        if (cls) cls[o] = hp.cls[o];
    }
    for (size_t c = 0; c < hp.classes.size(); ++c) {
        const OrbitClass& oc = hp.classes[c];
        for (int h = 0; h < 24; ++h) {
            if (canon) canon[24 * c + h] = oc.canon[h];
            for (int i = 0; i < 3; ++i)
                if (wrap) wrap[72 * c + 3 * h + i] = oc.wrap[h][i];
        }
        for (int e = 0; e < 576; ++e) {
            if (fwd) { fwd[2 * (576 * c + e)] = oc.fwd[e].real(); fwd[2 * (576 * c + e) + 1] = oc.fwd[e].imag(); }
            if (inv) { inv[2 * (576 * c + e)] = oc.inv[e].real(); inv[2 * (576 * c + e) + 1] = oc.inv[e].imag(); }
            if (adj) { adj[2 * (576 * c + e)] = oc.adj[e].real(); adj[2 * (576 * c + e) + 1] = oc.adj[e].imag(); }
        }
    }
    return FCC_OK;
}

fcc_status fcc_dct_weyl_group(int32_t* out) {
    if (!out) return fail(FCC_ERR_INVALID_ARG);
    const WeylGroup& G = weyl();
    for (int g = 0; g < 24; ++g)
        for (int j = 0; j < 9; ++j) out[9 * g + j] = G.m[g][j];
    return FCC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// fcc_dct_inverse_static: the inverse with a file-scope workspace.
// ---------------------------------------------------------------------------

namespace {

// The workspace of fcc_dct_inverse_static.  In host code this name is only a
// stand-in for the symbol; kernels receive the device address obtained with
// cudaGetSymbolAddress below.
static __device__ __align__(256) float2 g_static_scratch[FCC_STATIC_SCRATCH_BYTES / sizeof(float2)];

constexpr int kMaxDevices = 64;
std::atomic<float2*> g_static_addr[kMaxDevices];

// Device address of g_static_scratch on the current device (looked up once).
fcc_status static_scratch(int dev, float2** ptr) {
    if (dev < 0 || dev >= kMaxDevices) return FCC_ERR_UNSUPPORTED;
    float2* p = g_static_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        void* addr = nullptr;
        if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess || !addr) {
            cudaGetLastError();
            return FCC_ERR_CUDA;
        }
        p = (float2*)addr;
        g_static_addr[dev].store(p, std::memory_order_release);
    }
    *ptr = p;
    return FCC_OK;
}

// One chunk (a pair of real volumes, or one volume) at a time through the
// static workspace, on the caller's stream only.
fcc_status run_inverse_static(fcc_plan* p, const float* in, float* out, float2* ws, cudaStream_t st) {
    const bool rin = is_real_in(p->dtype);
    fcc_status s = FCC_OK;
    int v = 0;
    while (v < p->batch && !s) {
        int e = v + 1;
        while (e < p->batch && p->orders[e] == p->orders[v]) ++e;
        const OrderTables& t = p->tabs.at(p->orders[v]);
        const int64_t n3 = (int64_t)t.n * t.n * t.n;
        const float* y = in + p->offset[v] * 2;
        float* x = out + p->offset[v] * (rin ? 1 : 2);
        const int64_t nvol = e - v;
        const float scale = (float)(1.0 / (double)n3);
        if (t.n == 1) {
            // D = [1]: copy through the workspace in chunks of whole volumes
            const int64_t cap = FCC_STATIC_SCRATCH_BYTES / sizeof(float2);
            for (int64_t u = 0; u < nvol && !s; u += cap) {
                const int64_t nv = std::min(cap, nvol - u);
                s = launch_fft<float>(t, y + 2 * u, (float*)ws, nv, 0, -1, st);
                if (!s) s = launch_mix<float>(t, MODE_INV, false, rin, (const float*)ws, x + u * (rin ? 1 : 2), nv, 1.f, st);
            }
            v = e;
            continue;
        }
        const int64_t npairs = (rin && nvol >= 2) ? nvol / 2 : 0;
        for (int64_t q = 0; q < npairs && !s; ++q) {
            // pair merge fused into the first DFT pass where the buffers allow
            s = merge_dft3_pairs(t, y + q * 4 * n3, (float*)ws, 1, st);
            if (!s) s = launch_mix_tiled(t, MODE_INV, false, true, (const float*)ws, x + q * 2 * n3, 1, scale, st, true);
        }
        for (int64_t u = 2 * npairs; u < nvol && !s; ++u) {
            s = launch_dft3(t, -1, y + u * 2 * n3, (float*)ws, 1, st);
            if (!s) s = launch_mix_tiled(t, MODE_INV, false, rin, (const float*)ws, x + u * n3 * (rin ? 1 : 2), 1,
                                         scale, st);
        }
        v = e;
    }
    return s;
}

}  // namespace

extern "C" fcc_status fcc_dct_inverse_static(fcc_plan* p, const void* in, void* out, void* stream) {
    if (!p || !in || !out) return fail(FCC_ERR_INVALID_ARG);
    // a device-side timeout recorded by an earlier call of the plan surfaces
    // here, as in every other entry point
    if (*(volatile int*)p->h_status != 0) {
        *(volatile int*)p->h_status = 0;
        return fail(FCC_ERR_TIMEOUT);
    }
    if (!aligned16(in) || !aligned16(out)) return fail(FCC_ERR_INVALID_ARG);
    const uintptr_t a0 = (uintptr_t)in, a1 = a0 + in_bytes(p, 1);
    const uintptr_t b0 = (uintptr_t)out, b1 = b0 + out_bytes(p, 1);
    if (a0 < b1 && b0 < a1) return fail(FCC_ERR_INVALID_ARG);
    if ((p->dtype != FCC_R32 && p->dtype != FCC_C32) || p->skew || p->r2) return fail(FCC_ERR_UNSUPPORTED);
    for (int n : p->orders)
        if ((uint64_t)n * n * n * sizeof(float2) > FCC_STATIC_SCRATCH_BYTES) return fail(FCC_ERR_UNSUPPORTED);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return fail(FCC_ERR_CUDA); }
    if (cur != p->device && cudaSetDevice(p->device) != cudaSuccess) { cudaGetLastError(); return fail(FCC_ERR_CUDA); }
    float2* ws = nullptr;
    fcc_status s = static_scratch(p->device, &ws);
    if (!s) s = run_inverse_static(p, (const float*)in, (float*)out, ws, (cudaStream_t)stream);
    if (cur != p->device) cudaSetDevice(cur);
    return s == FCC_OK ? FCC_OK : fail(s);
}
