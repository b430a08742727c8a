// The radix-2x2x2 recursion of Sec. 4.B on the GPU (see radix2.h).
#include "radix2.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <map>
#include <memory>
#include <unordered_map>
#include <vector>

#include "plan.h"

namespace fcc {

namespace {

using cd = std::complex<double>;
using K3 = std::array<int, 3>;
constexpr double kPi2 = 6.283185307179586476925286766559;

// Moves an integer weight into the dominant chamber with the printed simple
// reflections s1, s2, s3 (T_{wk} = T_k, Prop. 1 (iii)).
K3 dominant(K3 k) {
    for (;;) {
        if (k[0] < 0) k = {-k[0], k[0] + k[1], k[2]};
        else if (k[1] < 0) k = {k[0] + k[1], -k[1], k[1] + k[2]};
        else if (k[2] < 0) k = {k[0], k[1] + k[2], -k[2]};
        else return k;
    }
}

K3 wapply(int g, const K3& k) {
    const int* m = weyl().m[g];
    return {m[0] * k[0] + m[1] * k[1] + m[2] * k[2], m[3] * k[0] + m[4] * k[1] + m[5] * k[2],
            m[6] * k[0] + m[7] * k[1] + m[8] * k[2]};
}

// exp(2 pi i num / den) with the numerator reduced exactly
cd root(int64_t num, int64_t den) {
    const int64_t r = ((num % den) + den) % den;
    return std::polar(1.0, kPi2 * (double)r / (double)den);
}

// T_k at theta = (v + d i) / (den) for the integer point i: the power form
// (1/24) sum_w exp(2 pi i (w k) . theta) with exact integer phases.
cd chebyshev_at(const K3& k, const int num[3], int den) {
    cd s = 0;
    for (int g = 0; g < 24; ++g) {
        const K3 wk = wapply(g, k);
        s += root((int64_t)wk[0] * num[0] + (int64_t)wk[1] * num[1] + (int64_t)wk[2] * num[2], den);
    }
    return s / 24.0;
}

// Distinct images W e_j of the unit weights, e_j first.
std::array<std::vector<K3>, 3> unit_orbits() {
    std::array<std::vector<K3>, 3> out;
    for (int j = 0; j < 3; ++j) {
        K3 e = {0, 0, 0};
        e[j] = 1;
        out[j].push_back(e);
        for (int g = 0; g < 24; ++g) {
            const K3 u = wapply(g, e);
            if (std::find(out[j].begin(), out[j].end(), u) == out[j].end()) out[j].push_back(u);
        }
    }
    return out;
}

using Sparse = std::vector<std::pair<int, cd>>;   // (box index, coefficient)

// T_k for a dominant k of any size as a combination of the basis b_n
// (indices in the box [0, n)^3), reducing with the ideal
// T_{n e_j} = sigma_j: from T_{n e_j} T_low = (1/|W e_j|) sum_{u in W e_j} T_{low + n u}
// (mother recurrence), the u whose dominant image is k itself is solved for;
// every other term is lower in dominance order.
struct Reducer {
    int n;
    cd sigma[3];
    std::array<std::vector<K3>, 3> orb;
    std::map<K3, Sparse> memo;

    const Sparse& red(const K3& k) {
        auto it = memo.find(k);
        if (it != memo.end()) return it->second;
        Sparse out;
        if (k[0] < n && k[1] < n && k[2] < n) {
            out.push_back({(k[0] * n + k[1]) * n + k[2], cd(1.0)});
        } else {
            const int j = k[0] >= n ? 0 : k[1] >= n ? 1 : 2;
            K3 low = k;
            low[j] -= n;
            std::unordered_map<int, cd> acc;
            const double osz = (double)orb[j].size();
            {
                const Sparse lo = red(low);   // copy: red() may grow the memo
                for (const auto& kv : lo) acc[kv.first] += osz * sigma[j] * kv.second;
            }
            int same = 0;
            for (const K3& u : orb[j]) {
                const K3 t = dominant({low[0] + n * u[0], low[1] + n * u[1], low[2] + n * u[2]});
                if (t == k) {
                    ++same;
                    continue;
                }
                const Sparse tt = red(t);
                for (const auto& kv : tt) acc[kv.first] -= kv.second;
            }
            for (const auto& kv : acc)
                if (kv.second != cd(0.0)) out.push_back({kv.first, kv.second / (double)same});
            std::sort(out.begin(), out.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        }
        return memo.emplace(k, std::move(out)).first->second;
    }
};

// B_n^{-1}(c), dense row-major N x N: column (efg, abc) = b_n coordinates of
// T_{abc} T_{m(e,f,g)} = (1/24) sum_w T_{(a,b,c) + w m(e,f,g)}.
std::vector<cd> basis_change_inverse(int n, const int v[3], int d) {
    const int m = n / 2, N = n * n * n, M = m * m * m;
    Reducer R;
    R.n = n;
    R.orb = unit_orbits();
    for (int j = 0; j < 3; ++j) {
        K3 e = {0, 0, 0};
        e[j] = 1;
        R.sigma[j] = chebyshev_at(e, v, d);
    }
    std::vector<cd> out((size_t)N * N, cd(0.0));
    for (int efg = 0; efg < 8; ++efg) {
        const K3 l = {m * (efg >> 2), m * ((efg >> 1) & 1), m * (efg & 1)};
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b)
                for (int c = 0; c < m; ++c) {
                    const int col = efg * M + (a * m + b) * m + c;
                    for (int g = 0; g < 24; ++g) {
                        const K3 wl = wapply(g, l);
                        const Sparse& s = R.red(dominant({a + wl[0], b + wl[1], c + wl[2]}));
                        for (const auto& kv : s) out[(size_t)kv.first * N + col] += kv.second / 24.0;
                    }
                }
    }
    return out;
}

// D_2(c): 8 x 8, row = point i in {0,1}^3, column = coefficient j in
// {0,1}^3, T_j((c + i)/2) (Def. 2 at order 2), lexicographic.
std::vector<cd> dct2(const int v[3], int d) {
    std::vector<cd> out(64);
    for (int i = 0; i < 8; ++i) {
        const int num[3] = {v[0] + d * (i >> 2), v[1] + d * ((i >> 1) & 1), v[2] + d * (i & 1)};
        for (int j = 0; j < 8; ++j) out[i * 8 + j] = chebyshev_at({j >> 2, (j >> 1) & 1, j & 1}, num, 2 * d);
    }
    return out;
}

// ---- device: Gauss-Jordan inversion (FP64, partial pivoting) --------------

// argmax over rows r >= k of |A[r][k]|^2 (one block)
__global__ void gj_pivot(const double2* A, int N, int k, int* piv) {
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    double best = -1.0;
    int arg = k;
    for (int r = k + threadIdx.x; r < N; r += blockDim.x) {
        const double2 a = A[(size_t)r * N + k];
        const double m = a.x * a.x + a.y * a.y;
        if (m > best) { best = m; arg = r; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = arg;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s && bv[threadIdx.x + s] > bv[threadIdx.x]) {
            bv[threadIdx.x] = bv[threadIdx.x + s];
            bi[threadIdx.x] = bi[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) piv[0] = bi[0];
}

// swap rows k and piv of A and I; then the reciprocal of the pivot
__global__ void gj_swap(double2* A, double2* I, int N, int k, const int* piv) {
    const int p = piv[0];
    if (p == k) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 2 * N; c += gridDim.x * blockDim.x) {
        double2* M = c < N ? A : I;
        const int cc = c < N ? c : c - N;
        const double2 t = M[(size_t)k * N + cc];
        M[(size_t)k * N + cc] = M[(size_t)p * N + cc];
        M[(size_t)p * N + cc] = t;
    }
}

__global__ void gj_recip(const double2* A, int N, int k, double2* pinv, int* status) {
    const double2 a = A[(size_t)k * N + k];
    const double m = a.x * a.x + a.y * a.y;
    if (!(m > 1e-200)) {
        status[0] = 1;
        pinv[0] = make_double2(0.0, 0.0);
    } else {
        pinv[0] = make_double2(a.x / m, -a.y / m);
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// row k of A and I times the reciprocal pivot; column k of A saved in f
__global__ void gj_scale(double2* A, double2* I, int N, int k, const double2* pinv, double2* f) {
    const double2 s = pinv[0];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 2 * N; c += gridDim.x * blockDim.x) {
        if (c < N) {
            f[c] = A[(size_t)c * N + k];   // column k (row c), read before any elimination
            A[(size_t)k * N + c] = cmul(A[(size_t)k * N + c], s);
        } else {
            I[(size_t)k * N + (c - N)] = cmul(I[(size_t)k * N + (c - N)], s);
        }
    }
}

// rows r != k: row_r -= f[r] row_k (A: columns >= k, I: all)
__global__ void gj_elim(double2* A, double2* I, int N, int k, const double2* f) {
    const int r = blockIdx.y;
    if (r == k) return;
    const double2 fr = f[r];
    if (fr.x == 0.0 && fr.y == 0.0) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < 2 * N; c += gridDim.x * blockDim.x) {
        if (c < N) {
            if (c < k) continue;
            const double2 t = cmul(fr, A[(size_t)k * N + c]);
            double2& x = A[(size_t)r * N + c];
            x.x -= t.x;
            x.y -= t.y;
        } else {
            const double2 t = cmul(fr, I[(size_t)k * N + (c - N)]);
            double2& x = I[(size_t)r * N + (c - N)];
            x.x -= t.x;
            x.y -= t.y;
        }
    }
}

__global__ void to_float2(const double2* a, float2* b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// ---- device: the recursion ---------------------------------------------------

template <typename T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

template <typename T>
struct Mat8 { typename C2<T>::t a[64]; };

template <typename V>
__device__ __forceinline__ V cfma(V acc, V a, V b) {
    acc.x += a.x * b.x - a.y * b.y;
    acc.y += a.x * b.y + a.y * b.x;
    return acc;
}

// Y[b][r] = sum_c B[r][c] X[b][c]: one warp per row, grid.y = batch
template <typename T>
__global__ void r2_matvec(const typename C2<T>::t* __restrict__ B, int N, const typename C2<T>::t* __restrict__ X,
                          int64_t xs, typename C2<T>::t* __restrict__ Y, int64_t ys) {
    using V = typename C2<T>::t;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (r >= N) return;
    const V* x = X + blockIdx.y * xs;
    V acc = {0, 0};
    for (int c = lane; c < N; c += 32) acc = cfma(acc, B[(size_t)r * N + c], x[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) Y[blockIdx.y * ys + r] = acc;
}

// (D_2 (x) 1_M): U[b][i M + k] = sum_e D2[i][e] X[b][e M + k]; one thread per (b, k)
template <typename T>
__global__ void r2_butterfly(const Mat8<T> D, int M, const typename C2<T>::t* __restrict__ X, int64_t xs,
                             typename C2<T>::t* __restrict__ U, int64_t us) {
    using V = typename C2<T>::t;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const V* x = X + blockIdx.y * xs;
    V in[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) in[e] = x[e * M + k];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        V acc = {0, 0};
#pragma unroll
        for (int e = 0; e < 8; ++e) acc = cfma(acc, D.a[i * 8 + e], in[e]);
        U[blockIdx.y * us + i * M + k] = acc;
    }
}

// the 8-point base transform D_2 of each of `batch` vectors
template <typename T>
__global__ void r2_base(const Mat8<T> D, const typename C2<T>::t* __restrict__ X, int64_t xs,
                        typename C2<T>::t* __restrict__ Y, int64_t ys, int batch) {
    using V = typename C2<T>::t;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= batch * 8) return;
    const int b = t >> 3, i = t & 7;
    V acc = {0, 0};
#pragma unroll
    for (int j = 0; j < 8; ++j) acc = cfma(acc, D.a[i * 8 + j], X[b * xs + j]);
    Y[b * ys + i] = acc;
}

// P_n: row (i, k) of the stacked sub-transforms -> grid point i + 2k
template <typename T>
__global__ void r2_scatter(int n, const typename C2<T>::t* __restrict__ Yc, int64_t cs,
                           typename C2<T>::t* __restrict__ Y, int64_t ys) {
    const int m = n / 2, M = m * m * m;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * M) return;
    const int i = t / M, k = t % M;
    const int k0 = k / (m * m), k1 = (k / m) % m, k2 = k % m;
    const int p = ((((i >> 2) + 2 * k0) * n) + (((i >> 1) & 1) + 2 * k1)) * n + ((i & 1) + 2 * k2);
    Y[blockIdx.y * ys + p] = Yc[blockIdx.y * cs + t];
}

}  // namespace

// One node of the recursion: D_n at the shift v / d.
struct R2Node {
    int n = 0;
    int v[3] = {0, 0, 0};
    int d = 1;
    void* B = nullptr;                 // B_n(c), N x N, double2 or float2 (n >= 4)
    std::vector<cd> d2;                // D_2(c), 8 x 8
    int child[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    double nnz_row = 0, max_abs = 0;   // of B_n
};

struct R2Plan {
    int n = 0, batch = 0;
    bool fp64 = true;
    std::vector<R2Node> nodes;         // nodes[0] is the whole transform
    // per order k >= 4: Xt, U, Yc buffers of batch * k^3 complex values
    std::map<int, std::array<void*, 3>> bufs;
    int launches = 0;
    double macs = 0;                   // complex multiply-adds of one transform
};

namespace {

template <typename T>
Mat8<T> mat8(const std::vector<cd>& m) {
    Mat8<T> out;
    for (int i = 0; i < 64; ++i) out.a[i] = {(T)m[i].real(), (T)m[i].imag()};
    return out;
}

// B_n = (B_n^{-1})^{-1} into dst (FP64) with Gauss-Jordan on the device;
// A, f, scalars: scratch.  Returns FCC_ERR_UNSUPPORTED when singular.
fcc_status invert_on_device(const std::vector<cd>& binv, int N, double2* dst, double2* A, double2* f, double2* pinv,
                            int* piv, int* status) {
    if (cudaMemcpy(A, binv.data(), (size_t)N * N * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess)
        return FCC_ERR_CUDA;
    std::vector<cd> eye((size_t)N * N, cd(0.0));
    for (int i = 0; i < N; ++i) eye[(size_t)i * N + i] = 1.0;
    if (cudaMemcpy(dst, eye.data(), (size_t)N * N * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(status, 0, sizeof(int)) != cudaSuccess)
        return FCC_ERR_CUDA;
    const int tb = 256, gb = std::max(1, std::min(1024, (2 * N + tb - 1) / tb));
    for (int k = 0; k < N; ++k) {
        gj_pivot<<<1, 1024>>>(A, N, k, piv);
        gj_swap<<<gb, tb>>>(A, dst, N, k, piv);
        gj_recip<<<1, 1>>>(A, N, k, pinv, status);
        gj_scale<<<gb, tb>>>(A, dst, N, k, pinv, f);
        gj_elim<<<dim3((unsigned)gb, (unsigned)N), tb>>>(A, dst, N, k, f);
    }
    int bad = 0;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&bad, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FCC_ERR_CUDA;
    return bad ? FCC_ERR_UNSUPPORTED : FCC_OK;
}

int add_node(R2Plan& r, int n, const int v[3], int d) {
    const int id = (int)r.nodes.size();
    r.nodes.emplace_back();
    R2Node& nd = r.nodes.back();
    nd.n = n;
    for (int i = 0; i < 3; ++i) nd.v[i] = v[i];
    nd.d = d;
    nd.d2 = dct2(v, d);
    if (n >= 4)
        for (int i = 0; i < 8; ++i) {
            const int vi[3] = {v[0] + d * (i >> 2), v[1] + d * ((i >> 1) & 1), v[2] + d * (i & 1)};
            const int c = add_node(r, n / 2, vi, 2 * d);   // (c + i) / 2
            r.nodes[id].child[i] = c;
        }
    return id;
}

template <typename T>
void forward_node(const R2Plan& r, int id, const void* X, int64_t xs, void* Y, int64_t ys, cudaStream_t st, int& launches) {
    using V = typename C2<T>::t;
    const R2Node& nd = r.nodes[id];
    const Mat8<T> D = mat8<T>(nd.d2);
    if (nd.n == 2) {
        const int t = r.batch * 8;
        r2_base<T><<<(t + 255) / 256, 256, 0, st>>>(D, (const V*)X, xs, (V*)Y, ys, r.batch);
        ++launches;
        return;
    }
    const int n = nd.n, N = n * n * n, M = N / 8;
    const auto& b = r.bufs.at(n);
    V* Xt = (V*)b[0];
    V* U = (V*)b[1];
    V* Yc = (V*)b[2];
    r2_matvec<T><<<dim3((unsigned)((N + 7) / 8), (unsigned)r.batch), 256, 0, st>>>((const V*)nd.B, N, (const V*)X, xs, Xt, N);
    r2_butterfly<T><<<dim3((unsigned)((M + 255) / 256), (unsigned)r.batch), 256, 0, st>>>(D, M, Xt, N, U, N);
    launches += 2;
    for (int i = 0; i < 8; ++i) forward_node<T>(r, nd.child[i], U + i * M, N, Yc + i * M, N, st, launches);
    r2_scatter<T><<<dim3((unsigned)((N + 255) / 256), (unsigned)r.batch), 256, 0, st>>>(n, Yc, N, (V*)Y, ys);
    ++launches;
}

}  // namespace

R2Plan* r2_build(int n, int batch, bool fp64, const int v[3], int d, R2Alloc alloc, void* ctx, fcc_status* st) {
    *st = FCC_OK;
    if (!(n == 2 || n == 4 || n == 8 || n == 16) || batch < 1 || batch > 65535 || d < 1) {
        *st = FCC_ERR_INVALID_ARG;
        return nullptr;
    }
    std::unique_ptr<R2Plan> r(new (std::nothrow) R2Plan());
    if (!r) { *st = FCC_ERR_ALLOC; return nullptr; }
    r->n = n;
    r->batch = batch;
    r->fp64 = fp64;
    add_node(*r, n, v, d);
    const size_t es = fp64 ? sizeof(double2) : sizeof(float2);
    // scratch of the inversion (the largest B_n^{-1} and its pivot column)
    const int Nmax = n >= 4 ? n * n * n : 0;
    double2 *A = nullptr, *f = nullptr, *sc = nullptr;
    if (Nmax > 0) {
        fcc_status s = alloc(ctx, (void**)&A, (size_t)Nmax * Nmax * sizeof(double2));
        if (!s) s = alloc(ctx, (void**)&f, (size_t)Nmax * sizeof(double2));
        if (!s) s = alloc(ctx, (void**)&sc, 4 * sizeof(double2));
        if (s) { *st = s; return nullptr; }
    }
    std::vector<double2> host;
    for (R2Node& nd : r->nodes) {
        if (nd.n < 4) {
            r->macs += 64;
            continue;
        }
        const int N = nd.n * nd.n * nd.n;
        double2* b64 = nullptr;
        fcc_status s = alloc(ctx, (void**)&b64, (size_t)N * N * sizeof(double2));
        if (!s) s = invert_on_device(basis_change_inverse(nd.n, nd.v, nd.d), N, b64, A, f, sc, (int*)(sc + 2), (int*)(sc + 3));
        if (s) { *st = s; return nullptr; }
        // statistics of B_n (the paper's cost claim: O(1) entries per row)
        host.resize((size_t)N * N);
        if (cudaMemcpy(host.data(), b64, host.size() * sizeof(double2), cudaMemcpyDeviceToHost) != cudaSuccess) {
            *st = FCC_ERR_CUDA;
            return nullptr;
        }
        double mx = 0;
        for (const double2& z : host) mx = std::max(mx, std::hypot(z.x, z.y));
        int64_t nnz = 0;
        for (const double2& z : host) nnz += std::hypot(z.x, z.y) > 1e-12 * mx ? 1 : 0;
        nd.nnz_row = (double)nnz / N;
        nd.max_abs = mx;
        r->macs += (double)nnz + 64.0 * (N / 8);
        if (fp64) {
            nd.B = b64;
        } else {
            float2* b32 = nullptr;
            if ((s = alloc(ctx, (void**)&b32, (size_t)N * N * sizeof(float2)))) { *st = s; return nullptr; }
            to_float2<<<1024, 256>>>(b64, b32, (size_t)N * N);
            nd.B = b32;
        }
        if (!r->bufs.count(nd.n)) {
            std::array<void*, 3> b = {nullptr, nullptr, nullptr};
            for (int i = 0; i < 3 && !s; ++i) s = alloc(ctx, &b[i], (size_t)batch * N * es);
            if (s) { *st = s; return nullptr; }
            r->bufs[nd.n] = b;
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) { cudaGetLastError(); *st = FCC_ERR_CUDA; return nullptr; }
    int launches = 0;
    // count the launches of one forward (the recursion's shape does not depend on the data)
    std::vector<int> stack = {0};
    while (!stack.empty()) {
        const int id = stack.back();
        stack.pop_back();
        if (r->nodes[id].n == 2) { ++launches; continue; }
        launches += 3;
        for (int i = 0; i < 8; ++i) stack.push_back(r->nodes[id].child[i]);
    }
    r->launches = launches;
    return r.release();
}

void r2_destroy(R2Plan* r) { delete r; }   // device memory belongs to the owning plan

fcc_status r2_forward(R2Plan* r, const void* in, void* out, cudaStream_t stream) {
    const int64_t N = (int64_t)r->n * r->n * r->n;
    int launches = 0;
    if (r->fp64) forward_node<double>(*r, 0, in, N, out, N, stream, launches);
    else forward_node<float>(*r, 0, in, N, out, N, stream, launches);
    return cudaGetLastError() == cudaSuccess ? FCC_OK : FCC_ERR_CUDA;
}

int r2_launches(const R2Plan* r) { return r ? r->launches : 0; }

int r2_stats(const R2Plan* r, int k, double* nnz_per_row, double* max_abs, double* macs_per_point) {
    if (!r) return -1;
    if (k == 0) {
        if (macs_per_point) *macs_per_point = r->macs / ((double)r->n * r->n * r->n);
        return 0;
    }
    double nz = 0, mx = 0;
    int cnt = 0;
    for (const R2Node& nd : r->nodes)
        if (nd.n == k && nd.n >= 4) {
            nz += nd.nnz_row;
            mx = std::max(mx, nd.max_abs);
            ++cnt;
        }
    if (!cnt) return -1;
    if (nnz_per_row) *nnz_per_row = nz / cnt;
    if (max_abs) *max_abs = mx;
    return cnt;
}

}  // namespace fcc
