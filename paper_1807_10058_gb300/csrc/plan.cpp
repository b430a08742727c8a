// Host-side plan builder: W, orbit partition of Z_n^3, class cores.
// See plan.h for the factorisation it implements.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

namespace fcc {

namespace {

// Generators of Sec. 3 (row-major).
const int kGen[3][9] = {
    {-1, 0, 0, 1, 1, 0, 0, 0, 1},
    {1, 1, 0, 0, -1, 0, 0, 1, 1},
    {1, 0, 0, 0, 1, 1, 0, 0, -1},
};
const int kV[3] = {1, 0, 3};  // 8 * (1/8, 0, 3/8)

void mat3(const int* a, const int* b, int* c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int s = 0;
            for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
}

WeylGroup make_weyl() {
    WeylGroup G{};
    std::vector<std::array<int, 9>> els;
    els.push_back({1, 0, 0, 0, 1, 0, 0, 0, 1});
    for (size_t head = 0; head < els.size(); ++head)
        for (int g = 0; g < 3; ++g) {
            std::array<int, 9> c;
            mat3(kGen[g], els[head].data(), c.data());
            if (std::find(els.begin(), els.end(), c) == els.end()) els.push_back(c);
        }
    // |W| = 24 for the printed generators; anything else is a build error.
    if (els.size() != 24) std::abort();
    for (int a = 0; a < 24; ++a) std::memcpy(G.m[a], els[a].data(), sizeof(G.m[a]));
    auto find = [&](const int* c) {
        for (int j = 0; j < 24; ++j)
            if (std::memcmp(c, G.m[j], sizeof(int) * 9) == 0) return j;
        std::abort();
    };
    for (int a = 0; a < 24; ++a)
        for (int b = 0; b < 24; ++b) {
            int c[9];
            mat3(G.m[a], G.m[b], c);
            G.mul[a][b] = find(c);
        }
    for (int a = 0; a < 24; ++a)
        for (int b = 0; b < 24; ++b)
            if (G.mul[a][b] == 0) G.inv[a] = b;
    for (int g = 0; g < 24; ++g)
        for (int j = 0; j < 3; ++j) {
            int s = 0;
            for (int i = 0; i < 3; ++i) s += G.m[g][3 * i + j] * kV[i];
            G.u[g][j] = s;
        }
    return G;
}

// exact 8th roots of unity w_8^e
cd root8(int e);

// w_d^e: exact when e / d in lowest terms has a denominator dividing 8,
// else from the reduced angle
cd root_d(int64_t e, int d) {
    e = ((e % d) + d) % d;
    const int64_t g = std::gcd(e, (int64_t)d);
    const int64_t dr = d / g;
    if (8 % dr == 0) return root8((int)((e / g) * (8 / dr)));
    return std::polar(1.0, 2.0 * M_PI * (double)e / (double)d);
}

cd root8(int e) {
    e = ((e % 8) + 8) % 8;
    const double h = std::sqrt(0.5);
    static const double re[8] = {1, 0, 0, 0, -1, 0, 0, 0};
    static const double im[8] = {0, 0, 1, 0, 0, 0, -1, 0};
    if (e % 2 == 0) return cd(re[e], im[e]);
    const double sr = (e == 1 || e == 7) ? h : -h;
    const double si = (e == 1 || e == 3) ? h : -h;
    return cd(sr, si);
}

// Gauss-Jordan inverse with partial pivoting; returns false if singular.
bool invert(std::vector<cd>& a, int s) {
    std::vector<cd> inv(s * s, cd(0));
    for (int i = 0; i < s; ++i) inv[i * s + i] = 1;
    for (int c = 0; c < s; ++c) {
        int p = c;
        for (int r = c + 1; r < s; ++r)
            if (std::abs(a[r * s + c]) > std::abs(a[p * s + c])) p = r;
        if (std::abs(a[p * s + c]) < 1e-12) return false;
        if (p != c)
            for (int j = 0; j < s; ++j) {
                std::swap(a[p * s + j], a[c * s + j]);
                std::swap(inv[p * s + j], inv[c * s + j]);
            }
        cd d = cd(1) / a[c * s + c];
        for (int j = 0; j < s; ++j) {
            a[c * s + j] *= d;
            inv[c * s + j] *= d;
        }
        for (int r = 0; r < s; ++r)
            if (r != c && a[r * s + c] != cd(0)) {
                cd f = a[r * s + c];
                for (int j = 0; j < s; ++j) {
                    a[r * s + j] -= f * a[c * s + j];
                    inv[r * s + j] -= f * inv[c * s + j];
                }
            }
    }
    a.swap(inv);
    return true;
}

using ClassKey = std::array<int8_t, 24 * 4>;

}  // namespace

const WeylGroup& weyl() {
    static const WeylGroup G = make_weyl();
    return G;
}

std::vector<int> fft_radices(int n) {
    std::vector<int> r;
    while (n % 4 == 0) { r.push_back(4); n /= 4; }
    while (n % 2 == 0) { r.push_back(2); n /= 2; }
    for (int p : {3, 5, 7, 11, 13}) {
        while (n % p == 0) { r.push_back(p); n /= p; }
    }
    if (n > 1) r.push_back(n);  // larger prime: generic radix
    return r;
}

int build_host_plan(int n, HostPlan& P, const int* v, int d) {
    if (n < 1 || n > kMaxOrder) return -1;
    if (!v) { v = kV; d = 8; }
    if (d < 1 || d > kMaxShiftDen) return -1;
    for (int i = 0; i < 3; ++i)
        if (v[i] < -kMaxShiftNum || v[i] > kMaxShiftNum) return -1;
    const WeylGroup& G = weyl();
    P = HostPlan();
    P.n = n;
    P.d = d;
    for (int i = 0; i < 3; ++i) P.v[i] = v[i];
    for (int g = 0; g < 24; ++g)
        for (int j = 0; j < 3; ++j) {
            int acc = 0;
            for (int i = 0; i < 3; ++i) acc += G.m[g][3 * i + j] * v[i];
            P.u[g][j] = acc;
        }
    P.points = (int64_t)n * n * n;
    std::vector<uint8_t> seen(P.points, 0);
    std::map<ClassKey, int> key2cls;
    std::vector<uint32_t> reps;
    std::vector<int> cls;
    int64_t covered = 0;

    for (int k1 = 0; k1 <= n; ++k1)
        for (int k2 = 0; k1 + k2 <= n; ++k2)
            for (int k3 = 0; k1 + k2 + k3 <= n; ++k3) {
                const int k[3] = {k1, k2, k3};
                int64_t flat[24];
                ClassKey key;
                int8_t canon[24];
                for (int h = 0; h < 24; ++h) {
                    int kap[3];
                    for (int i = 0; i < 3; ++i) {
                        const int p = G.m[h][3 * i] * k[0] + G.m[h][3 * i + 1] * k[1] + G.m[h][3 * i + 2] * k[2];
                        kap[i] = ((p % n) + n) % n;
                        key[3 * h + i] = (int8_t)((p - kap[i]) / n);
                    }
                    flat[h] = ((int64_t)kap[0] * n + kap[1]) * n + kap[2];
                    canon[h] = (int8_t)h;
                    for (int j = 0; j < h; ++j)
                        if (flat[j] == flat[h]) { canon[h] = canon[j]; break; }
                    key[72 + h] = canon[h];
                }
                if (seen[flat[0]]) continue;  // orbit already has a representative
                for (int h = 0; h < 24; ++h)
                    if (canon[h] == h) {
                        if (seen[flat[h]]) return -2;
                        seen[flat[h]] = 1;
                        ++covered;
                    }
                auto it = key2cls.find(key);
                int c;
                if (it == key2cls.end()) {
                    c = (int)P.classes.size();
                    key2cls[key] = c;
                    OrbitClass oc{};
                    std::memcpy(oc.wrap, key.data(), 72);
                    std::memcpy(oc.canon, canon, 24);
                    P.classes.push_back(oc);
                } else {
                    c = it->second;
                }
                const bool interior = k1 > 0 && k2 > 0 && k3 > 0 && k1 + k2 + k3 < n;
                bool all_distinct = true;
                for (int h = 0; h < 24; ++h) all_distinct &= canon[h] == h;
                if (interior && all_distinct) {
                    if (P.free_class < 0) P.free_class = c;
                    else if (P.free_class != c) return -2;  // the free core must be universal
                }
                reps.push_back((uint32_t)k1 | ((uint32_t)k2 << 10) | ((uint32_t)k3 << 20));
                cls.push_back(c);
            }
    if (covered != P.points) return -2;
    if (P.classes.size() > 255) return -2;

    // Class cores.
    for (auto& oc : P.classes) {
        int s = 0;
        oc.canon_mask = 0;
        for (int h = 0; h < 24; ++h)
            if (oc.canon[h] == h) {
                oc.dist[h] = (int8_t)s++;
                oc.canon_mask |= 1u << h;
            }
        for (int h = 0; h < 24; ++h) oc.dist[h] = oc.dist[oc.canon[h]];
        oc.distinct = s;
        oc.fwd.assign(576, cd(0));
        for (int g = 0; g < 24; ++g)
            for (int h = 0; h < 24; ++h) {
                const int w = G.mul[g][G.inv[h]];
                int64_t t = 0;
                for (int i = 0; i < 3; ++i) {
                    const int wm = G.m[w][3 * i] * oc.wrap[h][0] + G.m[w][3 * i + 1] * oc.wrap[h][1] +
                                   G.m[w][3 * i + 2] * oc.wrap[h][2];
                    t += (int64_t)wm * v[i];
                }
                oc.fwd[g * 24 + h] = root_d(-t, d) / 24.0;
            }
        // distinct-member block B (s x s): rows at canonical slots, columns
        // summed over slots holding the same member
        std::vector<cd> B(s * s, cd(0));
        for (int g = 0; g < 24; ++g) {
            if (oc.canon[g] != g) continue;
            for (int h = 0; h < 24; ++h) B[oc.dist[g] * s + oc.dist[h]] += oc.fwd[g * 24 + h];
        }
        std::vector<cd> Binv = B;
        const bool inv_ok = invert(Binv, s);
        P.invertible = P.invertible && inv_ok;
        oc.inv.assign(576, cd(0));
        oc.adj.assign(576, cd(0));
        for (int h = 0; h < 24; ++h)
            for (int g = 0; g < 24; ++g) {
                if (oc.canon[g] != g) continue;
                if (inv_ok) oc.inv[h * 24 + g] = Binv[oc.dist[h] * s + oc.dist[g]];
                oc.adj[h * 24 + g] = std::conj(B[oc.dist[g] * s + oc.dist[h]]);
            }
    }

    // Sort orbits by class (free class first), stable in enumeration order.
    const int ncls = (int)P.classes.size();
    std::vector<int> rank(ncls);
    {
        std::vector<int> order(ncls);
        for (int c = 0; c < ncls; ++c) order[c] = c;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (a == P.free_class) > (b == P.free_class);
        });
        // renumber classes so that class index == rank
        std::vector<OrbitClass> sorted(ncls);
        for (int r = 0; r < ncls; ++r) {
            rank[order[r]] = r;
            sorted[r] = P.classes[order[r]];
        }
        P.classes.swap(sorted);
        if (P.free_class >= 0) P.free_class = rank[P.free_class];
    }
    P.class_begin.assign(ncls, 0);
    P.class_count.assign(ncls, 0);
    for (int c : cls) P.class_count[rank[c]]++;
    for (int c = 1; c < ncls; ++c) P.class_begin[c] = P.class_begin[c - 1] + P.class_count[c - 1];
    std::vector<int64_t> pos = P.class_begin;
    P.reps.resize(reps.size());
    P.cls.resize(reps.size());
    for (size_t o = 0; o < reps.size(); ++o) {
        const int r = rank[cls[o]];
        const int64_t at = pos[r]++;
        P.reps[at] = reps[o];
        P.cls[at] = (uint8_t)r;
    }
    for (int c = 0; c < ncls; ++c) P.orbits_per_class_max = std::max(P.orbits_per_class_max, P.class_count[c]);

    // Tiles.
    struct Item { int64_t key; int a, b, c; uint32_t rep; uint8_t cls; int64_t local = 0; };
    std::vector<Item> items(P.reps.size());
    for (size_t o = 0; o < P.reps.size(); ++o) {
        const int k1 = P.reps[o] & 1023, k2 = (P.reps[o] >> 10) & 1023, k3 = (P.reps[o] >> 20) & 1023;
        const int a = k1 + k2 + k3, b = k1 + k2, c = k1;
        // super-box first so that consecutive tiles (one block) are neighbours
        const int64_t sk = ((int64_t)(a / kSuperA) * (n / kSuperB + 1) + b / kSuperB) * (n / kSuperC + 1) + c / kSuperC;
        const int sub = (((a % kSuperA) / kTileA) * (kSuperB / kTileB) + (b % kSuperB) / kTileB) * (kSuperC / kTileC) +
                        (c % kSuperC) / kTileC;
        // class-pure tiles: the free class first (boxes), then each boundary
        // class packed in runs of kTileMax along (a', b', c') (boundary orbits
        // lie on faces of the alcove, where boxes would be mostly empty)
        const int64_t crank = (P.cls[o] == (uint8_t)P.free_class) ? 0 : 1 + P.cls[o];
        const int64_t nsk = (int64_t)(n / kSuperA + 1) * (n / kSuperB + 1) * (n / kSuperC + 1);
        int64_t tk = (crank * nsk + sk) * 64 + sub;
        if (crank > 0) tk = (crank * nsk) * 64;   // one key per class; split into runs below
        // a' fastest inside the tile
        int64_t local = ((int64_t)(c % kTileC) * kTileB + b % kTileB) * kTileA + a % kTileA;
        // order inside a boundary class: by 4 x 4 x 4 boxes of (a', b', c'),
        // then lexicographic, so that a run of kTileMax is a compact patch of
        // the alcove face (or edge) the class lies on rather than a line
        // (CPU sector count at n = 128: 18 % fewer sectors per gathered value)
        if (crank > 0) {
            const int64_t m = n / 4 + 1, l = n + 1;
            const int64_t box = ((int64_t)(a / 4) * m + b / 4) * m + c / 4;
            local = box * l * l * l + ((int64_t)a * l + b) * l + c;
        }
        items[o] = {tk, a, b, c, P.reps[o], P.cls[o]};
        items[o].local = local;
    }
    std::sort(items.begin(), items.end(),
              [](const Item& x, const Item& y) { return x.key != y.key ? x.key < y.key : x.local < y.local; });
    // free class: a box of the tiling that the open alcove cuts (fewer than
    // kTileMax orbits) gives up its own tile; the orbits of such boxes, in box
    // order, fill tiles of kTileMax (full boxes stay tiles, so the tile order
    // stays a walk through neighbouring boxes).  Lanes of the kernels' warps
    // and rows of the tensor-core blocks then carry orbits instead of idling:
    // at n = 128 a fifth of the tiles go, at n = 32 over half, for the same
    // sectors per gathered value.
    {
        size_t nfree = 0;
        while (nfree < items.size() && items[nfree].cls == (uint8_t)P.free_class) ++nfree;
        std::vector<Item> out;
        out.reserve(nfree);
        std::vector<Item> pending;
        int64_t key = 0;
        auto emit = [&](std::vector<Item>& v, size_t cnt) {
            for (size_t t = 0; t < cnt; ++t) {
                v[t].key = key;
                v[t].local = (int64_t)t;
                out.push_back(v[t]);
            }
            v.erase(v.begin(), v.begin() + (std::ptrdiff_t)cnt);
            ++key;
        };
        size_t i0 = 0;
        while (i0 < nfree) {
            size_t e = i0;
            while (e < nfree && items[e].key == items[i0].key) ++e;
            std::vector<Item> box(items.begin() + (std::ptrdiff_t)i0, items.begin() + (std::ptrdiff_t)e);
            if (box.size() == (size_t)kTileMax) {
                emit(box, box.size());
            } else {
                pending.insert(pending.end(), box.begin(), box.end());
                while (pending.size() >= (size_t)kTileMax) emit(pending, (size_t)kTileMax);
            }
            i0 = e;
        }
        if (!pending.empty()) emit(pending, pending.size());
        std::copy(out.begin(), out.end(), items.begin());   // same orbits, keys 0.. in tile order
    }
    // boundary classes: consecutive runs of kTileMax orbits become tiles
    {
        size_t i0 = 0;
        while (i0 < items.size()) {
            size_t e = i0;
            while (e < items.size() && items[e].key == items[i0].key) ++e;
            if (items[i0].cls != (uint8_t)P.free_class)
                for (size_t t = i0; t < e; ++t) items[t].key += (int64_t)((t - i0) / kTileMax) + 1;
            i0 = e;
        }
    }
    P.tile_off.clear();
    P.tile_reps.resize(items.size());
    P.tile_cls.resize(items.size());
    P.tile_perm_b.resize(items.size());
    P.tile_perm_c.resize(items.size());
    size_t i = 0;
    while (i < items.size()) {
        size_t e = i;
        const int64_t tk = items[i].key;
        while (e < items.size() && items[e].key == tk) ++e;
        P.tile_off.push_back((int32_t)i);
        P.max_tile = std::max(P.max_tile, (int)(e - i));
        std::vector<int> ord(e - i);
        for (size_t t = i; t < e; ++t) {
            P.tile_reps[t] = items[t].rep;
            P.tile_cls[t] = items[t].cls;
            ord[t - i] = (int)(t - i);
        }
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
            const Item& X = items[i + x];
            const Item& Y = items[i + y];
            if (X.a != Y.a) return X.a < Y.a;
            if (X.c != Y.c) return X.c < Y.c;
            return X.b < Y.b;
        });
        for (size_t t = 0; t < ord.size(); ++t) P.tile_perm_b[i + t] = (uint8_t)ord[t];
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
            const Item& X = items[i + x];
            const Item& Y = items[i + y];
            if (X.a != Y.a) return X.a < Y.a;
            if (X.b != Y.b) return X.b < Y.b;
            return X.c < Y.c;
        });
        for (size_t t = 0; t < ord.size(); ++t) P.tile_perm_c[i + t] = (uint8_t)ord[t];
        i = e;
    }
    P.tile_off.push_back((int32_t)items.size());
    P.free_tiles = 0;
    for (size_t t = 0; t + 1 < P.tile_off.size(); ++t)
        if ((int)P.tile_cls[P.tile_off[t]] == P.free_class) P.free_tiles = (int)t + 1;
    return 0;
}

void slot_directions(int dir[24]) {
    const WeylGroup& G = weyl();
    // d1 = e3 (a'), d2 = (0,1,-1) (b'), d3 = (1,-1,0) (c')
    const int d[3][3] = {{0, 0, 1}, {0, 1, -1}, {1, -1, 0}};
    for (int g = 0; g < 24; ++g) {
        dir[g] = 3;
        for (int i = 0; i < 3; ++i) {
            int img[3];
            for (int r = 0; r < 3; ++r)
                img[r] = G.m[g][3 * r] * d[i][0] + G.m[g][3 * r + 1] * d[i][1] + G.m[g][3 * r + 2] * d[i][2];
            if (img[0] == 0 && img[1] == 0 && img[2] == 1) dir[g] = i;
        }
    }
}

}  // namespace fcc
