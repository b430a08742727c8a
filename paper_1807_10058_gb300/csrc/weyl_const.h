// Compile-time copy of the group W (Sec. 3): the closure of the printed
// generators s1, s2, s3, built in the same breadth-first order as the
// run-time plan builder (which checks that the two agree), plus the per-slot
// constants the mixing kernels need:
//   m[g]    the 3x3 matrix W_g (row-major),
//   u[g]    W_g^T (1, 0, 3), so that (W_g k).v = u_g . k,
//   dir[g]  0/1/2 if W_g maps d = e3 / (0,1,-1) / (1,-1,0) onto e3, else 3,
//   fw[g]   the wrap vector of slot g for representatives inside the open
//           alcove: -1 where row i of W_g is a negated positive form.
#pragma once

namespace fcc {
namespace wc {

struct Tab {
    int m[24][9];
    int u[24][3];
    int dir[24];
    int fw[24][3];
    int order;
};

constexpr Tab build() {
    Tab T{};
    const int gen[3][9] = {
        {-1, 0, 0, 1, 1, 0, 0, 0, 1},
        {1, 1, 0, 0, -1, 0, 0, 1, 1},
        {1, 0, 0, 0, 1, 1, 0, 0, -1},
    };
    for (int i = 0; i < 9; ++i) T.m[0][i] = (i % 4 == 0) ? 1 : 0;
    int cnt = 1;
    for (int head = 0; head < cnt; ++head) {
        for (int s = 0; s < 3; ++s) {
            int c[9] = {};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    int acc = 0;
                    for (int k = 0; k < 3; ++k) acc += gen[s][3 * i + k] * T.m[head][3 * k + j];
                    c[3 * i + j] = acc;
                }
            bool known = false;
            for (int e = 0; e < cnt && !known; ++e) {
                bool eq = true;
                for (int i = 0; i < 9; ++i) eq = eq && (T.m[e][i] == c[i]);
                known = eq;
            }
            if (!known && cnt < 24) {
                for (int i = 0; i < 9; ++i) T.m[cnt][i] = c[i];
                ++cnt;
            }
        }
    }
    T.order = cnt;
    const int v[3] = {1, 0, 3};
    const int d[3][3] = {{0, 0, 1}, {0, 1, -1}, {1, -1, 0}};
    for (int g = 0; g < 24; ++g) {
        for (int j = 0; j < 3; ++j) {
            int acc = 0;
            for (int i = 0; i < 3; ++i) acc += T.m[g][3 * i + j] * v[i];
            T.u[g][j] = acc;
        }
        T.dir[g] = 3;
        for (int q = 0; q < 3; ++q) {
            int img[3] = {};
            for (int r = 0; r < 3; ++r)
                img[r] = T.m[g][3 * r] * d[q][0] + T.m[g][3 * r + 1] * d[q][1] + T.m[g][3 * r + 2] * d[q][2];
            if (img[0] == 0 && img[1] == 0 && img[2] == 1) T.dir[g] = q;
        }
        for (int r = 0; r < 3; ++r) {
            const int s = T.m[g][3 * r] + T.m[g][3 * r + 1] + T.m[g][3 * r + 2];
            T.fw[g][r] = s < 0 ? -1 : 0;
        }
    }
    return T;
}

struct K {
    static constexpr Tab t = build();
};
static_assert(K::t.order == 24, "W must have order 24");

}  // namespace wc
}  // namespace fcc
