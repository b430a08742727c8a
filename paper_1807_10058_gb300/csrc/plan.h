// Host-side plan builder for the FCC cosine transform (no CUDA code here).
//
// The skew transform DCT_n(r,s,t) of Def. 2 (explicit matrix form, Sec. 4.A)
// factors exactly as
//
//   y = DCT_n x = F S x,
//
// where F is the unnormalised 3-D DFT with the + sign over Z_n^3 and S is
// block diagonal over the W-orbits of Z_n^3 (W = the group of Sec. 3
// generated by s1, s2, s3, acting on the coefficient index k from the left as
// in the power form).  This follows from the power form of T_k evaluated at
// theta = (c + idx)/n, c = (r, s, t) = v / d with v integer (the FCC cosine
// transform proper: v = (1, 0, 3), d = 8):
//
//   y[idx] = sum_kappa Z[kappa] w_n^{kappa.idx},
//   Z[kappa] = (1/24) sum_{(k,w): w k = kappa mod n} x_k w_{dn}^{(w k).v}.
//
// Each orbit O is described by an integer representative kO in the closed
// alcove {k >= 0, k1+k2+k3 <= n} and 24 "slots" h (one per group element):
// p_h = W_h kO, member kappa_h = p_h mod n, wrap m_h = (p_h - kappa_h)/n.
// Then, for every slot g,
//
//   Z[kappa_g] = R_g * sum_h E[g][h] x[kappa_h] / 24,
//   R_g = w_{dn}^{p_g.v},   E[g][h] = w_d^{-(W_g W_h^{-1} m_h).v}.
//
// E depends only on the wrap vectors and on which slots coincide, so orbits
// fall into a handful of classes; all free orbits (95% of the points at
// n = 128) share one class.  For d = 8 every core has 8th roots of unity as
// entries.  D = F S is invertible exactly when every class block is (F is);
// for most shifts other than (1/8, 0, 3/8) and the halved shifts of the
// radix-2 recursion, some block is singular.
#pragma once
#include <array>
#include <complex>
#include <cstdint>
#include <vector>

namespace fcc {

using cd = std::complex<double>;

struct WeylGroup {
    int m[24][9];     // row-major 3x3 integer matrices, m[0] = identity
    int inv[24];      // index of the inverse element
    int mul[24][24];  // index of m[a] * m[b]
    int u[24][3];     // W_g^T v, v = (1, 0, 3): (W_g k).v = u_g . k
};
const WeylGroup& weyl();

struct OrbitClass {
    int8_t wrap[24][3];   // m_h
    int8_t canon[24];     // first slot holding the same member as slot h
    int8_t dist[24];      // index of slot h's member among the distinct ones
    int distinct;         // number of distinct members s
    uint32_t canon_mask;  // bit h set if slot h is canonical (canon[h] == h)
    // 24 x 24 row-major cores:
    //   forward  Z_g = R_g * sum_h fwd[g][h] x_h                (all slots)
    //   inverse  x_h = sum_g inv[h][g] conj(R_g) Z_g            (canonical g)
    //   adjoint  x_h = sum_g adj[h][g] conj(R_g) G_g            (canonical g)
    std::vector<cd> fwd, inv, adj;
};

struct HostPlan {
    int n = 0;
    int v[3] = {1, 0, 3};           // shift c = v / d
    int d = 8;
    int u[24][3] = {};              // W_g^T v: (W_g k).v = u_g . k
    bool invertible = true;         // every class block invertible (else inv cores are zero)
    int64_t points = 0;             // n^3
    std::vector<uint32_t> reps;     // packed representative: k1 | k2 << 10 | k3 << 20
    std::vector<uint8_t> cls;       // class of each orbit
    std::vector<OrbitClass> classes;
    int free_class = -1;            // class of the free orbits in the open alcove
    int64_t orbits_per_class_max = 0;
    std::vector<int64_t> class_begin;  // orbits are sorted by class; [begin, begin+count)
    std::vector<int64_t> class_count;

    // Tiles for the locality-aware mixing kernel.  With
    //   a' = k1 + k2 + k3, b' = k1 + k2, c' = k1
    // the representative is k = a' e3 + b' (0,1,-1) + c' (1,-1,0) and the
    // closed alcove is n >= a' >= b' >= c' >= 0.  Free representatives are
    // grouped into boxes of kTileA x kTileB x kTileC in (a', b', c'): a full
    // box is a tile (a' fastest, then b', then c'); the orbits of boxes the
    // alcove cuts fill tiles of kTileMax in box order.  Boundary classes come
    // after, in runs of kTileMax per class.  perm_b / perm_c list each tile
    // with b' (resp. c') fastest, as indices into its order.
    std::vector<int32_t> tile_off;   // [ntiles + 1], offsets into tile_reps
    std::vector<uint32_t> tile_reps; // packed representatives, tile order
    std::vector<uint8_t> tile_cls;
    std::vector<uint8_t> tile_perm_b;
    std::vector<uint8_t> tile_perm_c;
    int max_tile = 0;
    int free_tiles = 0;              // tiles [0, free_tiles) hold free orbits only
};

constexpr int kTileA = 4, kTileB = 4, kTileC = 2;   // one warp per tile
constexpr int kTileMax = kTileA * kTileB * kTileC;
constexpr int kSuperA = 8, kSuperB = 8, kSuperC = 4;  // tiles of one block are adjacent

// For slot g, the direction in (a', b', c') along which consecutive
// representatives map to consecutive memory: 0 = a', 1 = b', 2 = c',
// 3 = none of the three (the fourth direction -e1).
void slot_directions(int dir[24]);

// Orders supported by the packing of representatives.
constexpr int kMaxOrder = 512;

// Returns 0 on success, -1 on invalid order or shift, -2 on an internal
// consistency failure (a member not covered exactly once).  v, d: the shift
// c = v / d (1 <= d <= kMaxShiftDen, |v_i| <= kMaxShiftNum); v = nullptr
// selects (1/8, 0, 3/8).  A singular class block clears `invertible`.
constexpr int kMaxShiftDen = 1024;
constexpr int kMaxShiftNum = 1 << 16;
int build_host_plan(int n, HostPlan& out, const int* v = nullptr, int d = 8);

// Factorisation of a DFT length into the radices the kernels implement.
std::vector<int> fft_radices(int n);

}  // namespace fcc
