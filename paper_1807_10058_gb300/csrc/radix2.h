// The paper's radix-2x2x2 factorisation of DCT_n(r,s,t) (Sec. 4.B, eq.
// FastAlgorithm) evaluated on the GPU: for n = 2m
//
//   D_n(c) = P_n . (direct sum over i in {0,1}^3 of D_m((c + i)/2))
//                . (D_2(c) (x) 1_{m^3}) . B_n(c),
//
// recursively down to the 8 x 8 transform D_2 of the definition.  The paper
// leaves the basis change B_n to future work; here it follows from its
// definition (radix2.cu): column (efg, abc) of B_n^{-1} holds the b_n
// coordinates of T_{abc} T_{m(e,f,g)}, the product expanded with the mother
// recurrence (Prop. 1 (iv)), indices moved to the dominant chamber (Prop. 1
// (iii)) and indices outside the box reduced with the ideal
// T_{n e_j} = T_{e_j}(c) (Lemma 2).  B_n^{-1} is assembled on the host in
// FP64 and inverted on the GPU (Gauss-Jordan with partial pivoting).  Orders
// 2, 4, 8, 16 (B_32 would be 32768^2 complex values); complex input, FP64 or
// FP32 arithmetic (the FP32 form shows how the recursion rounds).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fcc_dct.h"

namespace fcc {

struct R2Plan;

// Device allocation through the owning plan (counted and released with it).
using R2Alloc = fcc_status (*)(void* ctx, void** ptr, size_t bytes);

// Builds the plan (host algebra, device inversion); synchronises the device.
// v, d: the shift c = v / d.  Returns nullptr with *st set on failure
// (FCC_ERR_UNSUPPORTED for a singular B_n^{-1}).
R2Plan* r2_build(int n, int batch, bool fp64, const int v[3], int d, R2Alloc alloc, void* ctx, fcc_status* st);
void r2_destroy(R2Plan* r);
// y = D_n(c) x for `batch` complex volumes (interleaved, coefficients in,
// point values out), asynchronous on `stream`.
fcc_status r2_forward(R2Plan* r, const void* in, void* out, cudaStream_t stream);
int r2_launches(const R2Plan* r);
// Statistics of B_k(c') at level k of the recursion (k = n, n/2, ... >= 4,
// averaged over the level's shifts): non-zeros per row (|entry| > 1e-12 of
// the largest), largest |entry|; complex multiply-adds of one transform per
// point when k = 0.
int r2_stats(const R2Plan* r, int k, double* nnz_per_row, double* max_abs, double* macs_per_point);

}  // namespace fcc
