/*
 * FP64 oracle for the FCC cosine transform DCT_{n x n x n} (Seifert, Hueper,
 * Uhl, "Fast cosine transform for FCC lattices", 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA library.
 *
 * What it computes is the plain definition, written out term by term:
 *
 *   Weyl group W (Sec. 3, eq. of the generator matrices): the 24 integer
 *   3x3 matrices generated by the printed s1, s2, s3, acting on k from the
 *   left, so that the 24 exponent vectors of the power form of T_{n,m,l}
 *   (Sec. 3, "general power form") are exactly {w k : w in W}.
 *
 *   T_k(theta) = (1/24) sum_{w in W} exp(2 pi i (w k) . theta)
 *     (Def. 1 with the power form; theta in R^3 / Z^3)
 *
 *   Sample points (Lemma 1, Lemma 2, Def. 2): for the skew parameter
 *   (r,s,t) = (a1, a2, a3)/d and order n,
 *     theta_{i,l,q} = ((r+i)/n, (s+l)/n, (t+q)/n),   0 <= i,l,q < n.
 *   The FCC cosine transform uses (r,s,t) = (1/8, 0, 3/8), i.e. a=(1,0,3),
 *   d=8.  Then d*n*theta = a + d*idx is an integer vector, and every phase
 *   (w k) . theta = ((w k) . (a + d*idx)) / (d n) is an exact rational whose
 *   numerator is reduced modulo M = d*n before a single table lookup of
 *   cos/sin(2 pi e / M).  No angle error accumulates.
 *
 *   Matrix (Def. 2, explicit matrix form): rows are the n^3 sample points
 *   (i,l,q), columns the n^3 basis polynomials T_{j,k,p}, both in
 *   lexicographic order with the last index fastest:
 *     D[(i,l,q),(j,k,p)] = T_{(j,k,p)}(theta_{i,l,q}).
 *   The forward transform is y = D x (coefficients -> values at the
 *   points); the adjoint is D^H.
 *
 * Parallelism: optional OpenMP over output rows (the only reason for the
 * nthreads arguments); every row is the same serial sum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The three generators as printed in Sec. 3 (row-major). */
static const int GEN[3][9] = {
    {-1, 0, 0, 1, 1, 0, 0, 0, 1},
    {1, 1, 0, 0, -1, 0, 0, 1, 1},
    {1, 0, 0, 0, 1, 1, 0, 0, -1},
};

static void matmul3(const int* a, const int* b, int* c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int s = 0;
            for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
}

/* Closure of {s1,s2,s3} under multiplication, breadth first from the
 * identity.  Writes up to cap matrices (row-major, 9 ints each) and returns
 * the group order (24 for the printed generators). */
int fcc_oracle_weyl_group(int* out, int cap) {
    int* grp = (int*)malloc(sizeof(int) * 9 * 64);
    int count = 1;
    const int id[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(grp, id, sizeof id);
    for (int head = 0; head < count; ++head) {
        for (int g = 0; g < 3; ++g) {
            int c[9];
            matmul3(GEN[g], grp + 9 * head, c);
            int known = 0;
            for (int j = 0; j < count && !known; ++j)
                known = memcmp(c, grp + 9 * j, sizeof c) == 0;
            if (!known) {
                if (count == 64) { free(grp); return -1; }
                memcpy(grp + 9 * count, c, sizeof c);
                ++count;
            }
        }
    }
    for (int j = 0; j < count && j < cap; ++j) memcpy(out + 9 * j, grp + 9 * j, sizeof(int) * 9);
    free(grp);
    return count;
}

/* T_k(theta) at an arbitrary real theta, straight from the orbit sum. */
void fcc_oracle_chebyshev(const int* k, const double* theta, double* re, double* im) {
    int W[24 * 9];
    int m = fcc_oracle_weyl_group(W, 24);
    double sr = 0.0, si = 0.0;
    for (int g = 0; g < m; ++g) {
        const int* w = W + 9 * g;
        double ph = 0.0;
        for (int a = 0; a < 3; ++a) {
            int wk = w[3 * a + 0] * k[0] + w[3 * a + 1] * k[1] + w[3 * a + 2] * k[2];
            ph += wk * theta[a];
        }
        ph -= floor(ph);
        sr += cos(2.0 * M_PI * ph);
        si += sin(2.0 * M_PI * ph);
    }
    *re = sr / m;
    *im = si / m;
}

static int64_t mod64(int64_t a, int64_t m) {
    int64_t r = a % m;
    return r < 0 ? r + m : r;
}

typedef struct {
    int n, d, M;
    int a[3];
    int W[24 * 9];
    double* c; /* cos(2 pi e / M) */
    double* s; /* sin(2 pi e / M) */
} ctx_t;

static int ctx_init(ctx_t* cx, int n, const int* a, int d) {
    if (n < 1 || d < 1) return -1;
    cx->n = n;
    cx->d = d;
    cx->M = d * n;
    for (int j = 0; j < 3; ++j) cx->a[j] = a[j];
    if (fcc_oracle_weyl_group(cx->W, 24) != 24) return -1;
    cx->c = (double*)malloc(sizeof(double) * cx->M);
    cx->s = (double*)malloc(sizeof(double) * cx->M);
    for (int e = 0; e < cx->M; ++e) {
        cx->c[e] = cos(2.0 * M_PI * (double)e / (double)cx->M);
        cx->s[e] = sin(2.0 * M_PI * (double)e / (double)cx->M);
    }
    return 0;
}

static void ctx_free(ctx_t* cx) {
    free(cx->c);
    free(cx->s);
}

/* exponent numerator of (w k) . theta_idx, i.e. (w k) . (a + d*idx) mod M */
static inline int64_t phase_num(const ctx_t* cx, const int* w, const int* k, const int* idx) {
    int64_t e = 0;
    for (int r = 0; r < 3; ++r) {
        int64_t wk = (int64_t)w[3 * r + 0] * k[0] + (int64_t)w[3 * r + 1] * k[1] + (int64_t)w[3 * r + 2] * k[2];
        e += wk * (int64_t)(cx->a[r] + cx->d * idx[r]);
    }
    return mod64(e, cx->M);
}

/* T_k(theta_idx) for integer k and sample point idx (exact phases). */
static void cheb_at_point(const ctx_t* cx, const int* k, const int* idx, double* re, double* im) {
    double sr = 0.0, si = 0.0;
    for (int g = 0; g < 24; ++g) {
        int64_t e = phase_num(cx, cx->W + 9 * g, k, idx);
        sr += cx->c[e];
        si += cx->s[e];
    }
    *re = sr / 24.0;
    *im = si / 24.0;
}

static void unflat(int64_t f, int n, int* v) {
    v[2] = (int)(f % n);
    f /= n;
    v[1] = (int)(f % n);
    v[0] = (int)(f / n);
}

/* Dense D (N x N, N = n^3), row-major: D[row*N + col]. */
int fcc_oracle_matrix(int n, const int* a, int d, double* re, double* im, int nthreads) {
    ctx_t cx;
    if (ctx_init(&cx, n, a, d)) return -1;
    const int64_t N = (int64_t)n * n * n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t row = 0; row < N; ++row) {
        int idx[3], k[3];
        unflat(row, n, idx);
        for (int64_t col = 0; col < N; ++col) {
            unflat(col, n, k);
            cheb_at_point(&cx, k, idx, re + row * N + col, im + row * N + col);
        }
    }
    (void)nthreads;
    ctx_free(&cx);
    return 0;
}

/* y[r] = sum_k D[rows[r], k] x[k] for one volume x (n^3 complex, x_im may be
 * NULL for real input).  Cost 24 n^3 per requested row. */
int fcc_oracle_forward_rows(int n, const int* a, int d, const double* x_re, const double* x_im,
                            const int64_t* rows, int64_t nrows, double* y_re, double* y_im,
                            int nthreads) {
    ctx_t cx;
    if (ctx_init(&cx, n, a, d)) return -1;
    const int64_t N = (int64_t)n * n * n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t r = 0; r < nrows; ++r) {
        int idx[3], k[3];
        unflat(rows[r], n, idx);
        double sr = 0.0, si = 0.0;
        for (int64_t col = 0; col < N; ++col) {
            unflat(col, n, k);
            double tr, ti;
            cheb_at_point(&cx, k, idx, &tr, &ti);
            double xr = x_re[col], xi = x_im ? x_im[col] : 0.0;
            sr += tr * xr - ti * xi;
            si += tr * xi + ti * xr;
        }
        y_re[r] = sr;
        y_im[r] = si;
    }
    (void)nthreads;
    ctx_free(&cx);
    return 0;
}

/* (D^H g)[cols[c]] = sum_idx conj(D[idx, cols[c]]) g[idx], one volume. */
int fcc_oracle_adjoint_rows(int n, const int* a, int d, const double* g_re, const double* g_im,
                            const int64_t* cols, int64_t ncols, double* x_re, double* x_im,
                            int nthreads) {
    ctx_t cx;
    if (ctx_init(&cx, n, a, d)) return -1;
    const int64_t N = (int64_t)n * n * n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t c = 0; c < ncols; ++c) {
        int idx[3], k[3];
        unflat(cols[c], n, k);
        double sr = 0.0, si = 0.0;
        for (int64_t row = 0; row < N; ++row) {
            unflat(row, n, idx);
            double tr, ti;
            cheb_at_point(&cx, k, idx, &tr, &ti);
            double gr = g_re[row], gi = g_im ? g_im[row] : 0.0;
            /* conj(t) * g */
            sr += tr * gr + ti * gi;
            si += tr * gi - ti * gr;
        }
        x_re[c] = sr;
        x_im[c] = si;
    }
    (void)nthreads;
    ctx_free(&cx);
    return 0;
}

int fcc_oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
