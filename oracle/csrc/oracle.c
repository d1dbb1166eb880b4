/* Plain FP64 per-site correlator sums for the oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Nothing in the product library links this file.  It restates, in plain C and without
 * blocking or reordering, the sums of arXiv 2201.04269 Eq. 1 with the quark-level
 * contraction in its determinant form (Sec. 1), the canonical merged form (Sec. 3) and
 * the linearised factor-tree evaluation (Sec. 4, Fig. 5).  All arithmetic is complex
 * double; sums over terms use compensated (TwoSum, Knuth) accumulation.  The optional
 * OpenMP loop runs over independent sites only.
 *
 * Complex numbers are interleaved (re, im) doubles.  A 12x12 propagator is row-major,
 * row = sink spin-colour index, column = source index.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) {
    cplx r = { a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re };
    return r;
}

/* Complex division a / b, Smith's algorithm (R. L. Smith, CACM 5(8), 1962). */
static inline cplx cdiv(cplx a, cplx b) {
    cplx r;
    if (fabs(b.re) >= fabs(b.im)) {
        double q = b.im / b.re, d = b.re + b.im * q;
        r.re = (a.re + a.im * q) / d;
        r.im = (a.im - a.re * q) / d;
    } else {
        double q = b.re / b.im, d = b.re * q + b.im;
        r.re = (a.re * q + a.im) / d;
        r.im = (a.im * q - a.re) / d;
    }
    return r;
}

/* Compensated accumulator: value = hi + lo (TwoSum of each addend into hi). */
typedef struct { double hi, lo; } acc_t;
static inline void acc_add(acc_t* s, double x) {
    double t = s->hi + x;
    double bp = t - s->hi;
    s->lo += (s->hi - (t - bp)) + (x - bp);
    s->hi = t;
}

/* Determinant of an n x n complex matrix by LU with partial pivoting.
 * Pivot = largest |re| + |im| in the column (first on ties); a row swap flips the
 * sign; an exactly zero pivot gives 0. */
static cplx det_lu(int n, cplx* a) {
    cplx det = { 1.0, 0.0 };
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[k * n + k].re) + fabs(a[k * n + k].im);
        for (int i = k + 1; i < n; ++i) {
            double m = fabs(a[i * n + k].re) + fabs(a[i * n + k].im);
            if (m > best) { best = m; p = i; }
        }
        if (best == 0.0) { cplx z = { 0.0, 0.0 }; return z; }
        if (p != k) {
            for (int c = 0; c < n; ++c) { cplx t = a[k * n + c]; a[k * n + c] = a[p * n + c]; a[p * n + c] = t; }
            det.re = -det.re; det.im = -det.im;
        }
        det = cmul(det, a[k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            cplx f = cdiv(a[i * n + k], a[k * n + k]);
            for (int c = k + 1; c < n; ++c) {
                cplx g = cmul(f, a[k * n + c]);
                a[i * n + c].re -= g.re;
                a[i * n + c].im -= g.im;
            }
        }
    }
    return det;
}

/* det M[rows, cols] of a 12x12 matrix (ordered rows / cols, n <= 12; n = 0 gives 1). */
static cplx minor_det(const cplx* m, int n, const int8_t* rows, const int8_t* cols) {
    cplx a[144];
    if (n == 0) { cplx one = { 1.0, 0.0 }; return one; }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) a[i * n + k] = m[rows[i] * 12 + cols[k]];
    return det_lu(n, a);
}

void oracle_det(int n, const double* m, double* out) {
    cplx a[144];
    memcpy(a, m, sizeof(cplx) * (size_t)n * (size_t)n);
    cplx d = det_lu(n, a);
    out[0] = d.re; out[1] = d.im;
}

static int wick_sign(int n) { return ((n * (n - 1) / 2) % 2) ? -1 : 1; }

/* Eq. 1 by definition over the index set I of a factored weight
 *   W(a, a') = sum_{j,j'} P_jj' s_j(a) conj(r_j'(a')),
 * C_x = (-1)^{n(n-1)/2} sum_{(a, a') in I} W det U_x[a_u, a'_u] det D_x[a_d, a'_d].
 * snk_idx: [n_snk][n_u + n_d] flavour-grouped slot indices, snk_w complex, snk_off
 * [n_free + 1] offsets per free index (same for src). U, D: [n_sites][12][12] complex.
 * out: [n_sites] complex. */
void oracle_direct(int n_u, int n_d, int n_free,
                   const int8_t* snk_idx, const double* snk_w, const int64_t* snk_off,
                   const int8_t* src_idx, const double* src_w, const int64_t* src_off,
                   const double* proj, const double* U, const double* D,
                   int64_t n_sites, double* out, int n_threads) {
    const int nq = n_u + n_d;
    const cplx* sw = (const cplx*)snk_w;
    const cplx* rw = (const cplx*)src_w;
    const cplx* P = (const cplx*)proj;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t x = 0; x < n_sites; ++x) {
        const cplx* u = (const cplx*)U + x * 144;
        const cplx* d = (const cplx*)D + x * 144;
        acc_t re = { 0, 0 }, im = { 0, 0 };
        for (int j = 0; j < n_free; ++j)
            for (int k = 0; k < n_free; ++k) {
                cplx p = P[j * n_free + k];
                if (p.re == 0.0 && p.im == 0.0) continue;
                for (int64_t a = snk_off[j]; a < snk_off[j + 1]; ++a) {
                    cplx pa = cmul(p, sw[a]);
                    const int8_t* ia = snk_idx + a * nq;
                    for (int64_t b = src_off[k]; b < src_off[k + 1]; ++b) {
                        const int8_t* ib = src_idx + b * nq;
                        cplx rb = { rw[b].re, -rw[b].im };
                        cplx w = cmul(pa, rb);
                        cplx du = minor_det(u, n_u, ia, ib);
                        cplx dd = minor_det(d, n_d, ia + n_u, ib + n_u);
                        cplx t = cmul(w, cmul(du, dd));
                        acc_add(&re, t.re);
                        acc_add(&im, t.im);
                    }
                }
            }
        double s = (double)wick_sign(nq);
        out[2 * x] = s * (re.hi + re.lo);
        out[2 * x + 1] = s * (im.hi + im.lo);
    }
}

/* Canonical merged form (Sec. 3): C_x = sum_t W_t det U_x[mu_t] det D_x[md_t].
 * Minor m of flavour f has ascending rows rows_f[m][k] and columns cols_f[m][k]
 * (k = n_f entries).  W already folds the Wick sign.  Every distinct minor is
 * evaluated once per site by LU, then the terms are summed in list order. */
void oracle_canonical(int n_u, int n_d,
                      int64_t n_mu, const int8_t* rows_u, const int8_t* cols_u,
                      int64_t n_md, const int8_t* rows_d, const int8_t* cols_d,
                      int64_t n_terms, const int32_t* mu, const int32_t* md, const double* W,
                      const double* U, const double* D, int64_t n_sites, double* out, int n_threads) {
    const cplx* w = (const cplx*)W;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t x = 0; x < n_sites; ++x) {
        const cplx* u = (const cplx*)U + x * 144;
        const cplx* d = (const cplx*)D + x * 144;
        cplx* vu = (cplx*)malloc(sizeof(cplx) * (size_t)(n_mu + n_md + 1));
        cplx* vd = vu + n_mu;
        for (int64_t m = 0; m < n_mu; ++m) vu[m] = minor_det(u, n_u, rows_u + m * n_u, cols_u + m * n_u);
        for (int64_t m = 0; m < n_md; ++m) vd[m] = minor_det(d, n_d, rows_d + m * n_d, cols_d + m * n_d);
        acc_t re = { 0, 0 }, im = { 0, 0 };
        for (int64_t t = 0; t < n_terms; ++t) {
            cplx v = cmul(w[t], cmul(vu[mu[t]], vd[md[t]]));
            acc_add(&re, v.re);
            acc_add(&im, v.im);
        }
        out[2 * x] = re.hi + re.lo;
        out[2 * x + 1] = im.hi + im.lo;
        free(vu);
    }
}

/* Linearised factor tree (Sec. 4, Fig. 5): factors[] in depth-first order (factors[0]
 * is the root, ignored), children[] the child count of each vertex, coefficients[] the
 * leaf coefficients in depth-first order.  The value is the sum over root-to-leaf paths
 * of the product of the path's factor values times the leaf coefficient.  Factor id f
 * refers to fval[f] (per site: values[x][f]). */
void oracle_tree(int64_t n_nodes, const int32_t* factors, const int32_t* children,
                 const double* coefficients, int64_t n_factor_values, const double* values,
                 int64_t n_sites, double* out, int n_threads) {
    const cplx* c = (const cplx*)coefficients;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t x = 0; x < n_sites; ++x) {
        const cplx* fv = (const cplx*)values + x * n_factor_values;
        cplx prod[64];
        int64_t rem[64];
        int depth = 0;
        prod[0].re = 1.0; prod[0].im = 0.0;
        rem[0] = children[0];
        int64_t leaf = 0;
        acc_t re = { 0, 0 }, im = { 0, 0 };
        for (int64_t k = 1; k < n_nodes; ++k) {
            while (depth > 0 && rem[depth] == 0) --depth;   /* climb to the open parent */
            rem[depth] -= 1;
            cplx p = cmul(prod[depth], fv[factors[k]]);
            if (children[k] == 0) {
                cplx v = cmul(c[leaf++], p);
                acc_add(&re, v.re);
                acc_add(&im, v.im);
            } else {
                ++depth;
                prod[depth] = p;
                rem[depth] = children[k];
            }
        }
        out[2 * x] = re.hi + re.lo;
        out[2 * x + 1] = im.hi + im.lo;
    }
}

/* Minor tables for many sites: out[x][m] = det M_x[rows[m], cols[m]] (n x n). */
void oracle_minors(int n, int64_t n_minors, const int8_t* rows, const int8_t* cols,
                   const double* M, int64_t n_sites, double* out, int n_threads) {
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t x = 0; x < n_sites; ++x) {
        const cplx* m = (const cplx*)M + x * 144;
        cplx* o = (cplx*)out + x * n_minors;
        for (int64_t k = 0; k < n_minors; ++k) o[k] = minor_det(m, n, rows + k * n, cols + k * n);
    }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
