/*
 * Oracle (test infrastructure only): plain FP64 brute-force nearest
 * neighbours on the CPU.  Not part of the product path; only tests, the
 * smoke check and the benchmark's CPU-baseline leg call it.
 *
 * The brute-force primitive BF(Q, X) (Section 3): for every query q the
 * distance rho(q, x) to every database point x is computed and the closest
 * points are returned.  The k-NN form used here returns the k smallest
 * (rho, id) pairs in lexicographic order, so equal distances are broken by
 * the smaller database id.
 *
 * Metrics (Section 6): l2 rho = sqrt(sum_i (q_i - x_i)^2) evaluated in the
 * difference form, and l1 rho = sum_i |q_i - x_i|.  Inputs are float32, every
 * operation is carried out in double precision.
 *
 * Parallel over queries with OpenMP; each query is independent, so the
 * result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* rho(a, b) in double precision. metric 0 = l2, 1 = l1. */
static double oracle_rho(const float* a, const float* b, int32_t d, int32_t metric) {
    double s = 0.0;
    if (metric == 1) {
        for (int32_t i = 0; i < d; ++i) s += fabs((double)a[i] - (double)b[i]);
        return s;
    }
    for (int32_t i = 0; i < d; ++i) {
        double t = (double)a[i] - (double)b[i];
        s += t * t;
    }
    return sqrt(s);
}

/* (r1, i1) < (r2, i2) in lexicographic order */
static int pair_less(double r1, int64_t i1, double r2, int64_t i2) {
    return r1 < r2 || (r1 == r2 && i1 < i2);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * BF(Q, X) with k results per query.
 *   Q [m, d], X [n, d] row-major float32; out_ids [m, k] int64, out_dist [m, k]
 *   double.  If k > n the tail is filled with id -1 and distance +inf.
 *   nthreads <= 0 uses the OpenMP default.
 */
void oracle_bf(const float* Q, int64_t m, const float* X, int64_t n, int32_t d, int32_t k,
               int32_t metric, int64_t* out_ids, double* out_dist, int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < m; ++qi) {
        double* bd = out_dist + qi * (int64_t)k;
        int64_t* bi = out_ids + qi * (int64_t)k;
        int32_t filled = 0;
        for (int32_t j = 0; j < k; ++j) {
            bd[j] = INFINITY;
            bi[j] = -1;
        }
        const float* q = Q + qi * (int64_t)d;
        for (int64_t xi = 0; xi < n; ++xi) {
            double r = oracle_rho(q, X + xi * (int64_t)d, d, metric);
            if (filled == k && !pair_less(r, xi, bd[k - 1], bi[k - 1])) continue;
            /* insertion into the sorted list of the best k seen so far */
            int32_t pos = filled < k ? filled : k - 1;
            while (pos > 0 && pair_less(r, xi, bd[pos - 1], bi[pos - 1])) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = r;
            bi[pos] = xi;
            if (filled < k) ++filled;
        }
    }
}

/*
 * All pairwise distances D [m, n] (double), for small cases where the method
 * needs every rho(q, r) (the representative distances of the exact search).
 */
void oracle_dist(const float* Q, int64_t m, const float* X, int64_t n, int32_t d,
                 int32_t metric, double* out, int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(static)
    for (int64_t qi = 0; qi < m; ++qi)
        for (int64_t xi = 0; xi < n; ++xi)
            out[qi * n + xi] = oracle_rho(Q + qi * (int64_t)d, X + xi * (int64_t)d, d, metric);
}

/*
 * BF(Q, X[L]) for a per-query id list: query qi searches only the ids
 * list_ids[list_off[qi] .. list_off[qi+1]).  Same ordering rule as oracle_bf.
 */
void oracle_bf_lists(const float* Q, int64_t m, const float* X, int32_t d, int32_t k,
                     int32_t metric, const int64_t* list_off, const int64_t* list_ids,
                     int64_t* out_ids, double* out_dist, int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < m; ++qi) {
        double* bd = out_dist + qi * (int64_t)k;
        int64_t* bi = out_ids + qi * (int64_t)k;
        int32_t filled = 0;
        for (int32_t j = 0; j < k; ++j) {
            bd[j] = INFINITY;
            bi[j] = -1;
        }
        const float* q = Q + qi * (int64_t)d;
        for (int64_t t = list_off[qi]; t < list_off[qi + 1]; ++t) {
            int64_t xi = list_ids[t];
            double r = oracle_rho(q, X + xi * (int64_t)d, d, metric);
            if (filled == k && !pair_less(r, xi, bd[k - 1], bi[k - 1])) continue;
            int32_t pos = filled < k ? filled : k - 1;
            while (pos > 0 && pair_less(r, xi, bd[pos - 1], bi[pos - 1])) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = r;
            bi[pos] = xi;
            if (filled < k) ++filled;
        }
    }
}
