/*
 * FP64 brute-force oracle for Reverse k-Maximum Inner Product Search (RkMIPS).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA library.
 *
 * What it computes is the plain definition of the problem:
 *   Def. 1 (RkMIPS): u is in the answer for (q, k) iff q is among the k largest
 *   inner products of u over P u {q}.  The trivial approach of the Introduction
 *   (a linear scan over all items for every user) is the algorithm used here.
 *
 * Tie reading (the paper states none): Alg. 2 answers "no" only when
 * <u,q> < phi, and Alg. 5 prunes only when <u,q> < L and answers "yes" when
 * ||p_k|| <= <u,q>; all three keep q on ties.  Hence
 *     c_u(q) = #{ p in P : <u,p> > <u,q> }   (strictly greater)
 *     u in R(q,k)  <=>  c_u(q) < k.
 * Copies of q inside P are never strictly greater than <u,q>, so the answer is
 * the same whether q is kept in P, removed from it, or duplicated.
 *
 * Arithmetic: every inner product is accumulated in double, sequentially over
 * i = 0 .. d-1, from the float inputs promoted to double.  The product of two
 * floats is exact in double, so contraction into FMA cannot change a result;
 * the file is still compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double ip64(const float* a, const float* b, int32_t d) {
  double s = 0.0;
  for (int32_t i = 0; i < d; ++i) s += (double)a[i] * (double)b[i];
  return s;
}

int32_t oracle_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int32_t t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* <u,p> for every user and item: out is m x n, row-major (tiny cases only). */
void oracle_scores(const float* U, int64_t m, const float* P, int64_t n, int32_t d,
                   double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t u = 0; u < m; ++u)
    for (int64_t p = 0; p < n; ++p) out[u * n + p] = ip64(U + u * d, P + p * d, d);
}

/* <u,q> for every user and query: out is m x nq, row-major. */
void oracle_query_scores(const float* U, int64_t m, int32_t d, const float* Q, int64_t nq,
                         double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t u = 0; u < m; ++u)
    for (int64_t j = 0; j < nq; ++j) out[u * nq + j] = ip64(U + u * d, Q + j * d, d);
}

/* c_u(q) for the listed users (users == NULL: all m users, in order).
 * counts[i] belongs to users[i] (or to user i). */
void oracle_count_above(const float* U, int64_t m, const float* P, int64_t n, int32_t d,
                        const float* q, const int64_t* users, int64_t nusers,
                        int64_t* counts) {
  int64_t cnt = users ? nusers : m;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < cnt; ++i) {
    const float* u = U + (users ? users[i] : i) * d;
    double sq = ip64(u, q, d);
    int64_t c = 0;
    for (int64_t p = 0; p < n; ++p)
      if (ip64(u, P + p * d, d) > sq) ++c;
    counts[i] = c;
  }
}

/* RkMIPS(q, k) over all users: writes the user ids (ascending) to out_ids,
 * which must hold m entries, and returns how many there are. */
int64_t oracle_rkmips(const float* U, int64_t m, const float* P, int64_t n, int32_t d,
                      const float* q, int32_t k, int32_t* out_ids) {
  int64_t* counts = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  oracle_count_above(U, m, P, n, d, q, NULL, m, counts);
  int64_t r = 0;
  for (int64_t u = 0; u < m; ++u)
    if (counts[u] < (int64_t)k) out_ids[r++] = (int32_t)u;
  free(counts);
  return r;
}

static int cmp_desc(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x < y) - (x > y);
}

/* tau_u(j), j = 1..kmax: the j-th largest element of the multiset {<u,p> : p in P}
 * (-inf when j > n), for the listed users (users == NULL: all).  tau is
 * cnt x kmax, row-major.  One full descending sort per user. */
void oracle_tau(const float* U, int64_t m, const float* P, int64_t n, int32_t d,
                int32_t kmax, const int64_t* users, int64_t nusers, double* tau) {
  int64_t cnt = users ? nusers : m;
#pragma omp parallel
  {
    double* s = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < cnt; ++i) {
      const float* u = U + (users ? users[i] : i) * d;
      for (int64_t p = 0; p < n; ++p) s[p] = ip64(u, P + p * d, d);
      qsort(s, (size_t)n, sizeof(double), cmp_desc);
      for (int32_t j = 0; j < kmax; ++j) tau[i * kmax + j] = (j < n) ? s[j] : -INFINITY;
    }
    free(s);
  }
}

/* RkMIPS(q, k) from cached thresholds: u in R(q,k) <=> <u,q> >= tau_u(k).
 * tau is m x kmax from oracle_tau over all users; k must be <= kmax. */
int64_t oracle_rkmips_tau(const float* U, int64_t m, int32_t d, const double* tau,
                          int32_t kmax, const float* q, int32_t k, int32_t* out_ids) {
  int64_t r = 0;
  for (int64_t u = 0; u < m; ++u)
    if (ip64(U + u * d, q, d) >= tau[u * kmax + (k - 1)]) out_ids[r++] = (int32_t)u;
  return r;
}

/* margin_u = |<u,q> - tau_u(k)| / (||u|| ||q||) for the listed users. */
void oracle_margins(const float* U, int32_t d, const double* tau_rows, int32_t kmax,
                    const float* q, int32_t k, const int64_t* users, int64_t nusers,
                    double* out) {
  double nq = sqrt(ip64(q, q, d));
  for (int64_t i = 0; i < nusers; ++i) {
    const float* u = U + users[i] * d;
    double nu = sqrt(ip64(u, u, d));
    double t = tau_rows[i * kmax + (k - 1)];
    double den = nu * nq;
    out[i] = (den > 0.0 && isfinite(t)) ? fabs(ip64(u, q, d) - t) / den : INFINITY;
  }
}
