/* Binary64 enumeration of Eq. (1) on the host cores (OpenMP).
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY, like the rest of oracle/: it is
 * loaded by tests/ and by the CPU-baseline leg of bench.py, never by the
 * library.  It shares no code with the CUDA path.
 *
 * What it computes, in the order of the paper:
 *  - Definition 3, Eq. (1): the sum over all ascending column sequences
 *    j1 < ... < jm of (-1)^(r+s) det(A[:, J]), r = m(m+1)/2, s = j1+...+jm
 *    (1-based); 0 when m > n.
 *  - Section 5: the C(n,m) dictionary-order ranks are cut into contiguous
 *    runs, one per processor (here OpenMP threads, a few runs per thread);
 *    each run's first sequence comes from its rank (Section 4, in the closed
 *    form of the combinatorial number system) and the rest from the
 *    dictionary successor.
 *  - Each minor: Gaussian elimination with partial pivoting in binary64,
 *    det = +-prod(pivots).
 *  - Sums: plain binary64 addition per run, runs added in run order.
 * It is a plain statement of the method, not tuned: no blocking, no vector
 * intrinsics, no prefix sharing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define CPU_MAX_M 32
#define CPU_MAX_N 64

static uint64_t binom_u64(int n, int k) {
  if (k < 0 || k > n) return 0;
  if (k > n - k) k = n - k;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

/* rank q (0-based, dictionary order) -> 0-based ascending columns c[0..m-1] */
static void unrank(uint64_t q, int n, int m, int* c) {
  uint64_t r = binom_u64(n, m) - 1 - q;
  int v = n;
  for (int i = 0; i < m; ++i) {
    const int k = m - i;
    int w = v - 1;
    while (binom_u64(w, k) > r) --w;
    c[i] = n - 1 - w;
    r -= binom_u64(w, k);
    v = w;
  }
}

/* dictionary successor (must not be called on the last sequence) */
static void successor(int* c, int n, int m) {
  int pos = m - 1;
  while (c[pos] == n - m + pos) --pos;
  ++c[pos];
  for (int j = pos + 1; j < m; ++j) c[j] = c[j - 1] + 1;
}

static double minor_det(const double* A, int lda, int m, const int* c) {
  double a[CPU_MAX_M][CPU_MAX_M];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) a[i][j] = A[(long long)i * lda + c[j]];
  double det = 1.0;
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (fabs(a[i][k]) > fabs(a[p][k])) p = i;
    if (a[p][k] == 0.0) return 0.0;
    if (p != k) {
      for (int j = 0; j < m; ++j) {
        const double t = a[k][j];
        a[k][j] = a[p][j];
        a[p][j] = t;
      }
      det = -det;
    }
    det *= a[k][k];
    for (int i = k + 1; i < m; ++i) {
      const double l = a[i][k] / a[k][k];
      for (int j = k + 1; j < m; ++j) a[i][j] -= l * a[k][j];
    }
  }
  return det;
}

/* Sum of the signed minors with dictionary ranks q0 .. q0+count-1 (clipped to
 * C(n,m)); *abs_sum receives the sum of their magnitudes and *threads the
 * number of OpenMP threads used.  A: host, m x n row-major, leading
 * dimension lda.  Returns 0 (and *abs_sum = 0) for m > n or invalid sizes. */
double radic_cpu_sum(const double* A, int m, int n, int lda, uint64_t q0, uint64_t count, double* abs_sum,
                     int* threads) {
  *abs_sum = 0.0;
  *threads = 1;
  if (m < 1 || n < 1 || m > CPU_MAX_M || n > CPU_MAX_N || m > n || lda < n) return 0.0;
  const uint64_t total = binom_u64(n, m);
  if (q0 >= total) return 0.0;
  if (count > total - q0) count = total - q0;
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  const long long runs = (long long)nth * 8;  /* Section 5: contiguous runs */
  const uint64_t per = (count + (uint64_t)runs - 1) / (uint64_t)runs;
  double* part = (double*)calloc((size_t)runs * 2, sizeof(double));
  if (!part) return NAN;
  const int r_par = m * (m + 1) / 2 + m; /* r plus the "+1" of each 1-based index */
#pragma omp parallel for schedule(dynamic, 1)
  for (long long t = 0; t < runs; ++t) {
    const uint64_t a0 = q0 + (uint64_t)t * per;
    if (a0 >= q0 + count) continue;
    uint64_t a1 = a0 + per;
    if (a1 > q0 + count) a1 = q0 + count;
    int c[CPU_MAX_M];
    unrank(a0, n, m, c);
    double s = 0.0, sa = 0.0;
    for (uint64_t q = a0; q < a1; ++q) {
      int par = r_par;
      for (int i = 0; i < m; ++i) par += c[i];
      double d = minor_det(A, lda, m, c);
      if (par & 1) d = -d;
      s += d;
      sa += fabs(d);
      if (q + 1 < a1) successor(c, n, m);
    }
    part[2 * t] = s;
    part[2 * t + 1] = sa;
  }
  double s = 0.0, sa = 0.0;
  for (long long t = 0; t < runs; ++t) {
    s += part[2 * t];
    sa += part[2 * t + 1];
  }
  free(part);
  *abs_sum = sa;
  *threads = nth;
  return s;
}
