/*
 * TEST INFRASTRUCTURE ONLY: the oracle's doubling form of the stochastic KPM
 * moments (oracle/kpm_oracle.py, moments_doubling) restated in plain C for a
 * multi-core CPU baseline.  Only the tests and the benchmark's CPU-baseline
 * leg load it; it shares no code with the CUDA library.
 *
 * Paper (arXiv:1105.5481), Sec. II-A: H~ = (H - b)/a (Eq. (tilde)),
 * r_1 = H~ r_0, r_{n+1} = 2 H~ r_n - r_{n-1} (Eq. (rn)); moments by the
 * doubling identities of the cited KPM review (Eq. 34):
 *   mu_0^r = <v_0|v_0>/N, mu_1^r = Re<v_1|v_0>/N,
 *   mu_2n^r = 2<v_n|v_n>/N - mu_0^r, mu_2n+1^r = 2 Re<v_n+1|v_n>/N - mu_1^r,
 * averaged over the R vectors (Eq. (munr)).  FP64 throughout.
 *
 * Layout: CSR (rowptr[n+1], col[nnz], val[nnz] real or (re, im) pairs) and
 * N x R vector blocks, row-major with the R entries of a site contiguous
 * (complex: (re, im) pairs).  The products are parallel over rows (OpenMP),
 * the dot products over rows with one partial per thread.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* y = (H x - b x) / a for an N x R block; c = 1 (real) or 2 (complex) */
static void rescaled_apply(int64_t n, const int64_t* rowptr, const int64_t* col,
                           const double* val, int c, double a, double b, const double* x,
                           double* y, int R, int threads) {
  const int64_t w = (int64_t)R * c;
#pragma omp parallel for schedule(static) num_threads(threads)
  for (int64_t i = 0; i < n; ++i) {
    double* yi = y + i * w;
    const double* xi = x + i * w;
    for (int64_t e = 0; e < w; ++e) yi[e] = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const double* xj = x + col[k] * w;
      if (c == 1) {
        const double h = val[k];
        for (int r = 0; r < R; ++r) yi[r] += h * xj[r];
      } else {
        const double hr = val[2 * k], hi = val[2 * k + 1];
        for (int r = 0; r < R; ++r) {
          const double xr = xj[2 * r], xim = xj[2 * r + 1];
          yi[2 * r] += hr * xr - hi * xim;
          yi[2 * r + 1] += hr * xim + hi * xr;
        }
      }
    }
    for (int64_t e = 0; e < w; ++e) yi[e] = (yi[e] - b * xi[e]) / a;
  }
}

/* out[r] = Re<p|q>_r / n for the R columns (sum over sites) */
static void col_dots(int64_t n, int c, const double* p, const double* q, int R, int threads,
                     double* out) {
  const int64_t w = (int64_t)R * c;
  int nt = 1;
#ifdef _OPENMP
  nt = threads > 0 ? threads : omp_get_max_threads();
#endif
  double* part = (double*)calloc((size_t)nt * R, sizeof(double));
  if (!part) return;
#pragma omp parallel num_threads(nt)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double* acc = part + (size_t)t * R;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      const double* pi = p + i * w;
      const double* qi = q + i * w;
      for (int r = 0; r < R; ++r) {
        if (c == 1)
          acc[r] += pi[r] * qi[r];
        else
          acc[r] += pi[2 * r] * qi[2 * r] + pi[2 * r + 1] * qi[2 * r + 1];
      }
    }
  }
  for (int r = 0; r < R; ++r) {
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += part[(size_t)t * R + r];
    out[r] = s / (double)n;
  }
  free(part);
}

int kpm_cpu_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * mu[M] (mean over the R vectors) and, if mu_per_vec is not NULL,
 * mu_per_vec[R][M].  cplx selects complex (re, im) values and vectors.
 * threads <= 0: all available.  Returns 0, -1 for invalid arguments, -2 when
 * memory runs out.
 */
int kpm_cpu_moments(int64_t n, const int64_t* rowptr, const int64_t* col, const double* val,
                    int cplx, double a, double b, const double* v0, int R, int M, double* mu,
                    double* mu_per_vec, int threads) {
  if (n < 1 || R < 1 || M < 2 || (M & 1) || !(a > 0.0) || !rowptr || !v0 || !mu) return -1;
  const int c = cplx ? 2 : 1;
  int nt = 1;
#ifdef _OPENMP
  nt = threads > 0 ? threads : omp_get_max_threads();
#else
  (void)threads;
#endif
  const size_t len = (size_t)n * R * c;
  double* prev = (double*)malloc(len * sizeof(double));
  double* cur = (double*)malloc(len * sizeof(double));
  double* nxt = (double*)malloc(len * sizeof(double));
  double* out = (double*)calloc((size_t)R * M, sizeof(double));
  double* mu0 = (double*)malloc((size_t)R * sizeof(double));
  double* mu1 = (double*)malloc((size_t)R * sizeof(double));
  double* d = (double*)malloc((size_t)R * sizeof(double));
  if (!prev || !cur || !nxt || !out || !mu0 || !mu1 || !d) {
    free(prev); free(cur); free(nxt); free(out); free(mu0); free(mu1); free(d);
    return -2;
  }
  memcpy(prev, v0, len * sizeof(double));
  rescaled_apply(n, rowptr, col, val, c, a, b, prev, cur, R, nt);   /* v_1 = H~ v_0 */
  col_dots(n, c, prev, prev, R, nt, mu0);
  col_dots(n, c, cur, prev, R, nt, mu1);
  for (int r = 0; r < R; ++r) {
    out[(size_t)r * M] = mu0[r];
    out[(size_t)r * M + 1] = mu1[r];
  }
  for (int s = 1; s < M / 2; ++s) {
    rescaled_apply(n, rowptr, col, val, c, a, b, cur, nxt, R, nt);  /* H~ v_n */
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int64_t e = 0; e < (int64_t)len; ++e) nxt[e] = 2.0 * nxt[e] - prev[e];
    col_dots(n, c, cur, cur, R, nt, d);
    for (int r = 0; r < R; ++r) out[(size_t)r * M + 2 * s] = 2.0 * d[r] - mu0[r];
    col_dots(n, c, nxt, cur, R, nt, d);
    for (int r = 0; r < R; ++r) out[(size_t)r * M + 2 * s + 1] = 2.0 * d[r] - mu1[r];
    double* t = prev; prev = cur; cur = nxt; nxt = t;
  }
  for (int m = 0; m < M; ++m) {
    double s = 0.0;
    for (int r = 0; r < R; ++r) s += out[(size_t)r * M + m];
    mu[m] = s / (double)R;
  }
  if (mu_per_vec) memcpy(mu_per_vec, out, (size_t)R * M * sizeof(double));
  free(prev); free(cur); free(nxt); free(out); free(mu0); free(mu1); free(d);
  return 0;
}
