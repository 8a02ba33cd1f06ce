/* Oracle CSR x dense block product, FP64: Y[i, c] = sum_t val[t] * X[col[t], c].
 * Plain loop over rows (OpenMP), entries of a row in stored order.
 * Test infrastructure only; shares nothing with the CUDA path. */
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void oracle_csr_spmm(int64_t n, int64_t k, const int64_t* row_ptr, const int32_t* col, const double* val,
                     const double* X, double* Y) {
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    double acc[64];
    for (int64_t c = 0; c < k && c < 64; ++c) acc[c] = 0.0;
    for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {
      const double v = val[t];
      const double* x = X + (int64_t)col[t] * k;
      for (int64_t c = 0; c < k && c < 64; ++c) acc[c] = acc[c] + v * x[c];
    }
    for (int64_t c = 0; c < k && c < 64; ++c) Y[i * k + c] = acc[c];
  }
}
