/*
 * CSR sparse matrix-vector product of the oracle's assembled operator
 * (test infrastructure only: the timed CPU baseline; nothing in the library
 * calls it). y_i = sum_k data[k] x[indices[k]] over k = indptr[i] ..
 * indptr[i+1]-1, summed in index order, one row at a time: the full
 * assembly storage level of the operator (Sec. 4.2), applied as the plain
 * definition of the product. Rows are split statically over `threads`
 * OpenMP threads; every row is summed by one thread in the same order, so
 * the result does not depend on the thread count. Compiled with
 * -ffp-contract=off (no fused multiply-add), -O2, no machine-specific flags.
 */
#include <stdint.h>

int oracle_csr_spmv(int64_t n, const int64_t* indptr, const int32_t* indices, const double* data,
                    const double* x, double* y, int threads) {
  if (n < 0 || threads < 1) return 1;
#pragma omp parallel for schedule(static) num_threads(threads)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = indptr[i]; k < indptr[i + 1]; ++k) s += data[k] * x[indices[k]];
    y[i] = s;
  }
  return 0;
}
