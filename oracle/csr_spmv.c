/*
 * Plain compressed-row product y = A x in float64 for the CPU baseline of the
 * benchmark — TEST INFRASTRUCTURE ONLY (oracle/).  The same product as
 * oracle.spmv (Sec. 1.1: the sparse-matrix alternative the paper compares
 * the stencil apply with, Sec. 3): one pass over the rows, each row's entries
 * in stored order, no blocking.  Rows are split evenly across `threads`
 * threads (OpenMP static schedule) so that the oracle can also be timed on
 * all host cores.  Built with -ffp-contract=off: every product is rounded
 * before it is added, as in the scalar library loop.
 */
#include <stdint.h>

void oracle_csr_spmv(int64_t n_rows, const int64_t* indptr, const int32_t* indices, const double* data,
                     const double* x, double* y, int threads) {
#pragma omp parallel for schedule(static) num_threads(threads)
  for (int64_t i = 0; i < n_rows; ++i) {
    double acc = 0.0;
    for (int64_t k = indptr[i]; k < indptr[i + 1]; ++k) acc += data[k] * x[indices[k]];
    y[i] = acc;
  }
}
