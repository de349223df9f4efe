/*
 * Oracle for the sgemm dataflow graph: the plain definition in FP64.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this file;
 * only tests/, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header or constant with the CUDA library.
 *
 * What it computes (Section 6.1, the SgemmLeaf of the sgemm example, whose
 * arguments are A, lda, B, ldb, C, ldc, k, alpha, beta with A and B read-only
 * and C read and written, Section 2.3 on in/out attributes):
 *
 *     C[i,j] <- alpha * sum_{p<K} opA(i,p) * opB(p,j) + beta * C[i,j]
 *
 * for 0 <= i < M, 0 <= j < N. Storage is column-major: element (r,c) of a
 * matrix with leading dimension ld lives at r + c*ld. opA(i,p) is A(i,p) when
 * transA == 0 and A(p,i) when transA != 0; likewise opB(p,j) is B(p,j) or
 * B(j,p). FP32 inputs are widened to FP64 exactly; the sum runs in FP64 in
 * increasing p. When beta == 0, C is not read (a NaN in C does not
 * propagate). The result is written as FP64 into a separate column-major
 * buffer `out` with leading dimension ldo.
 *
 * Built with -ffp-contract=off so no multiply-add is fused: the result does
 * not depend on the host architecture.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline double op_elem(const float* X, int64_t ld, int trans,
                             int64_t r, int64_t c) {
  /* element (r, c) of op(X) */
  return trans ? (double)X[c + r * ld] : (double)X[r + c * ld];
}

/* Block [i0, i0+bm) x [j0, j0+bn) of the result.
 *
 * The rows of op(A) and the columns of op(B) that the block needs are first
 * copied (widened to FP64, no arithmetic) into contiguous panels so the sum
 * over p walks memory in order; the sum itself is the definition above.
 * Returns 0, or -1 when the panels cannot be allocated. */
int oracle_sgemm_block_f64(int transA, int transB, int64_t M, int64_t N,
                           int64_t K, double alpha, const float* A,
                           int64_t lda, const float* B, int64_t ldb,
                           double beta, const float* C, int64_t ldc,
                           int64_t i0, int64_t j0, int64_t bm, int64_t bn,
                           double* out, int64_t ldo) {
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i0 + bm > M) bm = M - i0;
  if (j0 + bn > N) bn = N - j0;
  if (bm <= 0 || bn <= 0) return 0;
  const int64_t kk = K > 0 ? K : 1;
  double* pa = (double*)malloc(sizeof(double) * (size_t)(bm * kk));
  double* pb = (double*)malloc(sizeof(double) * (size_t)(bn * kk));
  if (!pa || !pb) {
    free(pa);
    free(pb);
    return -1;
  }
  for (int64_t ii = 0; ii < bm; ++ii)
    for (int64_t p = 0; p < K; ++p)
      pa[ii * kk + p] = op_elem(A, lda, transA, i0 + ii, p);
  for (int64_t jj = 0; jj < bn; ++jj)
    for (int64_t p = 0; p < K; ++p)
      pb[jj * kk + p] = op_elem(B, ldb, transB, p, j0 + jj);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t jj = 0; jj < bn; ++jj) {
    const int64_t j = j0 + jj;
    const double* bcol = pb + jj * kk;
    for (int64_t ii = 0; ii < bm; ++ii) {
      const int64_t i = i0 + ii;
      const double* arow = pa + ii * kk;
      double s = 0.0;
      for (int64_t p = 0; p < K; ++p) s += arow[p] * bcol[p];
      double r = alpha * s;
      if (beta != 0.0) r += beta * (double)C[i + j * ldc];
      out[ii + jj * ldo] = r;
    }
  }
  free(pa);
  free(pb);
  return 0;
}

/* The whole M x N result. */
int oracle_sgemm_f64(int transA, int transB, int64_t M, int64_t N, int64_t K,
                      double alpha, const float* A, int64_t lda,
                      const float* B, int64_t ldb, double beta,
                      const float* C, int64_t ldc, double* out, int64_t ldo) {
  return oracle_sgemm_block_f64(transA, transB, M, N, K, alpha, A, lda, B, ldb,
                                beta, C, ldc, 0, 0, M, N, out, ldo);
}

/* Set the number of OpenMP threads (ignored when built without OpenMP). */
void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Number of OpenMP threads the loops above use (1 when built without it). */
int oracle_num_threads(void) {
#ifdef _OPENMP
  int n = 1;
#pragma omp parallel
  {
#pragma omp single
    n = omp_get_num_threads();
  }
  return n;
#else
  return 1;
#endif
}
