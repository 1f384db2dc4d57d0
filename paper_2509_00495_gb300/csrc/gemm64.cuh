// gemm64.cuh -- launcher interface of the FP64 DMMA matrix-product kernel.
#pragma once
#include <cuda_runtime.h>

// D = alpha op(A) op(B) + beta Cin (Cin may alias C; ignored when beta == 0).
// op(A) is m x k, op(B) is k x n, all column-major.  Matrix b of a batch
// starts at X + b * strideX.  sym != 0: m == n and the result is known to be
// symmetric; only tiles on or below the diagonal are computed and every lower
// entry is also written to its mirror position.
struct GemmArgs {
  int m, n, k;
  double alpha, beta;
  const double* A;
  int lda;
  long long strideA;
  const double* B;
  int ldb;
  long long strideB;
  const double* Cin;
  int ldcin;
  long long strideCin;
  double* C;
  int ldc;
  long long strideC;
  int sym;
};

cudaError_t mpj_gemm64_launch(const GemmArgs& g, bool transA, bool transB, int batch, cudaStream_t stream);

// Convenience: one product, no batch.
inline cudaError_t mpj_gemm64(bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
                              const double* B, int ldb, double beta, const double* Cin, int ldcin, double* C,
                              int ldc, int sym, cudaStream_t s) {
  GemmArgs g{m, n, k, alpha, beta, A, lda, 0, B, ldb, 0, Cin, ldcin, 0, C, ldc, 0, sym};
  return mpj_gemm64_launch(g, ta, tb, 1, s);
}
