// ozaki.cuh -- FP64 matrix products on the tcgen05 tensor cores from exact
// bf16 slices (ozaki.cu).  Internal interface: operands are sliced once into
// caller-provided device memory and can serve several products (X^T X uses
// the same slices on both sides); products never allocate or synchronize.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

// One sliced operand: the R "rows" of op(X) (rows of op(A) for the left
// operand, columns of op(B) for the right one), each over K values of the
// contraction index, as 8 bf16 slices on the grid of the row's largest
// exponent.  Rows are padded to a multiple of 128, K to a multiple of 256.
struct OzOperand {
  const __nv_bfloat16* slices;  // 8 x Rp x Kp, 64-row x 32-k canonical K-major tiles
  const int* exps;              // Rp row exponents (max |x(r,:)| < 2^e_r; 0 for zero rows)
  int R, K, Rp, Kp;
};

// Device bytes one sliced operand of R rows and K contraction values needs.
size_t mpj_oz_operand_bytes(int R, int K);

// Slice op(X): row r, contraction index k at X[r * rs + k * ks] (rs = 1,
// ks = ld for the rows of a column-major matrix; rs = ld, ks = 1 for its
// columns).  `buf` holds mpj_oz_operand_bytes(R, K) bytes (256-byte aligned).
cudaError_t mpj_oz_prepare(const double* X, long long rs, long long ks, int R, int K, void* buf, OzOperand* op,
                           cudaStream_t s);

// C(0:m, 0:n) = alpha op(A) op(B) + beta Cin, op(A) rows from `a` (a.R >= m),
// op(B) columns from `b` (b.R >= n), a.K == b.K.  Cin may alias C (ignored
// when beta == 0).  A tensor-core completion wait that runs out sets
// MPJ_FLAG_TIMEOUT in *flags (device word, may be null).  lower: only the
// 128 x 64 output tiles that meet the lower triangle (row >= column) are
// formed, the others are left untouched (for a symmetric result whose upper
// triangle the caller mirrors from the lower one).
cudaError_t mpj_oz_gemm(const OzOperand& a, const OzOperand& b, int m, int n, double alpha, double beta,
                        const double* Cin, int ldcin, double* C, int ldc, unsigned* flags, cudaStream_t s,
                        bool lower = false);

// Whether the FP64 products of the solver and of the adjoint run on this
// engine (default) or on the FP64 DMMA kernel (environment MPJ_GEMM_TC=0).
bool mpj_gemm_tc_enabled();
