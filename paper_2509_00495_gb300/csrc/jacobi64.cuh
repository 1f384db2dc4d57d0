// jacobi64.cuh -- FP64 Jacobi sweep driver and reductions (jacobi64.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

// Scratch (records, scales, reduction partials, V history) for mpj_jacobi64_run
// with the full 64-round V batching; _rv: with rv rounds per V batch.
// _ordering: what mpj_jacobi64_run needs for that ordering (the block
// ordering adds an n x n FP64 buffer and the digit tiles of the U_P).
size_t mpj_jacobi64_scratch_bytes(int n);
size_t mpj_jacobi64_scratch_bytes_rv(int n, int rv);
size_t mpj_jacobi64_scratch_bytes_ordering(int n, int ordering);

// Block round-robin FP64 sweeps with tensor-core block updates (blocked64.cu):
// outer round R is the subproblem solves (U_P into set R mod 2 of the
// scratch), then A <- U~^T A U~ (through the n x n buffer B) and V <- V U~,
// the two updates independent of each other; the scratch they need, rounds
// per sweep, and the end-of-sweep symmetrization.
size_t mpj_blocked_scratch_bytes(int n);
cudaError_t mpj_blocked_solve(const double* A, int lda, int n, int R, double skip, double skip_abs, void* scratch,
                              unsigned* nrot, cudaStream_t s);
cudaError_t mpj_blocked_update_A(double* A, int lda, double* B, int n, int R, void* scratch, unsigned* flags,
                                 cudaStream_t s);
cudaError_t mpj_blocked_update_V(double* V, int ldv, int n, int R, void* scratch, unsigned* flags, cudaStream_t s);
int mpj_blocked_rounds_per_sweep(int n);
cudaError_t mpj_blocked_symmetrize(double* A, int lda, int n, cudaStream_t s);

// FP64 sweeps in place (see mpjacobi.h, mpj_jacobi64).  Synchronizes `s` once
// per sweep to read off(A).  `scratch_bytes` bounds the V batching (at least
// mpj_jacobi64_scratch_bytes_rv(n, 1)).  skip_abs > 0 also skips pairs with
// |a_pq| <= skip_abs (threshold variant).  With side_stream (and n >= 256,
// room for two V batches, MPJ_JACOBI_OVERLAP not "0"), the batched V updates
// run on a private non-blocking stream, overlapping the next rounds; it is
// joined back into `s` before every scale fold, so V is complete in `s` order
// on return.  rotated_blocks_out (block ordering, if not null) receives the
// number of block-pair subproblems that rotated, summed over all rounds.
// Returns MPJ_OK / MPJ_NOT_CONVERGED / MPJ_ECUDA / MPJ_EWORKSPACE.
int mpj_jacobi64_run(int n, double* A, int lda, double* V, int ldv, double tol, int ordering, int max_sweeps,
                     int* sweeps_out, double* off_out, double* off_initial, void* scratch, size_t scratch_bytes,
                     cudaStream_t s, double skip_abs = 0.0, bool side_stream = true,
                     long long* rotated_blocks_out = nullptr);

// Sum of squares of A's entries (off_only: off-diagonal entries) into *out,
// through 256 per-CTA partials summed in a fixed order; sets
// MPJ_FLAG_NONFINITE in *flags (if not null) when an entry is NaN or Inf.
cudaError_t mpj_sumsq(const double* A, int lda, int n, bool off_only, double* partial, double* out, unsigned* flags,
                      cudaStream_t s);
cudaError_t mpj_sumsq32(const float* A, int lda, int n, double* partial, double* out, cudaStream_t s);
cudaError_t mpj_check_symmetric(const double* A, int lda, int n, unsigned* flags, cudaStream_t s);
