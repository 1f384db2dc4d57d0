// stage1.cuh -- FP32 block round-robin Jacobi (stage 1 of the mixed method).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

int mpj_stage1_padded(int n);     // N: n rounded up to a multiple of 32
size_t mpj_stage1_bytes(int n);   // workspace bytes for mpj_stage1_run

// Q_l = double(V32) from an FP32 Jacobi on fl32(A).  `work` holds
// mpj_stage1_bytes(n); `partial` (256 doubles) and `dscal` (1 double) are
// device scratch for the off(A32) reduction.  Synchronizes `s` once per sweep.
// half: the half-precision stage (values and rotation parameters rounded to
// binary16, skip test at 2^-11).  sparse: the products contract only over the
// indices of each block pair that rotated (for a nearly diagonal A, where
// rotations thin out; the same result as the dense products).
int mpj_stage1_run(int n, const double* A, int lda, double* Ql, int ldq, double tol32, int max_sweeps,
                   int* sweeps_out, double* off_out, void* work, double* partial, double* dscal, cudaStream_t s,
                   bool half = false, bool sparse = false);
