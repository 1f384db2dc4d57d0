// ns_fast.cuh -- FP32 evaluation of a tiny Newton-Schulz correction (ns_fast.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

// Scratch bytes for mpj_ns_fp32_correction.
size_t mpj_ns_fast_bytes(int n);

// Given M = X^T X (n x n FP64, ld n), overwrite M with E = I - M and, if
// max|E| <= 2^-31 / sqrt(n), write Y = X + X E / 2 with X E evaluated in FP32 and
// return 0.  Otherwise return 1 and leave Y untouched (M holds E).  Negative
// values are mpj_status errors.  *max_e (may be null) receives max|E|.
int mpj_ns_fp32_correction(int n, const double* X, double* M, double* Y, void* work, double* max_e, cudaStream_t s);
