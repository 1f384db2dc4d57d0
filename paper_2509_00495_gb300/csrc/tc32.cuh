// tc32.cuh -- FP32 block products of stage 1 on the tcgen05 tensor cores.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

// One "panel" product of a block round R of the stage-1 ordering (blocks of
// 16 indices, nb blocks, block pair q of round R covering the 32 indices
// I_q = block I_q.x ∪ block I_q.y):
//   Out[:, I_q] = In[:, I_q] * U_q        for every block pair q,
// with In, Out N x N column-major FP32 (N a multiple of 32) and U_q the
// 32 x 32 column-major orthogonal factors Ubuf + q*1024.  transpose_out
// stores Out^T instead (Out(I_q[j], r) = result(r, j)).  In2/Out2 (optional,
// same shape) get the same product in the same launch, stored untransposed.
// In and Out may alias only when transpose_out is 0 (each CTA reads its
// tile before writing it).  The products run as 3xTF32 (hi*hi + hi*lo +
// lo*hi) on tcgen05.mma with the accumulators in tensor memory.  Timeouts of
// the completion wait set MPJ_FLAG_TIMEOUT in *flags.
// no_commit (tests only) issues no MMA and no commit, so every CTA's bounded
// wait runs out: the kernel sets MPJ_FLAG_TIMEOUT, frees its tensor memory and
// returns without touching Out.
cudaError_t mpj_tc_panel(int N, int nb, int R, const float* Ubuf, const float* In, float* Out, int transpose_out,
                         const float* In2, float* Out2, unsigned* flags, cudaStream_t s, int no_commit = 0);
