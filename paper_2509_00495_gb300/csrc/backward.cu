// backward.cu -- eigen-adjoint of the symmetric eigensolver (not in the paper;
// the standard first-order perturbation result, e.g. Giles 2008, "Collected
// matrix derivative results"):
//   M = Q^T dQ,  G_ii = dW_i,  G_ij = M_ij / (w_j - w_i) (i != j),
//   dA = sym(Q G Q^T) = Q sym(G) Q^T,  sym(X) = (X + X^T)/2.
// Symmetrizing G first makes the last product symmetric in exact arithmetic,
// so dA is written exactly symmetric (its lower triangle mirrored).  The three
// products run as FP64-accurate products on the tensor cores (exact bf16
// slices, ozaki.cu; Q sliced once per matrix for the two products it enters
// from the same side), the matrices spread over side streams so that several
// small products share the GPU, or with MPJ_GEMM_TC=0 on the FP64 DMMA kernel,
// batched over blockIdx.z (the last one as a lower-tile product).
#include "common.cuh"
#include "gemm64.cuh"
#include "ozaki.cuh"

namespace {

// Gs = sym(G) from M (may be null: M = 0), w, dW (may be null: dW = 0).
__global__ void adjoint_core(const double* __restrict__ M, const double* __restrict__ W,
                             const double* __restrict__ dW, int n, double* __restrict__ Gs,
                             unsigned* __restrict__ flags) {
  const int b = blockIdx.z;
  const double* w = W + (size_t)b * n;
  const double* Mb = M ? M + (size_t)b * n * n : nullptr;
  double* G = Gs + (size_t)b * n * n;
  int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double g;
    if (i == j) {
      g = dW ? dW[(size_t)b * n + i] : 0.0;
    } else {
      double mij = Mb ? Mb[(size_t)j * n + i] : 0.0;  // M(i,j)
      double mji = Mb ? Mb[(size_t)i * n + j] : 0.0;  // M(j,i)
      double gap = w[j] - w[i];
      double gij = 0.0, gji = 0.0;
      if (gap == 0.0) {
        if (mij != 0.0 || mji != 0.0) atomicOr(flags, MPJ_FLAG_DEGENERATE);
      } else {
        gij = mij / gap;   // F_ij M_ij, F_ij = 1/(w_j - w_i)
        gji = mji / -gap;  // F_ji M_ji
      }
      g = 0.5 * (gij + gji);
    }
    G[(size_t)j * n + i] = g;
  }
}

// B(j, i) = B(i, j) for i > j (the lower triangle mirrored), batched over blockIdx.y
__global__ void bwd_mirror(double* __restrict__ B, int ldb, long long sb, int n) {
  double* Bb = B + (size_t)blockIdx.y * sb;
  const size_t total = (size_t)n * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    if (i > j) Bb[(size_t)i * ldb + j] = Bb[(size_t)j * ldb + i];
  }
}

}  // namespace

extern "C" int mpj_syev_backward(int batch, int n, const double* W, const double* Q, int ldq, const double* dW,
                                 const double* dQ, int lddq, double* dA, int ldda, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (batch < 0 || n < 0 || ldq < n || lddq < n || ldda < n || ldq < 1 || lddq < 1 || ldda < 1) return MPJ_EINVAL;
  if (batch == 0 || n == 0) return MPJ_OK;
  if (!W || !Q || !dA) return MPJ_EINVAL;
  size_t sq = (size_t)n * n;
  const bool tc = mpj_gemm_tc_enabled();
  // tensor-core products: matrices spread over up to BW side streams (one
  // product of a small matrix does not fill the GPU), three sliced operands each
  constexpr int BW = 8;
  const int nw = tc ? (batch < BW ? batch : BW) : 0;
  const size_t ob = tc ? (mpj_oz_operand_bytes(n, n) + 255) / 256 * 256 : 0;
  void* w = nullptr;
  size_t bytes = 2 * (size_t)batch * sq * sizeof(double) + 256 + 3 * ob * (size_t)nw;
  if (cudaMallocAsync(&w, bytes, s) != cudaSuccess) return MPJ_ENOMEM;
  mpj_count_alloc();
  double* M = (double*)w;
  double* T = M + (size_t)batch * sq;
  unsigned* flags = (unsigned*)(T + (size_t)batch * sq);
  char* obuf = (char*)flags + 256;  // three sliced operands per side stream (tensor-core products)
  int st = MPJ_OK;
  unsigned hflags = 0;
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned), s);
  cudaStream_t ws[BW] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[BW] = {};
  if (e == cudaSuccess && tc) {
    e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < nw && e == cudaSuccess; ++i) {
      e = cudaStreamCreateWithFlags(&ws[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_join[i], cudaEventDisableTiming);
    }
  }
  // side streams start after everything issued so far on s, and s continues
  // after all of them
  auto fork = [&]() -> cudaError_t {
    cudaError_t r = cudaEventRecord(ev_fork, s);
    for (int i = 0; i < nw && r == cudaSuccess; ++i) r = cudaStreamWaitEvent(ws[i], ev_fork, 0);
    return r;
  };
  auto join = [&]() -> cudaError_t {
    cudaError_t r = cudaSuccess;
    for (int i = 0; i < nw && r == cudaSuccess; ++i) {
      r = cudaEventRecord(ev_join[i], ws[i]);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(s, ev_join[i], 0);
    }
    return r;
  };
  long long sQ = (long long)ldq * n, sdQ = (long long)lddq * n, sA = (long long)ldda * n, sN = (long long)sq;
  if (e == cudaSuccess && dQ) {  // M = Q^T dQ
    if (tc) {
      e = fork();
      for (int b = 0; b < batch && e == cudaSuccess; ++b) {
        cudaStream_t sb = ws[b % nw];
        char* ob0 = obuf + 3 * ob * (size_t)(b % nw);
        OzOperand oq, od;  // rows of Q^T (columns of Q) and columns of dQ, over the row index
        e = mpj_oz_prepare(Q + b * sQ, ldq, 1, n, n, ob0, &oq, sb);
        if (e == cudaSuccess) e = mpj_oz_prepare(dQ + b * sdQ, lddq, 1, n, n, ob0 + ob, &od, sb);
        if (e == cudaSuccess) e = mpj_oz_gemm(oq, od, n, n, 1.0, 0.0, nullptr, n, M + b * sN, n, flags, sb);
      }
      if (e == cudaSuccess) e = join();
    } else {
      GemmArgs g{n, n, n, 1.0, 0.0, Q, ldq, sQ, dQ, lddq, sdQ, nullptr, n, 0, M, n, sN, 0};
      e = mpj_gemm64_launch(g, true, false, batch, s);
    }
  }
  if (e == cudaSuccess) {  // T = sym(G) (into T), then M = Q T, then dA = M Q^T (symmetric)
    dim3 grid((n + 255) / 256 > 8 ? 8 : (n + 255) / 256, n, batch);
    adjoint_core<<<grid, 256, 0, s>>>(dQ ? M : nullptr, W, dW, n, T, flags);
    mpj_count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && tc) {
    e = fork();
    for (int b = 0; b < batch && e == cudaSuccess; ++b) {
      cudaStream_t sb = ws[b % nw];
      char* ob0 = obuf + 3 * ob * (size_t)(b % nw);
      OzOperand oq, ot, om;  // rows of Q (left of Q T, right of M Q^T), columns of T, rows of M
      e = mpj_oz_prepare(Q + b * sQ, 1, ldq, n, n, ob0, &oq, sb);
      if (e == cudaSuccess) e = mpj_oz_prepare(T + b * sN, n, 1, n, n, ob0 + ob, &ot, sb);
      if (e == cudaSuccess) e = mpj_oz_gemm(oq, ot, n, n, 1.0, 0.0, nullptr, n, M + b * sN, n, flags, sb);
      if (e == cudaSuccess) e = mpj_oz_prepare(M + b * sN, 1, n, n, n, ob0 + 2 * ob, &om, sb);
      if (e == cudaSuccess) e = mpj_oz_gemm(om, oq, n, n, 1.0, 0.0, nullptr, n, dA + b * sA, ldda, flags, sb);
    }
    if (e == cudaSuccess) e = join();
    if (e == cudaSuccess) {
      const size_t blocks = (sq + 255) / 256;
      bwd_mirror<<<dim3((unsigned)(blocks > 1024 ? 1024 : blocks), batch), 256, 0, s>>>(dA, ldda, sA, n);
      mpj_count_launch();
      e = cudaGetLastError();
    }
  } else if (e == cudaSuccess) {
    GemmArgs g{n, n, n, 1.0, 0.0, Q, ldq, sQ, T, n, sN, nullptr, n, 0, M, n, sN, 0};
    e = mpj_gemm64_launch(g, false, false, batch, s);
    if (e == cudaSuccess) {
      GemmArgs g2{n, n, n, 1.0, 0.0, M, n, sN, Q, ldq, sQ, nullptr, n, 0, dA, ldda, sA, 1};
      e = mpj_gemm64_launch(g2, false, true, batch, s);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "mpj_syev_backward", __LINE__);
    st = MPJ_ECUDA;
  }
  if (tc && ev_fork) {
    // whatever the error path, s must not run ahead of the side streams'
    // work before the workspace is released
    for (int i = 0; i < nw; ++i)
      if (ws[i] && ev_join[i] && cudaEventRecord(ev_join[i], ws[i]) == cudaSuccess)
        cudaStreamWaitEvent(s, ev_join[i], 0);
  }
  cudaFreeAsync(w, s);
  e = cudaStreamSynchronize(s);
  for (int i = 0; i < nw; ++i) {
    if (ws[i]) cudaStreamDestroy(ws[i]);
    if (ev_join[i]) cudaEventDestroy(ev_join[i]);
  }
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (e != cudaSuccess && st >= 0) {
    mpj_set_cuda_error(e, "mpj_syev_backward sync", __LINE__);
    st = MPJ_ECUDA;
  }
  if (st == MPJ_OK && (hflags & MPJ_FLAG_DEGENERATE)) st = MPJ_EDEGENERATE;
  if (st == MPJ_OK && (hflags & MPJ_FLAG_TIMEOUT)) st = MPJ_ETIMEOUT;
  return st;
}
