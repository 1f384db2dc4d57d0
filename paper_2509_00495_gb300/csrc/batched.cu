// batched.cu -- many independent symmetric eigenproblems (sizes 1..256) in one
// persistent launch.  Not in the paper: each matrix runs the mixed method of
// Algorithm 9 (Sec. 5.1) on its own, inside one CTA.
//
// One CTA of 1024 threads per SM pulls matrix indices from an atomic work
// queue ordered by decreasing n (longest job first).  For its matrix the CTA
//   1. FP32 round-robin Jacobi on fl32(A) from V32 = I until
//      off(A32) <= n 2^-24 ||A||_F (cap max32), Q_l = double(V32);
//   2. Newton-Schulz X <- 1.5 X - 0.5 X (X^T X), ns_steps times (FP64 DMMA);
//   3. A_cond = X^T (A X) (FP64 DMMA, lower tiles mirrored);
//   4. FP64 round-robin Jacobi on A_cond from V = I until off <= tol (cap max64);
//   5. W = sorted diag, Q = X V (columns permuted), written to the caller.
// The round-robin ordering, the rotation records and the 2x2-block update
// are those of the single-matrix kernels (common.cuh); here one round is one
// __syncthreads-separated phase of the CTA.  The CTA's matrices live in a
// per-CTA slice of global workspace (L2-resident for the most part); FP64 is
// the bound: GB300 issues about 2 FP64 FMA per clock per SM, so the batch
// costs its total FP64 work over 152 SMs.
#include "common.cuh"

namespace {

constexpr int NTH = 1024;
constexpr int NMAX = 256;

struct CtaBufs {
  float* A32;
  float* V32;
  double* X;
  double* M;
  double* Y;
  double* Vp;  // aliases A32/V32 after stage 1
};

MPJ_DEV double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

MPJ_DEV void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// CTA-level D = alpha op(A) op(B) + beta Cin (n x n, column-major, ld n for
// A/B/C unless given), warp tasks of 16 x 16 outputs on m8n8k4 DMMA.
template <bool TA, bool TB>
MPJ_DEV void cta_gemm(int n, double alpha, const double* A, int lda, const double* B, int ldb, double beta,
                      const double* Cin, double* C, int ldc, bool sym) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int nt = (n + 15) / 16;
  for (int t = warp; t < nt * nt; t += nw) {
    int ti = t % nt, tj = t / nt;
    if (sym && ti < tj) continue;
    int m0 = ti * 16, n0 = tj * 16;
    double acc[2][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
    for (int k = 0; k < n; k += 4) {
      int kk = k + tig;
      double af[2], bf[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        int r = m0 + i * 8 + gid;
        af[i] = (r < n && kk < n) ? (TA ? A[(size_t)r * lda + kk] : A[(size_t)kk * lda + r]) : 0.0;
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        int c = n0 + j * 8 + gid;
        bf[j] = (c < n && kk < n) ? (TB ? B[(size_t)kk * ldb + c] : B[(size_t)c * ldb + kk]) : 0.0;
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          int r = m0 + i * 8 + gid, c = n0 + j * 8 + tig * 2 + e;
          if (r >= n || c >= n || (sym && r < c)) continue;
          double v = alpha * acc[i][j][e];
          if (beta != 0.0) v = fma(beta, Cin[(size_t)c * ldc + r], v);
          C[(size_t)c * ldc + r] = v;
          if (sym && r != c) C[(size_t)r * ldc + c] = v;
        }
  }
  __syncthreads();
}

// One round-robin Jacobi sweep at CTA level on a symmetric n x n matrix A
// (ld n) with vectors V (ld n).  rec: m/2 records in shared memory.
template <typename T>
MPJ_DEV void cta_rr_sweep(int n, T* A, T* V, RotRec<T>* rec, T skip) {
  const int m = n + (n & 1), h = m / 2;
  for (int r = 0; r < m - 1; ++r) {
    for (int i = threadIdx.x; i < h; i += blockDim.x) {
      int x, y;
      rr_slot(m, r, i, x, y);
      T dx = x < n ? A[(size_t)x * n + x] : T(0);
      T dy = y < n ? A[(size_t)y * n + y] : T(0);
      T axy = (x < n && y < n) ? A[(size_t)y * n + x] : T(0);
      RotRec<T> rr;
      rr_make_rec<T>(m, n, r, x, y, dx, dy, axy, skip, rr);
      rec[i] = rr;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < h * h; e += blockDim.x) {
      int a = e % h, b = e / h;
      if (a < b) continue;
      RotRec<T> ra = rec[a];
      bool rota = rec_rotated(ra.cm1, ra.sig);
      int xa, ya, xb, yb;
      rr_slot(m, r, a, xa, ya);
      if (a == b) {
        if (rota) {
          A[(size_t)xa * n + xa] = ra.dx;
          A[(size_t)ya * n + ya] = ra.dy;
          A[(size_t)ya * n + xa] = T(0);
          A[(size_t)xa * n + ya] = T(0);
        }
        continue;
      }
      RotRec<T> rb = rec[b];
      bool rotb = rec_rotated(rb.cm1, rb.sig);
      if (!rota && !rotb) continue;
      rr_slot(m, r, b, xb, yb);
      bool vxa = xa < n, vya = ya < n, vxb = xb < n, vyb = yb < n;
      T vxx = (vxa && vxb) ? A[(size_t)xb * n + xa] : T(0);
      T vxy = (vxa && vyb) ? A[(size_t)yb * n + xa] : T(0);
      T vyx = (vya && vxb) ? A[(size_t)xb * n + ya] : T(0);
      T vyy = (vya && vyb) ? A[(size_t)yb * n + ya] : T(0);
      if (rota) {
        rot_apply(ra.cm1, ra.sig, vxx, vyx);
        rot_apply(ra.cm1, ra.sig, vxy, vyy);
      }
      if (rotb) {
        rot_apply(rb.cm1, rb.sig, vxx, vxy);
        rot_apply(rb.cm1, rb.sig, vyx, vyy);
      }
      if (vxa && vxb) A[(size_t)xb * n + xa] = A[(size_t)xa * n + xb] = vxx;
      if (vxa && vyb) A[(size_t)yb * n + xa] = A[(size_t)xa * n + yb] = vxy;
      if (vya && vxb) A[(size_t)xb * n + ya] = A[(size_t)ya * n + xb] = vyx;
      if (vya && vyb) A[(size_t)yb * n + ya] = A[(size_t)ya * n + yb] = vyy;
    }
    for (int e = threadIdx.x; e < n * h; e += blockDim.x) {
      int row = e % n, b = e / n;
      RotRec<T> rb = rec[b];
      if (!rec_rotated(rb.cm1, rb.sig)) continue;
      int xb, yb;
      rr_slot(m, r, b, xb, yb);
      T vx = V[(size_t)xb * n + row], vy = V[(size_t)yb * n + row];
      rot_apply(rb.cm1, rb.sig, vx, vy);
      V[(size_t)xb * n + row] = vx;
      V[(size_t)yb * n + row] = vy;
    }
    __syncthreads();
  }
}

template <typename T>
MPJ_DEV double cta_off2(int n, const T* A, double* red) {
  double s = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e % n, j = e / n;
    if (i != j) {
      double x = (double)A[e];
      s += x * x;
    }
  }
  return block_sum(s, red);
}

__global__ void __launch_bounds__(NTH, 1)
    batched_syev(const int* __restrict__ order, const int* __restrict__ nvec, const double* const* __restrict__ Aptr,
                 double* const* __restrict__ Wptr, double* const* __restrict__ Qptr, int batch, double tol_in,
                 int max32, int max64, int ns_steps, char* __restrict__ work, size_t per_cta, int* __restrict__ counter,
                 int* __restrict__ sweeps_out, unsigned* __restrict__ flags) {
  __shared__ double red[33];
  __shared__ RotRec<double> rec64[NMAX / 2 + 1];
  __shared__ RotRec<float> rec32[NMAX / 2 + 1];
  __shared__ int job;
  __shared__ int rank_sh[NMAX];
  char* base = work + (size_t)blockIdx.x * per_cta;
  CtaBufs B;
  B.A32 = (float*)base;
  B.V32 = B.A32 + NMAX * NMAX;
  B.Vp = (double*)base;
  B.X = (double*)(base + 2 * (size_t)NMAX * NMAX * sizeof(float));
  B.M = B.X + NMAX * NMAX;
  B.Y = B.M + NMAX * NMAX;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) job = atomicAdd(counter, 1);
    __syncthreads();
    const int jb = job;
    __syncthreads();
    if (jb >= batch) break;
    const int idx = order[jb];
    const int n = nvec[idx];
    const double* A = Aptr[idx];
    double* W = Wptr[idx];
    double* Q = Qptr[idx];
    // a0: norms and finiteness
    double s = 0.0;
    bool bad = false;
    for (int e = tid; e < n * n; e += NTH) {
      double x = A[e];
      if (!isfinite(x)) bad = true;
      s += x * x;
    }
    if (bad) atomicOr(flags, MPJ_FLAG_NONFINITE);
    double normA = sqrt(block_sum(s, red));
    double tol = tol_in > 0 ? tol_in : (double)n * 0x1p-53 * normA;
    double tol32 = (double)n * 0x1p-24 * normA;
    // 1. stage 1 (FP32 round-robin)
    for (int e = tid; e < n * n; e += NTH) {
      B.A32[e] = (float)A[e];
      B.V32[e] = (e % n == e / n) ? 1.0f : 0.0f;
    }
    __syncthreads();
    for (int sw = 0; sw < max32; ++sw) {
      double off2 = cta_off2<float>(n, B.A32, red);
      if (!(off2 > tol32 * tol32)) break;
      cta_rr_sweep<float>(n, B.A32, B.V32, rec32, 0x1p-24f);
    }
    for (int e = tid; e < n * n; e += NTH) B.X[e] = (double)B.V32[e];
    __syncthreads();
    // 2. Newton-Schulz
    double* X = B.X;
    double* Y = B.Y;
    for (int k = 0; k < ns_steps; ++k) {
      cta_gemm<true, false>(n, 1.0, X, n, X, n, 0.0, nullptr, B.M, n, true);
      cta_gemm<false, false>(n, -0.5, X, n, B.M, n, 1.5, X, Y, n, false);
      double* t = X;
      X = Y;
      Y = t;
    }
    // 3. A_cond = X^T (A X) -> M
    cta_gemm<false, false>(n, 1.0, A, n, X, n, 0.0, nullptr, Y, n, false);
    cta_gemm<true, false>(n, 1.0, X, n, Y, n, 0.0, nullptr, B.M, n, true);
    // 4. FP64 sweeps, V = Y from I
    double* V = Y;
    for (int e = tid; e < n * n; e += NTH) V[e] = (e % n == e / n) ? 1.0 : 0.0;
    __syncthreads();
    int sweeps = 0;
    for (;;) {
      double off2 = cta_off2<double>(n, B.M, red);
      if (!(off2 > tol * tol) || n < 2) break;
      if (sweeps >= max64) {
        if (tid == 0) atomicOr(flags, MPJ_FLAG_TIMEOUT);  // cap reached: reported as not converged
        break;
      }
      cta_rr_sweep<double>(n, B.M, V, rec64, 0x1p-53);
      ++sweeps;
    }
    // 5. sort, permute, Q = X Vp
    for (int i = tid; i < n; i += NTH) {
      double wi = B.M[(size_t)i * n + i];
      int r = 0;
      for (int j = 0; j < n; ++j) {
        double wj = B.M[(size_t)j * n + j];
        r += (wj < wi) || (wj == wi && j < i);
      }
      rank_sh[i] = r;
      W[r] = wi;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += NTH) {
      int i = e % n, j = e / n;
      B.Vp[(size_t)rank_sh[j] * n + i] = V[e];
    }
    __syncthreads();
    cta_gemm<false, false>(n, 1.0, X, n, B.Vp, n, 0.0, nullptr, Q, n, false);
    if (tid == 0) sweeps_out[idx] = sweeps;
    __syncthreads();
  }
}

}  // namespace

extern "C" int mpj_syev_batched(int batch, const int* n_host, const double* const* A_dev, double* const* W_dev,
                                double* const* Q_dev, double tol, int* sweeps_host, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (batch < 0 || (batch > 0 && (!n_host || !A_dev || !W_dev || !Q_dev))) return MPJ_EINVAL;
  if (batch == 0) return MPJ_OK;
  for (int i = 0; i < batch; ++i)
    if (n_host[i] < 1 || n_host[i] > NMAX) return MPJ_EINVAL;
  int dev = 0, sms = 0;
  MPJ_CUDA_TRY(cudaGetDevice(&dev));
  MPJ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int grid = sms < batch ? sms : batch;
  // longest job first: order by decreasing n, ties by index
  int* order = (int*)malloc(sizeof(int) * (size_t)batch);
  for (int i = 0; i < batch; ++i) order[i] = i;
  // counting sort on n (1..NMAX), descending
  {
    int cnt[NMAX + 2] = {0};
    for (int i = 0; i < batch; ++i) cnt[n_host[i]]++;
    int start[NMAX + 2];
    int acc = 0;
    for (int v = NMAX; v >= 1; --v) {
      start[v] = acc;
      acc += cnt[v];
    }
    for (int i = 0; i < batch; ++i) order[start[n_host[i]]++] = i;
  }
  size_t per_cta = 2 * (size_t)NMAX * NMAX * sizeof(float) + 3 * (size_t)NMAX * NMAX * sizeof(double);
  size_t small = 2 * (size_t)batch * sizeof(int) + (size_t)batch * sizeof(int) + 64;
  void* w = nullptr;
  cudaError_t e = cudaMallocAsync(&w, per_cta * grid + small, s);
  if (e != cudaSuccess) {
    free(order);
    mpj_set_cuda_error(e, "batched workspace", __LINE__);
    return MPJ_ENOMEM;
  }
  char* work = (char*)w;
  int* d_order = (int*)(work + per_cta * grid);
  int* d_n = d_order + batch;
  int* d_sweeps = d_n + batch;
  int* d_counter = d_sweeps + batch;
  unsigned* d_flags = (unsigned*)(d_counter + 1);
  int st = MPJ_OK;
  unsigned hflags = 0;
  e = cudaMemcpyAsync(d_order, order, sizeof(int) * batch, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_n, n_host, sizeof(int) * batch, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) {
    batched_syev<<<grid, NTH, 0, s>>>(d_order, d_n, A_dev, W_dev, Q_dev, batch, tol, 15, 30, 2, work, per_cta,
                                      d_counter, d_sweeps, d_flags);
    mpj_count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && sweeps_host)
    e = cudaMemcpyAsync(sweeps_host, d_sweeps, sizeof(int) * batch, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "mpj_syev_batched", __LINE__);
    st = MPJ_ECUDA;
  }
  cudaFreeAsync(w, s);
  cudaStreamSynchronize(s);
  free(order);
  if (st == MPJ_OK) {
    if (hflags & MPJ_FLAG_NONFINITE)
      st = MPJ_ENONFINITE;
    else if (hflags & MPJ_FLAG_TIMEOUT)
      st = MPJ_NOT_CONVERGED;
  }
  return st;
}
