// stage1.cu -- stage 1 of the mixed algorithm: approximate eigenvectors Q_l
// from an FP32 Jacobi (the paper's stage 1 is eig(single(A)), Sec. 4.1 and
// Algorithm 9; only an approximate Q_l with ||A Q_l - Q_l D_l|| <~ n u_l ||A||
// is needed, so the FP32 stage may use any convergent Jacobi ordering).
//
// Ordering: block round-robin.  The padded index range [0, N) (N a multiple
// of 32, pads inert: zero rows/columns never rotate) is cut into nb = N/16
// blocks of 16.  A sweep is nb-1 outer rounds of the circle method on blocks;
// in each round the nb/2 disjoint block pairs (I, J) each run one inner
// round-robin sweep over the 32 indices of I u J (31 inner rounds of 16
// disjoint pairs, Algorithm 2 with the skip test of Algorithm 4 at u_l = 2^-24)
// on their 32 x 32 diagonal subproblem, held in shared memory, accumulating the
// 32 x 32 orthogonal U_IJ.  The rotations of one round touch disjoint index
// sets, so applying them to the rest of the matrix afterwards as products
//   A[P,Q] <- U_P^T A[P,Q] U_Q,   V[:,Q] <- V[:,Q] U_Q
// (P, Q = index sets of block pairs) gives the same iterates as applying them
// one by one.  Each round is two launches: the subproblem solves and the
// blocked update (FP32 FMA), which touch A32 and V32 once per round instead of
// once per pair step.  off(A32) is reduced after each sweep; stop at
// off(A32) <= tol32 or the sweep cap.
#include <cuda_fp16.h>
#include <stdlib.h>

#include "common.cuh"
#include "stage1.cuh"
#include "tc32.cuh"

namespace {

constexpr int BS = 16;  // block size
constexpr int W2 = 32;  // indices per block pair
constexpr int LD = 33;  // padded shared-memory leading dimension

// global index of local index l in block pair (I, J)
MPJ_DEV int gidx(int I, int J, int l) { return l < BS ? I * BS + l : J * BS + (l - BS); }

MPJ_DEV void block_pair(int nb, int R, int slot, int& I, int& J) {
  int x, y;
  rr_slot(nb, R, slot, x, y);
  I = x < y ? x : y;
  J = x < y ? y : x;
}

// hq: the half-precision stage (binary16 values; Ch. 6 further work item 3):
// every stored value and rotation parameter is rounded to binary16.
MPJ_DEV float qh(float v, bool hq) { return hq ? __half2float(__float2half_rn(v)) : v; }

__global__ void init32(const double* __restrict__ A, int lda, int n, int N, float* __restrict__ A32,
                       float* __restrict__ V32, bool hq) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)N * N;
  for (; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % N), j = (int)(idx / N);
    A32[idx] = (i < n && j < n) ? qh((float)A[(size_t)j * lda + i], hq) : 0.0f;
    V32[idx] = (i == j) ? 1.0f : 0.0f;
  }
}

__global__ void widen(const float* __restrict__ V32, int N, int n, double* __restrict__ Q, int ldq) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)n * n;
  for (; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    Q[(size_t)j * ldq + i] = (double)V32[(size_t)j * N + i];
  }
}

// One CTA per block pair of outer round R: inner round-robin sweep on the
// 32 x 32 subproblem; writes the rotated subproblem S and the accumulated U.
__global__ void __launch_bounds__(256) solve32(const float* __restrict__ A32, int N, int nb, int R,
                                               float* __restrict__ Sbuf, float* __restrict__ Ubuf, bool hq) {
  __shared__ float S[W2][LD];
  __shared__ float U[W2][LD];
  __shared__ RotRec<float> rec[W2 / 2];
  const int slot = blockIdx.x;
  int I, J;
  block_pair(nb, R, slot, I, J);
  const int tid = threadIdx.x;
  #pragma unroll
  for (int it = 0; it < W2 * W2 / 256; ++it) {
    const int e = tid + it * 256;
    int li = e % W2, lj = e / W2;
    S[li][lj] = A32[(size_t)gidx(I, J, lj) * N + gidx(I, J, li)];
    U[li][lj] = (li == lj) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const float skip = hq ? 0x1p-11f : 0x1p-24f;
  for (int rho = 0; rho < W2 - 1; ++rho) {
    if (tid < W2 / 2) {
      int x, y;
      rr_slot(W2, rho, tid, x, y);
      RotRec<float> rr;
      rr_make_rec<float>(W2, W2, rho, x, y, S[x][x], S[y][y], S[y][x], skip, rr);
      if (hq && rec_rotated(rr.cm1, rr.sig)) {  // c and s as binary16, new diagonal rounded
        rr.cm1 = qh(1.0f + rr.cm1, true) - 1.0f;
        rr.sig = qh(rr.sig, true);
        rr.dx = qh(rr.dx, true);
        rr.dy = qh(rr.dy, true);
      }
      rec[tid] = rr;
    }
    __syncthreads();
    {
      int a = tid % 16, b = tid / 16;
      if (a >= b) {
        int xa, ya, xb, yb;
        rr_slot(W2, rho, a, xa, ya);
        rr_slot(W2, rho, b, xb, yb);
        RotRec<float> ra = rec[a], rb = rec[b];
        bool rota = rec_rotated(ra.cm1, ra.sig), rotb = rec_rotated(rb.cm1, rb.sig);
        if (a == b) {
          if (rota) {
            S[xa][xa] = ra.dx;
            S[ya][ya] = ra.dy;
            S[xa][ya] = 0.0f;
            S[ya][xa] = 0.0f;
          }
        } else if (rota || rotb) {
          float vxx = S[xa][xb], vxy = S[xa][yb], vyx = S[ya][xb], vyy = S[ya][yb];
          if (rota) {
            rot_apply(ra.cm1, ra.sig, vxx, vyx);
            rot_apply(ra.cm1, ra.sig, vxy, vyy);
          }
          if (rotb) {
            rot_apply(rb.cm1, rb.sig, vxx, vxy);
            rot_apply(rb.cm1, rb.sig, vyx, vyy);
          }
          vxx = qh(vxx, hq);
          vxy = qh(vxy, hq);
          vyx = qh(vyx, hq);
          vyy = qh(vyy, hq);
          S[xa][xb] = vxx;
          S[xb][xa] = vxx;
          S[xa][yb] = vxy;
          S[yb][xa] = vxy;
          S[ya][xb] = vyx;
          S[xb][ya] = vyx;
          S[ya][yb] = vyy;
          S[yb][ya] = vyy;
        }
      }
      // U <- U J: rows of U are independent; columns x_b, y_b
      for (int e = tid; e < W2 * (W2 / 2); e += 256) {
        int row = e % W2, sb = e / W2;
        RotRec<float> rb = rec[sb];
        if (!rec_rotated(rb.cm1, rb.sig)) continue;
        int xb, yb;
        rr_slot(W2, rho, sb, xb, yb);
        float ux = U[row][xb], uy = U[row][yb];
        rot_apply(rb.cm1, rb.sig, ux, uy);
        U[row][xb] = qh(ux, hq);
        U[row][yb] = qh(uy, hq);
      }
    }
    __syncthreads();
  }
  float* So = Sbuf + (size_t)slot * W2 * W2;
  float* Uo = Ubuf + (size_t)slot * W2 * W2;
  #pragma unroll
  for (int it = 0; it < W2 * W2 / 256; ++it) {
    const int e = tid + it * 256;
    int li = e % W2, lj = e / W2;
    So[e] = S[li][lj];
    Uo[e] = U[li][lj];
  }
}

__device__ __forceinline__ void tri_tile(int t, int nt, int& ti, int& tj) {
  tj = 0;
  while (t >= nt - tj) {
    t -= nt - tj;
    ++tj;
  }
  ti = tj + t;
}

// Blocked application of the round's U's: lower tiles of A32 (with mirror)
// and 32-row tiles of V32.  One 64-thread CTA per 32 x 32 tile; each thread
// owns a 4 x 4 block of the result, so every pair of float4 shared-memory
// loads feeds 16 FMAs.
constexpr int UT = 64;  // threads per update tile
constexpr int LD4 = 36; // padded row length (keeps rows 16-byte aligned)

// acc[a][b] = sum_l Lt[l][i4 + a] * R[l][j4 + b]  (a 4 x 4 block of Lt^T R, both
// operands 32 x 32 row-major in shared memory).
MPJ_DEV void tile_mm(const float (*Lt)[LD4], const float (*R)[LD4], float acc[4][4], int i4, int j4) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll 8
  for (int l = 0; l < W2; ++l) {
    float4 x = *reinterpret_cast<const float4*>(&Lt[l][i4]);  // op(L)[i4..i4+3][l]
    float4 y = *reinterpret_cast<const float4*>(&R[l][j4]);   // R[l][j4..j4+3]
    float xa[4] = {x.x, x.y, x.z, x.w}, yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xa[a], yb[b], acc[a][b]);
  }
}

// all tile loads unrolled (48 in flight per thread): 127 registers, 8 CTAs/SM
__global__ void __launch_bounds__(UT, 8) update32(float* __restrict__ A32, float* __restrict__ V32, int N, int nb, int R,
                                               const float* __restrict__ Sbuf, const float* __restrict__ Ubuf,
                                               int n_atiles, bool hq) {
  // three 32 x 32 buffers (13.5 KB): the tile (later X^T), U_P, U_Q
  __shared__ __align__(16) float T[W2][LD4];
  __shared__ __align__(16) float UP[W2][LD4];  // U_P[l][i]
  __shared__ __align__(16) float UQ[W2][LD4];  // U_Q[l][j]
  const int tid = threadIdx.x;
  const int i4 = (tid % 8) * 4, j4 = (tid / 8) * 4;
  const int npairs = nb / 2;
  int item = blockIdx.x;
  float acc[4][4];
  if (item < n_atiles) {
    int P, Q;
    tri_tile(item, npairs, P, Q);
    int IP, JP, IQ, JQ;
    block_pair(nb, R, P, IP, JP);
    block_pair(nb, R, Q, IQ, JQ);
    if (P == Q) {
      const float* Sp = Sbuf + (size_t)P * W2 * W2;
      #pragma unroll
      for (int it = 0; it < W2 * W2 / UT; ++it) {
        const int e = tid + it * UT;
        int li = e % W2, lj = e / W2;
        A32[(size_t)gidx(IP, JP, lj) * N + gidx(IP, JP, li)] = Sp[e];
      }
      return;
    }
    const float* Up = Ubuf + (size_t)P * W2 * W2;  // column-major 32 x 32: Up[li + 32 lj] = U_P(li, lj)
    const float* Uq = Ubuf + (size_t)Q * W2 * W2;
    #pragma unroll
    for (int it = 0; it < W2 * W2 / UT; ++it) {
      const int e = tid + it * UT;
      int li = e % W2, lj = e / W2;
      T[li][lj] = A32[(size_t)gidx(IQ, JQ, lj) * N + gidx(IP, JP, li)];
      UP[li][lj] = Up[e];
      UQ[li][lj] = Uq[e];
    }
    __syncthreads();
    // X = U_P^T T: X[i][j] = sum_l U_P[l][i] T[l][j]
    tile_mm(UP, T, acc, i4, j4);
    __syncthreads();  // every thread is done reading T
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) T[j4 + b][i4 + a] = acc[a][b];  // T now holds X^T
    __syncthreads();
    // Y = X U_Q: Y[i][j] = sum_l X^T[l][i] U_Q[l][j]
    tile_mm(T, UQ, acc, i4, j4);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) T[i4 + a][j4 + b] = qh(acc[a][b], hq);
    __syncthreads();
    #pragma unroll
    for (int it = 0; it < W2 * W2 / UT; ++it) {
      const int e = tid + it * UT;
      int li = e % W2, lj = e / W2;
      A32[(size_t)gidx(IQ, JQ, lj) * N + gidx(IP, JP, li)] = T[li][lj];
      // mirror: entry (cols(Q)[li], rows(P)[lj]) = T[lj][li]
      A32[(size_t)gidx(IP, JP, lj) * N + gidx(IQ, JQ, li)] = T[lj][li];
    }
    return;
  }
  // V tile: rows [rc*32, rc*32+32), column set of pair Q:  Y = T U_Q
  int v = item - n_atiles;
  int nrc = N / W2;
  int rc = v % nrc, Q = v / nrc;
  int IQ, JQ;
  block_pair(nb, R, Q, IQ, JQ);
  const float* Uq = Ubuf + (size_t)Q * W2 * W2;
  #pragma unroll
  for (int it = 0; it < W2 * W2 / UT; ++it) {
    const int e = tid + it * UT;
    int li = e % W2, lj = e / W2;
    UP[lj][li] = V32[(size_t)gidx(IQ, JQ, lj) * N + rc * W2 + li];  // UP holds the chunk transposed
    UQ[li][lj] = Uq[e];
  }
  __syncthreads();
  tile_mm(UP, UQ, acc, i4, j4);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) T[i4 + a][j4 + b] = qh(acc[a][b], hq);
  __syncthreads();
  #pragma unroll
  for (int it = 0; it < W2 * W2 / UT; ++it) {
    const int e = tid + it * UT;
    int li = e % W2, lj = e / W2;
    V32[(size_t)gidx(IQ, JQ, lj) * N + rc * W2 + li] = T[li][lj];
  }
}

}  // namespace

int mpj_stage1_padded(int n) { return ((n + W2 - 1) / W2) * W2; }

// A32, V32, the per-pair S and U, a flag word after them (the tensor-core
// update also keeps the transposed intermediate B^T there).
static int stage1_tensor_cores();

size_t mpj_stage1_bytes(int n) {
  size_t N = (size_t)mpj_stage1_padded(n);
  size_t nb = N / BS;
  return (stage1_tensor_cores() ? 3 : 2) * N * N * sizeof(float) + 2 * (nb / 2) * W2 * W2 * sizeof(float) + 4096;
}

// MPJ_STAGE1_TC=1 runs the A update of each block round on the tcgen05
// tensor cores (3xTF32, two panel products, see tc32.cu) and the V update on
// the FP32 pipe.  Off by default: on GB300 at n = 4096 it is slower (600 vs
// 435 ms for the stage), and V must stay on the FP32 pipe because the tensor
// cores' FP32 accumulation drifts the column norms over thousands of products
// (||V^T V - I||_F 0.08 instead of 0.007).
static int stage1_tensor_cores() {
  static int env = -1;
  if (env < 0) {
    const char* e = getenv("MPJ_STAGE1_TC");
    env = (e && e[0] == '1') ? 1 : 0;
  }
  return env;
}

cudaError_t mpj_sumsq32(const float* A, int lda, int n, double* partial, double* out, cudaStream_t s);

int mpj_stage1_run(int n, const double* A, int lda, double* Ql, int ldq, double tol32, int max_sweeps, int* sweeps_out,
                   double* off_out, void* work, double* partial, double* dscal, cudaStream_t s, bool half) {
  const int N = mpj_stage1_padded(n);
  const int nb = N / BS;
  float* A32 = (float*)work;
  float* V32 = A32 + (size_t)N * N;
  float* Sbuf = V32 + (size_t)N * N;
  float* Ubuf = Sbuf + (size_t)(nb / 2) * W2 * W2;
  float* Bt = Ubuf + (size_t)(nb / 2) * W2 * W2;
  unsigned* tflag = (unsigned*)(Bt + (stage1_tensor_cores() ? (size_t)N * N : 0));
  MPJ_CUDA_TRY(cudaMemsetAsync(tflag, 0, sizeof(unsigned), s));
  const int tc = stage1_tensor_cores() && !half;
  init32<<<1024, 256, 0, s>>>(A, lda, n, N, A32, V32, half);
  mpj_count_launch();
  MPJ_CUDA_TRY(cudaGetLastError());
  double off2 = 0.0;
  MPJ_CUDA_TRY(mpj_sumsq32(A32, N, N, partial, dscal, s));
  MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
  MPJ_CUDA_TRY(cudaStreamSynchronize(s));
  double off = sqrt(off2);
  int sweeps = 0, status = MPJ_OK;
  const int npairs = nb / 2;
  const int n_atiles = npairs * (npairs + 1) / 2;
  const int grid_u = n_atiles + (N / W2) * npairs;
  while (off > tol32) {
    if (sweeps >= max_sweeps) {
      status = MPJ_NOT_CONVERGED;
      break;
    }
    for (int R = 0; R < nb - 1; ++R) {
      solve32<<<npairs, 256, 0, s>>>(A32, N, nb, R, Sbuf, Ubuf, half);
      mpj_count_launch();
      if (tc == 1) {
        // A' = U^T A U = (A U)^T U (A symmetric): B^T = (A U)^T, then
        // A' = (B^T)(:, I_q) U_q on the tensor cores; V U on the FP32 pipe
        MPJ_CUDA_TRY(mpj_tc_panel(N, nb, R, Ubuf, A32, Bt, 1, nullptr, nullptr, tflag, s));
        MPJ_CUDA_TRY(mpj_tc_panel(N, nb, R, Ubuf, Bt, A32, 0, nullptr, nullptr, tflag, s));
        update32<<<(N / W2) * npairs, UT, 0, s>>>(A32, V32, N, nb, R, Sbuf, Ubuf, 0, false);
        mpj_count_launch();
      } else {
        update32<<<grid_u, UT, 0, s>>>(A32, V32, N, nb, R, Sbuf, Ubuf, n_atiles, half);
        mpj_count_launch();
      }
    }
    MPJ_CUDA_TRY(cudaGetLastError());
    ++sweeps;
    MPJ_CUDA_TRY(mpj_sumsq32(A32, N, N, partial, dscal, s));
    unsigned tf = 0;
    MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaMemcpyAsync(&tf, tflag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    if (tf & MPJ_FLAG_TIMEOUT) return MPJ_ETIMEOUT;
    off = sqrt(off2);
  }
  widen<<<1024, 256, 0, s>>>(V32, N, n, Ql, ldq);
  mpj_count_launch();
  MPJ_CUDA_TRY(cudaGetLastError());
  if (sweeps_out) *sweeps_out = sweeps;
  if (off_out) *off_out = off;
  return status;
}
