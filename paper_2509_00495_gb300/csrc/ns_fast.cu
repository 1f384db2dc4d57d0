// ns_fast.cu -- the Newton-Schulz correction in FP32 once it is tiny.
//
// A Newton-Schulz step (Sec. 4.3.4) X <- X (3I - X^T X)/2 equals
// X <- X + X E / 2 with E = I - X^T X.  The library forms X^T X in FP64 (its
// error decides the orthogonality reached) and E = I - X^T X exactly enough
// in FP64.  An FP32 evaluation of X E errs per entry by about
// sqrt(n) u_l max|E| (entries of X are O(1/sqrt n)); when
// max|E| <= 2^-31 / sqrt(n) that is below u_d / 4, so the product runs on the
// FP32 pipe (about 60x the FP64 rate on this GPU) instead of the FP64 one.
// This holds for a polish step on an already orthogonal Q (||E|| ~ n u_d);
// the solver's own Newton-Schulz steps (||E|| ~ n u_l, then ~ (n u_l)^2) stay
// in FP64.
#include "common.cuh"
#include "ns_fast.cuh"

namespace {

// E = I - M (FP64, in place into M), E32 = fl32(E), X32 = fl32(X); per-CTA max|E|.
__global__ void ns_residual(double* __restrict__ M, const double* __restrict__ X, int n, float* __restrict__ E32,
                            float* __restrict__ X32, double* __restrict__ part_max) {
  double mx = 0.0;
  size_t total = (size_t)n * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    double e = (i == j ? 1.0 : 0.0) - M[idx];
    M[idx] = e;
    E32[idx] = (float)e;
    X32[idx] = (float)X[idx];
    mx = fmax(mx, fabs(e));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ double w[32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, w[k]);
    part_max[blockIdx.x] = m;
  }
}

__global__ void max_partials(const double* __restrict__ part, int count, double* __restrict__ out) {
  __shared__ double sh[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < count; i += 256) m = fmax(m, part[i]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// C = A B, all n x n FP32 column-major.  64 x 64 tiles, 256 threads, each a
// 4 x 4 block; k staged 16 at a time in shared memory.
constexpr int SB = 64, SK = 16;
__global__ void __launch_bounds__(256) sgemm_nn(const float* __restrict__ A, const float* __restrict__ B,
                                                float* __restrict__ C, int n) {
  __shared__ __align__(16) float As[SK][SB + 4];  // As[k][i] = A(i0 + i, k0 + k)
  __shared__ __align__(16) float Bs[SK][SB + 4];  // Bs[k][j] = B(k0 + k, j0 + j)
  const int i0 = blockIdx.x * SB, j0 = blockIdx.y * SB;
  const int tid = threadIdx.x;
  const int ti = (tid % 16) * 4, tj = (tid / 16) * 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += SK) {
    for (int e = tid; e < SB * SK; e += 256) {
      int i = e % SB, k = e / SB;  // A: consecutive threads along rows i
      int gi = i0 + i, gk = k0 + k;
      As[k][i] = (gi < n && gk < n) ? A[(size_t)gk * n + gi] : 0.0f;
      int kb = e % SK, j = e / SK;  // B: consecutive threads along k (column-major)
      int gkb = k0 + kb, gj = j0 + j;
      Bs[kb][j] = (gkb < n && gj < n) ? B[(size_t)gj * n + gkb] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SK; ++k) {
      float4 a = *reinterpret_cast<const float4*>(&As[k][ti]);
      float4 b = *reinterpret_cast<const float4*>(&Bs[k][tj]);
      float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int gi = i0 + ti + p, gj = j0 + tj + q;
      if (gi < n && gj < n) C[(size_t)gj * n + gi] = acc[p][q];
    }
}

// Y = X + C / 2 (FP64 + FP32 correction).
__global__ void ns_combine(const double* __restrict__ X, const float* __restrict__ C, double* __restrict__ Y, int n) {
  size_t total = (size_t)n * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x)
    Y[idx] = fma(0.5, (double)C[idx], X[idx]);
}

constexpr int RED = 256;

}  // namespace

static inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout: E32, X32, C32 (n^2 floats each), then the max partials (doubles);
// every part starts on a 256-byte boundary.
size_t mpj_ns_fast_bytes(int n) {
  return 3 * al256((size_t)n * n * sizeof(float)) + al256((RED + 1) * sizeof(double));
}

int mpj_ns_fp32_correction(int n, const double* X, double* M, double* Y, void* work, double* max_e,
                           cudaStream_t s) {
  const size_t fb = al256((size_t)n * n * sizeof(float));
  float* E32 = (float*)work;
  float* X32 = (float*)((char*)work + fb);
  float* C32 = (float*)((char*)work + 2 * fb);
  double* part = (double*)((char*)work + 3 * fb);
  double* dmax = part + RED;
  ns_residual<<<RED, 256, 0, s>>>(M, X, n, E32, X32, part);
  mpj_count_launch();
  max_partials<<<1, 256, 0, s>>>(part, RED, dmax);
  mpj_count_launch();
  double h = 0.0;
  MPJ_CUDA_TRY(cudaMemcpyAsync(&h, dmax, sizeof(double), cudaMemcpyDeviceToHost, s));
  MPJ_CUDA_TRY(cudaStreamSynchronize(s));
  if (max_e) *max_e = h;
  if (!(h <= 0x1p-31 / sqrt((double)n))) return 1;  // too large for FP32; M now holds E
  dim3 grid((n + SB - 1) / SB, (n + SB - 1) / SB);
  sgemm_nn<<<grid, 256, 0, s>>>(X32, E32, C32, n);
  mpj_count_launch();
  size_t total = (size_t)n * n;
  int blocks = (int)((total + 255) / 256 > 4096 ? 4096 : (total + 255) / 256);
  ns_combine<<<blocks, 256, 0, s>>>(X, C32, Y, n);
  mpj_count_launch();
  MPJ_CUDA_TRY(cudaGetLastError());
  return 0;
}
