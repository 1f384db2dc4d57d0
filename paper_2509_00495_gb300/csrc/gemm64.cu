// gemm64.cu -- FP64 matrix products on the FP64 tensor path (mma.sync
// m8n8k4 .f64, "DMMA"), for the dense products of the mixed algorithm:
// Newton-Schulz X^T X and X (3I - X^T X)/2 (Sec. 4.3.4, Algorithm 8), the
// transform Q_d^T A Q_d (Algorithm 9 step 3) and Q = Q_d V (step 4).
//
// D = alpha op(A) op(B) + beta Cin, column-major, op = identity or transpose.
// Tiles of 64 x 64 outputs per CTA (4 warps, 32 x 32 each), k staged through
// shared memory 16 at a time with cp.async double buffering.  On GB300 the
// FP64 pipe issues about 2 FMA per clock per SM for both DFMA and DMMA, so the
// kernel is FP64-pipe bound; shared memory and HBM are far from limits.
//
// sym != 0 computes only the tiles on or below the diagonal of a square
// result that is symmetric in exact arithmetic (X^T X, Q_d^T (A Q_d)) and
// writes each lower entry together with its mirror, so the result is exactly
// symmetric and costs half the flops.
#include "common.cuh"
#include "gemm64.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, PAD = 4;
constexpr int NT = 128;

MPJ_DEV void cp_async8(double* smem, const double* gmem, bool valid) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  int src_bytes = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
MPJ_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
MPJ_DEV void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
MPJ_DEV void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::); }

MPJ_DEV void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(NT) dgemm_kernel(GemmArgs g) {
  __shared__ __align__(16) double As[2][BK][BM + PAD];
  __shared__ __align__(16) double Bs[2][BK][BN + PAD];

  int ti, tj;
  if (g.sym) {
    // blockIdx.x enumerates lower-triangular tiles column by column
    int t = blockIdx.x, nt = (g.m + BM - 1) / BM;
    tj = 0;
    while (t >= nt - tj) {
      t -= nt - tj;
      ++tj;
    }
    ti = tj + t;
  } else {
    ti = blockIdx.x;
    tj = blockIdx.y;
  }
  const int batch = blockIdx.z;
  const double* A = g.A + (size_t)batch * g.strideA;
  const double* B = g.B + (size_t)batch * g.strideB;
  const double* Cin = g.Cin ? g.Cin + (size_t)batch * g.strideCin : nullptr;
  double* C = g.C + (size_t)batch * g.strideC;

  const int m0 = ti * BM, n0 = tj * BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int gid = lane >> 2, tig = lane & 3;

  auto load_tile = [&](int buf, int k0) {
#pragma unroll
    for (int j = 0; j < (BM * BK) / NT; ++j) {
      int idx = tid + j * NT;
      int mm, kk;
      if (!TA) {
        kk = idx / BM;
        mm = idx % BM;
      } else {
        mm = idx / BK;
        kk = idx % BK;
      }
      int gm = m0 + mm, gk = k0 + kk;
      bool v = gm < g.m && gk < g.k;
      const double* src = TA ? (A + (size_t)(v ? gm : 0) * g.lda + (v ? gk : 0))
                             : (A + (size_t)(v ? gk : 0) * g.lda + (v ? gm : 0));
      cp_async8(&As[buf][kk][mm], src, v);
    }
#pragma unroll
    for (int j = 0; j < (BN * BK) / NT; ++j) {
      int idx = tid + j * NT;
      int nn, kk;
      if (!TB) {
        nn = idx / BK;
        kk = idx % BK;
      } else {
        kk = idx / BN;
        nn = idx % BN;
      }
      int gn = n0 + nn, gk = k0 + kk;
      bool v = gn < g.n && gk < g.k;
      const double* src = TB ? (B + (size_t)(v ? gk : 0) * g.ldb + (v ? gn : 0))
                             : (B + (size_t)(v ? gn : 0) * g.ldb + (v ? gk : 0));
      cp_async8(&Bs[buf][kk][nn], src, v);
    }
    cp_async_commit();
  };

  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  const int ktiles = (g.k + BK - 1) / BK;
  if (ktiles > 0) load_tile(0, 0);
  for (int kt = 0; kt < ktiles; ++kt) {
    int buf = kt & 1;
    if (kt + 1 < ktiles) {
      load_tile(buf ^ 1, (kt + 1) * BK);
      cp_async_wait_1();
    } else {
      cp_async_wait_0();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) af[i] = As[buf][kk + tig][wm * 32 + i * 8 + gid];
#pragma unroll
      for (int j = 0; j < 4; ++j) bf[j] = Bs[buf][kk + tig][wn * 32 + j * 8 + gid];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
    }
    __syncthreads();
  }

  // epilogue
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        int r = m0 + wm * 32 + i * 8 + gid;
        int c = n0 + wn * 32 + j * 8 + tig * 2 + e;
        if (r >= g.m || c >= g.n) continue;
        if (g.sym && r < c) continue;
        double v = g.alpha * acc[i][j][e];
        if (g.beta != 0.0) v = fma(g.beta, Cin[(size_t)c * g.ldcin + r], v);
        C[(size_t)c * g.ldc + r] = v;
        if (g.sym && r != c) C[(size_t)r * g.ldc + c] = v;
      }
}

}  // namespace

cudaError_t mpj_gemm64_launch(const GemmArgs& g, bool ta, bool tb, int batch, cudaStream_t stream) {
  if (g.m <= 0 || g.n <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid;
  if (g.sym) {
    int nt = (g.m + BM - 1) / BM;
    grid = dim3(nt * (nt + 1) / 2, 1, batch);
  } else {
    grid = dim3((g.m + BM - 1) / BM, (g.n + BN - 1) / BN, batch);
  }
  if (!ta && !tb)
    dgemm_kernel<false, false><<<grid, NT, 0, stream>>>(g);
  else if (ta && !tb)
    dgemm_kernel<true, false><<<grid, NT, 0, stream>>>(g);
  else if (!ta && tb)
    dgemm_kernel<false, true><<<grid, NT, 0, stream>>>(g);
  else
    dgemm_kernel<true, true><<<grid, NT, 0, stream>>>(g);
  mpj_count_launch();
  return cudaGetLastError();
}
