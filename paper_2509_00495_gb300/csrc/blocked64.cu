// blocked64.cu -- FP64 Jacobi sweeps in block round-robin order with the
// block updates on the tcgen05 tensor cores (the block Jacobi procedure the
// paper names as further work, Ch. 6; the rotations themselves are the
// paper's Algorithm 2 with the skip test of Algorithm 4, in FP64).
//
// Ordering: the padded index range [0, N) (N = n rounded up to a multiple of
// 32; indices >= n are inert) is cut into nb = N/16 blocks of 16.  A sweep is
// nb - 1 outer rounds of the circle method on blocks; in round R the nb/2
// disjoint block pairs P = (I, J) each run one inner round-robin sweep (31
// inner rounds of 16 disjoint pairs) over the 32 indices of I u J on their
// 32 x 32 diagonal subproblem A[P, P], in FP64 in shared memory, accumulating
// the orthogonal U_P.  This is the rotation sequence of the block
// round-robin ordering one rotation at a time: the subproblem's rotations
// depend only on its own entries, and the pairs of one round are disjoint.
// The rest of the matrix then receives the round's rotations as products
//   A <- U~^T A U~,  V <- V U~,   U~ = blockdiag(U_P) (in index-set order),
// run as three block-diagonal right multiplications, each panel
// Y[:, P] = X_P U_P with X_P one of
//   A[:, P]          (B = A U~),
//   B[P, :]^T        (C = B^T U~ = U~^T A U~ for symmetric A, written to A),
//   V[:, P]          (V <- V U~, in place).
//
// The right multiplication is FP64-accurate on the bf16 tensor cores: each
// CTA takes 128 rows of X_P (K = 32 values each), finds each row's largest
// exponent e_r (max |x_rk| < 2^e_r), and cuts x_rk * 2^(56 - e_r), rounded to
// an integer Y (|Y| < 2^56; the rounding is below 2^(e_r - 57)), into seven
// signed 8-bit digits with integer arithmetic (d_0 in [-256, 256], the others
// in [-128, 128], each exactly a bf16).  U_P's columns are cut the same way
// when the subproblem is solved.  The digit products of levels
// L = i + j <= 6 (28 pairs) go to seven FP32 accumulators in tensor memory;
// over K = 32 every level sum is an integer of magnitude at most 2^22.2, so
// the accumulation is exact.  The epilogue reads the level sums, forms
// Z = sum_L s_L 2^(8 (6 - L)) exactly in two 64-bit integers, rounds Z to FP64
// once and scales by 2^(e_r + f_c - 64).  Dropped levels (L >= 7) are below
// 2^-55 of max|x_r.| max|u_.c| per term.
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include "common.cuh"
#include "jacobi64.cuh"

namespace {

constexpr int BS = 16;                 // block size
constexpr int W2 = 32;                 // indices per block pair (K and N of the products)
constexpr int LDS = 33;                // padded shared-memory leading dimension
constexpr int NSL = 7;                 // 8-bit digits per value
constexpr int NLEV = 7;                // levels 0..6 kept
constexpr int TM = 128;                // rows per CTA of the right multiplication
constexpr uint32_t TMEM_COLS = 256;    // >= NLEV * 32
constexpr int USL_BYTES = W2 * W2 * 2;          // one 32 x 32 bf16 digit tile
constexpr int XSL_BYTES = TM * W2 * 2;          // one 128 x 32 bf16 digit tile
constexpr long long WAIT_CYCLES = 4000000000LL;

MPJ_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

MPJ_DEV int gidx(int I, int J, int l) { return l < BS ? I * BS + l : J * BS + (l - BS); }

MPJ_DEV void block_pair(int nb, int R, int slot, int& I, int& J) {
  int x, y;
  rr_slot(nb, R, slot, x, y);
  I = x < y ? x : y;
  J = x < y ? y : x;
}

// byte offset of (row, k), k in [0, 32), in a K-major tile of 8-row x 16-byte
// core matrices (k-adjacent cores 128 bytes apart, 8-row groups 512 apart)
MPJ_DEV int kmaj16(int row, int k) { return (((row >> 3) * 4 + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1); }

// The seven signed 8-bit digits of x on the grid 2^e (|x| < 2^e):
// x = sum_i d_i 2^(e - 8 (i + 1)) + r, |r| <= 2^(e - 57).
MPJ_DEV void digits8x7(double x, int e, int d[NSL]) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  const long long mant = bits & 0xFFFFFFFFFFFFFLL;
  const long long M = ex ? (mant | (1LL << 52)) : mant;
  const int eb = ex ? ex : 1;
  const int sh = eb - 1019 - e;  // x 2^(56 - e) = M 2^sh, sh <= 3
  long long Y;
  if (sh >= 0)
    Y = M << sh;
  else if (sh > -62)
    Y = (M + (1LL << (-sh - 1))) >> (-sh);
  else
    Y = 0;
  if (bits < 0) Y = -Y;
#pragma unroll
  for (int i = NSL - 1; i >= 1; --i) {
    const long long r = ((Y + 128) & 255) - 128;
    d[i] = (int)r;
    Y = (Y - r) >> 8;
  }
  d[0] = (int)Y;
}

MPJ_DEV int exp_of_max(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

// ---------------------------------------------------------------- subproblems
// One CTA per block pair of round R: one inner round-robin sweep on the FP64
// 32 x 32 subproblem (the paper's row update, column update and vector update
// per rotation; the 16 disjoint rotations of an inner round are applied
// together), then U_P's columns cut into digits for the tensor products.
// Writes per block pair: NSL digit tiles (32 x 32 bf16, K-major over the
// rows of U_P, one "row" per column of U_P), 32 column exponents, and whether
// any rotation happened.
__global__ void __launch_bounds__(256) blk_solve(const double* __restrict__ A, int lda, int n, int nb, int R,
                                                 double skip, double skip_abs, __nv_bfloat16* __restrict__ Usl,
                                                 int* __restrict__ Uexp, int* __restrict__ rotated) {
  __shared__ double S[W2][LDS];
  __shared__ double U[W2][LDS];
  __shared__ double cs[W2 / 2][2];
  __shared__ int rot[W2 / 2];
  __shared__ int any;
  const int P = blockIdx.x, tid = threadIdx.x;
  int I, J;
  block_pair(nb, R, P, I, J);
  if (tid == 0) any = 0;
  for (int e = tid; e < W2 * W2; e += blockDim.x) {
    const int li = e % W2, lj = e / W2;
    const int gi = gidx(I, J, li), gj = gidx(I, J, lj);
    S[li][lj] = (gi < n && gj < n) ? A[(size_t)gj * lda + gi] : 0.0;
    U[li][lj] = (li == lj) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int rho = 0; rho < W2 - 1; ++rho) {
    if (tid < W2 / 2) {
      int x, y;
      rr_slot(W2, rho, tid, x, y);
      const int p = x < y ? x : y, q = x < y ? y : x;
      const double app = S[p][p], aqq = S[q][q], apq = S[p][q];
      int r = 0;
      double c = 1.0, s = 0.0;
      if (gidx(I, J, q) < n && fabs(apq) > skip * sqrt(fabs(app * aqq)) && fabs(apq) > skip_abs) {
        // Algorithm 2, stable form (Appendix A approach 2)
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : 1.0 / (tau - sqrt(1.0 + tau * tau));
        c = 1.0 / sqrt(1.0 + t * t);
        s = t * c;
        r = 1;
        any = 1;
      }
      cs[tid][0] = c;
      cs[tid][1] = s;
      rot[tid] = r;
    }
    __syncthreads();
    // rows: S([p q], :) = J^T S([p q], :)
    for (int e = tid; e < (W2 / 2) * W2; e += blockDim.x) {
      const int k = e / W2, j = e % W2;
      if (!rot[k]) continue;
      int x, y;
      rr_slot(W2, rho, k, x, y);
      const int p = x < y ? x : y, q = x < y ? y : x;
      const double c = cs[k][0], s = cs[k][1];
      const double sp = S[p][j], sq = S[q][j];
      S[p][j] = c * sp - s * sq;
      S[q][j] = s * sp + c * sq;
    }
    __syncthreads();
    // columns: S(:, [p q]) = S(:, [p q]) J;  vectors: U(:, [p q]) = U(:, [p q]) J
    for (int e = tid; e < (W2 / 2) * W2; e += blockDim.x) {
      const int k = e / W2, j = e % W2;
      if (!rot[k]) continue;
      int x, y;
      rr_slot(W2, rho, k, x, y);
      const int p = x < y ? x : y, q = x < y ? y : x;
      const double c = cs[k][0], s = cs[k][1];
      const double sp = S[j][p], sq = S[j][q];
      S[j][p] = c * sp - s * sq;
      S[j][q] = s * sp + c * sq;
      const double up = U[j][p], uq = U[j][q];
      U[j][p] = c * up - s * uq;
      U[j][q] = s * up + c * uq;
    }
    __syncthreads();
  }
  // digits of U_P's columns: column c is "row" c of the right operand, over k = row of U_P
  __nv_bfloat16* dst = Usl + (size_t)P * NSL * (USL_BYTES / 2);
  if (tid < W2) {
    const int c = tid;
    double m = 0.0;
    for (int k = 0; k < W2; ++k) m = fmax(m, fabs(U[k][c]));
    const int e = exp_of_max(m);
    Uexp[P * W2 + c] = e;
    for (int k0 = 0; k0 < W2; k0 += 8) {
      int d[8][NSL];
#pragma unroll
      for (int j = 0; j < 8; ++j) digits8x7(U[k0 + j][c], e, d[j]);
#pragma unroll
      for (int s = 0; s < NSL; ++s) {
        __align__(16) __nv_bfloat16 q8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) q8[j] = __float2bfloat16((float)d[j][s]);
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(dst + (size_t)s * (USL_BYTES / 2)) + kmaj16(c, k0)) =
            *reinterpret_cast<const uint4*>(q8);
      }
    }
  }
  if (tid == 0) rotated[P] = any;
}

// ---------------------------------------------------------------- right multiplication
MPJ_DEV uint64_t sdesc(uint32_t saddr) {
  // K-major, no swizzle: LBO = 128 bytes (k-adjacent cores), SBO = 512 bytes (8-row groups)
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: D F32, A and B bf16, both K-major
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

MPJ_DEV void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

MPJ_DEV bool mbar_test(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

#define BLK_LD32(taddr, v)                                                                                         \
  asm volatile(                                                                                                    \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18," \
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                               \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),           \
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),     \
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),   \
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])    \
      : "r"(taddr))

struct __align__(1024) RmulSmem {
  unsigned char xs[NSL][XSL_BYTES];  // digits of the 128 x 32 tile of X_P
  unsigned char us[NSL][USL_BYTES];  // digits of U_P
  int uexp[W2];
  uint64_t mbar;
  uint32_t tmem;
};

enum { XMODE_COLS = 0, XMODE_ROWS = 1 };

// Y[r, g_P(c)] = sum_k X_P(r, k) U_P(k, c) for the CTA's 128 rows r and block
// pair P = blockIdx.y; X_P(r, k) = X[r + g_P(k) ldx] (XMODE_COLS) or
// X[g_P(k) + r ldx] (XMODE_ROWS).  Y may alias X in XMODE_COLS (each CTA reads
// and writes only its own rows of its own panel).
__global__ void __launch_bounds__(TM, 2) blk_rmul(const double* X, int ldx, int xmode, double* Y, int ldy, int n,
                                                  int nb, int R, const __nv_bfloat16* __restrict__ Usl,
                                                  const int* __restrict__ Uexp, unsigned* __restrict__ flags) {
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  RmulSmem& sm = *reinterpret_cast<RmulSmem*>(dsm_raw + ((1024 - (smem_u32(dsm_raw) & 1023)) & 1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int P = blockIdx.y;
  const int row = blockIdx.x * TM + tid;
  int I, J;
  block_pair(nb, R, P, I, J);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar)) : "memory");
  // U_P digits (contiguous, NSL x 2 KB) and column exponents
  {
    const uint4* src = reinterpret_cast<const uint4*>(Usl + (size_t)P * NSL * (USL_BYTES / 2));
    uint4* dst = reinterpret_cast<uint4*>(sm.us[0]);
    for (int i = tid; i < NSL * USL_BYTES / 16; i += TM) dst[i] = src[i];
    if (tid < W2) sm.uexp[tid] = Uexp[P * W2 + tid];
  }
  // this thread's row of X_P: 32 values, its exponent and digits
  double x[W2];
  if (xmode == XMODE_COLS) {
#pragma unroll
    for (int k = 0; k < W2; ++k) {
      const int g = gidx(I, J, k);
      x[k] = (row < n && g < n) ? X[(size_t)g * ldx + row] : 0.0;
    }
  } else {
#pragma unroll
    for (int k = 0; k < W2; ++k) {
      const int g = gidx(I, J, k);
      x[k] = (row < n && g < n) ? X[(size_t)row * ldx + g] : 0.0;
    }
  }
  double m = 0.0;
#pragma unroll
  for (int k = 0; k < W2; ++k) m = fmax(m, fabs(x[k]));
  const int er = exp_of_max(m);
#pragma unroll
  for (int k0 = 0; k0 < W2; k0 += 8) {
    int d[8][NSL];
#pragma unroll
    for (int j = 0; j < 8; ++j) digits8x7(x[k0 + j], er, d[j]);
#pragma unroll
    for (int s = 0; s < NSL; ++s) {
      __align__(16) __nv_bfloat16 q8[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) q8[j] = __float2bfloat16((float)d[j][s]);
      *reinterpret_cast<uint4*>(sm.xs[s] + kmaj16(tid, k0)) = *reinterpret_cast<const uint4*>(q8);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem;
  const uint32_t mb = smem_u32(&sm.mbar);
  if (tid == 0) {
    constexpr uint32_t idesc = idesc_f16(TM, W2);
    uint32_t started = 0;
    for (int i = 0; i < NSL; ++i)
      for (int j = 0; i + j < NLEV; ++j) {
        const int l = i + j;
#pragma unroll
        for (int kk = 0; kk < W2 / 16; ++kk) {
          mma_f16(tmem + (uint32_t)(l * W2), sdesc(smem_u32(sm.xs[i]) + kk * 256), sdesc(smem_u32(sm.us[j]) + kk * 256),
                  idesc, (started >> l) & 1u);
          started |= 1u << l;
        }
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
  }
  // bounded wait for the products
  bool ok = true;
  {
    const long long t0 = clock64();
    while (!mbar_test(mb, 0)) {
      if (clock64() - t0 > WAIT_CYCLES) {
        ok = false;
        break;
      }
      __nanosleep(20);
    }
    if (!ok) {
      if (lane == 0 && flags) atomicOr(flags, MPJ_FLAG_TIMEOUT);
      const long long t1 = clock64();  // the products may still be in flight
      while (!mbar_test(mb, 0) && clock64() - t1 <= WAIT_CYCLES) __nanosleep(64);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // Z = sum_L s_L 2^(8 (6 - L)) = hi 2^32 + lo, hi = s0 2^16 + s1 2^8 + s2, lo = s3 2^24 + s4 2^16 + s5 2^8 + s6
    long long hi[W2], lo[W2];
#pragma unroll
    for (int c = 0; c < W2; ++c) {
      hi[c] = 0;
      lo[c] = 0;
    }
#pragma unroll 1
    for (int l = 0; l < NLEV; ++l) {
      uint32_t v[32];
      BLK_LD32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(l * W2), v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int sh = l < 3 ? 8 * (2 - l) : 8 * (6 - l);
#pragma unroll
      for (int c = 0; c < W2; ++c) {
        const long long q = (long long)__float2int_rz(__uint_as_float(v[c]));  // exact integer below 2^24
        if (l < 3)
          hi[c] += q << sh;
        else
          lo[c] += q << sh;
      }
    }
    if (row < n) {
#pragma unroll
      for (int c = 0; c < W2; ++c) {
        const int g = gidx(I, J, c);
        if (g < n) {
          const double z = fma((double)hi[c], 0x1p32, (double)lo[c]);  // Z rounded once
          Y[(size_t)g * ldy + row] = ldexp(z, er + sm.uexp[c] - 64);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t mpj_blocked_scratch_bytes(int n) {
  const int N = (n + 2 * BS - 1) / (2 * BS) * (2 * BS);
  const int npairs = N / (2 * BS);
  return al256((size_t)npairs * NSL * USL_BYTES) + al256((size_t)npairs * W2 * sizeof(int)) +
         al256((size_t)npairs * sizeof(int)) + 256;
}

cudaError_t mpj_blocked_round(double* A, int lda, double* V, int ldv, double* B, int n, int R, double skip,
                              double skip_abs, void* scratch, unsigned* flags, cudaStream_t s) {
  const int N = (n + 2 * BS - 1) / (2 * BS) * (2 * BS);
  const int nb = N / BS, npairs = nb / 2;
  char* base = (char*)scratch;
  __nv_bfloat16* Usl = (__nv_bfloat16*)base;
  int* Uexp = (int*)(base + al256((size_t)npairs * NSL * USL_BYTES));
  int* rotated = (int*)((char*)Uexp + al256((size_t)npairs * W2 * sizeof(int)));
  blk_solve<<<npairs, 256, 0, s>>>(A, lda, n, nb, R, skip, skip_abs, Usl, Uexp, rotated);
  mpj_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // at least 80 KB of shared memory per CTA: at most two CTAs per SM, the two
  // that the 512 TMEM columns hold (256 each), so no CTA waits in tcgen05.alloc
  const size_t smem = sizeof(RmulSmem) + 1024 > 80 * 1024 ? sizeof(RmulSmem) + 1024 : 80 * 1024;
  static bool attr_set = false;
  if (!attr_set) {
    e = cudaFuncSetAttribute(blk_rmul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const dim3 grid((n + TM - 1) / TM, npairs);
  // B = A U~ ; A = B^T U~ (= U~^T A U~) ; V = V U~
  blk_rmul<<<grid, TM, smem, s>>>(A, lda, XMODE_COLS, B, n, n, nb, R, Usl, Uexp, flags);
  mpj_count_launch();
  blk_rmul<<<grid, TM, smem, s>>>(B, n, XMODE_ROWS, A, lda, n, nb, R, Usl, Uexp, flags);
  mpj_count_launch();
  blk_rmul<<<grid, TM, smem, s>>>(V, ldv, XMODE_COLS, V, ldv, n, nb, R, Usl, Uexp, flags);
  mpj_count_launch();
  return cudaGetLastError();
}

int mpj_blocked_rounds_per_sweep(int n) {
  const int N = (n + 2 * BS - 1) / (2 * BS) * (2 * BS);
  return N / BS - 1;
}

// A = (A + A^T) / 2 (the paper's end-of-sweep symmetrization; the blocked
// update computes both triangles, which agree only to rounding).
__global__ void blk_symmetrize(double* __restrict__ A, int lda, int n) {
  const size_t total = (size_t)n * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    if (i > j) {
      const double v = 0.5 * (A[(size_t)j * lda + i] + A[(size_t)i * lda + j]);
      A[(size_t)j * lda + i] = v;
      A[(size_t)i * lda + j] = v;
    }
  }
}

cudaError_t mpj_blocked_symmetrize(double* A, int lda, int n, cudaStream_t s) {
  size_t b = ((size_t)n * n + 255) / 256;
  blk_symmetrize<<<(int)(b > 4096 ? 4096 : (b < 1 ? 1 : b)), 256, 0, s>>>(A, lda, n);
  mpj_count_launch();
  return cudaGetLastError();
}
