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
//   B[P, :]^T        (C = B^T U~ = U~^T A U~ for symmetric A, written to A:
//                     only its lower triangle is formed, each entry also
//                     written to its mirror, so A stays exactly symmetric),
//   V[:, P]          (V <- V U~, in place).
//
// The right multiplication is FP64-accurate on the bf16 tensor cores: each
// CTA takes 128 rows of X_P (K = 32 values each), finds each row's largest
// exponent e_r (max |x_rk| < 2^e_r), and cuts x_rk * 2^(56 - e_r), rounded to
// an integer (magnitude below 2^56; the rounding is below 2^(e_r - 57)), into
// seven signed digits of 8 bits (|d_0| <= 256, |d_i| <= 128, each exactly a
// bf16).  U_P's columns are cut the same way when the subproblem is solved.
// The digit products of levels L = i + j <= 6 (28 pairs) go to seven FP32
// accumulators in tensor memory; over K = 32 a level sum is an integer of
// magnitude at most (2 * 256 * 128 + 5 * 128^2) * 32 = 2^22.2.  Measured on
// this GPU: the tensor cores' FP32 accumulation of such integer sums is exact
// below 2^23 but not in [2^23, 2^24) (unsigned byte digits, whose level sums
// reach 2^23.8, lost accuracy), so every bound here is kept below 2^23.  The epilogue reads the level sums, forms
// Z = sum_L s_L 2^(8 (6 - L)) exactly in two 64-bit integers, rounds Z to FP64
// once and scales by 2^(e_r + f_c - 64).  Dropped levels (L >= 7) are below
// 2^-55 of max|x_r.| max|u_.c| per term.  The epilogue uses integer
// instructions only (no FP64: on this GPU an FP64 instruction costs 64 times
// an FP32 one), so the products cost tensor time plus integer work.
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

// The seven signed digits of x on the grid 2^e (|x| < 2^e): x = sum_i d_i
// 2^(e - 8 (i + 1)) + r, |r| <= 2^(e - 57), |d_0| <= 256, |d_i| <= 128 (i >= 1),
// returned as FP32 bit patterns (exact small integers; their top 16 bits are
// the bf16).  Y = round(|x| 2^(56 - e)) < 2^56; adding 128 to each of its six
// low bytes (one 64-bit add, carries included) makes byte j of the sum
// d_(6-j) + 128 for centred digits d in [-128, 127], and the part above bit 48
// d_0 in [0, 256].  A byte b becomes a float through the bit pattern of
// 2^23 + b (one byte permute), then one FMA gives sign(x) (b - 128).
// Centred digits keep every level sum of the products below 2^23 (see the
// file comment).
MPJ_DEV void digits_f32(double x, int e, uint32_t d[NSL]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  const unsigned long long mant = bits & 0xFFFFFFFFFFFFFULL;
  const unsigned long long M = ex ? (mant | (1ULL << 52)) : mant;
  const int sh = (ex ? ex : 1) - 1019 - e;  // |x| 2^(56 - e) = M 2^sh, sh <= 3
  unsigned long long Y;
  if (sh >= 0)
    Y = M << sh;
  else if (sh > -62)
    Y = (M + (1ULL << (-sh - 1))) >> (-sh);
  else
    Y = 0;
  const unsigned long long T = Y + 0x0000808080808080ULL;
  const uint32_t lo = (uint32_t)T, hi = (uint32_t)(T >> 32);
  const float sg = (bits >> 63) ? -1.0f : 1.0f;
  const float c128 = -8388736.0f * sg;  // -(2^23 + 128) sign(x)
  // bytes of lo: d6+128, d5+128, d4+128, d3+128; of hi: d2+128, d1+128; hi >> 16: d0
  d[6] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(lo, 0x4B00u, 0x5440)), sg, c128));
  d[5] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(lo, 0x4B00u, 0x5441)), sg, c128));
  d[4] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(lo, 0x4B00u, 0x5442)), sg, c128));
  d[3] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(lo, 0x4B00u, 0x5443)), sg, c128));
  d[2] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(hi, 0x4B00u, 0x5440)), sg, c128));
  d[1] = __float_as_uint(fmaf(__uint_as_float(__byte_perm(hi, 0x4B00u, 0x5441)), sg, c128));
  d[0] = __float_as_uint(fmaf(__uint_as_float(0x4B000000u | (hi >> 16)), sg, -8388608.0f * sg));
}

// Two FP32 digit patterns packed as two bf16 (a in the low half).
MPJ_DEV uint32_t pack_bf16x2(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x7632); }

// The same from the bit pattern of max|x| (a non-negative double), with
// integer instructions only: the smallest e with max|x| < 2^e (0 for zero).
MPJ_DEV int exp_of_maxbits(unsigned long long b) {
  if (b == 0) return 0;
  const int ex = (int)(b >> 52);
  if (ex > 0) return ex - 1022;                     // 1.m 2^(ex-1023) < 2^(ex-1022)
  return (64 - __clzll((long long)b)) - 1074;       // subnormal: mant 2^-1074
}

// v 2^E as a double, exact for |v| < 2^53 when the result is a normal
// number (integer instructions only); 0 for v = 0.
MPJ_DEV double exact_scaled(long long v, int E) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? (1ULL << 63) : 0ULL;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int p = 63 - __clzll((long long)a);  // leading bit, < 53
  const unsigned long long m = (a << (52 - p)) & ((1ULL << 52) - 1ULL);
  return __longlong_as_double((long long)(sign | ((unsigned long long)(p + E + 1023) << 52) | m));
}

// Z 2^E rounded to the nearest double (ties to even), Z = hi 2^32 + lo with
// |Z| < 2^72, using integer instructions only.  Results outside the normal
// range go through ldexp (never for the operands of the sweeps).
MPJ_DEV double z_to_double(long long hi, long long lo, int E) {
  unsigned long long zl = ((unsigned long long)hi << 32) + (unsigned long long)lo;
  long long zh = (hi >> 32) + (lo >> 63) + (zl < (unsigned long long)lo ? 1 : 0);
  const unsigned long long sign = zh < 0 ? (1ULL << 63) : 0ULL;
  if (zh < 0) {  // |Z|
    zl = ~zl + 1ULL;
    zh = ~zh + (zl == 0 ? 1 : 0);
  }
  const unsigned long long h = (unsigned long long)zh;
  if (h == 0 && zl == 0) return __longlong_as_double((long long)sign);
  const int pos = h ? 127 - __clzll((long long)h) : 63 - __clzll((long long)zl);  // leading bit
  unsigned long long mant;
  if (pos <= 52) {
    mant = zl << (52 - pos);
  } else {
    const int sh = pos - 52;  // 1 .. 72
    unsigned long long lo_part, rnd, sticky;
    if (sh < 64) {
      mant = (zl >> sh) | (sh ? (h << (64 - sh)) : 0ULL);
      rnd = (zl >> (sh - 1)) & 1ULL;
      sticky = (sh >= 2) ? (zl & ((1ULL << (sh - 1)) - 1ULL)) : 0ULL;
    } else {
      mant = h >> (sh - 64);
      rnd = (sh == 64) ? (zl >> 63) : ((h >> (sh - 65)) & 1ULL);
      lo_part = (sh == 64) ? (zl & ((1ULL << 63) - 1ULL)) : (zl | (sh > 65 ? (h & ((1ULL << (sh - 65)) - 1ULL)) : 0ULL));
      sticky = lo_part;
    }
    mant &= (1ULL << 53) - 1ULL;
    if (rnd && (sticky || (mant & 1ULL))) ++mant;
  }
  int p2 = pos;
  if (mant >> 53) {
    mant >>= 1;
    ++p2;
  }
  const int biased = p2 + E + 1023;
  if (biased <= 0 || biased >= 2047) return ldexp(__longlong_as_double((long long)(sign | (1023ULL << 52) |
                                                                                   (mant & ((1ULL << 52) - 1ULL)))),
                                                 p2 + E);
  return __longlong_as_double((long long)(sign | ((unsigned long long)biased << 52) | (mant & ((1ULL << 52) - 1ULL))));
}

// Algorithm 2 for the scaled subproblem rotations, with the skip test of
// Algorithm 4 (|a_pq| > skip sqrt|a_pp a_qq|, compared in squares, and the
// threshold |a_pq| > skip_abs): t as in the stable form, c = 1 / sqrt(1 + t^2)
// and h = 1 / c = (1 + t^2) c for the scale vector and its reciprocal.
MPJ_DEV bool rot_scaled(double app, double aqq, double apq, double skip, double skip_abs, double& t, double& c,
                        double& h) {
  if (!(apq * apq > (skip * skip) * fabs(app * aqq) && fabs(apq) > skip_abs)) return false;
  const double tau = (aqq - app) / (2.0 * apq);
  const double r = sqrt(fma(tau, tau, 1.0));
  t = (tau >= 0.0) ? 1.0 / (tau + r) : 1.0 / (tau - r);
  const double w = fma(t, t, 1.0);
  c = rsqrt(w);
  h = w * c;
  return true;
}

// ---------------------------------------------------------------- subproblems
// One CTA per block pair of round R: one inner round-robin sweep on the FP64
// 32 x 32 subproblem (the paper's row update, column update and vector update
// per rotation, in scaled form: one FMA per entry and side, the factors c kept
// in a scale vector; the 16 disjoint rotations of an inner round are applied
// together), then U_P's columns cut into digits for the tensor products.
// Writes per block pair: NSL digit tiles (32 x 32 bf16, K-major over the
// rows of U_P, one "row" per column of U_P), 32 column exponents, and whether
// any rotation happened.
constexpr int SOLVE_THREADS = 512;
__global__ void __launch_bounds__(SOLVE_THREADS) blk_solve(const double* __restrict__ A, int lda, int n, int nb, int R,
                                                 double skip, double skip_abs, __nv_bfloat16* __restrict__ Usl,
                                                 int* __restrict__ Uexp, int* __restrict__ rotated,
                                                 unsigned* __restrict__ nrot) {
  __shared__ double S[W2][LDS];
  __shared__ double U[W2][LDS];
  __shared__ int any;
  const int P = blockIdx.x, tid = threadIdx.x;
  int I, J;
  block_pair(nb, R, P, I, J);
  if (tid == 0) any = 0;
  pdl_wait();
  for (int e = tid; e < W2 * W2; e += blockDim.x) {
    const int li = e % W2, lj = e / W2;
    const int gi = gidx(I, J, li), gj = gidx(I, J, lj);
    S[li][lj] = (gi < n && gj < n) ? A[(size_t)gj * lda + gi] : 0.0;
    U[li][lj] = (li == lj) ? 1.0 : 0.0;
  }
  __syncthreads();
  // Scaled rotations (the scheme of the scalar round-robin sweeps): off the
  // diagonal S = D S~ D and U = U~ D with one scale vector d (and e = 1/d);
  // S's diagonal holds the true values.  A rotation (c, s = t c) of pair
  // p < q then costs one FMA per entry and side:
  //   x_p <- x_p - mx x_q,  x_q <- x_q + my x_p  (old values),
  //   mx = t d_q / d_p,  my = t d_p / d_q,  d_p, d_q <- c d_p, c d_q,
  // the pair's diagonal becomes a_pp - t a_pq, a_qq + t a_pq and a_pq 0.
  // Each inner round applies its 16 rotations to every 2 x 2 block of S
  // between two pairs a < b once (rows by pair a, then columns by pair b; the
  // mirror block is the same values transposed) and to the two columns of U~
  // of every pair.  The next round's rotations read only the diagonal entries
  // and the blocks (a, b) that hold one of its pairs: warp 0 sets the
  // diagonal blocks and updates those blocks first and then computes the next
  // round's rotations, while the other warps update the remaining blocks and
  // U~.  Each block is updated by exactly one thread.
  __shared__ double cs[2][W2 / 2][2];  // mx, my
  __shared__ double dg[2][W2 / 2][2];  // the pair's new true diagonal
  __shared__ int rot[2][W2 / 2];
  __shared__ int pq[2][W2 / 2][2];
  __shared__ int slot_of[2][W2];  // pair slot of each local index in the round
  __shared__ double dsc[W2], esc[W2];  // d and e = 1 / d
  const int warp = tid >> 5, lane = tid & 31;
  if (tid < W2) {
    dsc[tid] = 1.0;
    esc[tid] = 1.0;
  }
  __syncthreads();
  // Algorithm 2 with the skip test of Algorithm 4 for pair `k` of inner round
  // rho, on the true coupling; the pair's scales are updated here (its lane
  // is the only one that touches them this round)
  auto rotation = [&](int rho, int k, int buf) {
    int x, y;
    rr_slot(W2, rho, k, x, y);
    const int p = x < y ? x : y, q = x < y ? y : x;
    const double app = S[p][p], aqq = S[q][q];
    const double dp = dsc[p], dq = dsc[q];
    const double apq = S[p][q] * dp * dq;
    double t = 0.0, c = 1.0, h = 1.0;
    const int r = gidx(I, J, q) < n && rot_scaled(app, aqq, apq, skip, skip_abs, t, c, h);
    double mx = 0.0, my = 0.0;
    if (r) {
      any = 1;
      const double ep = esc[p], eq = esc[q];
      mx = t * dq * ep;
      my = t * dp * eq;
      dsc[p] = dp * c;
      dsc[q] = dq * c;
      esc[p] = ep * h;
      esc[q] = eq * h;
      dg[buf][k][0] = app - t * apq;
      dg[buf][k][1] = aqq + t * apq;
    }
    cs[buf][k][0] = mx;
    cs[buf][k][1] = my;
    rot[buf][k] = r;
    pq[buf][k][0] = p;
    pq[buf][k][1] = q;
    slot_of[buf][p] = k;
    slot_of[buf][q] = k;
  };
  // the pair's own 2 x 2 block: the new true diagonal and a zero coupling
  auto diag_update = [&](int a, int buf) {
    if (!rot[buf][a]) return;
    const int pa = pq[buf][a][0], qa = pq[buf][a][1];
    S[pa][pa] = dg[buf][a][0];
    S[qa][qa] = dg[buf][a][1];
    S[pa][qa] = 0.0;
    S[qa][pa] = 0.0;
  };
  // the 2 x 2 block between pairs a < b of the round in buffer `buf`
  auto block_update = [&](int a, int b, int buf) {
    if (!rot[buf][a] && !rot[buf][b]) return;
    const int pa = pq[buf][a][0], qa = pq[buf][a][1], pb = pq[buf][b][0], qb = pq[buf][b][1];
    double b00 = S[pa][pb], b01 = S[pa][qb], b10 = S[qa][pb], b11 = S[qa][qb];
    if (rot[buf][a]) {  // rows pa, qa
      const double mx = cs[buf][a][0], my = cs[buf][a][1];
      const double t00 = fma(-mx, b10, b00), t10 = fma(my, b00, b10);
      const double t01 = fma(-mx, b11, b01), t11 = fma(my, b01, b11);
      b00 = t00;
      b10 = t10;
      b01 = t01;
      b11 = t11;
    }
    if (rot[buf][b]) {  // columns pb, qb
      const double mx = cs[buf][b][0], my = cs[buf][b][1];
      const double t00 = fma(-mx, b01, b00), t01 = fma(my, b00, b01);
      const double t10 = fma(-mx, b11, b10), t11 = fma(my, b10, b11);
      b00 = t00;
      b01 = t01;
      b10 = t10;
      b11 = t11;
    }
    S[pa][pb] = b00;
    S[pa][qb] = b01;
    S[qa][pb] = b10;
    S[qa][qb] = b11;
    S[pb][pa] = b00;
    S[qb][pa] = b01;
    S[pb][qa] = b10;
    S[qb][qa] = b11;
  };
  if (warp == 0 && lane < W2 / 2) rotation(0, lane, 0);
  __syncthreads();
  for (int rho = 0; rho < W2 - 1; ++rho) {
    const int cur = rho & 1;
    const bool more = rho + 1 < W2 - 1;
    if (warp == 0) {
      // lanes 0-15: the pairs' own blocks; lanes 16-31: the block holding pair
      // lane - 16 of the next round (once, when two next pairs share a block)
      if (lane < W2 / 2) {
        diag_update(lane, cur);
      } else if (more) {
        int x, y;
        rr_slot(W2, rho + 1, lane - W2 / 2, x, y);
        int a = slot_of[cur][x], b = slot_of[cur][y];
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
          const int tx = x;
          x = y;
          y = tx;
        }
        // x is in pair a: the other index of a, if its next partner is in b,
        // gives the same block; the smaller of the two indices takes it
        const int o = pq[cur][a][0] == x ? pq[cur][a][1] : pq[cur][a][0];
        const bool dup = slot_of[cur][rr_partner(W2, rho + 1, o)] == b;
        if (a != b && (!dup || x < o)) block_update(a, b, cur);
      }
      __syncwarp();
      if (more && lane < W2 / 2) rotation(rho + 1, lane, cur ^ 1);
    } else {
      for (int task = tid - 32; task < 120 + (W2 / 2) * W2; task += blockDim.x - 32) {
        if (task < 120) {
          // pair indices a < b from the triangular task number
          int a = 0, rem = task;
          while (rem >= 15 - a) {
            rem -= 15 - a;
            ++a;
          }
          const int b = a + 1 + rem;
          if (more) {  // a block that holds a pair of the next round: warp 0
            const int na = rr_partner(W2, rho + 1, pq[cur][a][0]), nq = rr_partner(W2, rho + 1, pq[cur][a][1]);
            if (slot_of[cur][na] == b || slot_of[cur][nq] == b) continue;
          }
          block_update(a, b, cur);
        } else {
          const int e = task - 120, k = e / W2, j = e % W2;
          if (!rot[cur][k]) continue;
          const int p = pq[cur][k][0], q = pq[cur][k][1];
          const double up = U[j][p], uq = U[j][q];
          U[j][p] = fma(-cs[cur][k][0], uq, up);
          U[j][q] = fma(cs[cur][k][1], up, uq);
        }
      }
    }
    __syncthreads();
  }
  // U = U~ D
  for (int e = tid; e < W2 * W2; e += blockDim.x) {
    const int i = e % W2, j = e / W2;
    U[i][j] *= dsc[j];
  }
  __syncthreads();
  // One Newton-Schulz step on U_P (Sec. 4.3.4): U <- U - U E / 2, E = U^T U - I.
  // U_P carries the rounding of its 496 rotations; applied to all of A and V
  // every round, that departure from orthogonality would accumulate over the
  // sweeps, so each U_P is made orthogonal to working precision first.
  {
    // E is symmetric: the 528 entries i <= j, mirrored (S is free now: it holds E)
    constexpr int NE = (528 + SOLVE_THREADS - 1) / SOLVE_THREADS;
    double e3[NE];
    int ij[NE];
#pragma unroll
    for (int t = 0; t < NE; ++t) {
      const int idx = tid + t * SOLVE_THREADS;
      e3[t] = 0.0;
      ij[t] = -1;
      if (idx < 528) {
        int i = 0, rem = idx;
        while (rem >= W2 - i) {
          rem -= W2 - i;
          ++i;
        }
        const int j = i + rem;
        double acc = (i == j) ? -1.0 : 0.0;
        for (int k = 0; k < W2; ++k) acc = fma(U[k][i], U[k][j], acc);
        e3[t] = acc;
        ij[t] = i * W2 + j;
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < NE; ++t)
      if (ij[t] >= 0) {
        const int i = ij[t] / W2, j = ij[t] % W2;
        S[i][j] = e3[t];
        S[j][i] = e3[t];
      }
    __syncthreads();
    // |E| is at the rounding level, so U E is formed in FP32 (its relative
    // error 2^-24 of a 1e-15 correction is far below FP64 rounding); U and E
    // are rounded to FP32 once (FP64 conversions issue on the slow FP64 pipe)
    __shared__ float Uf[W2][W2 + 1], Ef[W2][W2 + 1];
    for (int e = tid; e < W2 * W2; e += SOLVE_THREADS) {
      const int i = e % W2, j = e / W2;
      Uf[i][j] = (float)U[i][j];
      Ef[i][j] = (float)S[i][j];
    }
    __syncthreads();
    constexpr int NU = W2 * W2 / SOLVE_THREADS;
    double u4[NU];
#pragma unroll
    for (int t = 0; t < NU; ++t) {
      const int idx = tid + t * SOLVE_THREADS, i = idx % W2, j = idx / W2;
      float acc = 0.0f;
      for (int k = 0; k < W2; ++k) acc = fmaf(Uf[i][k], Ef[k][j], acc);
      u4[t] = fma(-0.5, (double)acc, U[i][j]);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < NU; ++t) {
      const int idx = tid + t * SOLVE_THREADS, i = idx % W2, j = idx / W2;
      U[i][j] = u4[t];
    }
    __syncthreads();
  }
  // digits of U_P's columns: column c is "row" c of the right operand, over
  // k = row of U_P; four threads per column, eight values each
  __nv_bfloat16* dst = Usl + (size_t)P * NSL * (USL_BYTES / 2);
  if (tid < 4 * W2) {
    const int c = tid >> 2, k0 = (tid & 3) * 8;
    unsigned long long maxbits = 0;
    for (int k = 0; k < W2; ++k) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(U[k][c]) & 0x7FFFFFFFFFFFFFFFULL;
      maxbits = b > maxbits ? b : maxbits;
    }
    const int e = exp_of_maxbits(maxbits);
    if ((tid & 3) == 0) Uexp[P * W2 + c] = e;
    uint32_t d[8][NSL];
#pragma unroll
    for (int j = 0; j < 8; ++j) digits_f32(U[k0 + j][c], e, d[j]);
#pragma unroll
    for (int sl = 0; sl < NSL; ++sl) {
      uint4 q;
      q.x = pack_bf16x2(d[0][sl], d[1][sl]);
      q.y = pack_bf16x2(d[2][sl], d[3][sl]);
      q.z = pack_bf16x2(d[4][sl], d[5][sl]);
      q.w = pack_bf16x2(d[6][sl], d[7][sl]);
      *reinterpret_cast<uint4*>(reinterpret_cast<char*>(dst + (size_t)sl * (USL_BYTES / 2)) + kmaj16(c, k0)) = q;
    }
  }
  if (tid == 0) {
    rotated[P] = any;
    if (any && nrot) atomicAdd(nrot, 1u);
  }
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
  int rexp[TM];
  uint64_t mbar;
  uint32_t tmem;
};

enum { XMODE_COLS = 0, XMODE_ROWS = 1 };

// Y[r, g_Q(c)] = sum_k X_Q(r, k) U_Q(k, c) for block pair Q = blockIdx.y and
// the CTA's 128 rows r: the 32 indices of each of the block pairs
// a = 4 blockIdx.x .. +3 (rows 32 j .. +31 of the tile are pair 4 blockIdx.x + j,
// so epilogue warp w handles exactly pair 4 blockIdx.x + (w mod 4)).
// X_Q(r, k) = X[r + g_Q(k) ldx] (XMODE_COLS) or X[g_Q(k) + r ldx] (XMODE_ROWS).
// Y may alias X in XMODE_COLS (each CTA reads and writes only its own rows of
// its own panel).  Which tiles (a, Q) are formed:
//   TRI_ALL   every tile (V <- V U~);
//   TRI_FIRST tiles a <= Q (B = A U~: only the tiles the second step reads);
//   TRI_SECOND tiles a >= Q of C = B^T U~, written to Y and to the mirror
//             tile (Q, a); in the diagonal tile a = Q the entries on and below
//             the diagonal, mirrored.  So Y = U~^T A U~ stays exactly
//             symmetric, and the second step reads B only in tiles (Q, a),
//             Q <= a, the ones TRI_FIRST formed.
// 256 threads: thread t digitizes tile row t/2 over block half t%2 (the 16
// indices of block I or J of Q); warp w reads the TMEM lanes of rows
// 32 (w mod 4) .. +31 and the 16 output columns 16 (w / 4) .. +15 of each level.
constexpr int RM_THREADS = 256;
enum { TRI_ALL = 0, TRI_FIRST = 1, TRI_SECOND = 2 };

// The 16 values X_Q(row, k), k = g0 .. g0 + 15 (block I or J of Q); zeros for
// row < 0 (no such block pair or a tile that is not formed), row >= n, or
// indices >= n.
MPJ_DEV void load_xrow(const double* X, int ldx, int xmode, int n, int row, int g0, double x[BS]) {
  if (row < 0) {
#pragma unroll
    for (int k = 0; k < BS; ++k) x[k] = 0.0;
  } else if (xmode == XMODE_COLS) {
#pragma unroll
    for (int k = 0; k < BS; ++k) x[k] = (row < n && g0 + k < n) ? X[(size_t)(g0 + k) * ldx + row] : 0.0;
  } else if (row < n && g0 + BS <= n && ((((size_t)row * ldx + g0) & 1) == 0)) {
    const double2* src = reinterpret_cast<const double2*>(X + (size_t)row * ldx + g0);
#pragma unroll
    for (int k = 0; k < BS / 2; ++k) {
      const double2 v = src[k];
      x[2 * k] = v.x;
      x[2 * k + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < BS; ++k) x[k] = (row < n && g0 + k < n) ? X[(size_t)row * ldx + g0 + k] : 0.0;
  }
}

// the global index of tile row rl (pair 4 gx + rl / 32, index rl mod 32), or
// -1 when that pair does not exist
MPJ_DEV int tile_row(int nb, int R, int gx, int rl) {
  const int a = 4 * gx + (rl >> 5);
  if (a >= nb / 2) return -1;
  int I, J;
  block_pair(nb, R, a, I, J);
  return gidx(I, J, rl & 31);
}

MPJ_DEV bool tile_needed(int tri, int a, int Q) {
  return tri == TRI_ALL || (tri == TRI_FIRST ? a <= Q : a >= Q);
}

__global__ void __launch_bounds__(RM_THREADS, 2)
    blk_rmul(const double* X, int ldx, int xmode, double* Y, int ldy, int n, int nb, int R,
             const __nv_bfloat16* __restrict__ Usl, const int* __restrict__ Uexp, const int* __restrict__ rotated,
             unsigned* __restrict__ flags, int tri) {
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  RmulSmem& sm = *reinterpret_cast<RmulSmem*>(dsm_raw + ((1024 - (smem_u32(dsm_raw) & 1023)) & 1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Q = blockIdx.y, gx = blockIdx.x;
  const int a0 = 4 * gx, a1 = min(4 * gx + 3, nb / 2 - 1);
  pdl_wait();
  if (tri == TRI_FIRST && a0 > Q) return;
  if (tri == TRI_SECOND && a1 < Q) return;
  int I, J;
  block_pair(nb, R, Q, I, J);
  if (!rotated[Q]) {
    // no rotation in this block pair: U_Q = I exactly, Y_Q = X_Q (nothing to
    // do in place).  For A, a tile between two block pairs without rotations
    // keeps its values: the second step leaves it alone, so the first need not
    // copy it to B.
    if (X == Y && xmode == XMODE_COLS) return;
    const int rl = tid >> 1, half = tid & 1;
    const int a = a0 + (rl >> 5);
    const int row = tile_row(nb, R, gx, rl);
    const int g0 = (half ? J : I) * BS;
    if (row >= 0 && row < n && tile_needed(tri, a, Q) && (tri == TRI_ALL || rotated[a])) {
      double x[BS];
      load_xrow(X, ldx, xmode, n, row, g0, x);
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        const int g = g0 + c;
        if (g < n && (tri != TRI_SECOND || a > Q || row >= g)) {
          Y[(size_t)g * ldy + row] = x[c];
          if (tri == TRI_SECOND && (a > Q || row > g)) Y[(size_t)row * ldy + g] = x[c];
        }
      }
    }
    return;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar)) : "memory");
  // U_Q digits (contiguous, NSL x 2 KB) and column exponents
  {
    const uint4* src = reinterpret_cast<const uint4*>(Usl + (size_t)Q * NSL * (USL_BYTES / 2));
    uint4* dst = reinterpret_cast<uint4*>(sm.us[0]);
    for (int i = tid; i < NSL * USL_BYTES / 16; i += RM_THREADS) dst[i] = src[i];
    if (tid < W2) sm.uexp[tid] = Uexp[Q * W2 + tid];
  }
  // digits of X_Q: this thread's tile row, 16 values of one block (zeros for
  // rows of tiles that are not formed)
  {
    const int rl = tid >> 1, half = tid & 1;
    const int row = tile_row(nb, R, gx, rl);
    const int g0 = (half ? J : I) * BS;
    double x[BS];
    load_xrow(X, ldx, xmode, n, tile_needed(tri, a0 + (rl >> 5), Q) ? row : -1, g0, x);
    unsigned long long maxbits = 0;
#pragma unroll
    for (int k = 0; k < BS; ++k) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(x[k]) & 0x7FFFFFFFFFFFFFFFULL;
      maxbits = b > maxbits ? b : maxbits;
    }
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, maxbits, 1);
    maxbits = other > maxbits ? other : maxbits;
    const int er = exp_of_maxbits(maxbits);
    if (half == 0) sm.rexp[rl] = er;
#pragma unroll
    for (int k0 = 0; k0 < BS; k0 += 8) {
      uint32_t d[8][NSL];
#pragma unroll
      for (int j = 0; j < 8; ++j) digits_f32(x[k0 + j], er, d[j]);
#pragma unroll
      for (int s = 0; s < NSL; ++s) {
        uint4 q;
        q.x = pack_bf16x2(d[0][s], d[1][s]);
        q.y = pack_bf16x2(d[2][s], d[3][s]);
        q.z = pack_bf16x2(d[4][s], d[5][s]);
        q.w = pack_bf16x2(d[6][s], d[7][s]);
        *reinterpret_cast<uint4*>(sm.xs[s] + kmaj16(rl, half * BS + k0)) = q;
      }
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
  const int quad = warp & 3, ch = warp >> 2;
  const int a = a0 + quad;  // this warp's block pair (warp-uniform)
  if (ok && a < nb / 2 && tile_needed(tri, a, Q)) {
    const int rl = quad * 32 + lane;
    const int row = tile_row(nb, R, gx, rl);
    // Z = sum_L s_L 2^(8 (6 - L)) = hi 2^32 + lo, hi = s0 2^16 + (s1 2^8 + s2),
    // lo = (s3 2^8 + s4) 2^16 + (s5 2^8 + s6); the bracketed pairs fit 32 bits
    // (|s_L| < 2^22.2), so levels are read in pairs and combined in int32
    int t[4][BS];
#pragma unroll
    for (int c = 0; c < BS; ++c) t[0][c] = t[1][c] = t[2][c] = t[3][c] = 0;
#pragma unroll
    for (int l = 0; l < NLEV; ++l) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(l * W2 + ch * BS)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      // level l goes to partial (l + 1) / 2 with weight 2^8 if l is odd (l = 1, 3, 5), 1 otherwise
      const int slot = (l + 1) >> 1;
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        const int q = __float2int_rz(__uint_as_float(v[c]));  // exact integer below 2^23
        t[slot][c] = (l & 1) ? (q << 8) : t[slot][c] + q;
      }
    }
    if (row >= 0 && row < n) {
      const int er = sm.rexp[rl];
      const int g0 = (ch ? J : I) * BS;
      const bool diag = tri == TRI_SECOND && a == Q;
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        const int g = g0 + c;
        if (g < n && (!diag || row >= g)) {
          // hi 2^32 + lo from the partials, both exact as doubles (|hi| < 2^39, |lo| < 2^47);
          // one FP64 add rounds the sum once (the same as rounding Z)
          const int E = er + sm.uexp[ch * BS + c] - 64;
          const long long hi = ((long long)t[0][c] << 16) + t[1][c];
          const long long lo = ((long long)t[2][c] << 16) + t[3][c];
          const int bexp = 32 + E + 1023;
          const double v = (bexp > 60 && bexp < 2000) ? exact_scaled(hi, 32 + E) + exact_scaled(lo, E)
                                                      : z_to_double(hi, lo, E);
          Y[(size_t)g * ldy + row] = v;
          if (tri == TRI_SECOND && (!diag || row > g)) Y[(size_t)row * ldy + g] = v;  // the mirror entry
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

// One set of U_P digit tiles, exponents and rotation flags for a round.
static size_t uset_bytes(int npairs) {
  return al256((size_t)npairs * NSL * USL_BYTES) + al256((size_t)npairs * W2 * sizeof(int)) +
         al256((size_t)npairs * sizeof(int));
}

// Two sets (rounds alternate between them, so the V update of a round may
// still read its set while the next round's subproblems write the other).
size_t mpj_blocked_scratch_bytes(int n) {
  const int N = (n + 2 * BS - 1) / (2 * BS) * (2 * BS);
  return 2 * uset_bytes(N / (2 * BS)) + 256;
}

namespace {
struct USet {
  __nv_bfloat16* sl;
  int* ex;
  int* rot;
};
USet uset(void* scratch, int n, int parity) {
  const int N = (n + 2 * BS - 1) / (2 * BS) * (2 * BS);
  const int npairs = N / (2 * BS);
  char* base = (char*)scratch + (size_t)parity * uset_bytes(npairs);
  USet u;
  u.sl = (__nv_bfloat16*)base;
  u.ex = (int*)(base + al256((size_t)npairs * NSL * USL_BYTES));
  u.rot = (int*)((char*)u.ex + al256((size_t)npairs * W2 * sizeof(int)));
  return u;
}
size_t rmul_smem() {
  // at least 80 KB of shared memory per CTA: at most two CTAs per SM, the two
  // that the 512 TMEM columns hold (256 each), so no CTA waits in tcgen05.alloc
  return sizeof(RmulSmem) + 1024 > 80 * 1024 ? sizeof(RmulSmem) + 1024 : 80 * 1024;
}
cudaError_t rmul_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(blk_rmul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rmul_smem());
  if (e == cudaSuccess) done = true;
  return e;
}
}  // namespace

// Round R, step 1: the subproblems of the block pairs, U_P into set R mod 2;
// *nrot (if not null) counts the block pairs that rotated.
cudaError_t mpj_blocked_solve(const double* A, int lda, int n, int R, double skip, double skip_abs, void* scratch,
                              unsigned* nrot, cudaStream_t s) {
  const int N = (n + 2 * BS - 1) / (2 * BS) * (2 * BS);
  const int nb = N / BS;
  const USet u = uset(scratch, n, R & 1);
  return mpj_launch_pdl(blk_solve, dim3(nb / 2), dim3(SOLVE_THREADS), 0, s, A, lda, n, nb, R, skip, skip_abs, u.sl,
                        u.ex, u.rot, nrot);
}

// Round R, step 2: A <- U~^T A U~ through B (two right multiplications).
cudaError_t mpj_blocked_update_A(double* A, int lda, double* B, int n, int R, void* scratch, unsigned* flags,
                                 cudaStream_t s) {
  const int N = (n + 2 * BS - 1) / (2 * BS) * (2 * BS);
  const int nb = N / BS;
  const USet u = uset(scratch, n, R & 1);
  cudaError_t e = rmul_attr();
  if (e != cudaSuccess) return e;
  const dim3 grid((nb / 2 + 3) / 4, nb / 2);
  e = mpj_launch_pdl(blk_rmul, grid, dim3(RM_THREADS), rmul_smem(), s, (const double*)A, lda, (int)XMODE_COLS, B, n,
                     n, nb, R, (const __nv_bfloat16*)u.sl, (const int*)u.ex, (const int*)u.rot, flags, (int)TRI_FIRST);
  if (e != cudaSuccess) return e;
  return mpj_launch_pdl(blk_rmul, grid, dim3(RM_THREADS), rmul_smem(), s, (const double*)B, n, (int)XMODE_ROWS, A,
                        lda, n, nb, R, (const __nv_bfloat16*)u.sl, (const int*)u.ex, (const int*)u.rot, flags,
                        (int)TRI_SECOND);
}

// Round R, step 3: V <- V U~ (in place); independent of step 2.
cudaError_t mpj_blocked_update_V(double* V, int ldv, int n, int R, void* scratch, unsigned* flags, cudaStream_t s) {
  const int N = (n + 2 * BS - 1) / (2 * BS) * (2 * BS);
  const int nb = N / BS;
  const USet u = uset(scratch, n, R & 1);
  cudaError_t e = rmul_attr();
  if (e != cudaSuccess) return e;
  const dim3 grid((nb / 2 + 3) / 4, nb / 2);
  return mpj_launch_pdl(blk_rmul, grid, dim3(RM_THREADS), rmul_smem(), s, (const double*)V, ldv, (int)XMODE_COLS, V,
                        ldv, n, nb, R, (const __nv_bfloat16*)u.sl, (const int*)u.ex, (const int*)u.rot, flags,
                        (int)TRI_ALL);
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
