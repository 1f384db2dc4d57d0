// ozaki.cu -- FP64 matrix products on the tcgen05 tensor cores from exact
// bf16 slices (an Ozaki-type splitting; the paper's products are plain FP64,
// Sec. 4.3.4 and Algorithm 9, and GB300's FP64 tensor rate is no faster than
// its FP64 FMA pipe).
//
// C = alpha op(A) op(B) + beta C, all FP64.  Each row r of op(A) is written on
// the grid of its largest binary exponent e_r (max |a_rk| < 2^e_r) as
//   a_rk = sum_{i=1..8} q_i(r,k) 2^(e_r - 7 i) + (a remainder below 2^(e_r - 57)),
// with integers |q_1| <= 128 and |q_i| <= 64 (i > 1), each exactly a bf16; the
// same for each column c of op(B) with exponents f_c.  Then
//   (op(A) op(B))_rc = 2^(e_r + f_c) sum_L 2^(-7 L) s_L(r,c),
//   s_L(r,c) = sum_{i+j=L} sum_k q_i(r,k) q_j(k,c),
// for levels L = 2..9 (the dropped levels are below 2^-54 relative to
// max|a_r.| max|b_.c| per term).  Over a chunk of 256 values of k every level
// sum (and every partial sum of it) is an integer of magnitude below 2^24 (at
// most 2^23.33, for the top levels), so the tensor cores' FP32 accumulation
// of the bf16 products is exact.  The epilogue converts each chunk's level
// sums to integers and accumulates them exactly in two 64-bit integers per
// output (levels 2..5 and 6..9, weights 2^(7(5-L)) and 2^(7(9-L)): below
// 2^48 after 16 chunks, so a launch covers up to 4096 values of k exactly;
// longer K runs as several launches that add into C).  The result is
//   2^(e_r + f_c) (hi 2^-35 + lo 2^-63),
// one rounding in FP64 for the sum and an exact power-of-two scaling, so the
// exponent sum is applied once and no intermediate weight can underflow.
//
// Sliced operand layout in global memory: for slice s, the rows are cut into
// 64-row groups and k into 32-wide groups; tile (k-group g, row group t) is
// 64 x 32 bf16 in the canonical K-major no-swizzle layout (8-row x 16-byte
// core matrices, k-adjacent cores 128 bytes apart, 8-row groups 512 bytes
// apart) and tiles are stored k-group-major: tile index g * (Rp / 64) + t.
// The two 64-row tiles of a 128-row MMA operand are therefore adjacent, one
// 8 KB bulk copy; a 64-row operand is one 4 KB bulk copy.
//
// The product kernel: one CTA per 128 x 64 output tile (one CTA per SM: its
// 192 KB shared-memory ring and 512 TMEM columns), 10 warps:
//   warp 8 (one thread): producer -- cp.async.bulk copies of the 16 slice
//          tiles of a 32-wide k step into one of two ring stages, completion
//          counted by the stage's "full" mbarrier (transaction bytes);
//   warp 9 (one thread): issues the 36 x 2 tcgen05.mma (M = 128, N = 64,
//          K = 16) of a k step into the 8 level accumulators (8 x 64 TMEM
//          columns), then tcgen05.commit to the stage's "empty" mbarrier, and
//          to "tmem_full" after the last k step of a 256-wide chunk;
//   warps 0-7: epilogue -- wait "tmem_full", read the 8 levels (warp w reads
//          TMEM lanes 32 (w mod 4) .. +31, columns 32 (w / 4) .. +31 of each
//          level), arrive on "tmem_empty", accumulate in integers.
// Every wait is bounded (about 2 s); a wait that runs out sets
// MPJ_FLAG_TIMEOUT, stops the other roles, waits (bounded) for work in
// flight, frees TMEM and leaves C untouched.
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include "common.cuh"
#include <stdlib.h>

#include "ozaki.cuh"

namespace {

constexpr int OZ_S = 8;              // slices per value
constexpr int OZ_TM = 128;           // output rows per CTA (MMA M)
constexpr int OZ_TN = 64;            // output columns per CTA (MMA N)
constexpr int OZ_KS = 32;            // k values per ring stage
constexpr int OZ_KC = 256;           // k values per exact chunk
constexpr int OZ_LEVELS = 8;         // L = 2..9
constexpr int OZ_PASS_SUBS = 4096 / OZ_KS;  // k steps per launch (exact integer accumulation)
constexpr uint32_t OZ_TMEM_COLS = 512;
constexpr int OZ_TILE64 = 64 * OZ_KS;                       // bf16 elements of a 64-row tile
constexpr uint32_t OZ_A_BYTES = OZ_TM * OZ_KS * 2;          // 8 KB per slice
constexpr uint32_t OZ_B_BYTES = OZ_TN * OZ_KS * 2;          // 4 KB per slice
constexpr uint32_t OZ_STAGE_BYTES = OZ_S * (OZ_A_BYTES + OZ_B_BYTES);  // 96 KB
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = (OZ_EPI_WARPS + 2) * 32;
constexpr long long OZ_WAIT_CYCLES = 4000000000LL;
constexpr int OZ_GROUP_M = 8;

MPJ_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, k) inside a 64- or 128-row x 32 K-major tile (k in [0, 32))
__host__ __device__ inline int kmaj16(int row, int k) {
  return (((row >> 3) * 4 + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

MPJ_DEV uint64_t oz_desc(uint32_t saddr) {
  // start address, LBO = 128 bytes (k-adjacent cores), SBO = 512 bytes (8-row
  // groups), tcgen05 descriptor version 1, no swizzle
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: D F32, A and B bf16, both K-major
__host__ __device__ constexpr uint32_t oz_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

MPJ_DEV void oz_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

MPJ_DEV void oz_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
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

MPJ_DEV void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

MPJ_DEV void mbar_arrive(uint32_t mbar) {
  uint64_t st;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(st) : "r"(mbar) : "memory");
  (void)st;
}

MPJ_DEV void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  uint64_t st;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;" : "=l"(st) : "r"(mbar), "r"(bytes) : "memory");
  (void)st;
}

MPJ_DEV void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// Bounded wait for the phase of parity `parity`; false when the budget runs
// out (then the CTA's abort word is set) or another role aborted.
MPJ_DEV bool oz_wait(uint32_t mbar, uint32_t parity, volatile int* abort_flag, unsigned* gflags) {
  const long long t0 = clock64();
  while (!mbar_test(mbar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > OZ_WAIT_CYCLES) {
      *abort_flag = 1;
      if (gflags) atomicOr(gflags, MPJ_FLAG_TIMEOUT);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// The same without the abort word (used to drain work in flight on abort).
MPJ_DEV void oz_drain(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(mbar, parity) && clock64() - t0 <= OZ_WAIT_CYCLES) __nanosleep(64);
}

#define OZ_LD32(taddr, v)                                                                                          \
  asm volatile(                                                                                                    \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18," \
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                               \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),           \
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),     \
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),   \
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])    \
      : "r"(taddr))

// ---- slicing ----------------------------------------------------------------
// The slicing uses integer and FP32 instructions only (an FP64 instruction
// costs 64 FP32 ones on this GPU).

// |x| as the bit pattern of a non-negative double (ordered like the value)
MPJ_DEV unsigned long long oz_absbits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}

// The smallest e with max|x| < 2^e from the bit pattern of max|x| (0 for
// zero): the exponent frexp returns.
MPJ_DEV int oz_exp_of(unsigned long long b) {
  if (b == 0) return 0;
  const int ex = (int)(b >> 52);
  if (ex > 0) return ex - 1022;
  return (64 - __clzll((long long)b)) - 1074;  // subnormal
}

// The 8 slices of x on the grid 2^e (|x| < 2^e) as FP32 bit patterns of
// small integers (their top 16 bits are the bf16): x = sum_i q_i 2^(e - 7 i) + r
// with |q_1| <= 128, |q_i| <= 64 (i > 1), |r| <= 2^(e - 57).  Y = |x| 2^(56 - e)
// rounded to an integer (half up; Y < 2^56), then balanced base-128 digits:
// adding 64 to each of Y's seven low 7-bit groups (one 64-bit add, carries
// included) makes group j equal d + 64 for a digit d in [-64, 63] of weight
// 128^j, and the part above bit 49 the top digit in [0, 128].  A group g
// becomes a float through the bit pattern of 2^23 + g; one FMA gives
// sign(x) (g - 64).
MPJ_DEV void oz_digits(double x, int e, uint32_t q[OZ_S]) {
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
  const unsigned long long T = Y + 0x0001020408102040ULL;  // 64 * (1 + 128 + ... + 128^6)
  const float sg = (bits >> 63) ? -1.0f : 1.0f;
  const float c64 = -8388672.0f * sg;  // -(2^23 + 64) sign(x)
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const uint32_t g = (uint32_t)(T >> (7 * j)) & 127u;
    q[OZ_S - 1 - j] = __float_as_uint(fmaf(__uint_as_float(0x4B000000u | g), sg, c64));
  }
  q[0] = __float_as_uint(fmaf(__uint_as_float(0x4B000000u | (uint32_t)(T >> 49)), sg, -8388608.0f * sg));
}

// Two FP32 digit patterns packed as two bf16 (a in the low half).
MPJ_DEV uint32_t oz_pack2(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x7632); }

// Largest |x(r, k)| per row as the bit pattern of a non-negative double
// (ordered like the value), combined with atomicMax.  Rows of a column-major
// matrix (rs == 1): one thread per row over a strip of k, coalesced across rows.
__global__ void oz_rowmax_cols(const double* __restrict__ X, long long ks, int R, int K, int kstrip,
                               unsigned long long* __restrict__ mx) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int k0 = blockIdx.y * kstrip, k1 = min(K, k0 + kstrip);
  unsigned long long m = 0;  // max of the magnitudes' bit patterns (integer compares, no FP64)
  for (int k = k0; k < k1; ++k) m = max(m, oz_absbits(X[r + (long long)k * ks]));
  if (m) atomicMax(mx + r, m);
}

// Rows stored contiguously (or any other stride): one warp per row.
__global__ void oz_rowmax_warp(const double* __restrict__ X, long long rs, long long ks, int R, int K,
                               unsigned long long* __restrict__ mx) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= R) return;
  unsigned long long m = 0;
  for (int k = lane; k < K; k += 32) m = max(m, oz_absbits(X[(long long)warp * rs + (long long)k * ks]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) mx[warp] = m;
}

// The 8 slices of 8 consecutive k values of one row per thread, written as
// one 16-byte core-matrix row per slice.  rows_fast: consecutive threads take
// consecutive rows (coalesced reads of column-major rows).
__global__ void oz_slice(const double* __restrict__ X, long long rs, long long ks, int R, int K, int Rp, int Kp,
                         int rows_fast, const unsigned long long* __restrict__ mx, int* __restrict__ exps,
                         __nv_bfloat16* __restrict__ S) {
  const long long total = (long long)Rp * (Kp / 8);
  const long long slice_elems = (long long)Rp * Kp;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int r, g;
    if (rows_fast) {
      r = (int)(idx % Rp);
      g = (int)(idx / Rp);
    } else {
      g = (int)(idx % (Kp / 8));
      r = (int)(idx / (Kp / 8));
    }
    const int k0 = g * 8;
    const int e = r < R ? oz_exp_of(mx[r]) : 0;  // every |x(r, k)| < 2^e
    if (g == 0) exps[r] = e;
    uint32_t d[8][OZ_S];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + j;
      const double x = (r < R && k < K) ? X[(long long)r * rs + (long long)k * ks] : 0.0;
      oz_digits(x, e, d[j]);
    }
    const long long tile = (long long)(k0 / OZ_KS) * (Rp / 64) + r / 64;
    const long long off = tile * OZ_TILE64 + (kmaj16(r & 63, k0 & 31) >> 1);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      uint4 q;
      q.x = oz_pack2(d[0][s], d[1][s]);
      q.y = oz_pack2(d[2][s], d[3][s]);
      q.z = oz_pack2(d[4][s], d[5][s]);
      q.w = oz_pack2(d[6][s], d[7][s]);
      *reinterpret_cast<uint4*>(S + s * slice_elems + off) = q;
    }
  }
}

// ---- the product ------------------------------------------------------------
struct __align__(1024) OzSmem {
  unsigned char stage[2][OZ_STAGE_BYTES];  // per stage: 8 A slices (8 KB), then 8 B slices (4 KB)
  uint64_t full[2], empty[2], tmem_full, tmem_empty;
  int colexp[OZ_TN];
  uint32_t tmem;
  int abort_flag;
};

__global__ void __maxnreg__(168)
    oz_gemm_kernel(const __nv_bfloat16* __restrict__ SA, const int* __restrict__ ea, int Rpa,
                   const __nv_bfloat16* __restrict__ SB, const int* __restrict__ eb, int Rpb, int Kp, int sub0,
                   int nsub, int m, int n, double alpha, double beta, const double* Cin, int ldcin, double* C,
                   int ldc, unsigned* gflags, int lower) {
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  OzSmem& sm = *reinterpret_cast<OzSmem*>(dsm_raw + ((1024 - (smem_u32(dsm_raw) & 1023)) & 1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tile order: groups of OZ_GROUP_M row tiles share the B tiles in L2
  const int ntm = (m + OZ_TM - 1) / OZ_TM, ntn = (n + OZ_TN - 1) / OZ_TN;
  const int id = blockIdx.x;
  const int group = id / (OZ_GROUP_M * ntn);
  const int first_m = group * OZ_GROUP_M;
  const int gsz = min(ntm - first_m, OZ_GROUP_M);
  const int local = id % (OZ_GROUP_M * ntn);
  const int mt = first_m + local % gsz, nt = local / gsz;
  // lower: only tiles that meet the lower triangle (row >= column) are formed
  if (lower && mt * OZ_TM + OZ_TM - 1 < nt * OZ_TN) return;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&sm.full[s]), 1);
      mbar_init(smem_u32(&sm.empty[s]), 1);
    }
    mbar_init(smem_u32(&sm.tmem_full), 1);
    mbar_init(smem_u32(&sm.tmem_empty), OZ_EPI_WARPS * 32);
    sm.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < OZ_TN) {
    const int c = nt * OZ_TN + tid;
    sm.colexp[tid] = (c < n) ? eb[c] : 0;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem;
  volatile int* abort_flag = &sm.abort_flag;
  const uint32_t stage0 = smem_u32(sm.stage[0]);

  if (warp == OZ_EPI_WARPS) {
    // ---------------- producer
    if (lane == 0) {
      int issued = 0;
      for (int sub = 0; sub < nsub; ++sub) {
        const int st = sub & 1;
        if (sub >= 2 && !oz_wait(smem_u32(&sm.empty[st]), ((sub >> 1) - 1) & 1, abort_flag, gflags)) break;
        const uint32_t fb = smem_u32(&sm.full[st]);
        mbar_expect_tx(fb, OZ_STAGE_BYTES);
        const uint32_t dA = stage0 + st * OZ_STAGE_BYTES, dB = dA + OZ_S * OZ_A_BYTES;
        const long long ta = ((long long)(sub0 + sub) * (Rpa / 64) + 2 * mt) * OZ_TILE64;
        const long long tb = ((long long)(sub0 + sub) * (Rpb / 64) + nt) * OZ_TILE64;
#pragma unroll 1
        for (int s = 0; s < OZ_S; ++s) {
          bulk_g2s(dA + s * OZ_A_BYTES, SA + (long long)s * Rpa * Kp + ta, OZ_A_BYTES, fb);
          bulk_g2s(dB + s * OZ_B_BYTES, SB + (long long)s * Rpb * Kp + tb, OZ_B_BYTES, fb);
        }
        issued = sub + 1;
      }
      if (*abort_flag) {
        // copies in flight still land in this CTA's shared memory: wait for them
        for (int sub = (issued > 2 ? issued - 2 : 0); sub < issued; ++sub)
          oz_drain(smem_u32(&sm.full[sub & 1]), (sub >> 1) & 1);
      }
    }
  } else if (warp == OZ_EPI_WARPS + 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = oz_idesc(OZ_TM, OZ_TN);
      int last_commit_sub = -1;
      for (int sub = 0; sub < nsub; ++sub) {
        const int st = sub & 1;
        const int chunk = sub / (OZ_KC / OZ_KS);
        const bool chunk_start = (sub % (OZ_KC / OZ_KS)) == 0;
        if (!oz_wait(smem_u32(&sm.full[st]), (sub >> 1) & 1, abort_flag, gflags)) break;
        if (chunk_start && chunk > 0 && !oz_wait(smem_u32(&sm.tmem_empty), (chunk - 1) & 1, abort_flag, gflags))
          break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t aB = stage0 + st * OZ_STAGE_BYTES, bB = aB + OZ_S * OZ_A_BYTES;
        uint32_t started = chunk_start ? 0u : 0xFFu;
        for (int i = 1; i <= OZ_S; ++i)
          for (int j = 1; i + j <= OZ_S + 1; ++j) {
            const int l = i + j - 2;
            const uint32_t d = tmem + (uint32_t)(l * OZ_TN);
#pragma unroll
            for (int kk = 0; kk < OZ_KS / 16; ++kk) {
              oz_mma(d, oz_desc(aB + (i - 1) * OZ_A_BYTES + kk * 256), oz_desc(bB + (j - 1) * OZ_B_BYTES + kk * 256),
                     idesc, (started >> l) & 1u);
              started |= 1u << l;
            }
          }
        oz_commit(smem_u32(&sm.empty[st]));
        last_commit_sub = sub;
        if ((sub + 1) % (OZ_KC / OZ_KS) == 0 || sub + 1 == nsub) oz_commit(smem_u32(&sm.tmem_full));
      }
      if (*abort_flag && last_commit_sub >= 0)  // MMAs in flight still use TMEM and the ring
        oz_drain(smem_u32(&sm.empty[last_commit_sub & 1]), (last_commit_sub >> 1) & 1);
    }
  } else {
    // ---------------- epilogue: warps 0-7
    const int quad = warp & 3, half = warp >> 2;
    const int row = mt * OZ_TM + quad * 32 + lane;
    const int nchunks = nsub / (OZ_KC / OZ_KS);
    long long hi[32], lo[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      hi[c] = 0;
      lo[c] = 0;
    }
    bool ok = true;
    for (int chunk = 0; chunk < nchunks; ++chunk) {
      if (!oz_wait(smem_u32(&sm.tmem_full), chunk & 1, abort_flag, gflags)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int l = 0; l < OZ_LEVELS; ++l) {
        uint32_t v[32];
        OZ_LD32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(l * OZ_TN + half * 32), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (l == OZ_LEVELS - 1) {
          // every level of this chunk is in registers: the MMAs of the next chunk may start
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(smem_u32(&sm.tmem_empty));
        }
        const int sh = 7 * (3 - (l & 3));
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const long long q = (long long)__float2int_rz(__uint_as_float(v[c]));  // an exact integer below 2^24
          if (l < 4)
            hi[c] += q << sh;
          else
            lo[c] += q << sh;
        }
      }
    }
    if (ok && !*abort_flag && row < m) {
      const int er = ea[row];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int cl = half * 32 + c;
        const int col = nt * OZ_TN + cl;
        if (col < n) {
          const double v = fma((double)hi[c], 0x1p-35, (double)lo[c] * 0x1p-63);
          double out = alpha * ldexp(v, er + sm.colexp[cl]);
          if (beta != 0.0) out = fma(beta, Cin[(long long)col * ldcin + row], out);
          C[(long long)col * ldc + row] = out;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
}

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
inline int pad_rows(int R) { return (R + OZ_TM - 1) / OZ_TM * OZ_TM; }
inline int pad_k(int K) { return (K + OZ_KC - 1) / OZ_KC * OZ_KC; }

}  // namespace

bool mpj_gemm_tc_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("MPJ_GEMM_TC");
    v = (e && e[0] == '0') ? 0 : 1;
  }
  return v == 1;
}

size_t mpj_oz_operand_bytes(int R, int K) {
  const size_t Rp = (size_t)pad_rows(R), Kp = (size_t)pad_k(K);
  return al256((size_t)OZ_S * Rp * Kp * 2) + al256(Rp * sizeof(int)) + al256(Rp * sizeof(unsigned long long));
}

cudaError_t mpj_oz_prepare(const double* X, long long rs, long long ks, int R, int K, void* buf, OzOperand* op,
                           cudaStream_t s) {
  const int Rp = pad_rows(R), Kp = pad_k(K);
  char* b = (char*)buf;
  __nv_bfloat16* S = (__nv_bfloat16*)b;
  int* exps = (int*)(b + al256((size_t)OZ_S * Rp * Kp * 2));
  unsigned long long* mx = (unsigned long long*)((char*)exps + al256((size_t)Rp * sizeof(int)));
  cudaError_t e = cudaMemsetAsync(mx, 0, (size_t)Rp * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (rs == 1) {
    const int kstrip = 64;
    dim3 grid((R + 127) / 128, (K + kstrip - 1) / kstrip);
    oz_rowmax_cols<<<grid, 128, 0, s>>>(X, ks, R, K, kstrip, mx);
  } else {
    oz_rowmax_warp<<<(R + 7) / 8, 256, 0, s>>>(X, rs, ks, R, K, mx);
  }
  mpj_count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "oz_rowmax launch", __LINE__);
    return e;
  }
  const long long total = (long long)Rp * (Kp / 8);
  const int blocks = (int)((total + 255) / 256 > 8192 ? 8192 : (total + 255) / 256);
  oz_slice<<<blocks, 256, 0, s>>>(X, rs, ks, R, K, Rp, Kp, rs == 1 ? 1 : 0, mx, exps, S);
  mpj_count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "oz_slice launch", __LINE__);
    return e;
  }
  op->slices = S;
  op->exps = exps;
  op->R = R;
  op->K = K;
  op->Rp = Rp;
  op->Kp = Kp;
  return cudaSuccess;
}

cudaError_t mpj_oz_gemm(const OzOperand& a, const OzOperand& b, int m, int n, double alpha, double beta,
                        const double* Cin, int ldcin, double* C, int ldc, unsigned* flags, cudaStream_t s,
                        bool lower) {
  if (a.Kp != b.Kp || m > a.R || n > b.R || m < 1 || n < 1) return cudaErrorInvalidValue;
  const size_t smem = sizeof(OzSmem) + 1024;
  cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int ntm = (m + OZ_TM - 1) / OZ_TM, ntn = (n + OZ_TN - 1) / OZ_TN;
  const int total = a.Kp / OZ_KS;
  for (int sub0 = 0; sub0 < total; sub0 += OZ_PASS_SUBS) {
    const int ns = total - sub0 < OZ_PASS_SUBS ? total - sub0 : OZ_PASS_SUBS;
    const bool first = sub0 == 0;
    oz_gemm_kernel<<<ntm * ntn, OZ_THREADS, smem, s>>>(a.slices, a.exps, a.Rp, b.slices, b.exps, b.Rp, a.Kp, sub0, ns,
                                                        m, n, alpha, first ? beta : 1.0, first ? Cin : C,
                                                        first ? ldcin : ldc, C, ldc, flags, lower ? 1 : 0);
    mpj_count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      cudaFuncAttributes fa;
      char what[160];
      if (cudaFuncGetAttributes(&fa, oz_gemm_kernel) == cudaSuccess)
        snprintf(what, sizeof what, "oz_gemm_kernel launch (regs %d, max threads %d, static smem %zu, dyn smem %zu)",
                 fa.numRegs, fa.maxThreadsPerBlock, fa.sharedSizeBytes, smem);
      else
        snprintf(what, sizeof what, "oz_gemm_kernel launch");
      mpj_set_cuda_error(e, what, __LINE__);
      return e;
    }
  }
  return cudaSuccess;
}

extern "C" int mpj_dgemm_tc(char transa, char transb, int m, int n, int k, double alpha, const double* A, int lda,
                            const double* B, int ldb, double beta, double* C, int ldc, void* stream) {
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && !(transa == 'N' || transa == 'n')) return MPJ_EINVAL;
  if (!tb && !(transb == 'N' || transb == 'n')) return MPJ_EINVAL;
  if (m < 1 || n < 1 || k < 1 || !A || !B || !C) return MPJ_EINVAL;
  if (lda < (ta ? k : m) || ldb < (tb ? n : k) || ldc < m) return MPJ_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ba = mpj_oz_operand_bytes(m, k), bb = mpj_oz_operand_bytes(n, k);
  const size_t bytes = ba + bb + 256;
  char* w = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&w, bytes, s);
  mpj_count_alloc();
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "mpj_dgemm_tc workspace", __LINE__);
    return MPJ_ENOMEM;
  }
  unsigned* flag = (unsigned*)(w + ba + bb);
  // op(A)(r, kk) = A[r*rs + kk*ks]; op(B)^T(c, kk) = op(B)(kk, c)
  const long long ars = ta ? lda : 1, aks = ta ? 1 : lda;
  const long long brs = tb ? 1 : ldb, bks = tb ? ldb : 1;
  OzOperand oa, ob;
  e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = mpj_oz_prepare(A, ars, aks, m, k, w, &oa, s);
  if (e == cudaSuccess) e = mpj_oz_prepare(B, brs, bks, n, k, w + ba, &ob, s);
  if (e == cudaSuccess) e = mpj_oz_gemm(oa, ob, m, n, alpha, beta, C, ldc, C, ldc, flag, s);
  const bool described = e != cudaSuccess;  // the failing step already recorded its message
  unsigned h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(w, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    if (!described) mpj_set_cuda_error(e, "mpj_dgemm_tc", __LINE__);
    return MPJ_ECUDA;
  }
  return (h & MPJ_FLAG_TIMEOUT) ? MPJ_ETIMEOUT : MPJ_OK;
}
