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
//   (op(A) op(B))_rc = sum_L 2^(e_r + f_c - 7 L) sum_{i+j=L} sum_k q_i(r,k) q_j(k,c)
// for levels L = 2..9 (the dropped levels are below 2^-57 relative).  Over a
// chunk of 256 values of k every level sum (and every partial sum of it) is
// an integer below 2^24 (at most 2^23.33 for the top levels), so the tensor
// cores' FP32 accumulation of the bf16 products is exact whatever its rounding; each chunk's level sums are read back from tensor memory,
// converted to FP64 exactly and accumulated in FP64.
//
// Layout of the slices in global memory: for slice s and a tile of TR rows
// and 32 values of k, TR x 32 bf16 in the canonical K-major no-swizzle layout
// (8-row x 16-byte core matrices; cores adjacent in k 128 bytes apart, 8-row
// groups 512 bytes apart), so a tile is one contiguous copy into shared memory.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace {

constexpr int OZ_S = 8;                 // slices per value
constexpr int OZ_TM = 128;              // output rows per CTA (MMA M)
constexpr int OZ_TN = 64;               // output columns per CTA (MMA N)
constexpr int OZ_KS = 32;               // k values per staged sub-chunk
constexpr int OZ_KC = 256;              // k values per exact chunk
constexpr int OZ_LEVELS = 8;            // L = 2..9
constexpr uint32_t OZ_TMEM_COLS = 512;  // OZ_LEVELS x OZ_TN FP32 columns
constexpr long long OZ_WAIT_CYCLES = 4000000000LL;

// bytes of one slice tile of TR rows x OZ_KS values
__host__ __device__ constexpr int tile_bytes(int tr) { return tr * OZ_KS * 2; }

MPJ_DEV uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, k) inside a TR x 32 K-major tile (k in [0, 32))
MPJ_DEV int kmaj16(int row, int k) { return (((row >> 3) * 4 + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1); }

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

MPJ_DEV bool oz_test(uint32_t mbar, uint32_t parity) {
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

MPJ_DEV bool oz_wait(uint32_t mbar, uint32_t parity) {
  long long t0 = clock64();
  while (!oz_test(mbar, parity)) {
    if (clock64() - t0 > OZ_WAIT_CYCLES) return false;
    __nanosleep(64);
  }
  return true;
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

// Exponent e with max_k |x(r,k)| < 2^e for each of R rows (x(r,k) = X[r*rs + k*ks]);
// one warp per row.  Rows of zeros get e = 0 (their slices are zero).
__global__ void oz_rowexp(const double* __restrict__ X, long long rs, long long ks, int R, int K, int* __restrict__ e) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= R) return;
  double mx = 0.0;
  for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(X[(long long)warp * rs + (long long)k * ks]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    int ex = 0;
    if (mx > 0.0) frexp(mx, &ex);  // mx = f 2^ex, f in [0.5, 1): mx < 2^ex
    e[warp] = ex;
  }
}

// The 8 slices of every value into the tiled layout (rows padded to a
// multiple of TR, k to a multiple of OZ_KC; padding is zero).
__global__ void oz_slice(const double* __restrict__ X, long long rs, long long ks, int R, int K, int Rp, int Kp, int tr,
                         const int* __restrict__ e, __nv_bfloat16* __restrict__ S) {
  const long long total = (long long)Rp * Kp;
  const long long slice_elems = total;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Kp), r = (int)(idx / Kp);
    double y = (r < R && k < K) ? X[(long long)r * rs + (long long)k * ks] : 0.0;
    if (r < R) y = ldexp(y, -e[r]);  // |y| < 1
    // tile (r / tr, k / 32), then (row, k) inside it
    const long long tile = (long long)(r / tr) * (Kp / OZ_KS) + (k / OZ_KS);
    const long long off = tile * (tr * OZ_KS) + (kmaj16(r % tr, k % OZ_KS) >> 1);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      y *= 128.0;
      const double q = rint(y);
      y -= q;  // exact: y and q share the grid of y's last bit
      S[(long long)s * slice_elems + off] = __double2bfloat16((double)q);  // |q| <= 128: exact
    }
  }
}

struct __align__(16) OzSmem {
  unsigned char a[OZ_S][tile_bytes(OZ_TM)];  // 8 x 8 KB
  unsigned char b[OZ_S][tile_bytes(OZ_TN)];  // 8 x 4 KB
  double colscale[OZ_TN];
  uint64_t mbar;
  uint32_t tmem;
};

__global__ void __launch_bounds__(128, 1)
    oz_gemm(int M, int N, int Kp, const __nv_bfloat16* __restrict__ SA, const __nv_bfloat16* __restrict__ SB,
            long long slice_a, long long slice_b, const int* __restrict__ ea, const int* __restrict__ eb, double alpha,
            double beta, const double* Cin, double* C, int ldc, unsigned* flags) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  OzSmem& sm = *reinterpret_cast<OzSmem*>(dsm);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, nt = blockIdx.y;
  const int row = mt * OZ_TM + warp * 32 + lane;  // the output row this thread accumulates
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.tmem)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.mbar)) : "memory");
  if (tid < OZ_TN) {
    const int c = nt * OZ_TN + tid;
    sm.colscale[tid] = (c < N) ? ldexp(1.0, eb[c]) : 0.0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem;
  const uint32_t mb = smem_addr(&sm.mbar);
  const int er = (row < M) ? ea[row] : 0;

  double acc[OZ_TN];
#pragma unroll
  for (int c = 0; c < OZ_TN; ++c) acc[c] = 0.0;

  const int nsub = Kp / OZ_KS;
  const int ktiles = Kp / OZ_KS;
  uint32_t phase = 0;
  bool ok = true;
  for (int sub = 0; sub < nsub && ok; ++sub) {
    // stage the 8 A slices and 8 B slices of this 32-wide k range
    const long long ta = ((long long)mt * ktiles + sub) * (tile_bytes(OZ_TM) / 2);
    const long long tb = ((long long)nt * ktiles + sub) * (tile_bytes(OZ_TN) / 2);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      const uint4* ga = reinterpret_cast<const uint4*>(SA + s * slice_a + ta);
      uint4* da = reinterpret_cast<uint4*>(sm.a[s]);
      for (int i = tid; i < tile_bytes(OZ_TM) / 16; i += 128) da[i] = ga[i];
      const uint4* gb = reinterpret_cast<const uint4*>(SB + s * slice_b + tb);
      uint4* db = reinterpret_cast<uint4*>(sm.b[s]);
      for (int i = tid; i < tile_bytes(OZ_TN) / 16; i += 128) db[i] = gb[i];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool chunk_start = (sub % (OZ_KC / OZ_KS)) == 0;
    if (tid == 0) {
      constexpr uint32_t idesc = oz_idesc(OZ_TM, OZ_TN);
      bool first[OZ_LEVELS];
#pragma unroll
      for (int l = 0; l < OZ_LEVELS; ++l) first[l] = chunk_start;
      for (int i = 1; i <= OZ_S; ++i)
        for (int j = 1; i + j <= OZ_S + 1; ++j) {
          const int l = i + j - 2;
          const uint32_t d = tmem + (uint32_t)(l * OZ_TN);
#pragma unroll
          for (int kk = 0; kk < OZ_KS / 16; ++kk) {  // K = 16 per instruction: two 16-byte core columns
            oz_mma(d, oz_desc(smem_addr(sm.a[i - 1]) + kk * 256), oz_desc(smem_addr(sm.b[j - 1]) + kk * 256), idesc,
                   first[l] ? 0u : 1u);
            first[l] = false;
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    ok = oz_wait(mb, phase);
    if (!ok) {
      if (flags && lane == 0) atomicOr(flags, MPJ_FLAG_TIMEOUT);
      oz_wait(mb, phase);  // the products may still be in flight
    }
    ok = __all_sync(0xffffffffu, ok);
    ok = __syncthreads_and(ok);
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // end of a chunk: read the level sums (exact integers) and add them in FP64
    if (ok && ((sub + 1) % (OZ_KC / OZ_KS) == 0 || sub + 1 == nsub)) {
#pragma unroll 1
      for (int l = 0; l < OZ_LEVELS; ++l) {
        const double w = ldexp(1.0, er - 7 * (l + 2));
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          uint32_t v[32];
          OZ_LD32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(l * OZ_TN + half * 32), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int c = 0; c < 32; ++c) acc[half * 32 + c] = fma((double)__uint_as_float(v[c]), w, acc[half * 32 + c]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // every level is read before the next chunk overwrites it
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
  }
  if (ok && row < M) {
#pragma unroll
    for (int c = 0; c < OZ_TN; ++c) {
      const int col = nt * OZ_TN + c;
      if (col < N) {
        double v = alpha * (acc[c] * sm.colscale[c]);
        if (beta != 0.0) v = fma(beta, Cin[(long long)col * ldc + row], v);
        C[(long long)col * ldc + row] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
}

}  // namespace

extern "C" int mpj_dgemm_tc(char transa, char transb, int m, int n, int k, double alpha, const double* A, int lda,
                            const double* B, int ldb, double beta, double* C, int ldc, void* stream) {
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && !(transa == 'N' || transa == 'n')) return MPJ_EINVAL;
  if (!tb && !(transb == 'N' || transb == 'n')) return MPJ_EINVAL;
  if (m < 1 || n < 1 || k < 1 || !A || !B || !C) return MPJ_EINVAL;
  if (lda < (ta ? k : m) || ldb < (tb ? n : k) || ldc < m) return MPJ_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int Mp = (m + OZ_TM - 1) / OZ_TM * OZ_TM, Np = (n + OZ_TN - 1) / OZ_TN * OZ_TN;
  const int Kp = (k + OZ_KC - 1) / OZ_KC * OZ_KC;
  const long long slice_a = (long long)Mp * Kp, slice_b = (long long)Np * Kp;
  const size_t bytes = (size_t)OZ_S * (slice_a + slice_b) * 2 + (size_t)(Mp + Np) * sizeof(int) + 256;
  char* w = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&w, bytes, s);
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "mpj_dgemm_tc workspace", __LINE__);
    return MPJ_ENOMEM;
  }
  __nv_bfloat16* SA = (__nv_bfloat16*)w;
  __nv_bfloat16* SB = SA + OZ_S * slice_a;
  int* ea = (int*)(SB + OZ_S * slice_b);
  int* eb = ea + Mp;
  unsigned* flag = (unsigned*)(eb + Np);
  // op(A)(r, kk) = A[r*rs + kk*ks]; op(B)^T(c, kk) = op(B)(kk, c)
  const long long ars = ta ? lda : 1, aks = ta ? 1 : lda;
  const long long brs = tb ? 1 : ldb, bks = tb ? ldb : 1;
  const size_t smem = sizeof(OzSmem) + 1024;
  e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    oz_rowexp<<<(m + 7) / 8, 256, 0, s>>>(A, ars, aks, m, k, ea);
    mpj_count_launch();
    oz_rowexp<<<(n + 7) / 8, 256, 0, s>>>(B, brs, bks, n, k, eb);
    mpj_count_launch();
    oz_slice<<<4096, 256, 0, s>>>(A, ars, aks, m, k, Mp, Kp, OZ_TM, ea, SA);
    mpj_count_launch();
    oz_slice<<<4096, 256, 0, s>>>(B, brs, bks, n, k, Np, Kp, OZ_TN, eb, SB);
    mpj_count_launch();
    e = cudaFuncSetAttribute(oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (e == cudaSuccess) {
    dim3 grid(Mp / OZ_TM, Np / OZ_TN);
    oz_gemm<<<grid, 128, smem, s>>>(m, n, Kp, SA, SB, slice_a, slice_b, ea, eb, alpha, beta, C, C, ldc, flag);
    mpj_count_launch();
    e = cudaGetLastError();
  }
  unsigned h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(w, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "mpj_dgemm_tc", __LINE__);
    return MPJ_ECUDA;
  }
  return (h & MPJ_FLAG_TIMEOUT) ? MPJ_ETIMEOUT : MPJ_OK;
}
