// tc32.cu -- 3xTF32 panel products on the tcgen05 tensor cores for the
// blocked update of the stage-1 FP32 Jacobi (Sec. 4.1 asks only for an
// approximate Q_l; the block ordering is described in stage1.cu).
//
// One CTA (4 warps) computes a 128-row tile of Out[:, I_q] = In[:, I_q] U_q
// for QPC block pairs q.  Operands are staged by the threads into shared
// memory in the canonical K-major layout without swizzle (8-row x 16-byte
// core matrices; core matrices adjacent in K are 128 bytes apart, 8-row
// groups 1024 bytes apart), each split into a TF32 head and an FP32 tail
// (x = hi + lo exactly, hi = x rounded to TF32).  One thread issues, per
// block pair, 3 x 4 tcgen05.mma (M = 128, N = 32, K = 8 each) for
// hi*hi + hi*lo + lo*hi into 32 tensor-memory columns, commits them to an
// mbarrier, and the four warps read their 32 accumulator lanes back with
// tcgen05.ld.  The lo*lo term (2^-22 relative) is dropped: the result is
// accurate to about 2^-21 relative per product, which is what an FP32 stage
// needs (its rotations are themselves FP32).
#include <stdint.h>

#include "common.cuh"
#include "tc32.cuh"

namespace {

constexpr int TM = 128;             // rows per tile (MMA M)
constexpr int KQ = 32;              // indices per block pair (MMA K and N)
constexpr int QPC = 2;              // block pairs per CTA
constexpr int TPB = 128;            // threads per CTA
constexpr uint32_t TMEM_COLS = 64;  // QPC x 32 FP32 accumulator columns
constexpr int X_FLOATS = TM * KQ;   // one operand tile (16 KB)
constexpr int U_FLOATS = KQ * KQ;   // one U_q (4 KB)
// shared memory: xh[QPC], xl[QPC], uh[QPC], ul[QPC], then mbarrier + TMEM address
constexpr size_t SMEM_BYTES = (size_t)(2 * QPC * X_FLOATS + 2 * QPC * U_FLOATS) * 4 + 64;
constexpr long long WAIT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz

MPJ_DEV int bgidx(int I, int J, int l) { return l < 16 ? I * 16 + l : J * 16 + (l - 16); }

MPJ_DEV void block_pair_tc(int nb, int R, int slot, int& I, int& J) {
  int x, y;
  rr_slot(nb, R, slot, x, y);
  I = x < y ? x : y;
  J = x < y ? y : x;
}

// float offset of element (row r, column k) of a K-major tile with 32 columns
MPJ_DEV int kmaj(int r, int k) { return (((r >> 3) * 8 + (k >> 2)) << 5) + ((r & 7) << 2) + (k & 3); }

MPJ_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// x = hi + lo with hi the TF32 rounding of x (low 13 mantissa bits zero)
MPJ_DEV void split_tf32(float x, float& hi, float& lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  // round the tail too: the tensor cores would otherwise truncate it (a bias
  // that accumulates over thousands of products)
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hi));
  lo = __uint_as_float(l);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K)
// byte offset, stride (M/N) byte offset, all >> 4; bits 46-47 = 1 (the
// tcgen05 descriptor version); base offset 0; no swizzle.
MPJ_DEV uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

MPJ_DEV void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
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

// Wait for phase `parity` of the mbarrier for at most WAIT_CYCLES.
MPJ_DEV bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  long long t0 = clock64();
  while (!mbar_test(mbar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
    __nanosleep(64);
  }
  return true;
}

#define TC_LD32(taddr, v)                                                                                          \
  asm volatile(                                                                                                    \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18," \
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                               \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),           \
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),     \
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),   \
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])    \
      : "r"(taddr))

__global__ void __launch_bounds__(TPB) tc_panel_kernel(int N, int nb, int R, const float* __restrict__ Ubuf,
                                                       const float* In, float* Out, int transpose_out,
                                                       const float* In2, float* Out2, unsigned* flags,
                                                       int no_commit) {
  extern __shared__ __align__(1024) float sm[];
  float* xh = sm;                          // [QPC][X_FLOATS]
  float* xl = xh + QPC * X_FLOATS;         // [QPC][X_FLOATS]
  float* uh = xl + QPC * X_FLOATS;         // [QPC][U_FLOATS]
  float* ul = uh + QPC * U_FLOATS;         // [QPC][U_FLOATS]
  uint64_t* mbar = (uint64_t*)(ul + QPC * U_FLOATS);
  uint32_t* tmem_slot = (uint32_t*)(mbar + 1);

  const bool second = blockIdx.z == 1;
  const float* src = second ? In2 : In;
  float* dst = second ? Out2 : Out;
  const int tr = second ? 0 : transpose_out;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * TM;
  const int npairs = nb / 2;
  const int q0 = blockIdx.y * QPC;
  const int nq = min(QPC, npairs - q0);

  // tensor memory for the accumulators (warp 0 allocates and frees)
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
  }

  // stage the operands: row r = tid of the tile, 4 columns at a time
  const int r = row0 + tid;
  for (int qi = 0; qi < nq; ++qi) {
    int I, J;
    block_pair_tc(nb, R, q0 + qi, I, J);
    float* th = xh + qi * X_FLOATS;
    float* tl = xl + qi * X_FLOATS;
#pragma unroll
    for (int kc = 0; kc < KQ / 4; ++kc) {
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int gc = bgidx(I, J, 4 * kc + e);
        v[e] = (r < N) ? src[(size_t)gc * N + r] : 0.0f;
      }
      float4 h, l;
      split_tf32(v[0], h.x, l.x);
      split_tf32(v[1], h.y, l.y);
      split_tf32(v[2], h.z, l.z);
      split_tf32(v[3], h.w, l.w);
      int off = kmaj(tid, 4 * kc);
      *reinterpret_cast<float4*>(th + off) = h;
      *reinterpret_cast<float4*>(tl + off) = l;
    }
    // U_q as the B operand (N x K, K-major): element (n, k) = U_q(k, n)
    const float* U = Ubuf + (size_t)(q0 + qi) * U_FLOATS;
    for (int e = tid; e < U_FLOATS / 4; e += TPB) {
      int nn = e >> 3, kc = e & 7;
      float4 u = *reinterpret_cast<const float4*>(U + 32 * nn + 4 * kc);
      float4 h, l;
      split_tf32(u.x, h.x, l.x);
      split_tf32(u.y, h.y, l.y);
      split_tf32(u.z, h.z, l.z);
      split_tf32(u.w, h.w, l.w);
      int off = kmaj(nn, 4 * kc);
      *reinterpret_cast<float4*>(uh + qi * U_FLOATS + off) = h;
      *reinterpret_cast<float4*>(ul + qi * U_FLOATS + off) = l;
    }
  }
  // make the generic-proxy shared stores visible to the tensor cores
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t mb = smem_u32(mbar);

  if (tid == 0 && !no_commit) {  // no_commit: failure-detection test, nothing is issued
    constexpr uint32_t idesc = idesc_tf32(TM, KQ);
    for (int qi = 0; qi < nq; ++qi) {
      const uint32_t d = tmem + (uint32_t)(qi * KQ);
      const uint32_t a_h = smem_u32(xh + qi * X_FLOATS), a_l = smem_u32(xl + qi * X_FLOATS);
      const uint32_t b_h = smem_u32(uh + qi * U_FLOATS), b_l = smem_u32(ul + qi * U_FLOATS);
      const uint32_t as[3] = {a_h, a_h, a_l}, bs[3] = {b_h, b_l, b_h};
#pragma unroll
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int ks = 0; ks < KQ / 8; ++ks)  // K = 8 per instruction: two 16-byte core columns
          mma_tf32(d, sdesc(as[t] + ks * 256, 128, 1024), sdesc(bs[t] + ks * 256, 128, 1024), idesc,
                   (t > 0 || ks > 0) ? 1u : 0u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                 : "memory");
  }
  bool ok = mbar_wait_bounded(mb, 0);
  if (!ok) {
    if (flags && lane == 0) atomicOr(flags, MPJ_FLAG_TIMEOUT);
    ok = mbar_wait_bounded(mb, 0);  // the products may still be in flight
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective

  if (ok) {
    for (int qi = 0; qi < nq; ++qi) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(qi * KQ);
      TC_LD32(taddr, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      int I, J;
      block_pair_tc(nb, R, q0 + qi, I, J);
      const int rr = row0 + warp * 32 + lane;
      if (rr < N) {
        if (!tr) {
#pragma unroll
          for (int j = 0; j < KQ; ++j) dst[(size_t)bgidx(I, J, j) * N + rr] = __uint_as_float(v[j]);
        } else {
          float* o = dst + (size_t)rr * N;
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            *reinterpret_cast<float4*>(o + I * 16 + j) = make_float4(
                __uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
            *reinterpret_cast<float4*>(o + J * 16 + j) =
                make_float4(__uint_as_float(v[16 + j]), __uint_as_float(v[17 + j]), __uint_as_float(v[18 + j]),
                            __uint_as_float(v[19 + j]));
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace

cudaError_t mpj_tc_panel(int N, int nb, int R, const float* Ubuf, const float* In, float* Out, int transpose_out,
                         const float* In2, float* Out2, unsigned* flags, cudaStream_t s, int no_commit) {
  if (N <= 0 || N % 32 || nb != N / 16 || !Ubuf || !In || !Out) return cudaErrorInvalidValue;
  if (transpose_out && In == Out) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(tc_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int npairs = nb / 2;
  dim3 grid((N + TM - 1) / TM, (npairs + QPC - 1) / QPC, (In2 && Out2) ? 2 : 1);
  tc_panel_kernel<<<grid, TPB, SMEM_BYTES, s>>>(N, nb, R, Ubuf, In, Out, transpose_out, In2, Out2, flags, no_commit);
  mpj_count_launch();
  return cudaGetLastError();
}

extern "C" int mpj_stage1_panel(int N, int R, const float* U, const float* In, float* Out, int mode,
                                void* stream) {
  const int transpose_out = mode & 1, no_commit = (mode >> 1) & 1;
  if (N < 32 || N % 32 || R < 0 || R >= N / 16 - 1 || !U || !In || !Out || (mode & ~3)) return MPJ_EINVAL;
  if (no_commit && N > 256) return MPJ_EINVAL;  // the test form runs one small wave only
  if (transpose_out && In == Out) return MPJ_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* flag = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&flag, sizeof(unsigned), s);
  mpj_count_alloc();
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = mpj_tc_panel(N, N / 16, R, U, In, Out, transpose_out, nullptr, nullptr, flag, s, no_commit);
  unsigned h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (flag) cudaFreeAsync(flag, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "mpj_stage1_panel", __LINE__);
    return MPJ_ECUDA;
  }
  return (h & MPJ_FLAG_TIMEOUT) ? MPJ_ETIMEOUT : MPJ_OK;
}
