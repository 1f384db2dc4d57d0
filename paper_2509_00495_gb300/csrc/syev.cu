// syev.cu -- host driver and C ABI of libmpjacobi: the mixed precision
// Jacobi eigensolver of Algorithm 9 (Sec. 5.1) and the plain FP64 Jacobi.
//
//   mixed:  A --(stage 1, FP32 block round-robin Jacobi)--> Q_l
//             --(Newton-Schulz x ns_steps, FP64 DMMA)--> Q_d
//             --(A_cond = Q_d^T (A Q_d), FP64 DMMA, symmetric)--> A_cond
//             --(FP64 Jacobi sweeps, V from I, until off <= tol)--> diag, V
//             --> W = diag (sorted), Q = Q_d V (columns permuted to match)
//   plain:  FP64 Jacobi sweeps on a copy of A with V from I; W = diag, Q = V.
//
// Workspace (mixed, n): three n x n FP64 buffers (X = Q_l/Q_d, M = X^T X then
// A_cond, Y = NS temporary then V), the stage-1 FP32 buffers (A32, V32 and
// the per-pair S, U; reused for the permuted V at the end), two sliced
// operands of the tensor-core products (16 n^2 bytes each) and a small
// scratch area.  About 56 n^2 + 8 N^2 bytes: 1 GiB at n = 4096.  The solve
// allocates nothing when the caller passes a workspace.
#include <stdio.h>
#include <string.h>

#include <cmath>

#include "common.cuh"
#include "gemm64.cuh"
#include "jacobi64.cuh"
#include "ns_fast.cuh"
#include "ozaki.cuh"
#include "stage1.cuh"

#include <atomic>

static thread_local char g_cuda_err[256] = "";
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_allocs{0};

void mpj_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void mpj_count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void mpj_count_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

void mpj_set_cuda_error(cudaError_t e, const char* what, int line) {
  snprintf(g_cuda_err, sizeof g_cuda_err, "%s (%d) in %s [syev line %d]", cudaGetErrorString(e), (int)e, what, line);
}

namespace {

inline size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t X, M, Y, Z, S1, OZ0, OZ1, scratch, small, total;
};

// Z (a fourth n x n buffer) only exists when a second preconditioning pass is
// run; the sweep scratch depends on the FP64 ordering.
Layout layout(int n, int passes, int ordering) {
  Layout L;
  size_t sq = al((size_t)n * n * sizeof(double));
  size_t off = 0;
  L.X = off;
  off += sq;
  L.M = off;
  off += sq;
  L.Y = off;
  off += sq;
  L.Z = off;
  if (passes >= 2) off += sq;
  L.S1 = off;
  // stage-1 buffers, or later an n x n FP64 temporary plus the FP32 Newton-Schulz scratch
  size_t s1 = al(mpj_stage1_bytes(n));
  size_t s1b = sq + al(mpj_ns_fast_bytes(n));
  if (s1 < s1b) s1 = s1b;
  off += s1;
  // the two sliced operands of the tensor-core products
  L.OZ0 = off;
  off += al(mpj_oz_operand_bytes(n, n));
  L.OZ1 = off;
  off += al(mpj_oz_operand_bytes(n, n));
  L.scratch = off;
  off += al(mpj_jacobi64_scratch_bytes_ordering(n, ordering));
  L.small = off;
  // flags + scalar (256 B), partials (2048 B), ranks (4n B, then rounded up to 256), w (8n B),
  // two n-vectors of the premise check
  off += al(2560 + 256 + (size_t)n * (sizeof(int) + sizeof(double))) + al((size_t)2 * n * sizeof(double));
  L.total = off;
  return L;
}

// small area: [0] flags (unsigned), [8] dscal (double), [256..] partials (256 doubles),
// [2304..] ranks (int n), then w (double n)
struct Small {
  unsigned* flags;
  double* dscal;
  double* partial;
  int* rank;
  double* w;
  double* vec;
};

Small small_ptrs(char* base, int n) {
  Small s;
  s.flags = (unsigned*)base;
  s.dscal = (double*)(base + 8);
  s.partial = (double*)(base + 256);
  s.rank = (int*)(base + 256 + 256 * sizeof(double));
  s.w = (double*)(base + al(256 + 256 * sizeof(double) + (size_t)n * sizeof(int)));
  s.vec = (double*)(base + al(2560 + 256 + (size_t)n * (sizeof(int) + sizeof(double))));
  return s;
}

__global__ void set_identity(double* V, int ldv, int n) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)n * n;
  for (; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    V[(size_t)j * ldv + i] = (i == j) ? 1.0 : 0.0;
  }
}

__global__ void copy_mat(const double* __restrict__ A, int lda, double* __restrict__ B, int ldb, int n) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)n * n;
  for (; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    B[(size_t)j * ldb + i] = A[(size_t)j * lda + i];
  }
}

// B(j, i) = B(i, j) for i > j: the lower triangle mirrored (exact symmetry).
__global__ void mirror_lower(double* __restrict__ B, int ldb, int n) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)n * n;
  for (; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    if (i > j) B[(size_t)i * ldb + j] = B[(size_t)j * ldb + i];
  }
}

// The Newton-Schulz and A_cond products run on the tensor cores (exact bf16
// slices, ozaki.cu) unless MPJ_GEMM_TC=0 selects the FP64 DMMA kernel.
bool gemm_tensor_cores() { return mpj_gemm_tc_enabled(); }

// rank_i = #{j : w_j < w_i or (w_j == w_i and j < i)}  (ascending, stable)
__global__ void rank_diag(const double* __restrict__ Ac, int ldc, int n, int sort, int* __restrict__ rank,
                          double* __restrict__ w) {
  extern __shared__ double sw[];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double wi = i < n ? Ac[(size_t)i * ldc + i] : 0.0;
  int r = 0;
  for (int j0 = 0; j0 < n; j0 += blockDim.x) {
    __syncthreads();
    int j = j0 + threadIdx.x;
    if (j < n) sw[threadIdx.x] = Ac[(size_t)j * ldc + j];
    __syncthreads();
    int lim = min((int)blockDim.x, n - j0);
    if (i < n && sort)
      for (int k = 0; k < lim; ++k) {
        double wj = sw[k];
        int jj = j0 + k;
        r += (wj < wi) || (wj == wi && jj < i);
      }
  }
  if (i < n) {
    rank[i] = sort ? r : i;
    w[i] = wi;
  }
}

// Vp(:, rank_j) = V(:, j);  W(rank_j) = w_j
__global__ void permute_cols(const double* __restrict__ V, int ldv, double* __restrict__ Vp, int ldp, int n,
                             const int* __restrict__ rank, const double* __restrict__ w, double* __restrict__ W) {
  int j = blockIdx.y;
  int rj = rank[j];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    Vp[(size_t)rj * ldp + i] = V[(size_t)j * ldv + i];
  if (blockIdx.x == 0 && threadIdx.x == 0) W[rj] = w[j];
}

int blocks_for(size_t total) {
  size_t b = (total + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

// CUDA events around the stages; marks that an early exit skipped are
// recorded at the end so every elapsed-time query sees recorded events.
struct Timer {
  cudaEvent_t ev[7];
  bool rec[7] = {false, false, false, false, false, false, false};
  bool on = false;
  cudaStream_t s;
  void start(cudaStream_t st) {
    s = st;
    on = true;
    for (auto& e : ev) cudaEventCreate(&e);
    cudaEventRecord(ev[0], s);
    rec[0] = true;
  }
  void mark(int i) {
    if (on) {
      cudaEventRecord(ev[i], s);
      rec[i] = true;
    }
  }
  void finish(mpj_info* info) {
    if (!on) return;
    for (int i = 1; i < 7; ++i)
      if (!rec[i]) cudaEventRecord(ev[i], s);
    cudaEventSynchronize(ev[6]);
    if (info) {
      for (int i = 0; i < 5; ++i) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
        info->ms_stage[i] = ms;
      }
      float tot = 0;
      cudaEventElapsedTime(&tot, ev[0], ev[6]);
      info->ms_stage[5] = tot;
    }
    for (auto& e : ev) cudaEventDestroy(e);
  }
};

// Newton-Schulz steps for a Q_l with unit roundoff ul: the paper bounds
// ||X_k - U|| by (sqrt(1 + n ul) - 1)^(2^k) (Sec. 4.3.4) and its code takes 2
// steps below n = 52000 for single precision, 3 above; the half-precision
// stage takes the smallest k whose bound is at most n 2^-53.
int ns_steps_for(int n, bool half) {
  if (!half) return n < 52000 ? 2 : 3;
  const double e0 = std::sqrt(1.0 + (double)n * 0x1p-11) - 1.0, target = (double)n * 0x1p-53;
  double e = e0;
  int k = 0;
  while (e > target && k < 8) {
    e *= e;
    ++k;
  }
  return k < 1 ? 1 : k;
}

int fill_opts(int n, const mpj_opts* in, mpj_opts* o) {
  if (in)
    *o = *in;
  else
    mpj_opts_default(o);
  if (o->max_sweeps64 <= 0) o->max_sweeps64 = 30;
  if (o->max_sweeps32 <= 0) o->max_sweeps32 = 15;
  if (o->ns_steps <= 0) o->ns_steps = ns_steps_for(n, o->stage1_half != 0);
  if (o->ordering != MPJ_ORDER_CYCLIC && o->ordering != MPJ_ORDER_ROUND_ROBIN && o->ordering != MPJ_ORDER_BLOCK)
    return MPJ_EINVAL;
  if (o->method != MPJ_METHOD_MIXED && o->method != MPJ_METHOD_PLAIN) return MPJ_EINVAL;
  return MPJ_OK;
}

// y = E x / ||x|| for the symmetric n x n E (column i of E dotted with x, one
// warp per column); partial[0..n) is y, the norm of x comes from *nrm.
__global__ void pow_step(const double* __restrict__ E, int n, const double* __restrict__ x,
                         const double* __restrict__ nrm, double* __restrict__ y) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  double t = 0.0;
  for (int j = lane; j < n; j += 32) t = fma(E[(size_t)i * n + j], x[j], t);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  const double nx = *nrm;
  if (lane == 0) y[i] = nx > 0.0 ? t / nx : 0.0;  // E x = 0 exactly: the estimate stays 0
}

// *nrm = ||y|| (one CTA, fixed order)
__global__ void pow_norm(const double* __restrict__ y, int n, double* __restrict__ nrm) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s = fma(y[i], y[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *nrm = sqrt(sh[0]);
}

__global__ void pow_init(double* __restrict__ x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = 1.0 + 0.5 * sin((double)i);
}

// Estimate of ||E||_2 for symmetric E by 30 steps of the power iteration on
// two n-vectors in `vec` (2n doubles) and one scalar.
int premise_norm(int n, const double* E, double* vec, double* scal, double* out, cudaStream_t s) {
  double* x = vec;
  double* y = vec + n;
  pow_init<<<(n + 255) / 256, 256, 0, s>>>(x, n);
  mpj_count_launch();
  pow_norm<<<1, 256, 0, s>>>(x, n, scal);
  mpj_count_launch();
  for (int it = 0; it < 30; ++it) {
    pow_step<<<(n + 7) / 8, 256, 0, s>>>(E, n, x, scal, y);
    mpj_count_launch();
    pow_norm<<<1, 256, 0, s>>>(y, n, scal);
    mpj_count_launch();
    double* t = x;
    x = y;
    y = t;
  }
  MPJ_CUDA_TRY(cudaGetLastError());
  MPJ_CUDA_TRY(cudaMemcpyAsync(out, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  MPJ_CUDA_TRY(cudaStreamSynchronize(s));
  return MPJ_OK;
}

// Device memory the tensor-core products use: two sliced-operand buffers
// (mpj_oz_operand_bytes(n, n) each) and the flags word where a completion
// wait that ran out is recorded.
struct OzWork {
  void* b0;
  void* b1;
  unsigned* flags;
};

int oz_fail(cudaError_t e, const char* what, int line) {
  mpj_set_cuda_error(e, what, line);
  return MPJ_ECUDA;
}

// C = alpha op(A) op(B) + beta Cin (n x n operands, ld n unless given) on the
// selected engine.  op(A) rows and op(B) columns are sliced into w.b0 / w.b1.
int product_run(bool ta, bool tb, int n, double alpha, const double* A, int lda, const double* B, int ldb,
                double beta, const double* Cin, double* C, const OzWork& w, cudaStream_t s) {
  if (!gemm_tensor_cores()) {
    cudaError_t e = mpj_gemm64(ta, tb, n, n, n, alpha, A, lda, B, ldb, beta, Cin, n, C, n, 0, s);
    return e == cudaSuccess ? MPJ_OK : oz_fail(e, "DMMA product", __LINE__);
  }
  OzOperand oa, ob;
  cudaError_t e = mpj_oz_prepare(A, ta ? lda : 1, ta ? 1 : lda, n, n, w.b0, &oa, s);
  if (e == cudaSuccess) e = mpj_oz_prepare(B, tb ? 1 : ldb, tb ? ldb : 1, n, n, w.b1, &ob, s);
  if (e == cudaSuccess) e = mpj_oz_gemm(oa, ob, n, n, alpha, beta, Cin, n, C, n, w.flags, s);
  return e == cudaSuccess ? MPJ_OK : oz_fail(e, "tensor-core product", __LINE__);
}

// Newton-Schulz X <- X (3I - X^T X) / 2, written X <- X + X E / 2 with
// E = I - X^T X: the symmetric product M = X^T X (tensor cores: the columns of
// X sliced once serve both operands, so M is exactly symmetric; DMMA: lower
// tiles mirrored), E in FP64, then X E either in FP32 when
// max|E| <= 2^-31 / sqrt(n) (ns_fast.cu) or as an FP64-accurate product.
// X, M, Y are n x n with ld n; `fp32work` holds mpj_ns_fast_bytes(n).  The
// result ends in *X.  With e0_out set, the first step also estimates
// ||E||_2 (premise_norm on `vec`, 2n doubles, and `dscal`) and stops with
// MPJ_EPREMISE when it is 2 or more.
int ns_steps_run(int n, double** X, double* M, double** Y, int steps, void* fp32work, const OzWork& w,
                 cudaStream_t s, double* e0_out = nullptr, double* vec = nullptr, double* dscal = nullptr) {
  const bool tc = gemm_tensor_cores();
  for (int k = 0; k < steps; ++k) {
    if (tc) {
      OzOperand ox;
      // X^T X is symmetric: the tiles of its lower triangle, mirrored
      cudaError_t e = mpj_oz_prepare(*X, n, 1, n, n, w.b0, &ox, s);  // column j of X = row j of X^T
      if (e == cudaSuccess) e = mpj_oz_gemm(ox, ox, n, n, 1.0, 0.0, nullptr, n, M, n, w.flags, s, true);
      if (e != cudaSuccess) return oz_fail(e, "Newton-Schulz X^T X", __LINE__);
      mirror_lower<<<blocks_for((size_t)n * n), 256, 0, s>>>(M, n, n);
      mpj_count_launch();
    } else {
      MPJ_CUDA_TRY(mpj_gemm64(true, false, n, n, n, 1.0, *X, n, *X, n, 0.0, nullptr, n, M, n, 1, s));
    }
    int r = mpj_ns_fp32_correction(n, *X, M, *Y, fp32work, nullptr, s);
    if (r < 0) return r;
    if (k == 0 && e0_out) {
      // M now holds E = I - X^T X: the premise ||E||_2 < 2 (Sec. 4.3.4), its
      // largest |eigenvalue|, estimated by 30 power-iteration steps
      double lam = 0.0;
      int rp = premise_norm(n, M, vec, dscal, &lam, s);
      if (rp != MPJ_OK) return rp;
      *e0_out = lam;
      if (!(lam < 2.0)) return MPJ_EPREMISE;
    }
    if (r == 1 && tc) {  // Y = X + X E / 2
      MPJ_CUDA_TRY(cudaMemcpyAsync(*Y, *X, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      int rt = product_run(false, false, n, 0.5, *X, n, M, n, 1.0, *Y, *Y, w, s);
      if (rt != MPJ_OK) return rt;
    } else if (r == 1) {
      MPJ_CUDA_TRY(mpj_gemm64(false, false, n, n, n, 0.5, *X, n, M, n, 1.0, *X, n, *Y, n, 0, s));
    }
    double* t = *X;
    *X = *Y;
    *Y = t;
  }
  return MPJ_OK;
}

// Algorithm 9 step 3: Ac = Qd^T (A Qd), written exactly symmetric (lower
// triangle mirrored); Y (n x n, ld n) receives A Qd.  Tensor cores: the
// columns of Qd are sliced once and serve as the right operand of A Qd and
// the left operand of Qd^T Y.
int transform_run(int n, const double* A, int lda, const double* Qd, int ldq, double* Y, double* Ac, int ldc,
                  const OzWork& w, cudaStream_t s) {
  if (gemm_tensor_cores()) {
    OzOperand oa, oq, oy;
    cudaError_t e = mpj_oz_prepare(A, 1, lda, n, n, w.b0, &oa, s);                 // rows of A
    if (e == cudaSuccess) e = mpj_oz_prepare(Qd, ldq, 1, n, n, w.b1, &oq, s);      // columns of Qd
    if (e == cudaSuccess) e = mpj_oz_gemm(oa, oq, n, n, 1.0, 0.0, nullptr, n, Y, n, w.flags, s);
    if (e == cudaSuccess) e = mpj_oz_prepare(Y, n, 1, n, n, w.b0, &oy, s);         // columns of A Qd
    if (e == cudaSuccess) e = mpj_oz_gemm(oq, oy, n, n, 1.0, 0.0, nullptr, n, Ac, ldc, w.flags, s, true);
    if (e != cudaSuccess) return oz_fail(e, "transform", __LINE__);
    mirror_lower<<<blocks_for((size_t)n * n), 256, 0, s>>>(Ac, ldc, n);
    mpj_count_launch();
    return MPJ_OK;
  }
  if (mpj_gemm64(false, false, n, n, n, 1.0, A, lda, Qd, ldq, 0.0, nullptr, n, Y, n, 0, s) != cudaSuccess ||
      mpj_gemm64(true, false, n, n, n, 1.0, Qd, ldq, Y, n, 0.0, nullptr, n, Ac, ldc, 1, s) != cudaSuccess)
    return oz_fail(cudaGetLastError(), "transform", __LINE__);
  return MPJ_OK;
}

}  // namespace

// =========================================================================== C ABI
extern "C" {

void mpj_opts_default(mpj_opts* o) {
  memset(o, 0, sizeof *o);
  o->ordering = MPJ_ORDER_BLOCK;
  o->method = MPJ_METHOD_MIXED;
  o->sort = 1;
  o->threshold = -1;
}

const char* mpj_status_str(int st) {
  switch (st) {
    case MPJ_OK: return "MPJ_OK";
    case MPJ_NOT_CONVERGED: return "MPJ_NOT_CONVERGED";
    case MPJ_EINVAL: return "MPJ_EINVAL";
    case MPJ_ENOTSYM: return "MPJ_ENOTSYM";
    case MPJ_ENONFINITE: return "MPJ_ENONFINITE";
    case MPJ_ECUDA: return "MPJ_ECUDA";
    case MPJ_ENOMEM: return "MPJ_ENOMEM";
    case MPJ_EDEGENERATE: return "MPJ_EDEGENERATE";
    case MPJ_EWORKSPACE: return "MPJ_EWORKSPACE";
    case MPJ_ETIMEOUT: return "MPJ_ETIMEOUT";
    case MPJ_ETOOLARGE: return "MPJ_ETOOLARGE";
    case MPJ_EPREMISE: return "MPJ_EPREMISE";
    default: return "MPJ_UNKNOWN";
  }
}

const char* mpj_last_cuda_error(void) { return g_cuda_err; }

long long mpj_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

long long mpj_device_allocations(void) { return g_allocs.load(std::memory_order_relaxed); }

size_t mpj_syev_workspace(int n, const mpj_opts* o) {
  (void)o;
  if (n <= 0) return 0;
  int passes = (o && o->precond_passes >= 2 && o->method == MPJ_METHOD_MIXED) ? 2 : 1;
  return layout(n, passes, o ? o->ordering : MPJ_ORDER_BLOCK).total;
}

int mpj_syev_ex(int n, const double* A, int lda, double* W, double* Q, int ldq, const mpj_opts* opts_in,
                mpj_info* info, void* work, size_t work_bytes, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  mpj_opts o;
  if (info) memset(info, 0, sizeof *info);
  if (n < 0 || (n > 0 && (!A || !W || !Q)) || lda < (n > 1 ? n : 1) || ldq < (n > 1 ? n : 1)) return MPJ_EINVAL;
  if (fill_opts(n, opts_in, &o) != MPJ_OK) return MPJ_EINVAL;
  if (n == 0) return MPJ_OK;
  const int passes = (o.method == MPJ_METHOD_MIXED && o.precond_passes >= 2) ? 2 : 1;
  Layout L = layout(n, passes, o.ordering);
  bool own = false;
  if (work) {
    if (work_bytes < L.total) return MPJ_EWORKSPACE;
  } else {
    cudaError_t e = cudaMallocAsync(&work, L.total, s);
    mpj_count_alloc();
    if (e != cudaSuccess) {
      mpj_set_cuda_error(e, "cudaMallocAsync(workspace)", __LINE__);
      return MPJ_ENOMEM;
    }
    own = true;
  }
  int st = MPJ_OK;
  char* base = (char*)work;
  unsigned flags_end = 0;
  double* X = (double*)(base + L.X);
  double* M = (double*)(base + L.M);
  double* Y = (double*)(base + L.Y);
  double* Z = (double*)(base + L.Z);
  void* S1 = base + L.S1;
  void* scratch = base + L.scratch;
  Small sm = small_ptrs(base + L.small, n);
  const OzWork ozw{base + L.OZ0, base + L.OZ1, sm.flags};
  Timer tm;
  double norm2 = 0.0;
  unsigned flags = 0;
  double tol = 0.0;
  int sweeps32 = 0, sweeps32b = 0, sweeps64 = 0;
  double off32 = 0.0, offc = 0.0, offf = 0.0, ns_e0 = 0.0;
  double* Ac = nullptr;
  double* V = nullptr;
  double* Qd = nullptr;

  tm.start(s);
  // a0: validation and norms
  {
    cudaError_t e = cudaMemsetAsync(sm.flags, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = mpj_sumsq(A, lda, n, false, sm.partial, sm.dscal, sm.flags, s);
    if (e == cudaSuccess && o.check_symmetry) e = mpj_check_symmetric(A, lda, n, sm.flags, s);
    if (e != cudaSuccess) {
      mpj_set_cuda_error(e, "validation", __LINE__);
      st = MPJ_ECUDA;
      goto done;
    }
  }
  cudaMemcpyAsync(&norm2, sm.dscal, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&flags, sm.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    mpj_set_cuda_error(cudaGetLastError(), "validation", __LINE__);
    st = MPJ_ECUDA;
    goto done;
  }
  if (flags & MPJ_FLAG_NONFINITE) {
    st = MPJ_ENONFINITE;
    goto done;
  }
  if (flags & MPJ_FLAG_NOTSYM) {
    st = MPJ_ENOTSYM;
    goto done;
  }
  {
    double normA = std::sqrt(norm2);
    tol = o.tol > 0 ? o.tol : (double)n * 0x1p-53 * normA;
    double tol32 = o.tol32 > 0 ? o.tol32 : (double)n * (o.stage1_half ? 0x1p-11 : 0x1p-24) * normA;
    if (info) {
      info->norm_fro = normA;
      info->tol = tol;
    }
    if (o.method == MPJ_METHOD_MIXED) {
      // stage 1 -> X = Q_l
      int r1 = mpj_stage1_run(n, A, lda, X, n, tol32, o.max_sweeps32, &sweeps32, &off32, S1, sm.partial, sm.dscal, s,
                              o.stage1_half != 0);
      if (r1 < 0) {
        st = r1;
        goto done;
      }
      tm.mark(1);
      // stage 2: Newton-Schulz -> X = Q_d
      double* Xp = X;
      double* Yp = Y;
      if ((st = ns_steps_run(n, &Xp, M, &Yp, o.ns_steps, S1, ozw, s, &ns_e0, sm.vec, sm.dscal)) != MPJ_OK)
        goto done;
      tm.mark(2);
      // stage 3: A_cond = Q_d^T (A Q_d) -> M (symmetric), Yp = A Q_d
      if ((st = transform_run(n, A, lda, Xp, n, Yp, M, n, ozw, s)) != MPJ_OK) goto done;
      Qd = Xp;
      Ac = M;
      V = Yp;
      if (passes >= 2) {
        // second pass (not in the paper): stages 1-3 on A_cond.  Its FP32
        // rounding is relative to each entry, so the FP32 Jacobi resolves the
        // eigenvalues that stage 1 on A could not separate.
        double offc2 = 0.0;
        if (mpj_sumsq(M, n, n, true, sm.partial, sm.dscal, nullptr, s) != cudaSuccess ||
            cudaMemcpyAsync(&offc2, sm.dscal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          mpj_set_cuda_error(cudaGetLastError(), "pass-2 off", __LINE__);
          st = MPJ_ECUDA;
          goto done;
        }
        double tol32b = (double)n * 0x1p-24 * std::sqrt(offc2);
        double* Ql2 = Yp;  // A Q_d (pass 1) is no longer needed
        // the second FP32 pass resolves the groups stage 1 could not separate;
        // each of its sweeps costs about a quarter of an FP64 sweep and saves
        // about one, up to the point where two FP64 sweeps remain (nine sweeps
        // at n = 4096), hence the cap
        int cap2 = o.max_sweeps32_pass2 > 0 ? o.max_sweeps32_pass2 : (o.max_sweeps32 < 9 ? o.max_sweeps32 : 9);
        int r1b = mpj_stage1_run(n, M, n, Ql2, n, tol32b, cap2, &sweeps32b, nullptr, S1, sm.partial, sm.dscal, s,
                                 false, true);
        if (r1b < 0) {
          st = r1b;
          goto done;
        }
        double* X2 = Ql2;
        double* Y2 = (double*)S1;  // the stage-1 area is free again
        if ((st = ns_steps_run(n, &X2, Z, &Y2, o.ns_steps, (char*)S1 + al((size_t)n * n * sizeof(double)), ozw,
                               s)) != MPJ_OK)
          goto done;
        // A_cond2 = Q_d2^T (A_cond Q_d2): A_cond Q_d2 into Z, then Q_d2^T Z into M (A_cond is
        // consumed); then Q_d = Q_d1 Q_d2 into Z
        if ((st = transform_run(n, M, n, X2, n, Z, M, n, ozw, s)) != MPJ_OK) goto done;
        if ((st = product_run(false, false, n, 1.0, Xp, n, X2, n, 0.0, nullptr, Z, ozw, s)) != MPJ_OK) goto done;
        Qd = Z;   // Q_d = Q_d1 Q_d2
        Ac = M;
        V = Xp;   // Q_d1 is folded into Z
      }
      tm.mark(3);
    } else {
      tm.mark(1);
      tm.mark(2);
      copy_mat<<<blocks_for((size_t)n * n), 256, 0, s>>>(A, lda, M, n, n);
      mpj_count_launch();
      tm.mark(3);
      Ac = M;
      V = Y;
    }
    // stage 4: FP64 sweeps.  Plain: V from I.  Mixed: the rotations are applied
    // to Q_d's columns directly (Q = Q_d V by associativity), which saves the
    // final n x n x n product.
    if (o.method == MPJ_METHOD_PLAIN) {
      set_identity<<<blocks_for((size_t)n * n), 256, 0, s>>>(V, n, n);
      mpj_count_launch();
    } else {
      V = Qd;
    }
    {
      const bool thr = o.threshold > 0 || (o.threshold < 0 && o.ordering != MPJ_ORDER_CYCLIC);
      long long rb = 0;
      int r4 = mpj_jacobi64_run(n, Ac, n, V, n, tol, o.ordering, o.max_sweeps64, &sweeps64, &offf, &offc, scratch,
                                mpj_jacobi64_scratch_bytes_ordering(n, o.ordering), s, thr ? tol / n : 0.0, true, &rb);
      if (info) info->rotated_blocks64 = rb;
      if (r4 < 0) {
        st = r4;
        goto done;
      }
      if (r4 == MPJ_NOT_CONVERGED) st = MPJ_NOT_CONVERGED;
    }
    tm.mark(4);
    // stage 5: W = diag(A_cond), sorted; Q = V (= Q_d V for the mixed method) with columns permuted
    {
      rank_diag<<<(n + 255) / 256, 256, 256 * sizeof(double), s>>>(Ac, n, n, o.sort, sm.rank, sm.w);
      mpj_count_launch();
      double* Vp = (double*)S1;  // the stage-1 area is free now
      permute_cols<<<dim3((n + 255) / 256 > 16 ? 16 : (n + 255) / 256, n), 256, 0, s>>>(V, n, Q, ldq, n, sm.rank,
                                                                                          sm.w, W);
      mpj_count_launch();
      if (o.polish) {
        // one more Newton-Schulz step on Q (not in the paper)
        double* T = (o.method == MPJ_METHOD_PLAIN) ? X : Vp;
        double* Qc = (o.method == MPJ_METHOD_PLAIN) ? Y : M;  // Q with ld n (M is reused for Q^T Q below)
        if (o.method != MPJ_METHOD_PLAIN) Qc = X;               // Q_d is no longer needed
        copy_mat<<<blocks_for((size_t)n * n), 256, 0, s>>>(Q, ldq, Qc, n, n);
        mpj_count_launch();
        double* Qp = Qc;
        double* Tp = T;
        if ((st = ns_steps_run(n, &Qp, M, &Tp, 1, (char*)S1 + al((size_t)n * n * sizeof(double)), ozw, s)) !=
            MPJ_OK)
          goto done;
        copy_mat<<<blocks_for((size_t)n * n), 256, 0, s>>>(Qp, n, Q, ldq, n);
        mpj_count_launch();
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        mpj_set_cuda_error(e, "finalize", __LINE__);
        st = MPJ_ECUDA;
        goto done;
      }
    }
    tm.mark(5);
  }
done:
  tm.mark(6);
  // device-side conditions of the products (a completion wait that ran out)
  // are read here, at the single synchronization that ends the call
  cudaMemcpyAsync(&flags_end, sm.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  tm.finish(info);
  if (own) cudaFreeAsync(work, s);
  {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st >= 0) {
      mpj_set_cuda_error(e, "final sync", __LINE__);
      st = MPJ_ECUDA;
    }
    if (st >= 0 && (flags_end & MPJ_FLAG_TIMEOUT)) st = MPJ_ETIMEOUT;
  }
  if (info) {
    info->status = st;
    info->sweeps32 = sweeps32;
    info->sweeps32_pass2 = sweeps32b;
    info->sweeps64 = sweeps64;
    info->ns_steps = (o.method == MPJ_METHOD_MIXED) ? o.ns_steps : 0;
    info->off32 = off32;
    info->off_final = offf;
    info->off_cond = offc;
    info->ns_e0 = ns_e0;
  }
  return st;
}

int mpj_syev(int n, const double* A, int lda, double* W, double* Q, double tol, void* stream) {
  mpj_opts o;
  mpj_opts_default(&o);
  o.tol = tol;
  return mpj_syev_ex(n, A, lda, W, Q, n, &o, nullptr, nullptr, 0, stream);
}

// ----------------------------------------------------------------- stage entry points
int mpj_stage1(int n, const double* A, int lda, double* Ql, int ldq, double tol32, int max_sweeps, int* sweeps,
               double* off32, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 0 || !A || !Ql || lda < n || ldq < n) return MPJ_EINVAL;
  size_t bytes = al(mpj_stage1_bytes(n)) + 4096;
  void* w = nullptr;
  if (cudaMallocAsync(&w, bytes, s) != cudaSuccess) return MPJ_ENOMEM;
  mpj_count_alloc();
  double* partial = (double*)((char*)w + al(mpj_stage1_bytes(n)));
  double* dscal = partial + 256;
  int st = MPJ_OK;
  double norm2 = 0;
  if (tol32 <= 0) {
    if (mpj_sumsq(A, lda, n, false, partial, dscal, nullptr, s) != cudaSuccess ||
        cudaMemcpyAsync(&norm2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = MPJ_ECUDA;
    tol32 = (double)n * 0x1p-24 * std::sqrt(norm2);
  }
  if (st == MPJ_OK)
    st = mpj_stage1_run(n, A, lda, Ql, ldq, tol32, max_sweeps > 0 ? max_sweeps : 15, sweeps, off32, w, partial, dscal,
                        s);
  cudaFreeAsync(w, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st >= 0) st = MPJ_ECUDA;
  return st;
}

int mpj_newton_schulz(int n, double* X, int ldx, int steps, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 0 || !X || ldx < n || steps < 0) return MPJ_EINVAL;
  void* w = nullptr;
  const size_t sq = al((size_t)n * n * sizeof(double));
  const size_t ozb = al(mpj_oz_operand_bytes(n, n));
  if (cudaMallocAsync(&w, 3 * sq + al(mpj_ns_fast_bytes(n)) + 2 * ozb + 256, s) != cudaSuccess) return MPJ_ENOMEM;
  mpj_count_alloc();
  char* b = (char*)w;
  double* Xc = (double*)b;
  double* M = (double*)(b + sq);
  double* Y = (double*)(b + 2 * sq);
  void* fp32work = b + 3 * sq;
  char* oz = b + 3 * sq + al(mpj_ns_fast_bytes(n));
  unsigned* flag = (unsigned*)(oz + 2 * ozb);
  const OzWork ozw{oz, oz + ozb, flag};
  unsigned h = 0;
  int st = cudaMemsetAsync(flag, 0, sizeof(unsigned), s) == cudaSuccess ? MPJ_OK : MPJ_ECUDA;
  double* Xp = Xc;
  double* Yp = Y;
  if (st == MPJ_OK) {
    copy_mat<<<blocks_for((size_t)n * n), 256, 0, s>>>(X, ldx, Xc, n, n);
    mpj_count_launch();
    st = ns_steps_run(n, &Xp, M, &Yp, steps, fp32work, ozw, s);
  }
  if (st == MPJ_OK) {
    copy_mat<<<blocks_for((size_t)n * n), 256, 0, s>>>(Xp, n, X, ldx, n);
    mpj_count_launch();
  }
  cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(w, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st >= 0) st = MPJ_ECUDA;
  if (st == MPJ_OK && (h & MPJ_FLAG_TIMEOUT)) st = MPJ_ETIMEOUT;
  return st;
}

int mpj_precondition(int n, const double* A, int lda, const double* Qd, int ldq, double* Ac, int ldc, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 0 || !A || !Qd || !Ac || lda < n || ldq < n || ldc < n) return MPJ_EINVAL;
  void* w = nullptr;
  const size_t sq = al((size_t)n * n * sizeof(double));
  const size_t ozb = al(mpj_oz_operand_bytes(n, n));
  if (cudaMallocAsync(&w, sq + 2 * ozb + 256, s) != cudaSuccess) return MPJ_ENOMEM;
  mpj_count_alloc();
  char* b = (char*)w;
  double* Wt = (double*)b;
  unsigned* flag = (unsigned*)(b + sq + 2 * ozb);
  const OzWork ozw{b + sq, b + sq + ozb, flag};
  unsigned h = 0;
  int st = cudaMemsetAsync(flag, 0, sizeof(unsigned), s) == cudaSuccess ? MPJ_OK : MPJ_ECUDA;
  if (st == MPJ_OK) st = transform_run(n, A, lda, Qd, ldq, Wt, Ac, ldc, ozw, s);
  cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(w, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st >= 0) st = MPJ_ECUDA;
  if (st == MPJ_OK && (h & MPJ_FLAG_TIMEOUT)) st = MPJ_ETIMEOUT;
  return st;
}

int mpj_jacobi64(int n, double* A, int lda, double* V, int ldv, double tol, int ordering, int max_sweeps, int* sweeps,
                 double* off_final, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 0 || !A || !V || lda < n || ldv < n) return MPJ_EINVAL;
  if (ordering != MPJ_ORDER_CYCLIC && ordering != MPJ_ORDER_ROUND_ROBIN && ordering != MPJ_ORDER_BLOCK)
    return MPJ_EINVAL;
  void* w = nullptr;
  size_t wbytes = mpj_jacobi64_scratch_bytes_ordering(n, ordering) + 4096;
  if (cudaMallocAsync(&w, wbytes, s) != cudaSuccess) return MPJ_ENOMEM;
  mpj_count_alloc();
  int st = MPJ_OK;
  if (tol <= 0) {
    double* partial = (double*)w;
    double* dscal = partial + 256;
    double norm2 = 0;
    if (mpj_sumsq(A, lda, n, false, partial, dscal, nullptr, s) != cudaSuccess ||
        cudaMemcpyAsync(&norm2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = MPJ_ECUDA;
    tol = (double)n * 0x1p-53 * std::sqrt(norm2);
  }
  if (st == MPJ_OK)
    st = mpj_jacobi64_run(n, A, lda, V, ldv, tol, ordering, max_sweeps > 0 ? max_sweeps : 30, sweeps, off_final, nullptr,
                          w, wbytes, s);
  cudaFreeAsync(w, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st >= 0) st = MPJ_ECUDA;
  return st;
}

int mpj_dgemm(char transa, char transb, int m, int n, int k, double alpha, const double* A, int lda, const double* B,
              int ldb, double beta, double* C, int ldc, void* stream) {
  bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && !(transa == 'N' || transa == 'n')) return MPJ_EINVAL;
  if (!tb && !(transb == 'N' || transb == 'n')) return MPJ_EINVAL;
  if (m < 0 || n < 0 || k < 0 || !A || !B || !C) return MPJ_EINVAL;
  if (lda < (ta ? k : m) || ldb < (tb ? n : k) || ldc < m || lda < 1 || ldb < 1 || ldc < 1) return MPJ_EINVAL;
  cudaError_t e = mpj_gemm64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "mpj_dgemm", __LINE__);
    return MPJ_ECUDA;
  }
  return MPJ_OK;
}

}  // extern "C"
