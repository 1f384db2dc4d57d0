// jacobi64.cu -- FP64 Jacobi sweeps (Algorithm 4 of the paper, Sec. 3.3) on a
// symmetric matrix held in full column-major storage, accumulating V <- V J.
//
// Two orderings:
//  * round-robin (the fast form): each sweep is m-1 rounds of m/2 disjoint
//    pairs (circle method, see rr_slot); one kernel launch per round updates
//    the whole matrix.  The matrix splits into 2x2 blocks indexed by
//    (slot a, slot b); block (a,b) becomes J_a^T B J_b.  Blocks with a >= b
//    are computed (in 16x16-slot tiles) and written together with their mirror,
//    so A stays exactly symmetric and the FP64 work is 2 FMA per entry of the
//    lower half per rotation side.  The same launch also builds the rotation
//    records of the next round: the coupling a_ij of a next-round pair (i,j) is
//    an entry of some block updated here, and the new diagonals come from this
//    round's records, so each round needs one launch and no extra pass.
//  * cyclic-by-row (the paper's ordering, the faithful form): pairs
//    (0,1),(0,2),...,(n-2,n-1) one after another, each applied as the paper's
//    row update, then column update, then vector update, with the paper's
//    formulas; (A + A^T)/2 after each sweep.  One CTA per matrix: every
//    rotation depends on the previous one.  It exists for fidelity checks and
//    is slow by construction.
//
// off(A) (Sec. 3.1, direct form) is reduced after every sweep with a fixed
// reduction order, so repeated runs are bitwise identical.
#include "common.cuh"
#include "jacobi64.cuh"

namespace {

constexpr int TS = 16;       // slots per tile side (a 32 x 32 entry region)
constexpr int VROWS = 256;   // rows of V per V work item
constexpr int VSLOTS = 8;    // slots per V work item
constexpr int RED_CTAS = 256;

__global__ void rr_init_params(const double* __restrict__ A, int lda, int n, int m, int r, double skip,
                               RotRec<double>* __restrict__ rec) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m / 2) return;
  int x, y;
  rr_slot(m, r, i, x, y);
  double dx = x < n ? A[(size_t)x * lda + x] : 0.0;
  double dy = y < n ? A[(size_t)y * lda + y] : 0.0;
  double axy = (x < n && y < n) ? A[(size_t)y * lda + x] : 0.0;
  RotRec<double> rr;
  rr_make_rec<double>(m, n, r, x, y, dx, dy, axy, skip, rr);
  rec[i] = rr;
}

__device__ __forceinline__ void tri_tile(int t, int nt, int& ti, int& tj) {
  // t enumerates the lower-triangular tiles column by column
  tj = 0;
  while (t >= nt - tj) {
    t -= nt - tj;
    ++tj;
  }
  ti = tj + t;
}

__global__ void __launch_bounds__(256) rr_step64(double* __restrict__ A, int lda, double* __restrict__ V, int ldv,
                                                 int n, int m, int r, double skip,
                                                 const RotRec<double>* __restrict__ rec,
                                                 RotRec<double>* __restrict__ rec_next, int nt, int n_atiles,
                                                 int v_row_chunks) {
  const int half = m / 2;
  const int rn = (r + 1 == m - 1) ? 0 : r + 1;  // next round (wraps into the next sweep)
  int item = blockIdx.x;
  if (item < n_atiles) {
    int ti, tj;
    tri_tile(item, nt, ti, tj);
    int a = ti * TS + (threadIdx.x % TS);
    int b = tj * TS + (threadIdx.x / TS);
    if (a >= half || b >= half || a < b) return;
    int xa, ya, xb, yb;
    rr_slot(m, r, a, xa, ya);
    rr_slot(m, r, b, xb, yb);
    RotRec<double> ra = rec[a];
    bool rota = rec_rotated(ra.cm1, ra.sig);
    bool vxa = xa < n, vya = ya < n;
    if (a == b) {
      // the pair's own 2x2 block: new diagonal from the record, a_xy annihilated
      double axy;
      if (rota) {
        A[(size_t)xa * lda + xa] = ra.dx;
        A[(size_t)ya * lda + ya] = ra.dy;
        A[(size_t)ya * lda + xa] = 0.0;
        A[(size_t)xa * lda + ya] = 0.0;
        axy = 0.0;
      } else {
        axy = (vxa && vya) ? A[(size_t)ya * lda + xa] : 0.0;
      }
      // next-round records that this block owns:
      // (1) the unpaired index of round rn when n is odd (slot 0 pairs it with the dummy)
      if ((n & 1) && (xa == rn || ya == rn)) {
        RotRec<double> z;
        z.cm1 = 0.0;
        z.sig = 0.0;
        z.dx = (xa == rn) ? ra.dx : ra.dy;
        z.dy = 0.0;
        rec_next[0] = z;
      }
      // (2) m == 2: the same pair again in the next sweep
      if (vxa && vya && rr_partner(m, rn, xa) == ya) {
        RotRec<double> nr;
        int s = rr_make_rec<double>(m, n, rn, xa, ya, ra.dx, ra.dy, axy, skip, nr);
        rec_next[s] = nr;
      }
      return;
    }
    RotRec<double> rb = rec[b];
    bool rotb = rec_rotated(rb.cm1, rb.sig);
    bool vxb = xb < n, vyb = yb < n;
    size_t cxb = (size_t)xb * lda, cyb = (size_t)yb * lda;
    double vxx = (vxa && vxb) ? A[cxb + xa] : 0.0;
    double vxy = (vxa && vyb) ? A[cyb + xa] : 0.0;
    double vyx = (vya && vxb) ? A[cxb + ya] : 0.0;
    double vyy = (vya && vyb) ? A[cyb + ya] : 0.0;
    if (rota) {  // rows x_a, y_a: J_a^T
      rot_apply(ra.cm1, ra.sig, vxx, vyx);
      rot_apply(ra.cm1, ra.sig, vxy, vyy);
    }
    if (rotb) {  // columns x_b, y_b: J_b
      rot_apply(rb.cm1, rb.sig, vxx, vxy);
      rot_apply(rb.cm1, rb.sig, vyx, vyy);
    }
    if (rota || rotb) {
      if (vxa && vxb) {
        A[cxb + xa] = vxx;
        A[(size_t)xa * lda + xb] = vxx;
      }
      if (vxa && vyb) {
        A[cyb + xa] = vxy;
        A[(size_t)xa * lda + yb] = vxy;
      }
      if (vya && vxb) {
        A[cxb + ya] = vyx;
        A[(size_t)ya * lda + xb] = vyx;
      }
      if (vya && vyb) {
        A[cyb + ya] = vyy;
        A[(size_t)ya * lda + yb] = vyy;
      }
    }
    // next-round records owned by this block
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      int i = side ? ya : xa;
      if (i >= n) continue;
      int j = rr_partner(m, rn, i);
      if (j >= n || (j != xb && j != yb)) continue;
      double di = side ? ra.dy : ra.dx;
      double dj = (j == xb) ? rb.dx : rb.dy;
      double aij = side ? ((j == xb) ? vyx : vyy) : ((j == xb) ? vxx : vxy);
      RotRec<double> nr;
      int s = rr_make_rec<double>(m, n, rn, i, j, di, dj, aij, skip, nr);
      rec_next[s] = nr;
    }
    return;
  }
  // V work item: rows [rc*VROWS, +VROWS), slots [sc*VSLOTS, +VSLOTS)
  int v = item - n_atiles;
  int rc = v % v_row_chunks, sc = v / v_row_chunks;
  int i = rc * VROWS + threadIdx.x;
  if (i >= n) return;
#pragma unroll 2
  for (int k = 0; k < VSLOTS; ++k) {
    int b = sc * VSLOTS + k;
    if (b >= half) break;
    RotRec<double> rb = rec[b];
    if (!rec_rotated(rb.cm1, rb.sig)) continue;
    int xb, yb;
    rr_slot(m, r, b, xb, yb);
    double* px = V + (size_t)xb * ldv + i;
    double* py = V + (size_t)yb * ldv + i;
    double vx = *px, vy = *py;
    rot_apply(rb.cm1, rb.sig, vx, vy);
    *px = vx;
    *py = vy;
  }
}

// ---- off(A)^2 and ||A||_F^2 with a fixed reduction order --------------------
template <typename T, bool OFF_ONLY>
__global__ void __launch_bounds__(256) sumsq_partial(const T* __restrict__ A, int lda, int n,
                                                     double* __restrict__ partial, unsigned* __restrict__ flags) {
  double s = 0.0;
  bool bad = false;
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    const T* col = A + (size_t)j * lda;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double x = (double)col[i];
      if (OFF_ONLY && i == j) continue;
      if (!isfinite(x)) bad = true;
      s += x * x;
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  if (bad && flags) atomicOr(flags, MPJ_FLAG_NONFINITE);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void reduce_partials(const double* __restrict__ partial, int count, double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += 256) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void check_symmetric(const double* __restrict__ A, int lda, int n, unsigned* __restrict__ flags) {
  for (int j = blockIdx.x; j < n; j += gridDim.x)
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
      if (A[(size_t)j * lda + i] != A[(size_t)i * lda + j]) atomicOr(flags, MPJ_FLAG_NOTSYM);
}

// ---- cyclic-by-row, one CTA per matrix (the paper's ordering and update) ----
__global__ void __launch_bounds__(1024) cyclic_sweep64(double* __restrict__ A, int lda, double* __restrict__ V,
                                                       int ldv, int n, double skip, int* __restrict__ rotated) {
  __shared__ double cs[2];
  __shared__ int go;
  int any = 0;
  for (int p = 0; p < n - 1; ++p)
    for (int q = p + 1; q < n; ++q) {
      if (threadIdx.x == 0) {
        double app = A[(size_t)p * lda + p], aqq = A[(size_t)q * lda + q], apq = A[(size_t)q * lda + p];
        go = 0;
        if (fabs(apq) > skip * sqrt(fabs(app * aqq))) {
          // Algorithm 2, stable form (Appendix A approach 2)
          double tau = (aqq - app) / (2.0 * apq);
          double t = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : 1.0 / (tau - sqrt(1.0 + tau * tau));
          double c = 1.0 / sqrt(1.0 + t * t);
          cs[0] = c;
          cs[1] = t * c;
          go = 1;
        }
      }
      __syncthreads();
      if (go) {
        any = 1;
        double c = cs[0], s = cs[1];
        for (int k = threadIdx.x; k < n; k += blockDim.x) {  // rows: A([p q],:) = J^T A([p q],:)
          double ap = A[(size_t)k * lda + p], aq = A[(size_t)k * lda + q];
          A[(size_t)k * lda + p] = c * ap - s * aq;
          A[(size_t)k * lda + q] = s * ap + c * aq;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) {  // columns: A(:,[p q]) = A(:,[p q]) J
          double ap = A[(size_t)p * lda + k], aq = A[(size_t)q * lda + k];
          A[(size_t)p * lda + k] = c * ap - s * aq;
          A[(size_t)q * lda + k] = s * ap + c * aq;
          double vp = V[(size_t)p * ldv + k], vq = V[(size_t)q * ldv + k];
          V[(size_t)p * ldv + k] = c * vp - s * vq;
          V[(size_t)q * ldv + k] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
  // A = (A + A^T)/2 after a sweep with a rotation
  if (any) {
    for (int j = 0; j < n; ++j)
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
        double v = (A[(size_t)j * lda + i] + A[(size_t)i * lda + j]) / 2.0;
        A[(size_t)j * lda + i] = v;
        A[(size_t)i * lda + j] = v;
      }
  }
  if (threadIdx.x == 0) *rotated = any;
}

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t mpj_sumsq(const double* A, int lda, int n, bool off_only, double* partial, double* out, unsigned* flags,
                      cudaStream_t s) {
  if (off_only)
    sumsq_partial<double, true><<<RED_CTAS, 256, 0, s>>>(A, lda, n, partial, flags);
  else
    sumsq_partial<double, false><<<RED_CTAS, 256, 0, s>>>(A, lda, n, partial, flags);
  mpj_count_launch();
  reduce_partials<<<1, 256, 0, s>>>(partial, RED_CTAS, out);
  mpj_count_launch();
  return cudaGetLastError();
}

cudaError_t mpj_sumsq32(const float* A, int lda, int n, double* partial, double* out, cudaStream_t s) {
  sumsq_partial<float, true><<<RED_CTAS, 256, 0, s>>>(A, lda, n, partial, nullptr);
  mpj_count_launch();
  reduce_partials<<<1, 256, 0, s>>>(partial, RED_CTAS, out);
  mpj_count_launch();
  return cudaGetLastError();
}

cudaError_t mpj_check_symmetric(const double* A, int lda, int n, unsigned* flags, cudaStream_t s) {
  check_symmetric<<<RED_CTAS, 256, 0, s>>>(A, lda, n, flags);
  mpj_count_launch();
  return cudaGetLastError();
}

size_t mpj_jacobi64_scratch_bytes(int n) {
  int m = n + (n & 1);
  size_t recs = 2 * (size_t)(m / 2 + 1) * sizeof(RotRec<double>);
  // records, then (256-aligned) the reduction partials, two scalars and an int flag
  return ((recs + 255) & ~(size_t)255) + RED_CTAS * sizeof(double) + 4 * sizeof(double) + 256;
}

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int mpj_jacobi64_run(int n, double* A, int lda, double* V, int ldv, double tol, int ordering, int max_sweeps,
                     int* sweeps_out, double* off_out, double* off_initial, void* scratch, cudaStream_t s) {
  const double skip = 0x1p-53;
  int m = n + (n & 1);
  char* base = (char*)scratch;
  RotRec<double>* rec0 = (RotRec<double>*)base;
  RotRec<double>* rec1 = rec0 + (m / 2 + 1);
  double* partial = (double*)(base + align256(2 * (size_t)(m / 2 + 1) * sizeof(RotRec<double>)));
  double* dscal = partial + RED_CTAS;
  int* iscal = (int*)(dscal + 2);

  double off2 = 0.0;
  MPJ_CUDA_TRY(mpj_sumsq(A, lda, n, true, partial, dscal, nullptr, s));
  MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
  MPJ_CUDA_TRY(cudaStreamSynchronize(s));
  double off = sqrt(off2);
  if (off_initial) *off_initial = off;
  int sweeps = 0;
  int status = MPJ_OK;
  if (ordering == MPJ_ORDER_ROUND_ROBIN) {
    const int half = m / 2;
    const int nt = (half + TS - 1) / TS;
    const int n_atiles = nt * (nt + 1) / 2;
    const int vrc = (n + VROWS - 1) / VROWS;
    const int vsc = (half + VSLOTS - 1) / VSLOTS;
    const int grid = n_atiles + vrc * vsc;
    long long k = 0;  // global step counter (record buffer parity)
    if (off > tol && n > 1) {
      rr_init_params<<<(half + 127) / 128, 128, 0, s>>>(A, lda, n, m, 0, skip, rec0);
      mpj_count_launch();
      MPJ_CUDA_TRY(cudaGetLastError());
    }
    while (off > tol && n > 1) {
      if (sweeps >= max_sweeps) {
        status = MPJ_NOT_CONVERGED;
        break;
      }
      for (int r = 0; r < m - 1; ++r, ++k) {
        RotRec<double>* cur = (k & 1) ? rec1 : rec0;
        RotRec<double>* nxt = (k & 1) ? rec0 : rec1;
        rr_step64<<<grid, 256, 0, s>>>(A, lda, V, ldv, n, m, r, skip, cur, nxt, nt, n_atiles, vrc);
        mpj_count_launch();
      }
      MPJ_CUDA_TRY(cudaGetLastError());
      ++sweeps;
      MPJ_CUDA_TRY(mpj_sumsq(A, lda, n, true, partial, dscal, nullptr, s));
      MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
      MPJ_CUDA_TRY(cudaStreamSynchronize(s));
      off = sqrt(off2);
    }
  } else {
    while (off > tol && n > 1) {
      if (sweeps >= max_sweeps) {
        status = MPJ_NOT_CONVERGED;
        break;
      }
      cyclic_sweep64<<<1, 1024, 0, s>>>(A, lda, V, ldv, n, skip, iscal);
      mpj_count_launch();
      MPJ_CUDA_TRY(cudaGetLastError());
      int rotated = 0;
      ++sweeps;
      MPJ_CUDA_TRY(mpj_sumsq(A, lda, n, true, partial, dscal, nullptr, s));
      MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
      MPJ_CUDA_TRY(cudaMemcpyAsync(&rotated, iscal, sizeof(int), cudaMemcpyDeviceToHost, s));
      MPJ_CUDA_TRY(cudaStreamSynchronize(s));
      off = sqrt(off2);
      if (!rotated) break;
    }
  }
  if (sweeps_out) *sweeps_out = sweeps;
  if (off_out) *off_out = off;
  return status;
}

// ---------------------------------------------------------------------------
// Allocation-free entry point (see mpj_jacobi64_noalloc in mpjacobi.h): the
// sweep scratch lives in this file-scope device array instead of memory from
// cudaMallocAsync.  In host code `g_noalloc_scratch` names a host-side shadow,
// not device memory, so the kernels get the device address looked up with
// cudaGetSymbolAddress, once per device, with that device current.
#include <mutex>

static __device__ __align__(256) unsigned char g_noalloc_scratch[MPJ_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

int noalloc_scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    mpj_set_cuda_error(e, "cudaGetDevice", __LINE__);
    return MPJ_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return MPJ_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      mpj_set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __LINE__);
      return MPJ_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return MPJ_OK;
}
}  // namespace

extern "C" int mpj_jacobi64_noalloc(int n, double* A, int lda, double* V, int ldv, double tol, int ordering,
                                    int max_sweeps, int* sweeps, double* off_final, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 0 || !A || !V || lda < n || ldv < n) return MPJ_EINVAL;
  if (ordering != MPJ_ORDER_CYCLIC && ordering != MPJ_ORDER_ROUND_ROBIN) return MPJ_EINVAL;
  if (n > MPJ_NOALLOC_MAX_N || mpj_jacobi64_scratch_bytes(n) > (size_t)MPJ_NOALLOC_SCRATCH_BYTES)
    return MPJ_ETOOLARGE;
  void* w = nullptr;
  int st = noalloc_scratch_for_current_device(&w);
  if (st != MPJ_OK) return st;
  if (tol <= 0) {
    // default tolerance n 2^-53 ||A||_F; the reduction uses the front of the scratch
    double* partial = (double*)w;
    double* dscal = partial + RED_CTAS;
    double norm2 = 0;
    cudaError_t e = mpj_sumsq(A, lda, n, false, partial, dscal, nullptr, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&norm2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      mpj_set_cuda_error(e, "mpj_jacobi64_noalloc norm", __LINE__);
      return MPJ_ECUDA;
    }
    tol = (double)n * 0x1p-53 * sqrt(norm2);
  }
  st = mpj_jacobi64_run(n, A, lda, V, ldv, tol, ordering, max_sweeps > 0 ? max_sweeps : 30, sweeps, off_final, nullptr,
                        w, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && st >= 0) {
    mpj_set_cuda_error(e, "mpj_jacobi64_noalloc sync", __LINE__);
    st = MPJ_ECUDA;
  }
  return st;
}
