// common.cuh -- device helpers shared by the libmpjacobi kernels (sm_103a).
//
// Rotation parameters follow Algorithm 2 (jacobi_pair, Sec. 3.1.2) in its
// stable form (Appendix A, approach 2): tau = (a_qq - a_pp) / (2 a_pq),
// t = 1 / (tau + sign(tau) sqrt(1 + tau^2)) (tau >= 0 takes '+'),
// c = 1 / sqrt(1 + t^2), s = t c.  The rotation J = [c s; -s c] is applied as
// rows J^T A, columns A J, vectors V J (Sec. 3.2.2).  Two rounding-level
// departures, both identical in exact arithmetic:
//   * the update x' = c x - s y is evaluated as x' = (x - s y) + (c - 1) x with
//     c - 1 = -t^2 / (h (1 + h)), h = sqrt(1 + t^2), so that tiny rotations do
//     not round c to 1 and inflate column norms by t^2 each time;
//   * after a rotation the pair's diagonal becomes a_pp - t a_pq, a_qq + t a_pq
//     and a_pq becomes exactly 0 (the annihilated entry of Sec. 3.1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpjacobi.h"

#define MPJ_DEV __device__ __forceinline__

// Error flags written by kernels into a device word (bitwise OR).
enum : unsigned {
  MPJ_FLAG_NONFINITE = 1u,
  MPJ_FLAG_NOTSYM = 2u,
  MPJ_FLAG_TIMEOUT = 4u,
  MPJ_FLAG_DEGENERATE = 8u,
};

// Rotation record of one pair slot in one round-robin step, oriented to the
// slot's (x, y) indices (see rr_slot): the update of the index pair is
//   new_x = (v_x - sig v_y) + cm1 v_x,   new_y = (v_y + sig v_x) + cm1 v_y,
// i.e. sig = s when x < y (x plays p) and sig = -s otherwise.  dx, dy are the
// diagonal entries of x and y after the step (the old ones when no rotation).
// cm1 == 0 && sig == 0 means "not rotated".
template <typename T>
struct RotRec {
  T cm1, sig, dx, dy;
};

// Algorithm 2 with the skip test of Algorithm 4: rotate iff
// |a_pq| > skip * sqrt(|a_pp a_qq|) and (threshold variant) |a_pq| > skip_abs.
// Outputs t, c - 1, s (for the (p,q) order) and the rotated flag.
template <typename T>
MPJ_DEV bool jacobi_pair(T app, T aqq, T apq, T skip, T& t, T& cm1, T& s, T skip_abs = T(0)) {
  if (!(fabs(apq) > skip * sqrt(fabs(app * aqq)) && fabs(apq) > skip_abs)) {
    t = T(0);
    cm1 = T(0);
    s = T(0);
    return false;
  }
  T tau = (aqq - app) / (T(2) * apq);
  T r = sqrt(T(1) + tau * tau);
  t = (tau >= T(0)) ? T(1) / (tau + r) : T(1) / (tau - r);
  T h = sqrt(T(1) + t * t);
  T c = T(1) / h;
  cm1 = -(t * t) / (h * (T(1) + h));
  s = t * c;
  return true;
}

// Scale factor update of the scaled ("fast") rotations: d' = d (1 + cm1),
// d = d.x + d.y in double-double (Fast2Sum renormalization, |cm1| < 0.3), so
// that factors c = 1 + cm1 that round to 1 in FP64 still shrink d exactly.
MPJ_DEV double2 dd_scale(double2 d, double cm1) {
  double sum = fma(cm1, d.x, fma(cm1, d.y, d.y));
  double hi = d.x + sum;
  double lo = sum - (hi - d.x);
  return make_double2(hi, lo);
}

// Apply a rotation record to a pair of values (rows or columns x, y).
template <typename T>
MPJ_DEV void rot_apply(T cm1, T sig, T& vx, T& vy) {
  T nx = fma(cm1, vx, fma(-sig, vy, vx));
  T ny = fma(cm1, vy, fma(sig, vx, vy));
  vx = nx;
  vy = ny;
}

// ---- round-robin (circle method) ordering on m = n + (n & 1) indices -------
// Round r in [0, m-1): slot 0 pairs (r, m-1); slot i in [1, m/2) pairs
// x = (r + i) mod (m-1) with y = (r - i) mod (m-1).  When n is odd, index
// m-1 == n is a dummy and its pair is never rotated.  Every unordered pair of
// indices occurs in exactly one round of a sweep.
MPJ_DEV void rr_slot(int m, int r, int i, int& x, int& y) {
  if (i == 0) {
    x = r;
    y = m - 1;
  } else {
    x = r + i;
    if (x >= m - 1) x -= m - 1;
    y = r - i;
    if (y < 0) y += m - 1;
  }
}

MPJ_DEV int rr_partner(int m, int r, int idx) {
  if (idx == m - 1) return r;
  if (idx == r) return m - 1;
  int v = 2 * r - idx;  // in (-(m-1), 2(m-1)): one correction at most
  if (v < 0) v += m - 1;
  if (v >= m - 1) v -= m - 1;
  return v;
}

// Slot of index idx in round r, and whether it is the slot's y.
MPJ_DEV void rr_slot_of(int m, int r, int idx, int& slot, int& is_y) {
  if (idx == m - 1) {
    slot = 0;
    is_y = 1;
    return;
  }
  int d = idx - r;
  if (d < 0) d += m - 1;
  if (d == 0) {
    slot = 0;
    is_y = 0;
  } else if (d <= m / 2 - 1) {
    slot = d;
    is_y = 0;
  } else {
    slot = m - 1 - d;
    is_y = 1;
  }
}

// Build the rotation record of the pair (i, j) of round r from the current
// diagonal entries di = a_ii, dj = a_jj and the coupling aij.  Returns the
// slot index.  n is the true size (indices >= n are dummies).
template <typename T>
MPJ_DEV int rr_make_rec(int m, int n, int r, int i, int j, T di, T dj, T aij, T skip, RotRec<T>& rec,
                        T skip_abs = T(0)) {
  int slot, iy;
  rr_slot_of(m, r, i, slot, iy);
  int p = i < j ? i : j, q = i < j ? j : i;
  T app = (p == i) ? di : dj, aqq = (p == i) ? dj : di;
  T t, cm1, s;
  bool rot = (q < n) && jacobi_pair<T>(app, aqq, aij, skip, t, cm1, s, skip_abs);
  T np = app, nq = aqq;
  if (rot) {
    np = app - t * aij;
    nq = aqq + t * aij;
  }
  // orientation: x is the slot's first index
  int x = iy ? j : i;
  T sig = (x == p) ? s : -s;
  rec.cm1 = rot ? cm1 : T(0);
  rec.sig = rot ? sig : T(0);
  rec.dx = (x == p) ? np : nq;
  rec.dy = (x == p) ? nq : np;
  return slot;
}

// bit test rather than FP64 compares (those issue on the slow FP64 pipe);
// "not rotated" records hold +0.0 exactly
MPJ_DEV bool rec_rotated(double cm1, double sig) {
  return (__double_as_longlong(cm1) | __double_as_longlong(sig)) != 0;
}
MPJ_DEV bool rec_rotated(float cm1, float sig) { return cm1 != 0.0f || sig != 0.0f; }

// Loads that bypass L1 (data written by other CTAs earlier in the same
// persistent launch must not be served from a stale L1 line).
MPJ_DEV double ld_cg(const double* p) { return __ldcg(p); }
MPJ_DEV float ld_cg(const float* p) { return __ldcg(p); }

#define MPJ_CUDA_TRY(expr)                      \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) {                    \
      mpj_set_cuda_error(e_, #expr, __LINE__);  \
      return MPJ_ECUDA;                         \
    }                                           \
  } while (0)

// Host-side helpers implemented in syev.cu
void mpj_set_cuda_error(cudaError_t e, const char* what, int line);
// Counts every kernel this library enqueues (diagnostic, mpj_kernel_launches);
// mpj_count_launches adds k at once (a graph replay; negative for kernels
// that were only captured).
void mpj_count_launch();
void mpj_count_launches(long long k);

// Programmatic dependent launch.  A kernel launched by mpj_launch_pdl may have
// its CTAs scheduled while the previous kernel in the stream drains (once all
// of that kernel's CTAs have started); it calls pdl_wait() before touching
// global memory, which returns when the previous kernel has completed and its
// writes are visible.  pdl_wait() also lets the next such kernel start early.
MPJ_DEV void pdl_wait() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t mpj_launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                           Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
  mpj_count_launch();
  return e;
}

// Side stream and events for overlapping the V updates with the rotation
// rounds; released when the solve returns.  On every exit (also an early
// error return) the owner stream is first made to wait for the side stream,
// so stream-ordered reuse or freeing of the scratch stays after the last V
// update (owner = null: the caller has joined it, e.g. inside a captured graph).
struct SideStream {
  cudaStream_t owner = nullptr;
  cudaStream_t sv = nullptr;
  cudaEvent_t ready = nullptr, done[2] = {nullptr, nullptr};
  bool ok = false;
  explicit SideStream(cudaStream_t s) : owner(s) {
    ok = cudaStreamCreateWithFlags(&sv, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&done[0], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&done[1], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) (void)cudaGetLastError();
  }
  ~SideStream() {
    if (ok && owner && cudaEventRecord(ready, sv) == cudaSuccess) (void)cudaStreamWaitEvent(owner, ready, 0);
    if (done[1]) cudaEventDestroy(done[1]);
    if (done[0]) cudaEventDestroy(done[0]);
    if (ready) cudaEventDestroy(ready);
    if (sv) cudaStreamDestroy(sv);
  }
};

// Whether the V updates of the Jacobi sweeps (FP32 and FP64) may run on a
// side stream (environment MPJ_JACOBI_OVERLAP=0 keeps them on the caller's).
bool mpj_v_overlap_enabled();

// Counts every device (or pinned host) allocation the library makes
// (diagnostic, mpj_device_allocations).
void mpj_count_alloc();
