// jacobi64.cu -- FP64 Jacobi sweeps (Algorithm 4 of the paper, Sec. 3.3) on a
// symmetric matrix held in full column-major storage, accumulating V <- V J.
//
// Two orderings:
//  * round-robin (the fast form): each sweep is m-1 rounds of m/2 disjoint
//    pairs (circle method, see rr_slot).  The matrix splits into 2x2 blocks
//    indexed by (slot a, slot b); block (a,b) becomes J_a^T B J_b.  Blocks with
//    a >= b are computed in 16x16-slot tiles and written with their mirror, so
//    A stays exactly symmetric.  Rotations are applied in scaled form: off the
//    diagonal A = D At D and V = Vt D with one scale vector d (kept in
//    double-double), so a rotation costs one FMA per entry and side,
//      At_x <- At_x - mx At_y,   At_y <- At_y + my At_x,
//    mx = tau d_y / d_x, my = tau d_x / d_y, tau = +-t, while d_x, d_y take the
//    factor c = 1/sqrt(1 + t^2) (the paper's rotation, Sec. 3.1.1, with the
//    scaling split off).  The true diagonal is kept in A's diagonal entries.
//    One launch per round updates A and, from the coupling entries it has
//    just written, builds the next round's rotation records.  V is updated in
//    batches: each round's multipliers go to a history buffer and a second
//    kernel applies up to 64 rounds to row chunks of V held in shared memory,
//    so V is read and written once per batch instead of once per round.
//    Every 512 rounds and at the end of a sweep the scales are folded back
//    into A and V (d = 1), which keeps d far from underflow.
//  * cyclic-by-row (the paper's ordering, the faithful form): pairs
//    (0,1),(0,2),...,(n-2,n-1) in the paper's order, each applied as the
//    paper's row update, then column update, then vector update, with the
//    paper's formulas.  The sweep runs as 2n - 3 wavefronts of mutually
//    independent rotations (pairs with equal p + q), which is the same
//    rotation sequence (see cyc_wave_update).
//
// off(A) (Sec. 3.1, direct form) is reduced after every sweep with a fixed
// reduction order, so repeated runs are bitwise identical.
#include <memory>
#include <cstdlib>

#include "common.cuh"
#include "jacobi64.cuh"

namespace {

constexpr int TS = 16;        // slots per tile side (a 32 x 32 entry region)
constexpr int RED_CTAS = 256;
constexpr int RV_MAX = 64;    // rounds per batched V update
constexpr int RS = 512;       // rounds between scale folds

// Scaled-rotation record of one slot (see the file comment); mx == my == 0
// means "not rotated".  cm1 = c - 1 of the rotation (for the scale update),
// dx, dy: true diagonal entries after the rotation.
// 48 bytes (padded) so that (mx, my) load as one aligned 16-byte access.
struct __align__(16) FRec {
  double mx, my, cm1, dx, dy, pad;
};

// The multipliers of a record (the only fields every block reads), and the
// rotated test as a bit test instead of an FP64 compare: on this GPU FP64
// compares issue on the same slow FP64 pipe as the FMAs.  "Not rotated"
// records hold +0.0 exactly.
MPJ_DEV double2 frec_m(const FRec* __restrict__ p) { return __ldg(reinterpret_cast<const double2*>(p)); }
MPJ_DEV bool m_rotated(double2 mm) { return (__double_as_longlong(mm.x) | __double_as_longlong(mm.y)) != 0; }


// c - 1 of a record, computed once per slot when the record is built (kept in
// the record so the per-entry path never evaluates sqrt or a division).
MPJ_DEV double frec_cm1(const FRec& r) { return r.cm1; }


// Record of pair (i, j) of round r from true diagonals di, dj, true coupling
// aij and the scales si, sj the round will see.  Returns the slot.
MPJ_DEV int rr_make_frec(int m, int n, int r, int i, int j, double di, double dj, double aij, double si, double sj,
                         double skip, FRec& rec, double skip_abs) {
  int slot, iy;
  rr_slot_of(m, r, i, slot, iy);
  int p = i < j ? i : j, q = i < j ? j : i;
  double app = (p == i) ? di : dj, aqq = (p == i) ? dj : di;
  double t, cm1, s;
  bool rot = (q < n) && jacobi_pair<double>(app, aqq, aij, skip, t, cm1, s, skip_abs);
  double np = app, nq = aqq;
  if (rot) {
    np = app - t * aij;
    nq = aqq + t * aij;
  }
  int x = iy ? j : i;
  double tau = (x == p) ? t : -t;
  double sx = (x == i) ? si : sj, sy = (x == i) ? sj : si;
  rec.mx = rot ? tau * (sy / sx) : 0.0;
  rec.my = rot ? tau * (sx / sy) : 0.0;
  rec.cm1 = rot ? cm1 : 0.0;
  rec.dx = (x == p) ? np : nq;
  rec.dy = (x == p) ? nq : np;
  rec.pad = 0.0;
  return slot;
}

// Records of round r from A's true entries when all scales are 1.
__global__ void rr_init_frec(const double* __restrict__ A, int lda, int n, int m, int r, double skip,
                             double skip_abs, FRec* __restrict__ rec) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m / 2) return;
  int x, y;
  rr_slot(m, r, i, x, y);
  double dx = x < n ? A[(size_t)x * lda + x] : 0.0;
  double dy = y < n ? A[(size_t)y * lda + y] : 0.0;
  double axy = (x < n && y < n) ? A[(size_t)y * lda + x] : 0.0;
  FRec fr;
  rr_make_frec(m, n, r, x, y, dx, dy, axy, 1.0, 1.0, skip, fr, skip_abs);
  rec[i] = fr;
}

__global__ void d_reset(double2* __restrict__ d, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = make_double2(1.0, 0.0);
}

// Lower-triangular tiles (ti >= tj) enumerated row by row: t = ti (ti+1)/2 + tj.
__device__ __forceinline__ void tri_tile(int t, int& ti, int& tj) {
  int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > t) --r;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  ti = r;
  tj = t - r * (r + 1) / 2;
}

// Inputs of one next-round record, queued in shared memory by the thread whose
// 2 x 2 block holds the pair's coupling after this round.
struct HostIn {
  int i, j;            // pair (i, j) of the next round, i from this block's rows
  double di, dj, aij;  // true diagonals after this round, scaled coupling
  double cmi, cmj;     // c - 1 of this round's rotations of i and j (scale update)
};
// Queue length per CTA.  Entries come only from the row side of a block: the
// next-round partner of x_a (and of y_a) lies in exactly one slot, so each of
// a CTA's 16 row slots queues at most 2 entries: at most 32 per CTA.
constexpr int HMAX = 2 * TS;

MPJ_DEV void build_next_rec(const HostIn& h, int m, int n, int rn, double skip, double skip_abs,
                            const double2* __restrict__ dcur, FRec* __restrict__ rec_next) {
  double si = dd_scale(dcur[h.i], h.cmi).x;
  double sj = dd_scale(dcur[h.j], h.cmj).x;
  FRec nr;
  int sl = rr_make_frec(m, n, rn, h.i, h.j, h.di, h.dj, h.aij * si * sj, si, sj, skip, nr, skip_abs);
  rec_next[sl] = nr;
}

// One 2 x 2 block (rows x_a, y_a; columns x_b, y_b) of a round, with the
// diagonal blocks' scale and record work; next-round record inputs hosted by
// the block go to the CTA's shared-memory queue.
MPJ_DEV void rr_block(int a, int b, double* __restrict__ A, int lda, int n, int m, int r, int rn, int half,
                      double skip, double skip_abs, const FRec* __restrict__ rec, FRec* __restrict__ rec_next,
                      const double2* __restrict__ dcur, double2* __restrict__ dnext, double2* __restrict__ hist_row,
                      HostIn* hq, int* hcount) {
  if (a < half && b < half && a >= b) {
    int xa, ya;
    rr_slot(m, r, a, xa, ya);
    const FRec* pa = rec + a;
    const double2 ma = frec_m(pa);
    const bool rota = m_rotated(ma);
    const bool vxa = xa < n, vya = ya < n;
    if (a == b) {
      const FRec ra = *pa;
      const double cm1 = rota ? frec_cm1(ra) : 0.0;
      double2 sx = vxa ? dd_scale(dcur[xa], cm1) : make_double2(1.0, 0.0);
      double2 sy = vya ? dd_scale(dcur[ya], cm1) : make_double2(1.0, 0.0);
      if (vxa) dnext[xa] = sx;
      if (vya) dnext[ya] = sy;
      hist_row[a] = make_double2(ra.mx, ra.my);
      double axy_s;  // scaled coupling after the round
      if (rota) {
        A[(size_t)xa * lda + xa] = ra.dx;
        A[(size_t)ya * lda + ya] = ra.dy;
        A[(size_t)ya * lda + xa] = 0.0;
        A[(size_t)xa * lda + ya] = 0.0;
        axy_s = 0.0;
      } else {
        axy_s = (vxa && vya) ? A[(size_t)ya * lda + xa] : 0.0;
      }
      // the unpaired index of round rn when n is odd (slot 0 pairs it with the dummy)
      if ((n & 1) && (xa == rn || ya == rn)) {
        FRec z;
        z.mx = 0.0;
        z.my = 0.0;
        z.cm1 = 0.0;
        z.dx = (xa == rn) ? ra.dx : ra.dy;
        z.dy = 0.0;
        z.pad = 0.0;
        rec_next[0] = z;
      }
      // m == 2: the same pair again in the next sweep
      if (vxa && vya && rr_partner(m, rn, xa) == ya) {
        FRec nr;
        int sl = rr_make_frec(m, n, rn, xa, ya, ra.dx, ra.dy, axy_s * sx.x * sy.x, sx.x, sy.x, skip, nr, skip_abs);
        rec_next[sl] = nr;
      }
    } else {
      int xb, yb;
      rr_slot(m, r, b, xb, yb);
      const FRec* pb = rec + b;
      const double2 mb = frec_m(pb);
      const bool rotb = m_rotated(mb);
      const bool vxb = xb < n, vyb = yb < n;
      // next-round pairs hosted by this block: (x_a or y_a) with (x_b or y_b)
      int jx = vxa ? rr_partner(m, rn, xa) : -1;
      int jy = vya ? rr_partner(m, rn, ya) : -1;
      bool nx = jx >= 0 && jx < n && (jx == xb || jx == yb);
      bool ny = jy >= 0 && jy < n && (jy == xb || jy == yb);
      if (rota || rotb || nx || ny) {
        size_t cxb = (size_t)xb * lda, cyb = (size_t)yb * lda;
        double vxx = (vxa && vxb) ? A[cxb + xa] : 0.0;
        double vxy = (vxa && vyb) ? A[cyb + xa] : 0.0;
        double vyx = (vya && vxb) ? A[cxb + ya] : 0.0;
        double vyy = (vya && vyb) ? A[cyb + ya] : 0.0;
        if (rota) {  // rows x_a, y_a
          double t0 = fma(-ma.x, vyx, vxx), t1 = fma(ma.y, vxx, vyx);
          double t2 = fma(-ma.x, vyy, vxy), t3 = fma(ma.y, vxy, vyy);
          vxx = t0;
          vyx = t1;
          vxy = t2;
          vyy = t3;
        }
        if (rotb) {  // columns x_b, y_b
          double t0 = fma(-mb.x, vxy, vxx), t1 = fma(mb.y, vxx, vxy);
          double t2 = fma(-mb.x, vyy, vyx), t3 = fma(mb.y, vyx, vyy);
          vxx = t0;
          vxy = t1;
          vyx = t2;
          vyy = t3;
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
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          if (side == 0 && !nx) continue;
          if (side == 1 && !ny) continue;
          HostIn h;
          h.i = side ? ya : xa;
          h.j = side ? jy : jx;
          h.di = side ? pa->dy : pa->dx;
          h.dj = (h.j == xb) ? pb->dx : pb->dy;
          h.aij = side ? ((h.j == xb) ? vyx : vyy) : ((h.j == xb) ? vxx : vxy);
          h.cmi = rota ? pa->cm1 : 0.0;
          h.cmj = rotb ? pb->cm1 : 0.0;
          int slot = atomicAdd(hcount, 1);
          if (slot < HMAX) hq[slot] = h;  // always true (see HMAX)
        }
      }
    }
  }
}


// One round on A (scaled form) + next round's records + this round's V
// multipliers.  A CTA of 128 threads takes a 16 x 16 tile of the lower slot
// triangle; each thread owns two 2 x 2 blocks (row slots a and a + 8, column
// slot b).  Off-diagonal tiles load both blocks' four entries before any
// arithmetic or store (eight loads in flight per thread); diagonal tiles take
// the general per-block path.  The n/2 records of the next round need a
// square root and divisions each; their inputs are queued in shared memory
// and built by the CTA's first warp with all lanes busy, instead of by one
// lane of many warps (FP64 instructions issue at 1/64 of the FP32 rate on
// this GPU).  80 registers, 6 CTAs per SM.
__global__ void __launch_bounds__(128, 6) rr_step64(double* __restrict__ A, int lda, int n, int m, int r,
                                                      double skip, double skip_abs, const FRec* __restrict__ rec,
                                                      FRec* __restrict__ rec_next,
                                                      const double2* __restrict__ dcur, double2* __restrict__ dnext,
                                                      double2* __restrict__ hist_row) {
  __shared__ HostIn hq[HMAX];
  __shared__ int hcount;
  const int half = m / 2;
  const int rn = (r + 1 == m - 1) ? 0 : r + 1;
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int b = tj * TS + (threadIdx.x >> 3);
  const int a0 = ti * TS + (threadIdx.x & 7);
  if (threadIdx.x == 0) hcount = 0;
  // Programmatic dependent launch: once every CTA of this round has started,
  // the next round's CTAs may be scheduled into the slots this round frees;
  // each waits here until the previous round has completed and its writes
  // are visible (no global memory is touched before the wait).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  if (ti == tj) {
#pragma unroll 1
    for (int k = 0; k < 2; ++k)
      rr_block(a0 + 8 * k, b, A, lda, n, m, r, rn, half, skip, skip_abs, rec, rec_next, dcur, dnext, hist_row, hq,
               &hcount);
  } else if (b < half) {  // a > b for both blocks
    int xb, yb;
    rr_slot(m, r, b, xb, yb);
    const FRec* pb = rec + b;
    const double2 mb = frec_m(pb);
    const bool rotb = m_rotated(mb);
    const bool vxb = xb < n, vyb = yb < n;
    const size_t cxb = (size_t)xb * lda, cyb = (size_t)yb * lda;
    int xa[2], ya[2], jx[2], jy[2];
    bool need[2], rota[2], nx[2], ny[2], vxa[2], vya[2];
    double2 ma[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int a = a0 + 8 * k;
      need[k] = false;
      rota[k] = nx[k] = ny[k] = vxa[k] = vya[k] = false;
      xa[k] = ya[k] = jx[k] = jy[k] = 0;
      ma[k] = make_double2(0.0, 0.0);
      if (a < half) {
        rr_slot(m, r, a, xa[k], ya[k]);
        ma[k] = frec_m(rec + a);
        rota[k] = m_rotated(ma[k]);
        vxa[k] = xa[k] < n;
        vya[k] = ya[k] < n;
        jx[k] = vxa[k] ? rr_partner(m, rn, xa[k]) : -1;
        jy[k] = vya[k] ? rr_partner(m, rn, ya[k]) : -1;
        nx[k] = jx[k] >= 0 && jx[k] < n && (jx[k] == xb || jx[k] == yb);
        ny[k] = jy[k] >= 0 && jy[k] < n && (jy[k] == xb || jy[k] == yb);
        need[k] = rota[k] || rotb || nx[k] || ny[k];
      }
    }
    double v[2][4];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      v[k][0] = (need[k] && vxa[k] && vxb) ? A[cxb + xa[k]] : 0.0;
      v[k][1] = (need[k] && vxa[k] && vyb) ? A[cyb + xa[k]] : 0.0;
      v[k][2] = (need[k] && vya[k] && vxb) ? A[cxb + ya[k]] : 0.0;
      v[k][3] = (need[k] && vya[k] && vyb) ? A[cyb + ya[k]] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!need[k]) continue;
      double vxx = v[k][0], vxy = v[k][1], vyx = v[k][2], vyy = v[k][3];
      if (rota[k]) {
        double t0 = fma(-ma[k].x, vyx, vxx), t1 = fma(ma[k].y, vxx, vyx);
        double t2 = fma(-ma[k].x, vyy, vxy), t3 = fma(ma[k].y, vxy, vyy);
        vxx = t0;
        vyx = t1;
        vxy = t2;
        vyy = t3;
      }
      if (rotb) {
        double t0 = fma(-mb.x, vxy, vxx), t1 = fma(mb.y, vxx, vxy);
        double t2 = fma(-mb.x, vyy, vyx), t3 = fma(mb.y, vyx, vyy);
        vxx = t0;
        vxy = t1;
        vyx = t2;
        vyy = t3;
      }
      const int xk = xa[k], yk = ya[k];
      if (rota[k] || rotb) {
        if (vxa[k] && vxb) {
          A[cxb + xk] = vxx;
          A[(size_t)xk * lda + xb] = vxx;
        }
        if (vxa[k] && vyb) {
          A[cyb + xk] = vxy;
          A[(size_t)xk * lda + yb] = vxy;
        }
        if (vya[k] && vxb) {
          A[cxb + yk] = vyx;
          A[(size_t)yk * lda + xb] = vyx;
        }
        if (vya[k] && vyb) {
          A[cyb + yk] = vyy;
          A[(size_t)yk * lda + yb] = vyy;
        }
      }
      const FRec* pa = rec + a0 + 8 * k;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        if (side == 0 && !nx[k]) continue;
        if (side == 1 && !ny[k]) continue;
        HostIn h;
        h.i = side ? yk : xk;
        h.j = side ? jy[k] : jx[k];
        h.di = side ? pa->dy : pa->dx;
        h.dj = (h.j == xb) ? pb->dx : pb->dy;
        h.aij = side ? ((h.j == xb) ? vyx : vyy) : ((h.j == xb) ? vxx : vxy);
        h.cmi = rota[k] ? pa->cm1 : 0.0;
        h.cmj = rotb ? pb->cm1 : 0.0;
        int slot = atomicAdd(&hcount, 1);
        if (slot < HMAX) hq[slot] = h;  // always true (see HMAX)
      }
    }
  }
  __syncthreads();
  const int cnt = hcount < HMAX ? hcount : HMAX;
  if (threadIdx.x < 32)
    for (int k = threadIdx.x; k < cnt; k += 32) build_next_rec(hq[k], m, n, rn, skip, skip_abs, dcur, rec_next);
}

// Apply rounds r0 .. r0+nr-1 of the history to a chunk of ROWS consecutive
// rows of Vt held in shared memory as S[row * n + col]; one thread per slot
// and round, looping over the chunk's rows (2 FMA per row).
template <int ROWS>
__global__ void __launch_bounds__(512) v_apply_rounds(double* __restrict__ V, int ldv, int n, int m, int r0, int nr,
                                                      const double2* __restrict__ hist) {
  extern __shared__ double S[];
  const int half = m / 2;
  const int row0 = blockIdx.x * ROWS;
  const int rc = min(ROWS, n - row0);
  for (int e = threadIdx.x; e < n * ROWS; e += blockDim.x) {
    int col = e / ROWS, row = e % ROWS;
    S[row * n + col] = (row < rc) ? V[(size_t)col * ldv + row0 + row] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < nr; ++k) {
    const int r = r0 + k;
    const double2* h = hist + (size_t)k * half;
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      double2 mm = h[b];
      if ((__double_as_longlong(mm.x) | __double_as_longlong(mm.y)) == 0) continue;
      int x, y;
      rr_slot(m, r, b, x, y);
#pragma unroll
      for (int row = 0; row < ROWS; ++row) {
        double vx = S[row * n + x], vy = S[row * n + y];
        S[row * n + x] = fma(-mm.x, vy, vx);
        S[row * n + y] = fma(mm.y, vx, vy);
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * ROWS; e += blockDim.x) {
    int col = e / ROWS, row = e % ROWS;
    if (row < rc) V[(size_t)col * ldv + row0 + row] = S[row * n + col];
  }
}

template <int ROWS>
static cudaError_t launch_v_apply(double* V, int ldv, int n, int m, int r0, int nr, const double2* hist,
                                  cudaStream_t s) {
  size_t smem = (size_t)ROWS * n * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(v_apply_rounds<ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  v_apply_rounds<ROWS><<<(n + ROWS - 1) / ROWS, 512, smem, s>>>(V, ldv, n, m, r0, nr, hist);
  mpj_count_launch();
  return cudaGetLastError();
}

// rows of V per CTA: as many as fit in about 200 KB of shared memory (<= 8)
static cudaError_t v_apply(double* V, int ldv, int n, int m, int r0, int nr, const double2* hist, cudaStream_t s) {
  int rows = (200 * 1024) / (8 * (n > 0 ? n : 1));
  if (rows >= 8) return launch_v_apply<8>(V, ldv, n, m, r0, nr, hist, s);
  if (rows >= 6) return launch_v_apply<6>(V, ldv, n, m, r0, nr, hist, s);
  if (rows >= 4) return launch_v_apply<4>(V, ldv, n, m, r0, nr, hist, s);
  if (rows >= 2) return launch_v_apply<2>(V, ldv, n, m, r0, nr, hist, s);
  return launch_v_apply<1>(V, ldv, n, m, r0, nr, hist, s);
}

// Fold the scales into A (off the diagonal) and V: A_ij *= d_i d_j, V_ij *= d_j.
__global__ void fold_scales(double* __restrict__ A, int lda, double* __restrict__ V, int ldv, int n,
                            const double2* __restrict__ d) {
  size_t total = (size_t)n * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    double2 dj = d[j];
    double sj = dj.x + dj.y;
    if (i != j) {
      double2 di = d[i];
      double si = di.x + di.y;
      A[(size_t)j * lda + i] = (A[(size_t)j * lda + i] * si) * sj;
    }
    V[(size_t)j * ldv + i] *= sj;
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

// ---- cyclic-by-row as wavefronts (the paper's ordering and update) ----------
// In the cyclic-by-row order (0,1),(0,2),...,(0,n-1),(1,2),...,(n-2,n-1) the
// rotation of pair (p,q) depends only on the earlier rotations that touch p
// or q.  Giving (p,q) the time t = p + q, those earlier rotations all have
// smaller t, the later ones that touch p or q all have larger t, and the
// pairs of one time t are disjoint (p + q = p' + q', p < p' forces q > q',
// and p = q' or q = p' would contradict p < q, p' < q').  So the sweep runs
// as 2n - 3 wavefronts t = 1 .. 2n-3 of the pairs (p, t - p),
// p = max(0, t-n+1) .. (t-1)/2, applying exactly the paper's rotation
// sequence; only the interleaving of commuting updates of disjoint pairs
// changes.  Each rotation is Algorithm 2 with the paper's row update, then
// column update, then vector update (J = [c s; -s c]).  An entry (i, j)
// between two pairs a < b of one wavefront (i in a, j in b) becomes
// ((J_a^T B) J_b)(i, j), B = A([p_a q_a], [p_b q_b]): the sequential algorithm
// applies a's row update and then b's column update to it, and the mirror
// entry gets the same value bit for bit, so both triangles stay equal.  A
// pair's own 2 x 2 block (J^T B J) is stored with its two off-diagonal values
// averaged, which is what the paper's end-of-sweep symmetrization does.

struct WaveRec {
  double c, s;
  int rot;
  int pad;
};

// Rotation parameters of the wavefront's pairs (skip rule of Algorithm 4).
__global__ void cyc_wave_params(const double* __restrict__ A, int lda, int n, int t, int plo, int k, double skip,
                                double skip_abs, WaveRec* __restrict__ rec, int* __restrict__ rotated) {
  const int kp = blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= k) return;
  const int p = plo + kp, q = t - p;
  const double app = A[(size_t)p * lda + p], aqq = A[(size_t)q * lda + q], apq = A[(size_t)p * lda + q];
  WaveRec r;
  r.c = 1.0;
  r.s = 0.0;
  r.rot = 0;
  r.pad = 0;
  if (fabs(apq) > skip * sqrt(fabs(app * aqq)) && fabs(apq) > skip_abs) {
    // Algorithm 2, stable form (Appendix A approach 2)
    const double tau = (aqq - app) / (2.0 * apq);
    const double tt = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : 1.0 / (tau - sqrt(1.0 + tau * tau));
    r.c = 1.0 / sqrt(1.0 + tt * tt);
    r.s = tt * r.c;
    r.rot = 1;
    *rotated = 1;
  }
  rec[kp] = r;
}

// new (x_p, x_q) = (c x_p - s x_q, s x_p + c x_q): the row update J^T x and
// the column / vector update x J of Sec. 3.2.2 have the same form.
MPJ_DEV void jrot(double c, double s, double& xp, double& xq) {
  const double np = c * xp - s * xq, nq = s * xp + c * xq;
  xp = np;
  xq = nq;
}

// One wavefront: CTA (chunk, kp) owns columns p, q of pair kp (rows
// j in its chunk) and of V.  Rows j outside the wavefront get the column
// update and its mirror (rows p, q of column j).  Rows of another pair kj of
// the wavefront: the thread of that pair's first index computes the whole
// 2 x 2 block of rows (p_j, q_j) in columns (p, q) in the canonical order
// (lower pair index first); the other pair's CTA computes the mirror block
// from the same operands in the same order.  Nothing a CTA reads is written
// by another CTA of the same launch.
__global__ void __launch_bounds__(256) cyc_wave_update(double* __restrict__ A, int lda, double* __restrict__ V,
                                                       int ldv, int n, int t, int plo, int phi,
                                                       const WaveRec* __restrict__ rec) {
  const int kp = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const WaveRec ra = rec[kp];
  const int p = plo + kp, q = t - p;
  if (j >= n) return;
  const size_t cp = (size_t)p * lda, cq = (size_t)q * lda;
  // vectors: V(:, [p q]) = V(:, [p q]) J
  if (ra.rot) {
    double vp = V[(size_t)p * ldv + j], vq = V[(size_t)q * ldv + j];
    jrot(ra.c, ra.s, vp, vq);
    V[(size_t)p * ldv + j] = vp;
    V[(size_t)q * ldv + j] = vq;
  }
  const int qlo = t - phi;
  const bool in_p = j >= plo && j <= phi;
  const bool in_q = j >= qlo && j <= t - plo;
  if (!in_p && !in_q) {
    if (!ra.rot) return;
    double xp = A[cp + j], xq = A[cq + j];
    jrot(ra.c, ra.s, xp, xq);
    A[cp + j] = xp;
    A[cq + j] = xq;
    A[(size_t)j * lda + p] = xp;
    A[(size_t)j * lda + q] = xq;
    return;
  }
  if (in_q) return;  // rows of a pair are handled by the thread of its first index
  const int kj = j - plo;
  const int pj = j, qj = t - j;
  const WaveRec rb = rec[kj];
  if (kj == kp) {
    if (!ra.rot) return;
    // own block: rows (J^T B), then columns (.. J)
    double bpp = A[cp + p], bqp = A[cp + q], bpq = A[cq + p], bqq = A[cq + q];
    jrot(ra.c, ra.s, bpp, bqp);  // column p of B: rows p, q
    jrot(ra.c, ra.s, bpq, bqq);  // column q of B
    jrot(ra.c, ra.s, bpp, bpq);  // row p: columns p, q
    jrot(ra.c, ra.s, bqp, bqq);  // row q
    const double off = 0.5 * (bpq + bqp);
    A[cp + p] = bpp;
    A[cq + q] = bqq;
    A[cp + q] = off;
    A[cq + p] = off;
    return;
  }
  if (!ra.rot && !rb.rot) return;
  // rows (pj, qj) x columns (p, q): B(r, c) = A[row + col * lda]
  double b00 = A[cp + pj], b10 = A[cp + qj], b01 = A[cq + pj], b11 = A[cq + qj];
  if (kj < kp) {
    // T = (J_kj^T B) J_kp, stored as is
    jrot(rb.c, rb.s, b00, b10);  // rows pj, qj of column p
    jrot(rb.c, rb.s, b01, b11);  // of column q
    jrot(ra.c, ra.s, b00, b01);  // columns p, q of row pj
    jrot(ra.c, ra.s, b10, b11);  // of row qj
  } else {
    // canonical order with kp first: T' = (J_kp^T B^T) J_kj, stored transposed;
    // B^T(r', c') has rows (p, q), columns (pj, qj): B^T = [b00 b10; b01 b11]
    double t00 = b00, t01 = b10, t10 = b01, t11 = b11;
    jrot(ra.c, ra.s, t00, t10);  // rows p, q of column pj
    jrot(ra.c, ra.s, t01, t11);  // of column qj
    jrot(rb.c, rb.s, t00, t01);  // columns pj, qj of row p
    jrot(rb.c, rb.s, t10, t11);  // of row q
    b00 = t00;
    b10 = t01;
    b01 = t10;
    b11 = t11;
  }
  A[cp + pj] = b00;
  A[cp + qj] = b10;
  A[cq + pj] = b01;
  A[cq + qj] = b11;
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

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch layout: 2 record arrays, 2 scale arrays (double2), reduction
// partials and scalars, then the V history (rv rounds of m/2 double2).
static size_t scratch_fixed(int n) {
  int m = n + (n & 1);
  return 2 * align256((size_t)(m / 2 + 1) * sizeof(FRec)) + 2 * align256((size_t)n * sizeof(double2)) +
         align256(RED_CTAS * sizeof(double) + 4 * sizeof(double) + 64);
}

size_t mpj_jacobi64_scratch_bytes_rv(int n, int rv) {
  int m = n + (n & 1);
  return scratch_fixed(n) + (size_t)rv * (m / 2) * sizeof(double2);
}

// Room for two halves of RV_MAX rounds each: the rotation kernels fill one
// half while the batched V update of the other half runs on a side stream.
size_t mpj_jacobi64_scratch_bytes(int n) { return mpj_jacobi64_scratch_bytes_rv(n, 2 * RV_MAX); }

// The block ordering needs, after the fixed part, an n x n FP64 buffer and the
// per-round digit tiles of the U_P.
size_t mpj_jacobi64_scratch_bytes_ordering(int n, int ordering) {
  if (ordering == MPJ_ORDER_BLOCK)
    return scratch_fixed(n) + align256((size_t)n * n * sizeof(double)) + align256(mpj_blocked_scratch_bytes(n));
  return mpj_jacobi64_scratch_bytes(n);
}

namespace {
// rr_step64 with programmatic stream serialization, so that consecutive
// rounds overlap their launch and ramp-up (the kernel waits in
// griddepcontrol.wait before touching memory).
cudaError_t launch_rr_step64(int grid, cudaStream_t s, double* A, int lda, int n, int m, int r, double skip,
                             double skip_abs, const FRec* rec, FRec* rec_next, const double2* dcur, double2* dnext,
                             double2* hist_row) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e =
      cudaLaunchKernelEx(&cfg, rr_step64, A, lda, n, m, r, skip, skip_abs, rec, rec_next, dcur, dnext, hist_row);
  mpj_count_launch();
  return e;
}

bool overlap_enabled(int n) { return mpj_v_overlap_enabled() && n >= 256; }
}  // namespace

bool mpj_v_overlap_enabled() {
  static int env = -1;
  if (env < 0) {
    const char* e = getenv("MPJ_JACOBI_OVERLAP");
    env = (e && e[0] == '0') ? 0 : 1;
  }
  return env == 1;
}

int mpj_jacobi64_run(int n, double* A, int lda, double* V, int ldv, double tol, int ordering, int max_sweeps,
                     int* sweeps_out, double* off_out, double* off_initial, void* scratch, size_t scratch_bytes,
                     cudaStream_t s, double skip_abs, bool side_stream, long long* rotated_blocks_out) {
  const double skip = 0x1p-53;
  const int m = n + (n & 1);
  const int half = m / 2;
  char* base = (char*)scratch;
  FRec* rec[2];
  double2* dsc[2];
  size_t off_b = 0;
  rec[0] = (FRec*)(base + off_b);
  off_b += align256((size_t)(half + 1) * sizeof(FRec));
  rec[1] = (FRec*)(base + off_b);
  off_b += align256((size_t)(half + 1) * sizeof(FRec));
  dsc[0] = (double2*)(base + off_b);
  off_b += align256((size_t)n * sizeof(double2));
  dsc[1] = (double2*)(base + off_b);
  off_b += align256((size_t)n * sizeof(double2));
  double* partial = (double*)(base + off_b);
  double* dscal = partial + RED_CTAS;
  int* iscal = (int*)(dscal + 2);
  off_b += align256(RED_CTAS * sizeof(double) + 4 * sizeof(double) + 64);
  double2* hist = (double2*)(base + off_b);
  if (ordering == MPJ_ORDER_BLOCK ? mpj_jacobi64_scratch_bytes_ordering(n, ordering) > scratch_bytes
                                  : mpj_jacobi64_scratch_bytes_rv(n, 1) > scratch_bytes)
    return MPJ_EWORKSPACE;
  // rounds of history that fit; with the side stream two halves of rv rounds
  const size_t cap = (scratch_bytes - scratch_fixed(n)) / ((size_t)half * sizeof(double2));
  bool overlap = side_stream && ordering == MPJ_ORDER_ROUND_ROBIN && overlap_enabled(n) && cap >= 16;
  int rv = RV_MAX;
  while (rv > 1 && (size_t)rv * (overlap ? 2 : 1) > cap) rv >>= 1;

  double off2 = 0.0;
  MPJ_CUDA_TRY(mpj_sumsq(A, lda, n, true, partial, dscal, nullptr, s));
  MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
  MPJ_CUDA_TRY(cudaStreamSynchronize(s));
  double off = sqrt(off2);
  if (off_initial) *off_initial = off;
  int sweeps = 0;
  int status = MPJ_OK;
  if (ordering == MPJ_ORDER_ROUND_ROBIN) {
    const int nt = (half + TS - 1) / TS;
    const int n_atiles = nt * (nt + 1) / 2;  // lower-triangular TS x TS-slot tiles
    const int fgrid = (int)(((size_t)n * n + 255) / 256 > 4096 ? 4096 : ((size_t)n * n + 255) / 256);
    int k = 0;  // buffer parity of records and scales
    bool need_init = true;
    std::unique_ptr<SideStream> side;
    if (overlap) {
      side.reset(new SideStream(s));
      if (!side->ok) overlap = false;
    }
    int hb = 0;                          // history half being filled
    bool used[2] = {false, false};       // a V update may still read that half
    double2* hcur = hist;
    while (off > tol && n > 1) {
      if (sweeps >= max_sweeps) {
        status = MPJ_NOT_CONVERGED;
        break;
      }
      if (need_init) {
        d_reset<<<(n + 255) / 256, 256, 0, s>>>(dsc[k], n);
        mpj_count_launch();
        rr_init_frec<<<(half + 127) / 128, 128, 0, s>>>(A, lda, n, m, 0, skip, skip_abs, rec[k]);
        mpj_count_launch();
      }
      int pending = 0, since_fold = 0;
      for (int r = 0; r < m - 1; ++r) {
        if (overlap && pending == 0 && used[hb])  // the V update reading this half must be done
          MPJ_CUDA_TRY(cudaStreamWaitEvent(s, side->done[hb], 0));
        MPJ_CUDA_TRY(launch_rr_step64(n_atiles, s, A, lda, n, m, r, skip, skip_abs, rec[k], rec[k ^ 1], dsc[k],
                                      dsc[k ^ 1], hcur + (size_t)pending * half));
        k ^= 1;
        ++pending;
        ++since_fold;
        const bool last = (r == m - 2);
        const bool fold = last || since_fold == RS;
        if (pending == rv || fold) {
          if (overlap) {
            MPJ_CUDA_TRY(cudaEventRecord(side->ready, s));
            MPJ_CUDA_TRY(cudaStreamWaitEvent(side->sv, side->ready, 0));
            MPJ_CUDA_TRY(v_apply(V, ldv, n, m, r - pending + 1, pending, hcur, side->sv));
            MPJ_CUDA_TRY(cudaEventRecord(side->done[hb], side->sv));
            used[hb] = true;
            if (fold) MPJ_CUDA_TRY(cudaStreamWaitEvent(s, side->done[hb], 0));  // V is rescaled next
            hb ^= 1;
            hcur = hist + (size_t)hb * rv * half;
          } else {
            MPJ_CUDA_TRY(v_apply(V, ldv, n, m, r - pending + 1, pending, hist, s));
          }
          pending = 0;
        }
        if (fold) {
          fold_scales<<<fgrid, 256, 0, s>>>(A, lda, V, ldv, n, dsc[k]);
          mpj_count_launch();
          since_fold = 0;
          if (!last) {  // records of round r+1 were built for the old scales
            d_reset<<<(n + 255) / 256, 256, 0, s>>>(dsc[k], n);
            mpj_count_launch();
            rr_init_frec<<<(half + 127) / 128, 128, 0, s>>>(A, lda, n, m, r + 1, skip, skip_abs, rec[k]);
            mpj_count_launch();
          }
        }
      }
      MPJ_CUDA_TRY(cudaGetLastError());
      need_init = true;
      ++sweeps;
      MPJ_CUDA_TRY(mpj_sumsq(A, lda, n, true, partial, dscal, nullptr, s));
      MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
      MPJ_CUDA_TRY(cudaStreamSynchronize(s));
      off = sqrt(off2);
    }
  } else if (ordering == MPJ_ORDER_BLOCK) {
    double* B = (double*)(base + scratch_fixed(n));
    void* bscratch = base + scratch_fixed(n) + align256((size_t)n * n * sizeof(double));
    unsigned* bflags = (unsigned*)(iscal + 1);
    unsigned* nrot = (unsigned*)(iscal + 2);
    unsigned hflags = 0, hnrot = 0;
    MPJ_CUDA_TRY(cudaMemsetAsync(bflags, 0, 2 * sizeof(unsigned), s));
    const int rounds = mpj_blocked_rounds_per_sweep(n);
    // V <- V U~ of round R runs on a private side stream, overlapping round
    // R+1's subproblems and A update; the U_P sets alternate between rounds,
    // and round R+2's subproblems wait for round R's V update before
    // overwriting its set.  The side stream is joined at every sweep end.
    std::unique_ptr<SideStream> side;
    if (side_stream && overlap_enabled(n)) {
      side.reset(new SideStream(s));
      if (!side->ok) side.reset();
    }
    bool vpending[2] = {false, false};
    while (off > tol && n > 1) {
      if (sweeps >= max_sweeps) {
        status = MPJ_NOT_CONVERGED;
        break;
      }
      for (int R = 0; R < rounds; ++R) {
        const int par = R & 1;
        if (side && vpending[par]) MPJ_CUDA_TRY(cudaStreamWaitEvent(s, side->done[par], 0));
        MPJ_CUDA_TRY(mpj_blocked_solve(A, lda, n, R, skip, skip_abs, bscratch, nrot, s));
        if (side) {
          MPJ_CUDA_TRY(cudaEventRecord(side->ready, s));
          MPJ_CUDA_TRY(cudaStreamWaitEvent(side->sv, side->ready, 0));
          MPJ_CUDA_TRY(mpj_blocked_update_V(V, ldv, n, R, bscratch, bflags, side->sv));
          MPJ_CUDA_TRY(cudaEventRecord(side->done[par], side->sv));
          vpending[par] = true;
        } else {
          MPJ_CUDA_TRY(mpj_blocked_update_V(V, ldv, n, R, bscratch, bflags, s));
        }
        MPJ_CUDA_TRY(mpj_blocked_update_A(A, lda, B, n, R, bscratch, bflags, s));
      }
      if (side) {
        for (int par = 0; par < 2; ++par)
          if (vpending[par]) MPJ_CUDA_TRY(cudaStreamWaitEvent(s, side->done[par], 0));
        vpending[0] = vpending[1] = false;
      }
      MPJ_CUDA_TRY(mpj_blocked_symmetrize(A, lda, n, s));
      ++sweeps;
      MPJ_CUDA_TRY(mpj_sumsq(A, lda, n, true, partial, dscal, nullptr, s));
      MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
      MPJ_CUDA_TRY(cudaMemcpyAsync(&hflags, bflags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
      MPJ_CUDA_TRY(cudaMemcpyAsync(&hnrot, nrot, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
      MPJ_CUDA_TRY(cudaStreamSynchronize(s));
      off = sqrt(off2);
      if (rotated_blocks_out) *rotated_blocks_out = hnrot;
      if (hflags & MPJ_FLAG_TIMEOUT) {
        status = MPJ_ETIMEOUT;
        break;
      }
    }
  } else {
    while (off > tol && n > 1) {
      if (sweeps >= max_sweeps) {
        status = MPJ_NOT_CONVERGED;
        break;
      }
      // one sweep = 2n - 3 wavefronts; the rotation records use the record area
      WaveRec* wrec = reinterpret_cast<WaveRec*>(rec[0]);
      MPJ_CUDA_TRY(cudaMemsetAsync(iscal, 0, sizeof(int), s));
      for (int t = 1; t <= 2 * n - 3; ++t) {
        const int plo = t - (n - 1) > 0 ? t - (n - 1) : 0;
        const int phi = (t - 1) / 2;
        const int k = phi - plo + 1;
        cyc_wave_params<<<(k + 127) / 128, 128, 0, s>>>(A, lda, n, t, plo, k, skip, skip_abs, wrec, iscal);
        mpj_count_launch();
        cyc_wave_update<<<dim3((n + 255) / 256, k), 256, 0, s>>>(A, lda, V, ldv, n, t, plo, phi, wrec);
        mpj_count_launch();
      }
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
  if (n > MPJ_NOALLOC_MAX_N || mpj_jacobi64_scratch_bytes_rv(n, 1) > (size_t)MPJ_NOALLOC_SCRATCH_BYTES)
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
                        w, (size_t)MPJ_NOALLOC_SCRATCH_BYTES, s, 0.0, /*side_stream=*/false);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && st >= 0) {
    mpj_set_cuda_error(e, "mpj_jacobi64_noalloc sync", __LINE__);
    st = MPJ_ECUDA;
  }
  return st;
}
