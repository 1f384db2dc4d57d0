/*
 * mpj_oracle.c -- plain, slow, obviously correct CPU oracle of the mixed
 * precision Jacobi eigensolver (Zhou, "A Mixed Precision Eigensolver Based on
 * the Jacobi Algorithm", arXiv 2509.00495).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call, link or
 * execute this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or constant table with
 * the CUDA path.
 *
 * Conventions: every matrix is column-major with a leading dimension,
 * A(i,j) = A[i + j*lda], indices 0-based.  Built with -O2 -ffp-contract=off so
 * that every multiply and add is rounded separately, in the order written.
 *
 * Each function names the passage of the paper it follows.  The pieces that the
 * paper does not define (round-robin ordering, the off(A) <= tol stopping rule,
 * the optional final polish, the eigen-adjoint) say where their definition
 * comes from.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CYCLIC 0      /* cyclic-by-row ordering, Sec. 3.3 (Algorithm 4)     */
#define ORC_ROUND_ROBIN 1 /* circle-method tournament ordering (not in the paper) */
#define ORC_BLOCK_RR 2    /* block round-robin ordering of the FP32 stage (not in the paper) */
#define ORC_BLK 16        /* block size of ORC_BLOCK_RR */

#define AT(M, ld, i, j) ((M)[(size_t)(i) + (size_t)(j) * (size_t)(ld)])

/* Rounding of an FP32 value to the nearest IEEE binary16 value (ties to
 * even), for the half-precision stage 1 (Ch. 6, further work item 3: "these
 * theories can apply to half precision as well").  Reading: a half-precision
 * Jacobi keeps A, V and the rotation parameters in binary16 and rounds every
 * update, computed in FP32 from binary16 operands, once to binary16.        */
float orc_round_half(float x) { return (float)(_Float16)x; }
static float rq(float x, int half) { return half ? orc_round_half(x) : x; }

/* ------------------------------------------------------------------------ */
/* Algorithm 2 (jacobi_pair, Sec. 3.1.1-3.1.2) in the stable form the paper
 * prefers (Sec. 3.1.2 and Appendix A, approach 2): tau = (a_qq - a_pp) / (2 a_pq),
 * t = 1 / (tau + sqrt(1 + tau^2)) for tau >= 0, t = 1 / (tau - sqrt(1 + tau^2))
 * otherwise, c = 1 / sqrt(1 + t^2), s = t c.  a_pq = 0 gives (c, s) = (1, 0).  */
void orc_jacobi_pair_d(double app, double aqq, double apq, double* c, double* s) {
  if (apq == 0.0) {
    *c = 1.0;
    *s = 0.0;
    return;
  }
  double tau = (aqq - app) / (2.0 * apq);
  double t;
  if (tau >= 0.0)
    t = 1.0 / (tau + sqrt(1.0 + tau * tau));
  else
    t = 1.0 / (tau - sqrt(1.0 + tau * tau));
  *c = 1.0 / sqrt(1.0 + t * t);
  *s = t * (*c);
}

void orc_jacobi_pair_f(float app, float aqq, float apq, float* c, float* s) {
  if (apq == 0.0f) {
    *c = 1.0f;
    *s = 0.0f;
    return;
  }
  float tau = (aqq - app) / (2.0f * apq);
  float t;
  if (tau >= 0.0f)
    t = 1.0f / (tau + sqrtf(1.0f + tau * tau));
  else
    t = 1.0f / (tau - sqrtf(1.0f + tau * tau));
  *c = 1.0f / sqrtf(1.0f + t * t);
  *s = t * (*c);
}

/* off(A): Frobenius norm of the off-diagonal part, in the direct form
 * sqrt(sum_{i != j} a_ij^2) of the definition in Sec. 3.1 (the form the
 * paper's `off` listing evaluates).  Summed in column order, in double.      */
double orc_off_d(int n, const double* A, int lda) {
  double s = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i)
      if (i != j) s += AT(A, lda, i, j) * AT(A, lda, i, j);
  return sqrt(s);
}

double orc_off_f(int n, const float* A, int lda) {
  double s = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i)
      if (i != j) {
        double x = (double)AT(A, lda, i, j);
        s += x * x;
      }
  return sqrt(s);
}

double orc_fro_d(int n, const double* A, int lda) {
  double s = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) s += AT(A, lda, i, j) * AT(A, lda, i, j);
  return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* One Jacobi rotation applied as the paper does it (the O(n) row/column
 * update of Sec. 3.2.2, used by Algorithm 4 in Sec. 3.3): with J = [c s; -s c],
 *   rows:    A([p q],:) = J^T A([p q],:)
 *   columns: A(:,[p q]) = A(:,[p q]) J
 *   vectors: V(:,[p q]) = V(:,[p q]) J                                         */
static void rotate_d(int n, double* A, int lda, double* V, int ldv, int p, int q, double c, double s) {
  for (int k = 0; k < n; ++k) {
    double ap = AT(A, lda, p, k), aq = AT(A, lda, q, k);
    AT(A, lda, p, k) = c * ap - s * aq;
    AT(A, lda, q, k) = s * ap + c * aq;
  }
  for (int k = 0; k < n; ++k) {
    double ap = AT(A, lda, k, p), aq = AT(A, lda, k, q);
    AT(A, lda, k, p) = c * ap - s * aq;
    AT(A, lda, k, q) = s * ap + c * aq;
  }
  for (int k = 0; k < n; ++k) {
    double vp = AT(V, ldv, k, p), vq = AT(V, ldv, k, q);
    AT(V, ldv, k, p) = c * vp - s * vq;
    AT(V, ldv, k, q) = s * vp + c * vq;
  }
}

static void rotate_f(int n, float* A, int lda, float* V, int ldv, int p, int q, float c, float s, int half) {
  for (int k = 0; k < n; ++k) {
    float ap = AT(A, lda, p, k), aq = AT(A, lda, q, k);
    AT(A, lda, p, k) = rq(c * ap - s * aq, half);
    AT(A, lda, q, k) = rq(s * ap + c * aq, half);
  }
  for (int k = 0; k < n; ++k) {
    float ap = AT(A, lda, k, p), aq = AT(A, lda, k, q);
    AT(A, lda, k, p) = rq(c * ap - s * aq, half);
    AT(A, lda, k, q) = rq(s * ap + c * aq, half);
  }
  for (int k = 0; k < n; ++k) {
    float vp = AT(V, ldv, k, p), vq = AT(V, ldv, k, q);
    AT(V, ldv, k, p) = rq(c * vp - s * vq, half);
    AT(V, ldv, k, q) = rq(s * vp + c * vq, half);
  }
}

/* Pair k of a sweep.  Cyclic-by-row (Sec. 3.3): (0,1),(0,2),...,(0,n-1),
 * (1,2),...,(n-2,n-1).  Round-robin (circle method; m = n rounded up to even,
 * index m-1 is a dummy when n is odd): in round r = 0..m-2 the pairs are
 * (r, m-1) and ((r+i) mod (m-1), (r-i) mod (m-1)) for i = 1..m/2-1, each pair
 * written with p < q; every unordered pair occurs in exactly one round.
 * Returns 0 for a pair that involves the dummy index.                         */
static int rr_pair(int n, int r, int i, int* p, int* q) {
  int m = n + (n & 1);
  int a, b;
  if (i == 0) {
    a = r;
    b = m - 1;
  } else {
    a = (r + i) % (m - 1);
    b = ((r - i) % (m - 1) + (m - 1)) % (m - 1);
  }
  if (a > b) {
    int t = a;
    a = b;
    b = t;
  }
  *p = a;
  *q = b;
  return b < n;
}

void orc_round_robin_pair(int n, int r, int i, int* p, int* q, int* valid) { *valid = rr_pair(n, r, i, p, q); }

/* Block round-robin ordering (the FP32 stage's ordering): indices padded to
 * N = n rounded up to a multiple of 2*ORC_BLK are cut into nb = N/ORC_BLK
 * blocks.  A sweep is nb-1 outer rounds of the circle method on blocks; in
 * outer round R, block pair P = (I, J), I < J, runs one inner circle-method
 * sweep (2*ORC_BLK - 1 inner rounds of ORC_BLK pairs) over the 2*ORC_BLK
 * indices of I u J, local index l < ORC_BLK meaning I*ORC_BLK + l and
 * l >= ORC_BLK meaning J*ORC_BLK + l - ORC_BLK.  This returns the global pair
 * (p < q) of inner pair i of inner round rho; 0 when q is a padding index.  */
int orc_block_pair(int n, int R, int P, int rho, int i, int* p, int* q) {
  int N = ((n + 2 * ORC_BLK - 1) / (2 * ORC_BLK)) * (2 * ORC_BLK);
  int nb = N / ORC_BLK;
  int I, J, lx, ly;
  rr_pair(nb, R, P, &I, &J);
  rr_pair(2 * ORC_BLK, rho, i, &lx, &ly);
  int gx = lx < ORC_BLK ? I * ORC_BLK + lx : J * ORC_BLK + (lx - ORC_BLK);
  int gy = ly < ORC_BLK ? I * ORC_BLK + ly : J * ORC_BLK + (ly - ORC_BLK);
  *p = gx < gy ? gx : gy;
  *q = gx < gy ? gy : gx;
  return *q < n;
}

static int block_nb(int n) { return ((n + 2 * ORC_BLK - 1) / (2 * ORC_BLK)) * 2; }

/* Symmetrize A = (A + A^T)/2, as the paper's cyclic listing does after every
 * sweep in which a rotation happened (Appendix B, jacobi_cyclic).           */
static void symmetrize_d(int n, double* A, int lda) {
  for (int j = 0; j < n; ++j)
    for (int i = j + 1; i < n; ++i) {
      double v = (AT(A, lda, i, j) + AT(A, lda, j, i)) / 2.0;
      AT(A, lda, i, j) = v;
      AT(A, lda, j, i) = v;
    }
}
static void symmetrize_f(int n, float* A, int lda, int half) {
  for (int j = 0; j < n; ++j)
    for (int i = j + 1; i < n; ++i) {
      float v = rq((AT(A, lda, i, j) + AT(A, lda, j, i)) / 2.0f, half);
      AT(A, lda, i, j) = v;
      AT(A, lda, j, i) = v;
    }
}

/* Timing sample of the oracle's inner loop (for the CPU-baseline estimate
 * only): the first `nrot` rotations of a cyclic-by-row sweep, each with its
 * Algorithm 2 parameters and the paper's row/column/vector update, in FP64
 * (dtype 0) or FP32 (dtype 1), without the skip test.                      */
void orc_sample_rotations(int n, void* A, int lda, void* V, int ldv, long long nrot, int dtype) {
  long long k = 0;
  for (int p = 0; p < n - 1 && k < nrot; ++p)
    for (int q = p + 1; q < n && k < nrot; ++q, ++k) {
      if (dtype == 0) {
        double* a = (double*)A;
        double c, s;
        orc_jacobi_pair_d(AT(a, lda, p, p), AT(a, lda, q, q), AT(a, lda, p, q), &c, &s);
        rotate_d(n, a, lda, (double*)V, ldv, p, q, c, s);
      } else {
        float* a = (float*)A;
        float c, s;
        orc_jacobi_pair_f(AT(a, lda, p, p), AT(a, lda, q, q), AT(a, lda, p, q), &c, &s);
        rotate_f(n, a, lda, (float*)V, ldv, p, q, c, s, 0);
      }
    }
}

/* Cyclic Jacobi, Algorithm 4, FP64.
 *  - skip rule: pair (p,q) is rotated iff |a_pq| > skip_tol * sqrt(|a_pp a_qq|)
 *    (Algorithm 4's test; skip_tol = 2^-53 in the paper's experiments) and,
 *    for the threshold variant (Sec. 6 future work: threshold Jacobi),
 *    |a_pq| > skip_abs (skip_abs = 0 disables it);
 *  - stopping: when paper_mode = 0, stop as soon as off(A) <= tol, tested
 *    before the first sweep and after each sweep (the reading of the stopping
 *    rule used by this library); when paper_mode = 1, stop after a sweep with
 *    no rotation (the paper's rule), counting only sweeps that rotated;
 *  - at most max_sweeps sweeps (the paper's maxiter; its default is 10).
 * V must hold the starting matrix (the identity for a plain solve).
 * Returns 1 when the loop ended because of the cap (off > tol), else 0.     */
int orc_jacobi_d(int n, double* A, int lda, double* V, int ldv, int ordering, double tol, double skip_tol,
                 int max_sweeps, int paper_mode, int* sweeps_out, long long* rotations_out, double* off_out,
                 double skip_abs) {
  int sweeps = 0;
  long long rot = 0;
  int capped = 0;
  int m = n + (n & 1);
  double off = orc_off_d(n, A, lda);
  for (;;) {
    if (!paper_mode && off <= tol) break;
    if (sweeps >= max_sweeps) {
      capped = 1;
      break;
    }
    int done_rot = 0;
    if (ordering == ORC_CYCLIC) {
      for (int p = 0; p < n - 1; ++p)
        for (int q = p + 1; q < n; ++q) {
          double apq = AT(A, lda, p, q);
          if (fabs(apq) > skip_tol * sqrt(fabs(AT(A, lda, p, p) * AT(A, lda, q, q))) && fabs(apq) > skip_abs) {
            double c, s;
            orc_jacobi_pair_d(AT(A, lda, p, p), AT(A, lda, q, q), apq, &c, &s);
            rotate_d(n, A, lda, V, ldv, p, q, c, s);
            done_rot = 1;
            ++rot;
          }
        }
    } else if (ordering == ORC_BLOCK_RR) {
      int nb = block_nb(n);
      for (int R = 0; R < nb - 1; ++R)
        for (int P = 0; P < nb / 2; ++P)
          for (int rho = 0; rho < 2 * ORC_BLK - 1; ++rho)
            for (int i = 0; i < ORC_BLK; ++i) {
              int p, q;
              if (!orc_block_pair(n, R, P, rho, i, &p, &q)) continue;
              double apq = AT(A, lda, p, q);
              if (fabs(apq) > skip_tol * sqrt(fabs(AT(A, lda, p, p) * AT(A, lda, q, q))) && fabs(apq) > skip_abs) {
                double c, s;
                orc_jacobi_pair_d(AT(A, lda, p, p), AT(A, lda, q, q), apq, &c, &s);
                rotate_d(n, A, lda, V, ldv, p, q, c, s);
                done_rot = 1;
                ++rot;
              }
            }
    } else {
      for (int r = 0; r < m - 1; ++r)
        for (int i = 0; i < m / 2; ++i) {
          int p, q;
          if (!rr_pair(n, r, i, &p, &q)) continue;
          double apq = AT(A, lda, p, q);
          if (fabs(apq) > skip_tol * sqrt(fabs(AT(A, lda, p, p) * AT(A, lda, q, q))) && fabs(apq) > skip_abs) {
            double c, s;
            orc_jacobi_pair_d(AT(A, lda, p, p), AT(A, lda, q, q), apq, &c, &s);
            rotate_d(n, A, lda, V, ldv, p, q, c, s);
            done_rot = 1;
            ++rot;
          }
        }
    }
    if (done_rot) {
      symmetrize_d(n, A, lda);
      ++sweeps;
    } else if (paper_mode) {
      break;
    } else {
      ++sweeps; /* a sweep ran; it found nothing to rotate */
      off = orc_off_d(n, A, lda);
      break;
    }
    off = orc_off_d(n, A, lda);
  }
  if (paper_mode) capped = (sweeps >= max_sweeps);
  *sweeps_out = sweeps;
  if (rotations_out) *rotations_out = rot;
  if (off_out) *off_out = off;
  return capped;
}

/* The same loop in FP32 (stage 1 of the mixed algorithm, where the paper
 * calls eig(single(A)) and this library runs an FP32 Jacobi instead).
 * off(A) and tol are evaluated in double from the float entries.          */
static int jacobi_low(int n, float* A, int lda, float* V, int ldv, int ordering, double tol, float skip_tol,
                      int max_sweeps, int* sweeps_out, long long* rotations_out, double* off_out, int half);

int orc_jacobi_f(int n, float* A, int lda, float* V, int ldv, int ordering, double tol, float skip_tol,
                 int max_sweeps, int* sweeps_out, long long* rotations_out, double* off_out) {
  return jacobi_low(n, A, lda, V, ldv, ordering, tol, skip_tol, max_sweeps, sweeps_out, rotations_out, off_out, 0);
}

/* The same loop in half precision: A and V hold binary16 values, the
 * rotation parameters are rounded to binary16, and every update is rounded
 * once to binary16 (see orc_round_half). */
int orc_jacobi_h(int n, float* A, int lda, float* V, int ldv, int ordering, double tol, float skip_tol,
                 int max_sweeps, int* sweeps_out, long long* rotations_out, double* off_out) {
  return jacobi_low(n, A, lda, V, ldv, ordering, tol, skip_tol, max_sweeps, sweeps_out, rotations_out, off_out, 1);
}

static int jacobi_low(int n, float* A, int lda, float* V, int ldv, int ordering, double tol, float skip_tol,
                      int max_sweeps, int* sweeps_out, long long* rotations_out, double* off_out, int half) {
  int sweeps = 0;
  long long rot = 0;
  int capped = 0;
  int m = n + (n & 1);
  double off = orc_off_f(n, A, lda);
  for (;;) {
    if (off <= tol) break;
    if (sweeps >= max_sweeps) {
      capped = 1;
      break;
    }
    int done_rot = 0;
    if (ordering == ORC_CYCLIC) {
      for (int p = 0; p < n - 1; ++p)
        for (int q = p + 1; q < n; ++q) {
          float apq = AT(A, lda, p, q);
          if (fabsf(apq) > skip_tol * sqrtf(fabsf(AT(A, lda, p, p) * AT(A, lda, q, q)))) {
            float c, s;
            orc_jacobi_pair_f(AT(A, lda, p, p), AT(A, lda, q, q), apq, &c, &s);
            c = rq(c, half);
            s = rq(s, half);
            rotate_f(n, A, lda, V, ldv, p, q, c, s, half);
            done_rot = 1;
            ++rot;
          }
        }
    } else if (ordering == ORC_BLOCK_RR) {
      int nb = block_nb(n);
      for (int R = 0; R < nb - 1; ++R)
        for (int P = 0; P < nb / 2; ++P)
          for (int rho = 0; rho < 2 * ORC_BLK - 1; ++rho)
            for (int i = 0; i < ORC_BLK; ++i) {
              int p, q;
              if (!orc_block_pair(n, R, P, rho, i, &p, &q)) continue;
              float apq = AT(A, lda, p, q);
              if (fabsf(apq) > skip_tol * sqrtf(fabsf(AT(A, lda, p, p) * AT(A, lda, q, q)))) {
                float c, s;
                orc_jacobi_pair_f(AT(A, lda, p, p), AT(A, lda, q, q), apq, &c, &s);
            c = rq(c, half);
            s = rq(s, half);
                rotate_f(n, A, lda, V, ldv, p, q, c, s, half);
                done_rot = 1;
                ++rot;
              }
            }
    } else {
      for (int r = 0; r < m - 1; ++r)
        for (int i = 0; i < m / 2; ++i) {
          int p, q;
          if (!rr_pair(n, r, i, &p, &q)) continue;
          float apq = AT(A, lda, p, q);
          if (fabsf(apq) > skip_tol * sqrtf(fabsf(AT(A, lda, p, p) * AT(A, lda, q, q)))) {
            float c, s;
            orc_jacobi_pair_f(AT(A, lda, p, p), AT(A, lda, q, q), apq, &c, &s);
            c = rq(c, half);
            s = rq(s, half);
            rotate_f(n, A, lda, V, ldv, p, q, c, s, half);
            done_rot = 1;
            ++rot;
          }
        }
    }
    ++sweeps;
    if (!done_rot) {
      off = orc_off_f(n, A, lda);
      break;
    }
    symmetrize_f(n, A, lda, half);
    off = orc_off_f(n, A, lda);
  }
  *sweeps_out = sweeps;
  if (rotations_out) *rotations_out = rot;
  if (off_out) *off_out = off;
  return capped;
}

/* ------------------------------------------------------------------------ */
/* Plain matrix products; the sum over k runs in ascending k for every entry. */

/* C = A^T B, A is k x m, B is k x n, C is m x n. */
void orc_gemm_tn_d(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += AT(A, lda, l, i) * AT(B, ldb, l, j);
      AT(C, ldc, i, j) = s;
    }
}

/* C = A B, A is m x k, B is k x n, C is m x n.  Accumulated column by column
 * (axpy form); for each entry the terms are still added in ascending k.     */
void orc_gemm_nn_d(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < m; ++i) AT(C, ldc, i, j) = 0.0;
    for (int l = 0; l < k; ++l) {
      double b = AT(B, ldb, l, j);
      for (int i = 0; i < m; ++i) AT(C, ldc, i, j) += AT(A, lda, i, l) * b;
    }
  }
}

/* C = A B^T, A is m x k, B is n x k. */
void orc_gemm_nt_d(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < m; ++i) AT(C, ldc, i, j) = 0.0;
    for (int l = 0; l < k; ++l) {
      double b = AT(B, ldb, j, l);
      for (int i = 0; i < m; ++i) AT(C, ldc, i, j) += AT(A, lda, i, l) * b;
    }
  }
}

/* Newton-Schulz, the iteration of Sec. 4.3.4 and Algorithm 8: X_{k+1} = 1/2 X_k (3I - X_k^T X_k),
 * `steps` times (the paper's newton_schulz uses 2 steps for n < 52000, else 3).
 * Evaluated literally: M = X^T X, B = 3I - M, Y = X B, X = Y / 2.              */
void orc_newton_schulz_d(int n, double* X, int ldx, int steps) {
  double* M = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* Y = (double*)malloc(sizeof(double) * (size_t)n * n);
  for (int it = 0; it < steps; ++it) {
    orc_gemm_tn_d(n, n, n, X, ldx, X, ldx, M, n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) AT(M, n, i, j) = (i == j ? 3.0 : 0.0) - AT(M, n, i, j);
    orc_gemm_nn_d(n, n, n, X, ldx, M, n, Y, n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) AT(X, ldx, i, j) = 0.5 * AT(Y, n, i, j);
  }
  free(M);
  free(Y);
}

/* Preconditioning, Algorithm 9 (Sec. 5.1) step 3: A_cond = Q_d^T A Q_d, as Q_d^T (A Q_d). */
void orc_precondition_d(int n, const double* A, int lda, const double* Qd, int ldq, double* Ac, int ldc) {
  double* W = (double*)malloc(sizeof(double) * (size_t)n * n);
  orc_gemm_nn_d(n, n, n, A, lda, Qd, ldq, W, n);
  orc_gemm_tn_d(n, n, n, Qd, ldq, W, n, Ac, ldc);
  free(W);
}

/* ------------------------------------------------------------------------ */
typedef struct {
  double tol;       /* FP64 stop: off(A) <= tol; <= 0 selects n 2^-53 ||A||_F  */
  double tol32;     /* FP32 stop: off(A32) <= tol32; <= 0 selects n 2^-24 ||A||_F */
  double skip_tol;  /* FP64 per-pair test, <= 0 selects 2^-53                   */
  double skip_tol32;/* FP32 per-pair test, <= 0 selects 2^-24                   */
  int max_sweeps64; /* <= 0 selects 30 */
  int max_sweeps32; /* <= 0 selects 15 */
  int ns_steps;     /* <= 0 selects 2 for n < 52000, else 3                      */
  int ordering32;   /* ORC_CYCLIC or ORC_ROUND_ROBIN */
  int ordering64;
  int polish;       /* 1: one more Newton-Schulz step on the final Q             */
  int sort;         /* 1: sort W ascending, permute Q's columns to match        */
  int threshold;    /* 1: FP64 sweeps also skip pairs with |a_pq| <= tol / n     */
  int precond_passes; /* 2: Algorithm 9's stages 1-3 applied a second time to
                         A_cond before the FP64 sweeps (not in the paper)        */
  int stage1_half;    /* 1: stage 1 in half precision (binary16, u = 2^-11)      */
} orc_opts;

typedef struct {
  int sweeps32, sweeps64, capped32, capped64;
  long long rotations32, rotations64;
  double normA_fro, off32, off_cond, off_final;
  int sweeps32_pass2;
  int ns_steps;     /* Newton-Schulz steps applied                                   */
  double ns_e0;     /* ||Q_l^T Q_l - I||_2 before Newton-Schulz (power estimate)     */
} orc_info;

/* Newton-Schulz steps for a low-precision Q_l with unit roundoff ul: the paper
 * bounds ||X_k - U|| by (sqrt(1 + n ul) - 1)^(2^k) (Sec. 4.3.4, the analysis
 * behind Algorithm 8) and stops once that is at most n u_d.  For single
 * precision the paper's code uses 2 steps below n = 52000 and 3 above; for
 * half precision (ul = 2^-11) the same bound is evaluated here.            */
int orc_ns_steps(int n, int half) {
  if (!half) return n < 52000 ? 2 : 3;
  const double ud = ldexp(1.0, -53), ul = ldexp(1.0, -11);
  const double e0 = sqrt(1.0 + (double)n * ul) - 1.0;
  double e = e0;
  int k = 0;
  while (e > (double)n * ud && k < 8) {
    e = e * e;
    ++k;
  }
  return k < 1 ? 1 : k;
}

static void sort_eig(int n, double* W, double* Q, int ldq) {
  /* insertion sort on (value, index): ascending, ties by original index */
  int* idx = (int*)malloc(sizeof(int) * (size_t)n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 1; i < n; ++i) {
    int v = idx[i];
    int j = i - 1;
    while (j >= 0 && (W[idx[j]] > W[v])) {
      idx[j + 1] = idx[j];
      --j;
    }
    idx[j + 1] = v;
  }
  double* W2 = (double*)malloc(sizeof(double) * (size_t)n);
  double* Q2 = (double*)malloc(sizeof(double) * (size_t)n * n);
  for (int j = 0; j < n; ++j) {
    W2[j] = W[idx[j]];
    for (int i = 0; i < n; ++i) AT(Q2, n, i, j) = AT(Q, ldq, i, idx[j]);
  }
  for (int j = 0; j < n; ++j) {
    W[j] = W2[j];
    for (int i = 0; i < n; ++i) AT(Q, ldq, i, j) = AT(Q2, n, i, j);
  }
  free(idx);
  free(W2);
  free(Q2);
}

static void defaults(int n, double normA, const orc_opts* o, orc_opts* r) {
  *r = *o;
  const int lowbits = r->stage1_half ? 11 : 24;  /* unit roundoff 2^-11 or 2^-24 */
  if (r->tol <= 0) r->tol = (double)n * ldexp(1.0, -53) * normA;
  if (r->tol32 <= 0) r->tol32 = (double)n * ldexp(1.0, -lowbits) * normA;
  if (r->skip_tol <= 0) r->skip_tol = ldexp(1.0, -53);
  if (r->skip_tol32 <= 0) r->skip_tol32 = ldexp(1.0, -lowbits);
  if (r->max_sweeps64 <= 0) r->max_sweeps64 = 30;
  if (r->max_sweeps32 <= 0) r->max_sweeps32 = 15;
  if (r->ns_steps <= 0) r->ns_steps = orc_ns_steps(n, r->stage1_half);
}

/* Stage 1 alone: A32 = fl32(A), FP32 Jacobi from V32 = I, Q_l = double(V32).
 * A32out (n x n float, may be NULL) receives the final FP32 matrix.        */
int orc_stage1(int n, const double* A, int lda, double* Ql, int ldq, const orc_opts* o, orc_info* info,
               float* A32out) {
  orc_opts d;
  double normA = orc_fro_d(n, A, lda);
  defaults(n, normA, o, &d);
  float* A32 = (float*)malloc(sizeof(float) * (size_t)n * n);
  float* V32 = (float*)malloc(sizeof(float) * (size_t)n * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      AT(A32, n, i, j) = rq((float)AT(A, lda, i, j), d.stage1_half);
      AT(V32, n, i, j) = (i == j) ? 1.0f : 0.0f;
    }
  int capped = d.stage1_half
                   ? orc_jacobi_h(n, A32, n, V32, n, d.ordering32, d.tol32, (float)d.skip_tol32, d.max_sweeps32,
                                  &info->sweeps32, &info->rotations32, &info->off32)
                   : orc_jacobi_f(n, A32, n, V32, n, d.ordering32, d.tol32, (float)d.skip_tol32, d.max_sweeps32,
                                  &info->sweeps32, &info->rotations32, &info->off32);
  info->capped32 = capped;
  info->normA_fro = normA;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) AT(Ql, ldq, i, j) = (double)AT(V32, n, i, j);
  if (A32out) memcpy(A32out, A32, sizeof(float) * (size_t)n * n);
  free(A32);
  free(V32);
  return capped;
}

/* Algorithm 9 (jacobi_precondi) with an FP32 Jacobi as its stage 1:
 *   1. Q_l from stage 1;  2. Q_d = newton_schulz(Q_l);
 *   3. A_cond = Q_d^T A Q_d;  4. FP64 Jacobi on A_cond from V = I;
 *   5. W = diag(A_cond after the sweeps), Q = Q_d V  (optionally polished, sorted).
 * Intermediates (each n x n, may be NULL): Ql_out, Qd_out, Acond_out (with
 * two passes: Q_d = Q_d1 Q_d2 and the second A_cond).  Returns 2 (and no
 * results) when Q_l violates the Newton-Schulz premise.
 * Returns 0, or 1 when the FP64 stage hit its sweep cap.                     */
int orc_syev_mixed(int n, const double* A, int lda, double* W, double* Q, int ldq, const orc_opts* o, orc_info* info,
                   double* Ql_out, double* Qd_out, double* Acond_out) {
  orc_opts d;
  double normA = orc_fro_d(n, A, lda);
  defaults(n, normA, o, &d);
  memset(info, 0, sizeof(*info));
  double* X = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* Ac = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* V = (double*)malloc(sizeof(double) * (size_t)n * n);
  orc_stage1(n, A, lda, X, n, &d, info, NULL);
  if (Ql_out) memcpy(Ql_out, X, sizeof(double) * (size_t)n * n);
  /* The Newton-Schulz iteration converges when the singular values of Q_l lie
   * in (0, sqrt(3)) (Sec. 4.3.4), i.e. ||Q_l^T Q_l - I||_2 < 2.  The 2-norm of
   * the symmetric E = Q_l^T Q_l - I is its largest |eigenvalue|, estimated by
   * 200 steps of the power iteration. */
  {
    double* E = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double g = (i == j) ? -1.0 : 0.0;
        for (int k = 0; k < n; ++k) g += AT(X, n, k, i) * AT(X, n, k, j);
        AT(E, n, i, j) = g;
      }
    for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.5 * sin((double)i);
    double lam = 0.0;
    for (int it = 0; it < 200; ++it) {
      double nx = 0.0, ny = 0.0;
      for (int i = 0; i < n; ++i) nx += x[i] * x[i];
      nx = sqrt(nx);
      if (nx == 0.0) { /* E x = 0 exactly: the estimate is 0 */
        lam = 0.0;
        break;
      }
      for (int i = 0; i < n; ++i) {
        double t = 0.0;
        for (int j = 0; j < n; ++j) t += AT(E, n, i, j) * x[j];
        y[i] = t / nx;
        ny += y[i] * y[i];
      }
      lam = sqrt(ny);
      for (int i = 0; i < n; ++i) x[i] = y[i];
    }
    info->ns_e0 = lam;
    free(E);
    free(x);
    free(y);
  }
  info->ns_steps = d.ns_steps;
  if (!(info->ns_e0 < 2.0)) {
    free(X);
    free(Ac);
    free(V);
    return 2;
  }
  orc_newton_schulz_d(n, X, n, d.ns_steps);
  orc_precondition_d(n, A, lda, X, n, Ac, n);
  if (d.precond_passes >= 2) {
    /* Second pass (not in the paper): stages 1-3 once more, on A_cond.  Its
     * FP32 rounding is relative to A_cond's own entries, so the FP32 Jacobi
     * separates eigenvalues that stage 1 on A could not.  Reading: stage 1 of
     * this pass stops at off(A32) <= n 2^-24 off(A_cond) or after
     * min(max_sweeps32, 9) sweeps; Q_d = Q_d1 Q_d2 and
     * A_cond <- Q_d2^T A_cond Q_d2.                                          */
    orc_opts d2 = d;
    orc_info i2;
    memset(&i2, 0, sizeof i2);
    d2.tol32 = (double)n * ldexp(1.0, -24) * orc_off_d(n, Ac, n);
    d2.max_sweeps32 = d.max_sweeps32 < 9 ? d.max_sweeps32 : 9;
    d2.stage1_half = 0; /* the second pass runs in single precision */
    d2.skip_tol32 = ldexp(1.0, -24);
    double* X2 = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* T = (double*)malloc(sizeof(double) * (size_t)n * n);
    orc_stage1(n, Ac, n, X2, n, &d2, &i2, NULL);
    info->sweeps32_pass2 = i2.sweeps32;
    orc_newton_schulz_d(n, X2, n, d.ns_steps);
    orc_precondition_d(n, Ac, n, X2, n, T, n);
    memcpy(Ac, T, sizeof(double) * (size_t)n * n);
    orc_gemm_nn_d(n, n, n, X, n, X2, n, T, n);
    memcpy(X, T, sizeof(double) * (size_t)n * n);
    free(X2);
    free(T);
  }
  if (Qd_out) memcpy(Qd_out, X, sizeof(double) * (size_t)n * n);
  if (Acond_out) memcpy(Acond_out, Ac, sizeof(double) * (size_t)n * n);
  info->off_cond = orc_off_d(n, Ac, n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) AT(V, n, i, j) = (i == j) ? 1.0 : 0.0;
  int capped = orc_jacobi_d(n, Ac, n, V, n, d.ordering64, d.tol, d.skip_tol, d.max_sweeps64, 0, &info->sweeps64,
                            &info->rotations64, &info->off_final, d.threshold ? d.tol / n : 0.0);
  info->capped64 = capped;
  for (int j = 0; j < n; ++j) W[j] = AT(Ac, n, j, j);
  orc_gemm_nn_d(n, n, n, X, n, V, n, Q, ldq);
  if (d.polish) orc_newton_schulz_d(n, Q, ldq, 1);
  if (d.sort) sort_eig(n, W, Q, ldq);
  free(X);
  free(Ac);
  free(V);
  return capped;
}

/* Plain FP64 Jacobi from V = I on A itself (the metric's denominator, the
 * paper's jacobi_eig(A, tol, 'Cyclic') of the timing experiment).         */
int orc_syev_plain(int n, const double* A, int lda, double* W, double* Q, int ldq, const orc_opts* o, orc_info* info) {
  orc_opts d;
  double normA = orc_fro_d(n, A, lda);
  defaults(n, normA, o, &d);
  memset(info, 0, sizeof(*info));
  info->normA_fro = normA;
  double* Ac = (double*)malloc(sizeof(double) * (size_t)n * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      AT(Ac, n, i, j) = AT(A, lda, i, j);
      AT(Q, ldq, i, j) = (i == j) ? 1.0 : 0.0;
    }
  info->off_cond = orc_off_d(n, Ac, n);
  int capped = orc_jacobi_d(n, Ac, n, Q, ldq, d.ordering64, d.tol, d.skip_tol, d.max_sweeps64, 0, &info->sweeps64,
                            &info->rotations64, &info->off_final, d.threshold ? d.tol / n : 0.0);
  info->capped64 = capped;
  for (int j = 0; j < n; ++j) W[j] = AT(Ac, n, j, j);
  if (d.polish) orc_newton_schulz_d(n, Q, ldq, 1);
  if (d.sort) sort_eig(n, W, Q, ldq);
  free(Ac);
  return capped;
}

/* Eigen-adjoint (not in the paper; the standard first-order eigenvector
 * perturbation result, e.g. Giles 2008, "Collected matrix derivative
 * results"): with M = Q^T dQ, G_ii = dW_i, G_ij = M_ij / (w_j - w_i) (i != j),
 * dA = Q G Q^T, returned symmetrized as (dA + dA^T)/2.  dW or dQ NULL means 0.
 * Returns -1 if some w_i == w_j (i != j) with a nonzero M_ij, else 0.       */
int orc_eigh_backward(int n, const double* W, const double* Q, int ldq, const double* dW, const double* dQ, int lddq,
                      double* dA, int ldda) {
  double* M = (double*)calloc((size_t)n * n, sizeof(double));
  double* T = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* R = (double*)malloc(sizeof(double) * (size_t)n * n);
  int rc = 0;
  if (dQ) orc_gemm_tn_d(n, n, n, Q, ldq, dQ, lddq, M, n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double g;
      if (i == j) {
        g = dW ? dW[i] : 0.0;
      } else {
        double gap = W[j] - W[i];
        if (gap == 0.0) {
          if (AT(M, n, i, j) != 0.0) rc = -1;
          g = 0.0;
        } else {
          g = AT(M, n, i, j) / gap;
        }
      }
      AT(M, n, i, j) = g;
    }
  orc_gemm_nn_d(n, n, n, Q, ldq, M, n, T, n);  /* T = Q G   */
  orc_gemm_nt_d(n, n, n, T, n, Q, ldq, R, n);  /* R = T Q^T */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) AT(dA, ldda, i, j) = (AT(R, n, i, j) + AT(R, n, j, i)) / 2.0;
  free(M);
  free(T);
  free(R);
  return rc;
}
