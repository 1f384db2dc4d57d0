// stage1.cu -- stage 1 of the mixed algorithm: approximate eigenvectors Q_l
// from an FP32 Jacobi (the paper's stage 1 is eig(single(A)), Sec. 4.1 and
// Algorithm 9; only an approximate Q_l with ||A Q_l - Q_l D_l|| <~ n u_l ||A||
// is needed, so the FP32 stage may use any convergent Jacobi ordering).
//
// Ordering: block round-robin.  The padded index range [0, N) (N a multiple
// of 32, pads inert: zero rows/columns never rotate) is cut into nb = N/16
// blocks of 16.  A sweep is nb-1 outer rounds of the circle method on blocks;
// in each round the nb/2 disjoint block pairs (I, J) each run one inner
// round-robin sweep over the 32 indices of I u J (31 inner rounds of 16
// disjoint pairs, Algorithm 2 with the skip test of Algorithm 4 at u_l = 2^-24)
// on their 32 x 32 diagonal subproblem, held in shared memory, accumulating the
// 32 x 32 orthogonal U_IJ.  The rotations of one round touch disjoint index
// sets, so applying them to the rest of the matrix afterwards as products
//   A[P,Q] <- U_P^T A[P,Q] U_Q,   V[:,Q] <- V[:,Q] U_Q
// (P, Q = index sets of block pairs) gives the same iterates as applying them
// one by one.  Each round is the subproblem solves and two block products
// (FP32 FMA, rmul32): V <- V U~ and A <- U~^T A U~ (the lower tiles, each
// formed once and mirrored), so that A32 and V32 are touched once per round
// instead of once per pair step.  off(A32) is reduced after each sweep; stop
// at off(A32) <= tol32 or the sweep cap.
#include <memory>
#include <mutex>
#include <vector>
#include <cuda_fp16.h>
#include <stdlib.h>

#include "common.cuh"
#include "stage1.cuh"
#include "tc32.cuh"

namespace {

constexpr int BS = 16;  // block size
constexpr int W2 = 32;  // indices per block pair
constexpr int LD = 33;  // padded shared-memory leading dimension

// global index of local index l in block pair (I, J)
MPJ_DEV int gidx(int I, int J, int l) { return l < BS ? I * BS + l : J * BS + (l - BS); }

MPJ_DEV void block_pair(int nb, int R, int slot, int& I, int& J) {
  int x, y;
  rr_slot(nb, R, slot, x, y);
  I = x < y ? x : y;
  J = x < y ? y : x;
}

// hq: the half-precision stage (binary16 values; Ch. 6 further work item 3):
// every stored value and rotation parameter is rounded to binary16.
MPJ_DEV float qh(float v, bool hq) { return hq ? __half2float(__float2half_rn(v)) : v; }

__global__ void init32(const double* __restrict__ A, int lda, int n, int N, float* __restrict__ A32,
                       float* __restrict__ V32, bool hq) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)N * N;
  for (; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % N), j = (int)(idx / N);
    A32[idx] = (i < n && j < n) ? qh((float)A[(size_t)j * lda + i], hq) : 0.0f;
    V32[idx] = (i == j) ? 1.0f : 0.0f;
  }
}

__global__ void widen(const float* __restrict__ V32, int N, int n, double* __restrict__ Q, int ldq) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)n * n;
  for (; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    Q[(size_t)j * ldq + i] = (double)V32[(size_t)j * N + i];
  }
}

// The record of slot (x, y) (x the slot's first index) for the FP32 inner
// sweep: Algorithm 2 with the skip test of Algorithm 4 (compared in squares),
// t in the stable form, c = 1 / sqrt(1 + t^2) by rsqrtf, c - 1 = -t^2 c / (1 + h)
// with h = 1 / c = (1 + t^2) c; the new diagonal a_pp - t a_pq, a_qq + t a_pq.
MPJ_DEV void rec32(int x, int y, float dxx, float dyy, float axy, float skip, RotRec<float>& rr) {
  const bool xp = x < y;
  const float app = xp ? dxx : dyy, aqq = xp ? dyy : dxx;
  rr.cm1 = 0.0f;
  rr.sig = 0.0f;
  rr.dx = dxx;
  rr.dy = dyy;
  if (!(axy * axy > (skip * skip) * fabsf(app * aqq)) || y >= W2 || x >= W2) return;
  const float tau = (aqq - app) / (2.0f * axy);
  const float r = sqrtf(fmaf(tau, tau, 1.0f));
  const float t = (tau >= 0.0f) ? 1.0f / (tau + r) : 1.0f / (tau - r);
  const float w = fmaf(t, t, 1.0f);
  const float c = rsqrtf(w);
  const float h = w * c;
  const float s = t * c;
  rr.cm1 = -(t * t) * c / (1.0f + h);
  rr.sig = xp ? s : -s;
  const float np = app - t * axy, nq = aqq + t * axy;
  rr.dx = xp ? np : nq;
  rr.dy = xp ? nq : np;
}

// One CTA per block pair of outer round R: inner round-robin sweep on the
// 32 x 32 subproblem; writes the rotated subproblem S (column-major), the
// accumulated U (row-major for the FP32 products, column-major, urow false,
// for the tensor-core panel) and the set T of its indices that rotated
// (Mbuf, bit l for local index l, if not null): U is the identity outside
// T x T.
constexpr int S32_THREADS = 512;
__global__ void __launch_bounds__(S32_THREADS) solve32(const float* __restrict__ A32, int N, int nb, int R,
                                               float* __restrict__ Sbuf, float* __restrict__ Ubuf, bool hq,
                                               bool urow, unsigned* __restrict__ Mbuf) {
  __shared__ float S[W2][LD];
  __shared__ float U[W2][LD];
  __shared__ RotRec<float> rec[W2 / 2];
  const int slot = blockIdx.x;
  int I, J;
  block_pair(nb, R, slot, I, J);
  const int tid = threadIdx.x;
  pdl_wait();
  #pragma unroll
  for (int it = 0; it < W2 * W2 / S32_THREADS; ++it) {
    const int e = tid + it * S32_THREADS;
    int li = e % W2, lj = e / W2;
    S[li][lj] = A32[(size_t)gidx(I, J, lj) * N + gidx(I, J, li)];
    U[li][lj] = (li == lj) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const float skip = hq ? 0x1p-11f : 0x1p-24f;
  unsigned tmask = 0u;  // thread 0: the indices that rotated so far
  for (int rho = 0; rho < W2 - 1; ++rho) {
    if (tid < W2 / 2) {
      int x, y;
      rr_slot(W2, rho, tid, x, y);
      RotRec<float> rr;
      rec32(x, y, S[x][x], S[y][y], S[y][x], skip, rr);
      if (hq && rec_rotated(rr.cm1, rr.sig)) {  // c and s as binary16, new diagonal rounded
        rr.cm1 = qh(1.0f + rr.cm1, true) - 1.0f;
        rr.sig = qh(rr.sig, true);
        rr.dx = qh(rr.dx, true);
        rr.dy = qh(rr.dy, true);
      }
      rec[tid] = rr;
      if (Mbuf) {
        const unsigned bits = rec_rotated(rr.cm1, rr.sig) ? ((1u << x) | (1u << y)) : 0u;
        tmask |= __reduce_or_sync(0x0000FFFFu, bits);  // the 16 record lanes of warp 0
      }
    }
    __syncthreads();
    {
      int a = tid % 16, b = tid / 16;
      if (b < 16 && a >= b) {
        int xa, ya, xb, yb;
        rr_slot(W2, rho, a, xa, ya);
        rr_slot(W2, rho, b, xb, yb);
        RotRec<float> ra = rec[a], rb = rec[b];
        bool rota = rec_rotated(ra.cm1, ra.sig), rotb = rec_rotated(rb.cm1, rb.sig);
        if (a == b) {
          if (rota) {
            S[xa][xa] = ra.dx;
            S[ya][ya] = ra.dy;
            S[xa][ya] = 0.0f;
            S[ya][xa] = 0.0f;
          }
        } else if (rota || rotb) {
          float vxx = S[xa][xb], vxy = S[xa][yb], vyx = S[ya][xb], vyy = S[ya][yb];
          if (rota) {
            rot_apply(ra.cm1, ra.sig, vxx, vyx);
            rot_apply(ra.cm1, ra.sig, vxy, vyy);
          }
          if (rotb) {
            rot_apply(rb.cm1, rb.sig, vxx, vxy);
            rot_apply(rb.cm1, rb.sig, vyx, vyy);
          }
          vxx = qh(vxx, hq);
          vxy = qh(vxy, hq);
          vyx = qh(vyx, hq);
          vyy = qh(vyy, hq);
          S[xa][xb] = vxx;
          S[xb][xa] = vxx;
          S[xa][yb] = vxy;
          S[yb][xa] = vxy;
          S[ya][xb] = vyx;
          S[xb][ya] = vyx;
          S[ya][yb] = vyy;
          S[yb][ya] = vyy;
        }
      }
      // U <- U J: rows of U are independent; columns x_b, y_b
      for (int e = tid; e < W2 * (W2 / 2); e += S32_THREADS) {
        int row = e % W2, sb = e / W2;
        RotRec<float> rb = rec[sb];
        if (!rec_rotated(rb.cm1, rb.sig)) continue;
        int xb, yb;
        rr_slot(W2, rho, sb, xb, yb);
        float ux = U[row][xb], uy = U[row][yb];
        rot_apply(rb.cm1, rb.sig, ux, uy);
        U[row][xb] = qh(ux, hq);
        U[row][yb] = qh(uy, hq);
      }
    }
    __syncthreads();
  }
  float* So = Sbuf + (size_t)slot * W2 * W2;
  float* Uo = Ubuf + (size_t)slot * W2 * W2;
  #pragma unroll
  for (int it = 0; it < W2 * W2 / S32_THREADS; ++it) {
    const int e = tid + it * S32_THREADS;
    int li = e % W2, lj = e / W2;
    So[e] = S[li][lj];
    Uo[e] = urow ? U[lj][li] : U[li][lj];
  }
  if (tid == 0 && Mbuf) Mbuf[slot] = tmask;
}


// Packed pairs of FP32 values (low word first) and the paired FMA
// d = a * b + d, each half rounded to nearest like fmaf.
MPJ_DEV unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
MPJ_DEV void unpk2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
MPJ_DEV void fma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// ---------------------------------------------------------------- block update
enum { R32_ALL = 0, R32_BOTH = 1 };
constexpr int RT = 128;
constexpr int XLD = 132;  // padded row length of the X tile (k-major), 16-byte aligned rows
constexpr int ULD = 40;   // padded row length of U_Q, 16-byte aligned rows

// The 32 x 32 product of one warp: acc(4 g + i, 8 h + j) = sum_k L(k, 4 g + i) R(k, 8 h + j)
// for lane (g, h) = (lane mod 8, lane / 8), L and R k-major in shared memory
// (row stride LDL, LDR floats); packed FP32 pairs, each half rounded as fmaf.
template <int LDL, int LDR>
MPJ_DEV void warp_mm32(const float* L, const float* R, int g, int h, float acc[4][8]) {
  unsigned long long acc2[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jp = 0; jp < 4; ++jp) acc2[i][jp] = 0ULL;
#pragma unroll 4
  for (int k = 0; k < W2; ++k) {
    const float4 x = *reinterpret_cast<const float4*>(L + k * LDL + 4 * g);
    const float4 u0 = *reinterpret_cast<const float4*>(R + k * LDR + 8 * h);
    const float4 u1 = *reinterpret_cast<const float4*>(R + k * LDR + 8 * h + 4);
    const float xa[4] = {x.x, x.y, x.z, x.w};
    const unsigned long long up[4] = {pk2(u0.x, u0.y), pk2(u0.z, u0.w), pk2(u1.x, u1.y), pk2(u1.z, u1.w)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const unsigned long long xx = pk2(xa[i], xa[i]);
#pragma unroll
      for (int jp = 0; jp < 4; ++jp) fma2(acc2[i][jp], xx, up[jp]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jp = 0; jp < 4; ++jp) unpk2(acc2[i][jp], acc[i][2 * jp], acc[i][2 * jp + 1]);
}

// warp_mm32 with the contraction restricted to the indices k in `mask` (in
// increasing order: the terms it leaves out are exact zeros, so the sums
// are those of the full contraction).
template <int LDL, int LDR>
MPJ_DEV void warp_mm32_masked(const float* L, const float* R, int g, int h, unsigned mask, float acc[4][8]) {
  unsigned long long acc2[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jp = 0; jp < 4; ++jp) acc2[i][jp] = 0ULL;
  for (unsigned m = mask; m; m &= m - 1) {
    const int k = __ffs(m) - 1;
    const float4 x = *reinterpret_cast<const float4*>(L + k * LDL + 4 * g);
    const float4 u0 = *reinterpret_cast<const float4*>(R + k * LDR + 8 * h);
    const float4 u1 = *reinterpret_cast<const float4*>(R + k * LDR + 8 * h + 4);
    const float xa[4] = {x.x, x.y, x.z, x.w};
    const unsigned long long up[4] = {pk2(u0.x, u0.y), pk2(u0.z, u0.w), pk2(u1.x, u1.y), pk2(u1.z, u1.w)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const unsigned long long xx = pk2(xa[i], xa[i]);
#pragma unroll
      for (int jp = 0; jp < 4; ++jp) fma2(acc2[i][jp], xx, up[jp]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jp = 0; jp < 4; ++jp) unpk2(acc2[i][jp], acc[i][2 * jp], acc[i][2 * jp + 1]);
}

// U(k, c) of block pair P (32 x 32 in Ubuf, row-major, or column-major when
// ucol) into Us[k][c]
MPJ_DEV void load_u(const float* __restrict__ Ubuf, int P, float (*Us)[ULD], int t, int nt, bool ucol) {
  const float* Uq = Ubuf + (size_t)P * W2 * W2;
  for (int e = 4 * t; e < W2 * W2; e += 4 * nt) {
    const float4 v = *reinterpret_cast<const float4*>(Uq + e);
    if (!ucol) {
      *reinterpret_cast<float4*>(&Us[e / W2][e % W2]) = v;
    } else {
      const int k = e % W2, c = e / W2;
      Us[k][c] = v.x;
      Us[k + 1][c] = v.y;
      Us[k + 2][c] = v.z;
      Us[k + 3][c] = v.w;
    }
  }
}

// The round's rotations applied to the rest of A32 and to V32 as block-diagonal
// right multiplications Y[:, g_Q(c)] = X_Q U_Q (FP32 FMA, K = 32) over tiles
// (a, Q): block pair Q and the 128 rows that are the 32 indices of each of
// the block pairs a = 4 gx .. 4 gx + 3.  Modes:
//   R32_ALL    V <- V U~ (every tile, in place);
//   R32_BOTH   A <- U~^T A U~ in one pass, in place: tile (a, Q), a > Q, gets
//              U_a^T (A[P_a, Q] U_Q) (the second product on the first one's
//              result in shared memory), written to both triangles; the
//              diagonal tiles a = Q are the solved subproblems S.  The tiles
//              read (a > Q) are only those their own CTA writes, the mirrors
//              (Q, a) are read by no CTA.
// 128 threads: the tile's 128 x 32 values of X_Q and U_Q in shared memory,
// then warp w forms the 32 x 32 block of tile rows 32 w .. +31 (block pair
// a0 + w) and lane (g, h) = (t mod 8, t / 8 mod 4) the 4 x 8 block of rows
// 32 w + 4 g .. +3 and columns 8 h .. +7: per k one float4 of X (8 distinct
// in a warp: one shared-memory wavefront) and two float4 of U_Q (4 distinct:
// one wavefront each) feed 32 FMAs.
template <int TRI, bool MASKED>
__global__ void __launch_bounds__(RT) rmul32(const float* X, float* Y, int N, int nb, int R,
                                             const float* __restrict__ Sbuf, const float* __restrict__ Ubuf, bool hq,
                                             bool ucol, const unsigned* __restrict__ Mbuf) {
  __shared__ __align__(16) float Xs[W2][XLD];  // Xs[k][r] = X_Q(r, k); R32_BOTH: then T = X_Q U_Q per warp
  __shared__ __align__(16) float Us[W2][ULD];  // Us[k][c] = U_Q(k, c)
  __shared__ __align__(16) float Ua[TRI == R32_BOTH ? 4 : 1][W2][ULD];  // U_a of each warp's pair
  const int tid = threadIdx.x;
  const int Q = blockIdx.y, gx = blockIdx.x, npairs = nb / 2;
  const int a0 = 4 * gx, a1 = min(4 * gx + 3, npairs - 1);
  pdl_wait();
  if (TRI == R32_BOTH && a1 < Q) return;
  const int warp = tid >> 5, lane = tid & 31;
  const int a = a0 + warp;  // this warp's block pair
  // the indices of block pairs Q and a that rotated (U is the identity
  // outside them); loaded together with the U blocks, used after them
  const unsigned mQ = MASKED ? Mbuf[Q] : 0xFFFFFFFFu;
  const unsigned ma = !MASKED ? 0xFFFFFFFFu : (TRI == R32_BOTH && a < npairs) ? Mbuf[a] : 0u;
  int IQ, JQ;
  block_pair(nb, R, Q, IQ, JQ);
  load_u(Ubuf, Q, Us, tid, RT, ucol);
  if (TRI == R32_BOTH && a < npairs && a > Q) load_u(Ubuf, a, Ua[warp], lane, 32, ucol);
  if (TRI == R32_ALL && mQ == 0u) return;  // V U~ leaves these columns as they are
  {
    // X_Q(r, k) = X[g_Q(k) N + row(r)]; thread t: tile rows 4 (t mod 32) .. +3
    // (consecutive rows of one block), contraction indices k = t / 32 + 4 i
    const int rq = tid & 31, ar = a0 + (rq >> 3);
    int row = -1;
    if (ar < npairs && (TRI != R32_BOTH || ar > Q)) {
      int I, J;
      block_pair(nb, R, ar, I, J);
      row = gidx(I, J, (4 * rq) & 31);
    }
#pragma unroll
    for (int i = 0; i < W2 / 4; ++i) {
      const int k = (tid >> 5) + 4 * i;
      if (TRI == R32_ALL && !((mQ >> k) & 1u)) continue;  // column not read (V U~ contracts over T_Q only)
      const float4 v = row >= 0 ? *reinterpret_cast<const float4*>(X + (size_t)gidx(IQ, JQ, k) * N + row)
                                : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      *reinterpret_cast<float4*>(&Xs[k][4 * rq]) = v;
    }
  }
  __syncthreads();
  const int g = lane & 7, h = lane >> 3;
  const int c0 = 8 * h;
  if (a >= npairs) return;
  if (TRI == R32_BOTH && a < Q) return;
  int I, J;
  block_pair(nb, R, a, I, J);
  const int row0 = gidx(I, J, 4 * g);  // rows row0 .. row0 + 3 (one block)
  const int col0 = gidx(IQ, JQ, c0);   // columns col0 .. col0 + 7 (one block)
  if (TRI == R32_BOTH && a == Q) {
    // the diagonal tile: the solved subproblem
    const float* Sq = Sbuf + (size_t)Q * W2 * W2;
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const float4 o = *reinterpret_cast<const float4*>(Sq + 4 * g + W2 * (c0 + cc));
      *reinterpret_cast<float4*>(Y + (size_t)(col0 + cc) * N + row0) = o;
    }
    return;
  }
  if (TRI == R32_BOTH && mQ == 0u && ma == 0u) return;  // U_a^T A U_Q = A on this tile
  // a column c outside T_Q: (X U_Q)(:, c) = X(:, c); else the contraction over T_Q
  float acc[4][8];
  if (mQ == 0xFFFFFFFFu) {
    warp_mm32<XLD, ULD>(&Xs[0][32 * warp], &Us[0][0], g, h, acc);
  } else {
    warp_mm32_masked<XLD, ULD>(&Xs[0][32 * warp], &Us[0][0], g, h, mQ, acc);
    if (TRI == R32_BOTH) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (!((mQ >> (c0 + j)) & 1u)) {
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i][j] = Xs[c0 + j][32 * warp + 4 * g + i];
        }
    }
  }
  if (TRI == R32_BOTH) {
    // T = X_Q U_Q over this warp's 32 x 32 block of Xs (T(i, c) at Xs[i][32 w + c]),
    // then U_a^T T (a row r outside T_a: (U_a^T T)(r, :) = T(r, :))
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      *reinterpret_cast<float4*>(&Xs[4 * g + i][32 * warp + c0]) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      *reinterpret_cast<float4*>(&Xs[4 * g + i][32 * warp + c0 + 4]) =
          make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
    __syncwarp();
    if (ma == 0xFFFFFFFFu) {
      warp_mm32<ULD, XLD>(&Ua[warp][0][0], &Xs[0][32 * warp], g, h, acc);
    } else {
      warp_mm32_masked<ULD, XLD>(&Ua[warp][0][0], &Xs[0][32 * warp], g, h, ma, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (!((ma >> (4 * g + i)) & 1u)) {
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = Xs[4 * g + i][32 * warp + c0 + j];
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = qh(acc[i][j], hq);
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (TRI == R32_BOTH || ((mQ >> (c0 + j)) & 1u))  // V: only the columns in T_Q change
      *reinterpret_cast<float4*>(Y + (size_t)(col0 + j) * N + row0) =
          make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
  if (TRI == R32_BOTH) {  // the mirror: rows col0 .. +7 of columns row0 .. +3
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      *reinterpret_cast<float4*>(Y + (size_t)(row0 + i) * N + col0) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      *reinterpret_cast<float4*>(Y + (size_t)(row0 + i) * N + col0 + 4) =
          make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
  }
}

}  // namespace

int mpj_stage1_padded(int n) { return ((n + W2 - 1) / W2) * W2; }

// A32, V32, two sets of the per-pair S and U (alternate rounds), the
// tensor-core update's transposed intermediate B^T, a flag word and two sets
// of the per-pair rotated-index masks.
static int stage1_tensor_cores();

size_t mpj_stage1_bytes(int n) {
  size_t N = (size_t)mpj_stage1_padded(n);
  size_t nb = N / BS;
  return 3 * N * N * sizeof(float) + 4 * (nb / 2) * W2 * W2 * sizeof(float) + 4096 + 2 * (nb / 2) * sizeof(unsigned);
}

// MPJ_STAGE1_TC=1 runs the A update of each block round on the tcgen05
// tensor cores (3xTF32, two panel products, see tc32.cu) and the V update on
// the FP32 pipe.  Off by default: on GB300 at n = 4096 it is slower (600 vs
// 435 ms for the stage), and V must stay on the FP32 pipe because the tensor
// cores' FP32 accumulation drifts the column norms over thousands of products
// (||V^T V - I||_F 0.08 instead of 0.007).
static int stage1_tensor_cores() {
  static int env = -1;
  if (env < 0) {
    const char* e = getenv("MPJ_STAGE1_TC");
    env = (e && e[0] == '1') ? 1 : 0;
  }
  return env;
}


cudaError_t mpj_sumsq32(const float* A, int lda, int n, double* partial, double* out, cudaStream_t s);


namespace {
// One stage-1 sweep (nb - 1 block rounds) enqueued on stream s.  V <- V U~ of
// round R runs on the side stream (when given), overlapping round R + 1's
// subproblems; the S/U sets alternate between rounds, round R + 2's
// subproblems wait for round R's V update before overwriting its set, and
// the side stream is joined into s at the end of the sweep.
struct Stage1Bufs {
  int N, nb;
  float *A32, *V32, *Sb[2], *Ub[2], *Bt;
  unsigned* tflag;
  unsigned* Mb[2];  // per-pair rotated-index masks, by round parity
  bool half;
  bool sparse;  // products over the rotated indices only (masked kernels)
  int tc;
};

cudaError_t stage1_sweep(const Stage1Bufs& b, cudaStream_t s, SideStream* side) {
  const int N = b.N, nb = b.nb, npairs = nb / 2;
  const dim3 g32((npairs + 3) / 4, npairs);
  bool vpending[2] = {false, false};
  cudaError_t e = cudaSuccess;
#define S1_TRY(x)                    \
  do {                               \
    e = (x);                         \
    if (e != cudaSuccess) return e;  \
  } while (0)
  for (int R = 0; R < nb - 1; ++R) {
    const int par = R & 1;
    float* Sbuf = b.Sb[par];
    float* Ubuf = b.Ub[par];
    if (side && vpending[par]) S1_TRY(cudaStreamWaitEvent(s, side->done[par], 0));
    unsigned* Mbuf = b.sparse ? b.Mb[par] : nullptr;
    S1_TRY(mpj_launch_pdl(solve32, dim3(npairs), dim3(S32_THREADS), 0, s, (const float*)b.A32, N, nb, R, Sbuf, Ubuf,
                          b.half, b.tc != 1, Mbuf));
    auto vmul = b.sparse ? rmul32<R32_ALL, true> : rmul32<R32_ALL, false>;
    // V <- V U~
    if (side) {
      S1_TRY(cudaEventRecord(side->ready, s));
      S1_TRY(cudaStreamWaitEvent(side->sv, side->ready, 0));
      S1_TRY(mpj_launch_pdl(vmul, g32, dim3(RT), 0, side->sv, (const float*)b.V32, b.V32, N, nb, R, (const float*)Sbuf,
                            (const float*)Ubuf, b.half, b.tc == 1, (const unsigned*)Mbuf));
      S1_TRY(cudaEventRecord(side->done[par], side->sv));
      vpending[par] = true;
    } else {
      S1_TRY(mpj_launch_pdl(vmul, g32, dim3(RT), 0, s, (const float*)b.V32, b.V32, N, nb, R, (const float*)Sbuf,
                            (const float*)Ubuf, b.half, b.tc == 1, (const unsigned*)Mbuf));
    }
    if (b.tc == 1) {
      // A' = U^T A U = (A U)^T U (A symmetric): B^T = (A U)^T, then
      // A' = (B^T)(:, I_q) U_q on the tensor cores; V U on the FP32 pipe
      S1_TRY(mpj_tc_panel(N, nb, R, Ubuf, b.A32, b.Bt, 1, nullptr, nullptr, b.tflag, s));
      S1_TRY(mpj_tc_panel(N, nb, R, Ubuf, b.Bt, b.A32, 0, nullptr, nullptr, b.tflag, s));
    } else {
      // A <- U~^T A U~ in one pass (tiles a > Q, mirrored; S on the diagonal)
      auto amul = b.sparse ? rmul32<R32_BOTH, true> : rmul32<R32_BOTH, false>;
      S1_TRY(mpj_launch_pdl(amul, g32, dim3(RT), 0, s, (const float*)b.A32, b.A32, N, nb, R, (const float*)Sbuf,
                            (const float*)Ubuf, b.half, false, (const unsigned*)Mbuf));
    }
  }
  if (side)
    for (int par = 0; par < 2; ++par)
      if (vpending[par]) S1_TRY(cudaStreamWaitEvent(s, side->done[par], 0));
#undef S1_TRY
  return cudaGetLastError();
}

// A sweep captured once as a CUDA graph (the fork to the side stream and the
// dependent launches become graph edges) and replayed for every sweep.  The
// kernels' arguments are the workspace addresses, so an executable graph is
// kept per (device, workspace, N, precision, update engine) and reused by
// later calls with the same workspace.
struct SweepGraph {
  int dev, N, tc;
  bool half, side, sparse;
  void* work;
  cudaGraphExec_t exec;
  long long launches;  // kernels in one sweep
  ~SweepGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};
// Shared ownership: an entry evicted by one thread stays valid for a solve
// that is replaying it on another.  The registry itself is never destroyed
// (no CUDA calls during static destruction at process exit).
std::mutex g_sweep_mu;
std::vector<std::shared_ptr<SweepGraph>>& sweep_registry() {
  static auto* r = new std::vector<std::shared_ptr<SweepGraph>>();
  return *r;
}
constexpr size_t kMaxSweepGraphs = 4;

bool sweep_graphs_enabled() {
  static int env = -1;
  if (env < 0) {
    const char* e = getenv("MPJ_STAGE1_GRAPH");
    env = (e && e[0] == '0') ? 0 : 1;
  }
  return env == 1;
}

// The executable graph of one sweep for these buffers (captured on first use),
// or null if capture is not possible (the sweep is then enqueued directly).
std::shared_ptr<SweepGraph> sweep_graph(const Stage1Bufs& b, void* work, bool use_side) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_sweep_mu);
  auto& reg = sweep_registry();
  for (const auto& g : reg)
    if (g->dev == dev && g->work == work && g->N == b.N && g->half == b.half && g->tc == b.tc && g->side == use_side &&
        g->sparse == b.sparse)
      return g;
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaSuccess;
  // kernels of one sweep: per round the subproblems, V U~ and the A update
  // (one launch, or two tensor-core panels)
  const long long per = (long long)(b.nb - 1) * (b.tc == 1 ? 4 : 3);
  {
    std::unique_ptr<SideStream> side;
    if (use_side) {
      side.reset(new SideStream(cap));
      if (!side->ok) e = cudaErrorUnknown;
      side->owner = nullptr;  // joined inside the captured sweep
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t eq = stage1_sweep(b, cap, side.get());
      e = cudaStreamEndCapture(cap, &graph);
      if (eq != cudaSuccess) e = eq;
    }
  }
  if (e == cudaSuccess) mpj_count_launches(-per);  // captured, not launched
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    return nullptr;
  }
  if (reg.size() >= kMaxSweepGraphs) reg.erase(reg.begin());
  auto g = std::make_shared<SweepGraph>();
  g->dev = dev;
  g->N = b.N;
  g->tc = b.tc;
  g->half = b.half;
  g->side = use_side;
  g->sparse = b.sparse;
  g->work = work;
  g->exec = exec;
  g->launches = per;
  reg.push_back(g);
  return g;
}
}  // namespace

int mpj_stage1_run(int n, const double* A, int lda, double* Ql, int ldq, double tol32, int max_sweeps, int* sweeps_out,
                   double* off_out, void* work, double* partial, double* dscal, cudaStream_t s, bool half,
                   bool sparse) {
  Stage1Bufs b;
  b.N = mpj_stage1_padded(n);
  b.nb = b.N / BS;
  const int N = b.N, nb = b.nb;
  b.A32 = (float*)work;
  b.V32 = b.A32 + (size_t)N * N;
  const size_t pset = (size_t)(nb / 2) * W2 * W2;
  b.Sb[0] = b.V32 + (size_t)N * N;
  b.Sb[1] = b.Sb[0] + pset;
  b.Ub[0] = b.Sb[1] + pset;
  b.Ub[1] = b.Ub[0] + pset;
  b.Bt = b.Ub[1] + pset;
  b.tflag = (unsigned*)(b.Bt + (size_t)N * N);
  b.Mb[0] = b.tflag + 64;
  b.Mb[1] = b.Mb[0] + nb / 2;
  b.half = half;
  b.sparse = sparse;
  b.tc = stage1_tensor_cores() && !half;
  float* A32 = b.A32;
  float* V32 = b.V32;
  MPJ_CUDA_TRY(cudaMemsetAsync(b.tflag, 0, sizeof(unsigned), s));
  init32<<<1024, 256, 0, s>>>(A, lda, n, N, A32, V32, half);
  mpj_count_launch();
  MPJ_CUDA_TRY(cudaGetLastError());
  double off2 = 0.0;
  MPJ_CUDA_TRY(mpj_sumsq32(A32, N, N, partial, dscal, s));
  MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
  MPJ_CUDA_TRY(cudaStreamSynchronize(s));
  double off = sqrt(off2);
  int sweeps = 0, status = MPJ_OK;
  const bool use_side = mpj_v_overlap_enabled() && nb / 2 >= 8;
  std::shared_ptr<SweepGraph> graph;
  std::unique_ptr<SideStream> side;
  while (off > tol32) {
    if (sweeps >= max_sweeps) {
      status = MPJ_NOT_CONVERGED;
      break;
    }
    if (sweeps == 0 && sweep_graphs_enabled()) graph = sweep_graph(b, work, use_side);
    if (graph) {
      MPJ_CUDA_TRY(cudaGraphLaunch(graph->exec, s));
      mpj_count_launches(graph->launches);
    } else {
      if (use_side && !side) {
        side.reset(new SideStream(s));
        if (!side->ok) side.reset();
      }
      MPJ_CUDA_TRY(stage1_sweep(b, s, side.get()));
    }
    ++sweeps;
    MPJ_CUDA_TRY(mpj_sumsq32(A32, N, N, partial, dscal, s));
    unsigned tf = 0;
    MPJ_CUDA_TRY(cudaMemcpyAsync(&off2, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaMemcpyAsync(&tf, b.tflag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    if (tf & MPJ_FLAG_TIMEOUT) return MPJ_ETIMEOUT;
    off = sqrt(off2);
  }
  widen<<<1024, 256, 0, s>>>(V32, N, n, Ql, ldq);
  mpj_count_launch();
  MPJ_CUDA_TRY(cudaGetLastError());
  if (sweeps_out) *sweeps_out = sweeps;
  if (off_out) *off_out = off;
  return status;
}
