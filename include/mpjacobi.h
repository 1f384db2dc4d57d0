/*
 * mpjacobi.h -- C ABI of libmpjacobi, a GB300 (sm_103a) implementation of the
 * mixed precision Jacobi eigensolver for real symmetric matrices of
 * Zhou, "A Mixed Precision Eigensolver Based on the Jacobi Algorithm"
 * (arXiv 2509.00495).
 *
 * Problem (Sec. 5.1, Algorithm 9): given a symmetric A in R^{n x n}, return an
 * orthogonal Q and a diagonal Lambda = diag(W) with A = Q Lambda Q^T, plus the
 * number of Jacobi sweeps used.  The mixed method computes
 *   1. Q_l: approximate eigenvectors from an FP32 Jacobi (the paper's stage 1
 *      is eig(single(A)); here an FP32 block round-robin Jacobi),
 *   2. Q_d: Newton-Schulz X <- X (3I - X^T X) / 2 in FP64 (Sec. 4.3.4, Alg. 8),
 *   3. A_cond = Q_d^T A Q_d in FP64 (Alg. 9 step 3),
 *   4. FP64 Jacobi sweeps on A_cond from V = I until off(A_cond) <= tol
 *      (Alg. 4, with the round-robin or the cyclic-by-row ordering),
 *   5. W = diag(A_cond), Q = Q_d V (formed by rotating the columns of Q_d
 *      directly, the same product by associativity).
 * The plain method is step 4 applied to A itself (the paper's jacobi_eig).
 *
 * Conventions for every entry point:
 *   - matrices are column-major FP64 with a leading dimension (ld >= n);
 *     A(i,j) = A[i + j*lda];  Q(:,j) is the eigenvector of W[j];
 *   - pointers named *_dev are CUDA device pointers owned by the caller; the
 *     library never frees or keeps them past the call;
 *   - `stream` is a cudaStream_t passed as void* (0 = legacy default stream);
 *     all work is enqueued on it;
 *   - errors are returned as mpj_status, never raised; argument errors are
 *     found on the host before anything is enqueued; conditions found on the
 *     device (non-finite input, sweep cap) are reported through mpj_info after
 *     the call returns (the solve entry points synchronize `stream`);
 *   - no entry point traps or asserts on the device; every device-side wait
 *     has an iteration or clock limit.
 *
 * Environment switches (read once per process):
 *   MPJ_JACOBI_OVERLAP=0  keep the V updates of the FP32 stage-1 rounds and
 *                         of the FP64 sweeps on `stream` (by default they
 *                         run on a private side stream joined back into
 *                         `stream`);
 *   MPJ_STAGE1_GRAPH=0    enqueue the stage-1 sweeps kernel by kernel (by
 *                         default one sweep is captured once per workspace
 *                         as a CUDA graph and replayed);
 *   MPJ_STAGE1_TC=1       run the stage-1 A update on the tcgen05 tensor
 *                         cores (3xTF32; slower on GB300, off by default);
 *   MPJ_GEMM_TC=0         run the Newton-Schulz and Q_d^T A Q_d products on
 *                         the FP64 DMMA kernel instead of the tensor cores
 *                         (the exact bf16-slice products of mpj_dgemm_tc, the
 *                         default);
 *   MPJ_AUTOTUNE_CACHE=f  file that keeps the batched group-size choices;
 *   MPJ_BATCHED_GROUP=g   fix the batched group size (256, 512 or 1024).
 */
#ifndef MPJACOBI_H
#define MPJACOBI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MPJ_OK = 0,
  MPJ_NOT_CONVERGED = 1,  /* results written, but off(A) > tol at the sweep cap */
  MPJ_EINVAL = -1,        /* bad size, leading dimension, null pointer or option */
  MPJ_ENOTSYM = -2,       /* opts.check_symmetry set and A(i,j) != A(j,i) somewhere */
  MPJ_ENONFINITE = -3,    /* A holds a NaN or an infinity */
  MPJ_ECUDA = -4,         /* a CUDA runtime call failed (see mpj_last_cuda_error) */
  MPJ_ENOMEM = -5,        /* workspace allocation failed */
  MPJ_EDEGENERATE = -6,   /* backward: w_i == w_j for i != j with a nonzero coupling */
  MPJ_EWORKSPACE = -7,    /* caller workspace too small (see mpj_syev_workspace) */
  MPJ_ETIMEOUT = -8,      /* a device-side barrier gave up after its iteration limit */
  MPJ_ETOOLARGE = -9,     /* n exceeds the fixed scratch of an allocation-free entry point */
  MPJ_EPREMISE = -10      /* ||Q_l^T Q_l - I||_2 >= 2: Q_l outside the Newton-Schulz convergence premise */
} mpj_status;

enum { MPJ_ORDER_CYCLIC = 0, MPJ_ORDER_ROUND_ROBIN = 1, MPJ_ORDER_BLOCK = 2 };
enum { MPJ_METHOD_MIXED = 0, MPJ_METHOD_PLAIN = 1 };

typedef struct {
  double tol;        /* FP64 stop: off(A) <= tol; <= 0 selects n * 2^-53 * ||A||_F              */
  double tol32;      /* stage-1 stop: off(A32) <= tol32; <= 0 selects n * 2^-24 * ||A||_F       */
  int max_sweeps64;  /* FP64 sweep cap; <= 0 selects 30 (the paper's default is 10)           */
  int max_sweeps32;  /* stage-1 sweep cap; <= 0 selects 15                                    */
  int ns_steps;      /* Newton-Schulz steps; <= 0 selects 2 for n < 52000, else 3 (Alg. 8)     */
  int ordering;      /* FP64 sweep ordering: MPJ_ORDER_BLOCK (default: block round-robin, blocks of
                        16, block updates on the tensor cores), MPJ_ORDER_ROUND_ROBIN, or
                        MPJ_ORDER_CYCLIC (the paper's cyclic-by-row)                          */
  int method;        /* MPJ_METHOD_MIXED (default) or MPJ_METHOD_PLAIN                        */
  int polish;        /* 1: one more FP64 Newton-Schulz step on the final Q (not in the paper) */
  int sort;          /* 1 (default): W ascending, Q's columns permuted to match              */
  int check_symmetry;/* 1: fail with MPJ_ENOTSYM unless A is exactly symmetric               */
  int threshold;     /* FP64 sweeps also skip pairs with |a_pq| <= tol / n (threshold Jacobi, the
                        paper's future work): 1 on, 0 off, -1 (default) on for the block and
                        round-robin orderings, off for cyclic-by-row.  Cannot stop the sweeps
                        early.                                                                */
  int precond_passes;/* mixed method: 1 (default) = Algorithm 9; 2 = stages 1-3 applied again to
                        A_cond (FP32 Jacobi on fl32(A_cond), Newton-Schulz, Q_d2^T A_cond Q_d2,
                        Q_d = Q_d1 Q_d2) before the FP64 sweeps -- not in the paper            */
  int stage1_half;   /* 1: stage 1 in half precision (binary16 values, skip test and tol32 at
                        2^-11; the paper's further work, Ch. 6); Newton-Schulz then takes the
                        smallest k with (sqrt(1 + n 2^-11) - 1)^(2^k) <= n 2^-53 steps (the
                        paper's bound of Sec. 4.3.4 with the half unit roundoff)              */
  int max_sweeps32_pass2; /* stage-1 sweep cap of the second preconditioning pass; <= 0 selects
                        min(9, the stage-1 cap)                                               */
} mpj_opts;

typedef struct {
  int status;        /* mpj_status of the solve                                               */
  int sweeps32;      /* stage-1 (FP32) sweeps                                                 */
  int sweeps32_pass2;/* stage-1 sweeps of the second preconditioning pass (0 if not run)      */
  int sweeps64;      /* FP64 sweeps (the quantity the paper reports as "iterations")          */
  int ns_steps;      /* Newton-Schulz steps applied                                           */
  double norm_fro;   /* ||A||_F                                                               */
  double tol;        /* FP64 tolerance used                                                   */
  double off32;      /* off(A32) at the end of stage 1                                        */
  double off_cond;   /* off(A_cond) before the FP64 sweeps                                    */
  double off_final;  /* off(A) after the last FP64 sweep                                      */
  float ms_stage[6]; /* device time per stage: stage1, NS, transform, sweeps, final, total   */
  double ns_e0;      /* ||Q_l^T Q_l - I||_2 before Newton-Schulz, a 30-step power-iteration
                        estimate (the iteration converges for ||Q_l^T Q_l - I||_2 < 2,
                        Sec. 4.3.4; the solve returns MPJ_EPREMISE when the estimate is 2 or
                        more)                                                                */
  long long rotated_blocks64; /* block ordering: block-pair subproblems (32 x 32) that rotated,
                        summed over all rounds of all FP64 sweeps (0 for the other orderings) */
} mpj_info;

/* Fills `o` with the defaults described in mpj_opts. */
void mpj_opts_default(mpj_opts* o);

/* Human-readable name of a status code (static storage). */
const char* mpj_status_str(int status);

/* Text of the last CUDA error seen by this thread inside the library. */
const char* mpj_last_cuda_error(void);

/* Diagnostic: number of CUDA kernels this library has enqueued since it was
 * loaded (all threads).  The difference around a call counts its launches. */
long long mpj_kernel_launches(void);

/* Diagnostic: number of device (and pinned host) allocations this library has
 * made since it was loaded (all threads; cudaMalloc, cudaMallocAsync,
 * cudaMallocHost).  The difference around a call counts its allocations: zero
 * for mpj_syev_ex with a caller workspace. */
long long mpj_device_allocations(void);

/* Bytes of device workspace mpj_syev_ex needs for size n under `o` (NULL: defaults). */
size_t mpj_syev_workspace(int n, const mpj_opts* o);

/* Mixed precision symmetric eigensolver (Alg. 9), default options.
 * A_dev: n x n input, read only.  W_dev: n eigenvalues (ascending).
 * Q_dev: n x n eigenvectors, ldq = n.  tol <= 0 selects n 2^-53 ||A||_F.
 * Allocates its workspace with cudaMallocAsync on `stream` and frees it before
 * returning; synchronizes `stream`.  Returns MPJ_OK, MPJ_NOT_CONVERGED, or an
 * error code. */
int mpj_syev(int n, const double* A_dev, int lda, double* W_dev, double* Q_dev, double tol, void* stream);

/* Same with explicit options, output leading dimension, optional host `info`
 * (may be NULL) and optional caller workspace (work_dev may be NULL: then the
 * library allocates it with cudaMallocAsync and frees it before returning;
 * else work_bytes >= mpj_syev_workspace(n, o) and the call allocates nothing:
 * every buffer, including the sliced operands of the tensor-core products,
 * is carved from work_dev).  Synchronizes `stream` once per sweep (to read
 * off(A)) and at the end; device-side conditions (a tensor-core completion
 * wait that ran out: MPJ_ETIMEOUT) are read at the final synchronization.
 * Returns MPJ_EWORKSPACE if work_bytes is too small. */
int mpj_syev_ex(int n, const double* A_dev, int lda, double* W_dev, double* Q_dev, int ldq, const mpj_opts* o,
                mpj_info* info, void* work_dev, size_t work_bytes, void* stream);

/* Batched solve of `batch` independent matrices (sizes 1 <= n_i <= 256) in one
 * persistent launch (not in the paper; each matrix runs Algorithm 9 in one
 * thread group).  n_host: host array of sizes.  A_dev, W_dev, Q_dev: device
 * arrays of `batch` device pointers (A read only, lda_i = n_i; Q_i is
 * n_i x n_i, ld n_i).  sweeps_host (may be NULL): receives the FP64 sweep count
 * per matrix.  tol <= 0 selects n_i 2^-53 ||A_i||_F per matrix.
 * The first call for a given (sizes, pointer arrays, tol) plans: it allocates
 * a workspace with cudaMalloc, orders the queue by decreasing n, picks the
 * thread-group size (256, 512 or 1024 threads per matrix) by timing each on
 * this batch unless the size histogram was tuned before (choices persist in
 * the file named by the environment variable MPJ_AUTOTUNE_CACHE, if set;
 * MPJ_BATCHED_GROUP=256|512|1024 fixes the size instead), and
 * captures [queue reset, kernel, result copies] in a CUDA graph.  Later calls
 * with the same sizes and pointer arrays only launch that graph on `stream`
 * (the pointed-to data may change); they may themselves be stream-captured,
 * the first one may not.  Up to 4 plans are kept (mpj_release_plans frees
 * them).  Synchronizes `stream`.  Returns MPJ_NOT_CONVERGED if any matrix hit
 * the sweep cap, MPJ_ENONFINITE if any input holds a NaN or an infinity. */
int mpj_syev_batched(int batch, const int* n_host, const double* const* A_dev, double* const* W_dev,
                     double* const* Q_dev, double tol, int* sweeps_host, void* stream);

/* Frees the workspaces and graphs of all cached batched plans. */
void mpj_release_plans(void);

/* The autotuned thread-group size recorded for this batch's size histogram
 * (256, 512 or 1024), or 0 if none has been tuned yet. */
int mpj_batched_group_size(int batch, const int* n_host);

/* Eigen-adjoint (not in the paper): with W, Q from a solve (Q n x n, ld ldq),
 * upstream gradients dW (n, may be NULL = 0) and dQ (n x n, ld lddq, may be
 * NULL = 0), writes dA = sym(Q (diag(dW) + F o (Q^T dQ)) Q^T), F_ij = 1/(w_j - w_i)
 * for i != j, F_ii = 0, sym(X) = (X + X^T)/2, into dA (ld ldda).
 * `batch` matrices of the same n are processed at once; matrix b starts at
 * offset b*n (W, dW) and b*ld*n (Q, dQ, dA).  Returns MPJ_EDEGENERATE if some
 * w_i == w_j (i != j) meets a nonzero (Q^T dQ)_ij (dA is then undefined). */
int mpj_syev_backward(int batch, int n, const double* W_dev, const double* Q_dev, int ldq, const double* dW_dev,
                      const double* dQ_dev, int lddq, double* dA_dev, int ldda, void* stream);

/* ---- stage entry points (each one step of Alg. 9, for stage-wise checks) ---- */

/* Stage 1: FP32 block round-robin Jacobi on fl32(A) from V32 = I; writes
 * Ql = double(V32) (n x n, ld ldq).  Stops at off(A32) <= tol32 (<= 0: default)
 * or after max_sweeps (<= 0: 15).  sweeps / off32 (host, may be NULL). */
int mpj_stage1(int n, const double* A_dev, int lda, double* Ql_dev, int ldq, double tol32, int max_sweeps,
               int* sweeps, double* off32, void* stream);

/* Newton-Schulz in place: X <- X (3I - X^T X)/2, `steps` times (Sec. 4.3.4);
 * products as in the solve (tensor cores unless MPJ_GEMM_TC=0). */
int mpj_newton_schulz(int n, double* X_dev, int ldx, int steps, void* stream);

/* Preconditioning: Ac = Qd^T A Qd (Alg. 9 step 3); Ac is written exactly
 * symmetric (lower triangle mirrored).  Products as in the solve: the
 * tensor-core exact-slice engine unless MPJ_GEMM_TC=0 selects the FP64 DMMA
 * kernel.  Allocates its scratch with cudaMallocAsync; synchronizes. */
int mpj_precondition(int n, const double* A_dev, int lda, const double* Qd_dev, int ldq, double* Ac_dev, int ldc,
                     void* stream);

/* FP64 Jacobi sweeps (Alg. 4) in place on the symmetric A (full storage, both
 * triangles kept equal) accumulating V <- V J (V holds the start matrix, e.g.
 * I), with ordering
 *   MPJ_ORDER_BLOCK        block round-robin (blocks of 16; one inner
 *                          round-robin sweep per 32 x 32 block-pair subproblem
 *                          in FP64; the rest of A and V updated by the
 *                          accumulated block rotations as FP64-accurate
 *                          tensor-core products; the paper's block Jacobi,
 *                          Ch. 6 further work),
 *   MPJ_ORDER_ROUND_ROBIN  scalar round-robin (circle method), or
 *   MPJ_ORDER_CYCLIC       the paper's cyclic-by-row ordering, run as
 *                          wavefronts of the pairs with equal p + q (the same
 *                          rotation sequence),
 * per-pair skip rule |a_pq| > 2^-53 sqrt(|a_pp a_qq|), stop at off(A) <= tol
 * (tol <= 0: n 2^-53 ||A||_F) or max_sweeps (<= 0: 30).  sweeps / off_final
 * (host, may be NULL).  Returns MPJ_NOT_CONVERGED at the cap, MPJ_ETIMEOUT if
 * a tensor-core completion wait ran out. */
int mpj_jacobi64(int n, double* A_dev, int lda, double* V_dev, int ldv, double tol, int ordering, int max_sweeps,
                 int* sweeps, double* off_final, void* stream);

/* Allocation-free variant of mpj_jacobi64 (the paper has no counterpart).
 * For callers that may not allocate device memory during the call: code that
 * runs with its whole memory budget already committed, latency-critical
 * loops that must stay clear of the allocator, or hosts where allocation
 * calls are not allowed at that point.  Same arguments, behaviour and results
 * as mpj_jacobi64, but the sweep's scratch (rotation records, scale vectors,
 * reduction partials and a batch of rotation multipliers for V: about
 * (80 + 8 r) n bytes with r rounds per V batch, r = 64 down to 1 as n grows)
 * lives in one fixed array of MPJ_NOALLOC_SCRATCH_BYTES bytes in device
 * memory, reserved in every GPU that loads the library until the process
 * exits; no cudaMalloc, cudaFree or
 * allocating library routine is called.  n > MPJ_NOALLOC_MAX_N returns
 * MPJ_ETOOLARGE before any work.  The first call on a device looks up the
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  All calls share the one array:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it and must be serialized by the caller.  Every scratch word is
 * written before it is read, so nothing carries over between calls.  The
 * looked-up address is kept for the life of the process: do not use this
 * entry point across a cudaDeviceReset (or anything else that recreates the
 * device's primary context).  Only the round-robin and cyclic orderings are
 * offered here (the block ordering needs an n x n buffer). */
#define MPJ_NOALLOC_MAX_N 8192
#define MPJ_NOALLOC_SCRATCH_BYTES 1048576
int mpj_jacobi64_noalloc(int n, double* A_dev, int lda, double* V_dev, int ldv, double tol, int ordering,
                         int max_sweeps, int* sweeps, double* off_final, void* stream);

/* FP64 matrix product on the library's DMMA kernel:
 * C = alpha op(A) op(B) + beta C, op(X) = X or X^T (trans = 'N' or 'T'),
 * op(A) m x k, op(B) k x n.  No symmetric shortcuts. */
int mpj_dgemm(char transa, char transb, int m, int n, int k, double alpha, const double* A_dev, int lda,
              const double* B_dev, int ldb, double beta, double* C_dev, int ldc, void* stream);

/* FP64 matrix product on the tcgen05 tensor cores (not in the paper; the
 * paper's products are FP64): C = alpha op(A) op(B) + beta C with the same
 * arguments as mpj_dgemm (m, n, k >= 1).  Each row of op(A) and column of
 * op(B) is split on the grid of its largest exponent into 8 slices of 7 bits
 * held exactly as bf16; slice products are summed exactly in the tensor cores'
 * FP32 accumulators over chunks of 256 values of k (all partial sums are
 * integers below 2^24 in their level's unit) and the chunks exactly in 64-bit
 * integers; the result is rounded once to FP64 and scaled by 2^(e_r + f_c)
 * in one step (no intermediate underflow).  The error is within a small
 * multiple of 2^-53 (|op(A)| |op(B)|)_rc plus k 2^-54 max|op(A)(r,:)|
 * max|op(B)(:,c)| per entry.  Allocates about 16 (m + n) k bytes of scratch
 * with cudaMallocAsync; synchronizes the stream.  Returns MPJ_EINVAL,
 * MPJ_ENOMEM, MPJ_ETIMEOUT (the tensor cores did not signal completion within
 * about 2 s) or MPJ_ECUDA on failure. */
int mpj_dgemm_tc(char transa, char transb, int m, int n, int k, double alpha, const double* A_dev, int lda,
                 const double* B_dev, int ldb, double beta, double* C_dev, int ldc, void* stream);

/* One product of the stage-1 blocked update on the tcgen05 tensor cores
 * (3xTF32; the stage is the approximate eigenvector step of Sec. 4.1, and the
 * paper has no blocked form of it).  N: a multiple of 32; block round R in
 * [0, N/16 - 1) of the circle method on the N/16 blocks of 16 indices; block
 * pair q of that round covers the 32 indices I_q (its lower block, then its
 * upper block).  For every pair q:
 *   Out[:, I_q] = In[:, I_q] * U_q       (mode bit 0 clear), or
 *   Out[I_q, :] = (In[:, I_q] * U_q)^T   (mode bit 0 set),
 * In, Out: N x N column-major FP32 device arrays (ld = N), distinct when
 * transposing; U_dev: N/32 column-major 32 x 32 FP32 factors, U_q at
 * U_dev + 1024 q.  Products are accurate to about 2^-21 relative.  Mode bit 1
 * (failure-detection test, N <= 256 only) issues no tensor-core work, so the
 * completion wait runs out: the call then returns MPJ_ETIMEOUT after about
 * 4 s with Out untouched and the device usable.  Returns MPJ_EINVAL for bad
 * arguments, MPJ_ETIMEOUT if the tensor cores did not signal completion within
 * about 2 s, MPJ_ECUDA on a launch error.  Synchronizes the stream. */
int mpj_stage1_panel(int N, int R, const float* U_dev, const float* In_dev, float* Out_dev, int mode, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPJACOBI_H */
