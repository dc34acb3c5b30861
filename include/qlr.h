/*
 * qlr.h -- C ABI of the GB300 (sm_103a) pass-efficient randomized quaternion low-rank library.
 *
 * Method: pass-efficient randomized low-rank approximation of quaternion matrices
 * (arXiv 2507.13731).  The hot path is the per-pass quaternion sketch product Y = A X or
 * Z = A^H Y, run v times by the arbitrary-pass range finder (Algorithm 2) or the flexible block
 * Krylov variant (Algorithm 4), with an orthonormalisation ("QR") after every pass and a small
 * truncated QSVD at the end.
 *
 * Conventions (all entry points)
 *  - Quaternion matrices are four real planes (real, i, j, k) -- the paper's X1..X4, Section 2.
 *    A pure quaternion matrix (zero real part) may pass plane[0] == NULL.
 *  - The large data matrix A is row-major (ld >= cols).  Thin matrices (Omega, Q, Y, Z, U, V)
 *    are column-major (ld >= rows).  All pointers inside qlr_qmat are DEVICE pointers.
 *  - Caller owns every matrix and output buffer.  The context owns its workspace (device
 *    memory it allocates with cudaMalloc on first need and grows on demand; qlr_reserve
 *    pre-sizes it so that later calls -- e.g. inside CUDA stream capture -- allocate nothing).
 *  - Calls are asynchronous on the context's stream.  Host-side validation errors are returned
 *    immediately.  Device-side conditions (Cholesky breakdown, Jacobi non-convergence, bounded
 *    waits) are recorded in a device error word; qlr_sync() waits for the stream and returns it.
 *  - A context is not thread-safe: its calls share one workspace, error word and launch
 *    statistics, so calls on one context must not overlap across host threads.  Use one context
 *    per host thread (each on its own stream).
 *  - Every function returns QLR_OK (0) or one of the QLR_E* codes below.
 */
#ifndef QLR_H
#define QLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------------------------ */
#define QLR_OK 0
#define QLR_EINVAL 1       /* bad argument (null pointer, bad enum, bad layout / dtype combination) */
#define QLR_ESHAPE 2       /* inconsistent sizes, or k + p > min(m, n) (hypothesis of Lemma 2)    */
#define QLR_ENOTPD 3       /* Cholesky pivot <= 0: Gram matrix not numerically positive definite  */
#define QLR_ENOCONV 4      /* core Jacobi QSVD did not converge within its sweep limit            */
#define QLR_ETIMEOUT 5     /* a bounded device-side wait gave up                                  */
#define QLR_ECUDA 6        /* a CUDA runtime / driver call failed                                  */
#define QLR_ENOMEM 7       /* workspace too small and growing it is not allowed (stream capture)  */
#define QLR_EUNSUPPORTED 8 /* combination not implemented (e.g. a size beyond a kernel's limit)   */

/* ---- storage types ---------------------------------------------------------------------- */
#define QLR_F64 0
#define QLR_F32 1
#define QLR_BF16 2

/* ---- layouts ----------------------------------------------------------------------------- */
#define QLR_ROW_MAJOR 0
#define QLR_COL_MAJOR 1

/* ---- arithmetic of the sketch products ------------------------------------------------- */
#define QLR_COMPUTE_AUTO 0   /* F64 storage -> F64, F32 -> TF32X3, BF16 -> BF16                 */
#define QLR_COMPUTE_F64 1    /* FP64 SIMT (cuda cores)                                          */
#define QLR_COMPUTE_F32 2    /* FP32 SIMT: the plain FP32 GPU path                              */
#define QLR_COMPUTE_TF32 3   /* tcgen05 kind::tf32, one product (FP32 storage)                  */
#define QLR_COMPUTE_TF32X3 4 /* tcgen05 kind::tf32, hi/lo split of both operands, three products */
#define QLR_COMPUTE_BF16 5   /* tcgen05 kind::f16 with BF16 operands (BF16 storage of A)         */
/* FP32 storage, algorithm calls only: the products whose result only feeds a later basis or
 * Krylov block (Algorithm 2's passes 1..v-1, Algorithm 4's views before the final pass) run one
 * TF32 product; the last pass, which forms the returned R, runs 3xTF32. */
#define QLR_COMPUTE_TF32_MIXED 6
/* tcgen05 kind::tf32, one product of operands rounded to the nearest TF32 value (the tensor cores
 * alone drop the 13 low mantissa bits, a bias toward zero), FP32 sums in chunks of 512 reduction
 * elements added with round-to-nearest: each operand carries a zero-mean error of at most 2^-11
 * relative.  In an algorithm call the products that only feed a later basis run plain TF32 (as in
 * QLR_COMPUTE_TF32_MIXED) and the last pass this product.  The singular values then move by up
 * to ~2^-12 relative where singular vectors are concentrated on few entries (each entry's
 * rounding acts directly), far less where they are spread over many (the errors average out). */
#define QLR_COMPUTE_TF32_RN 7

/* ---- sketch operator ------------------------------------------------------------------- */
#define QLR_OP_N 0 /* Y = A X     */
#define QLR_OP_H 1 /* Y = A^H X   */

/* ---- algorithm / side / orthonormalisation choices ------------------------------------- */
#define QLR_ALG1 1 /* Algorithm 1 (classical power scheme, q = passes/2 - 1; passes even)     */
#define QLR_ALG2 2 /* Algorithm 2 (arbitrary number of passes)                                */
#define QLR_ALG3 3 /* Algorithm 3 (classical block Krylov, q = passes/2 - 1; passes even)     */
#define QLR_ALG4 4 /* Algorithm 4 (flexible block Krylov, arbitrary views)                    */
#define QLR_SIDE_AUTO (-1)
#define QLR_SIDE_X 0
#define QLR_SIDE_XH 1
#define QLR_ORTH_CHOLQR2 0  /* CholeskyQR2, FP64-class Gram and Cholesky              */
#define QLR_ORTH_SCHOLQR3 1 /* shifted CholeskyQR3 (Fukaya et al. 2020) for ill-conditioned input */
/* opts.flags bit: run opts.orth at every pass, as Algorithms 2 and 4 write it.  Without it, a basis
 * that only feeds the next pass (Algorithm 2's passes 1..v-2, the blocks Algorithm 4 stacks or
 * discards) gets one shifted CholeskyQR step: its R is never used and the next product depends only
 * on its column space, so the result is the same in exact arithmetic.  The QR factors whose Q or R
 * reach U, S, V always use opts.orth. */
#define QLR_FLAG_QR_EVERY_PASS 1
/* opts.flags bit for batch plans: enqueue every kernel on each run instead of replaying the
 * CUDA graph captured at creation (ignored by the single-problem calls). */
#define QLR_FLAG_NO_GRAPH 2

typedef struct {
  void* plane[4];  /* device pointers: planes real, i, j, k; plane[0] == NULL => pure quaternion */
  int64_t rows;    /* number of rows                                                            */
  int64_t cols;    /* number of columns                                                         */
  int64_t ld;      /* leading dimension in elements (row stride if row-major, column stride if col-major) */
  int32_t layout;  /* QLR_ROW_MAJOR or QLR_COL_MAJOR                                            */
  int32_t dtype;   /* QLR_F64, QLR_F32 or QLR_BF16                                              */
} qlr_qmat;

typedef struct {
  int32_t compute; /* QLR_COMPUTE_*; AUTO picks from A's dtype                                  */
  int32_t side;    /* QLR_SIDE_*; AUTO applies Section 6's rule (even v and n > m: use X^H)     */
  int32_t orth;    /* QLR_ORTH_*; Algorithm 4's stacked basis always uses QLR_ORTH_SCHOLQR3    */
  int32_t flags;   /* 0 or a combination of QLR_FLAG_QR_EVERY_PASS and QLR_FLAG_NO_GRAPH        */
} qlr_opts;

typedef struct qlr_ctx qlr_ctx;

/* Create a context on CUDA device `device` issuing work on `stream` (a cudaStream_t, NULL for
 * the legacy default stream).  Allocates the device error word.  Returns QLR_ECUDA on failure. */
int qlr_create(qlr_ctx** ctx, int device, void* stream);
/* Synchronise, free the workspace and the context.  ctx may be NULL. */
int qlr_destroy(qlr_ctx* ctx);
/* Change the stream later calls are issued on. */
int qlr_set_stream(qlr_ctx* ctx, void* stream);
/* Make sure the workspace holds at least `bytes` bytes (cudaMalloc now, never inside a call). */
int qlr_reserve(qlr_ctx* ctx, size_t bytes);
/* Workspace bytes a qlr_qsvd_lowrank / qlr_qblock_krylov call with these sizes needs. */
size_t qlr_workspace_size(int64_t m, int64_t n, int k, int p, int passes, int algo, int compute);
/* Wait for the context's stream; return the first device-side error code (and clear it), or
 * QLR_ECUDA if the stream reported a CUDA error. */
int qlr_sync(qlr_ctx* ctx);
/* Static English text for an error code. */
const char* qlr_strerror(int code);

/* ---- launch statistics (no paper counterpart: measurement support) ----------------------
 * Kernel classes counted / timed by the library.  Launch counts are always kept; with timing
 * enabled every launch is bracketed by CUDA events recorded on the context stream (do not
 * enable inside stream capture).  qlr_stats waits for the stream and returns, for class `kid`,
 * the number of launches and the summed event time in milliseconds since the last reset. */
#define QLR_KID_SKETCH_TC 0   /* tcgen05 sketch product                     */
#define QLR_KID_SKETCH_SIMT 1 /* SIMT sketch product / thin GEMMs           */
#define QLR_KID_GRAM 2        /* FP64-class Gram (slices / partials, combine) */
#define QLR_KID_CHOL 3        /* quaternion Cholesky                         */
#define QLR_KID_TRIINV 4      /* triangular inverse                          */
#define QLR_KID_APPLY 5       /* Q = Y R^{-1}, lifts, projections            */
#define QLR_KID_JACOBI 6      /* core QSVD sweeps                            */
#define QLR_KID_REFINE 7      /* core QSVD FP64 evaluation + ranking         */
#define QLR_KID_MISC 8        /* conversions, operand staging, small products */
#define QLR_KID_SERIES 9      /* CholeskyQR2 second step by series (factor and inverse) */
#define QLR_KID_COMPLETE 10   /* matrix completion: masked low-rank update   */
#define QLR_KID_SKETCH_X3 11  /* tcgen05 sketch product in 3xTF32 (class 0 holds BF16 / TF32) */
#define QLR_KID_SKETCH_RN 12  /* tcgen05 sketch product in rounded TF32 (QLR_COMPUTE_TF32_RN)   */
#define QLR_KID_COUNT 13
int qlr_set_timing(qlr_ctx* ctx, int enable);
int qlr_reset_stats(qlr_ctx* ctx);
int qlr_stats(qlr_ctx* ctx, int kid, int64_t* launches, double* total_ms);

/* ---- throughput probes (no paper counterpart: the roofline denominators) ---------------
 * qlr_peak_probe runs one probe kernel on `device` (on a stream of its own, synchronously) and
 * returns the floating-point operations it executed and its CUDA-event time:
 *   QLR_PEAK_TF32_MMA / QLR_PEAK_BF16_MMA: one CTA per SM issues `iters` rounds of 8 tcgen05 MMAs
 *     (M = 128, N = 256, K = 8 kind::tf32 / K = 16 kind::f16 with BF16 operands) on operands
 *     staged once in shared memory; iters <= 400000 (the kernel's bounded wait must not expire);
 *   QLR_PEAK_FP32_FMA / QLR_PEAK_FP64_FMA: 8 CTAs of 256 threads per SM, each thread `iters`
 *     rounds of 8 independent fused multiply-adds;
 *   QLR_PEAK_TF32_MMA_N64 / QLR_PEAK_BF16_MMA_N64: the MMA loops with N = 64 (the width of a thin
 *     sketch's MMAs; an MMA of M = 128 takes about as long for N = 64 as for N ~ 100).
 * Dense peak = flops / ms.  Errors: QLR_EINVAL (kind, iters, null outputs), QLR_ECUDA,
 * QLR_ETIMEOUT (the MMA probe's bounded wait gave up). */
#define QLR_PEAK_TF32_MMA 0
#define QLR_PEAK_BF16_MMA 1
#define QLR_PEAK_FP32_FMA 2
#define QLR_PEAK_FP64_FMA 3
#define QLR_PEAK_TF32_MMA_N64 4   /* the MMA loops with N = 64 (thin sketches' MMA width) */
#define QLR_PEAK_BF16_MMA_N64 5
int qlr_peak_probe(int kind, int device, int64_t iters, double* flops, float* ms);

/* ---- the Gaussian test matrix from a seed (Def. 2) ---------------------------------------
 * Def. 2's test matrix Omega has four independent standard normal components per entry; the
 * paper fixes no generator.  These calls reproduce, from a seed, the Omega that this library's
 * tests and benchmarks give both the GPU path and the FP64 oracle: a counter-based SplitMix64
 * (draw t of the stream with seed s is SplitMix64's finaliser applied to s + (t + 1) *
 * 0x9E3779B97F4A7C15) and the Box-Muller transform (normals 2p, 2p + 1 from uniforms u, w = the
 * top 53 bits of draws 2p, 2p + 1 times 2^-53: r cos(2 pi w), r sin(2 pi w), r = sqrt(-2 ln(1 - u))),
 * entry (c, i, j) of a rows x cols matrix being normal number c rows cols + j rows + i.
 * qlr_splitmix64 -- draw `counter` of the stream with seed `seed` (derives stream seeds: the test
 *   matrix of a workload with base seed b is drawn with seed qlr_splitmix64(b, 6)).
 * qlr_gaussian_qmat_host -- fills `out` (host, 4 planes of rows x cols doubles, column-major, plane c
 *   at out + c rows cols) with the Gaussian quaternion matrix of stream `seed`; real_only != 0 draws
 *   plane 0 only (the real Gaussian matrix of the experiments, Section 8) and zeroes the others.
 *   No device work.  QLR_EINVAL for a null out or negative sizes.
 * qlr_fill_omega -- the same matrix written into the device matrix `omega` (column-major, F64 or
 *   F32, 4 planes) on the context's stream; synchronises the stream (host-to-device copies). */
uint64_t qlr_splitmix64(uint64_t seed, uint64_t counter);
int qlr_gaussian_qmat_host(uint64_t seed, int64_t rows, int64_t cols, int real_only, double* out);
int qlr_fill_omega(qlr_ctx* ctx, uint64_t seed, int real_only, qlr_qmat* omega);

/*
 * qlr_qsketch -- one sketch pass (the products X Q2 / X^H Q1 of Algorithm 2 and Algorithm 4,
 * and the Hamilton product of eq. (1), Section 2, summed over the inner index).
 *   op == QLR_OP_N:  Y (m x l) = A (m x n) X (n x l)
 *   op == QLR_OP_H:  Y (n x l) = A^H X (m x l), with A^H = A1^T - A2^T i - A3^T j - A4^T k (Section 2)
 * A: row-major, dtype F64 / F32 / BF16 (pure allowed).  X: column-major, 4 planes; its dtype
 * must be F64 for COMPUTE_F64, F32 for F32 / TF32 / TF32X3 / TF32_RN, F32 or BF16 for BF16 (F32 input is
 * rounded to BF16 on the device).  Y: column-major, F64 (COMPUTE_F64) or F32.  A is read once.
 * Degenerate sizes: an empty Y (no rows or no columns) launches nothing; an empty inner
 * dimension (n = 0 for op N, m = 0 for op H) writes Y = 0.
 * Errors: QLR_EINVAL (null/dtype/layout), QLR_ESHAPE (size mismatch), QLR_EUNSUPPORTED.
 */
int qlr_qsketch(qlr_ctx* ctx, int op, const qlr_qmat* A, const qlr_qmat* X, qlr_qmat* Y, int compute);

/*
 * qlr_qgram -- G = Y^H Y with FP64-class accuracy (the Gram step of CholeskyQR; the "QR" of
 * Algorithms 1-4, Def. 1 eq. QQR).  F64 Y: FP64 arithmetic.  F32 Y: on the tensor cores by an
 * exact splitting of every column into 6-bit BF16 slices below its largest entry (error about
 * 2^-45 of max|y_i| max|y_j| m), or, when the workspace cannot hold the slices, double-FP32 sums
 * on the FP32 pipes.  Y: m x l column-major F32 or F64.  G: device, FP64, l x l x 4 planes,
 * column-major (G[c*l*l + j*l + i]), full Hermitian matrix written.
 */
int qlr_qgram(qlr_ctx* ctx, const qlr_qmat* Y, double* G);

/*
 * qlr_qchol -- upper-triangular R with real positive diagonal and G = R^H R (quaternion
 * Cholesky, FP64).  G, R: device FP64 l x l x 4 column-major (may not alias).  Lower triangle of
 * R is written as zero.  A non-positive pivot records QLR_ENOTPD in the device error word and
 * continues with a tiny positive pivot so later kernels see finite numbers.
 */
int qlr_qchol(qlr_ctx* ctx, int l, const double* G, double* R);

/*
 * qlr_cholqr -- thin QR Y = Q R (Def. 1, eq. QQR) by CholeskyQR2 (orth = QLR_ORTH_CHOLQR2) or
 * shifted CholeskyQR3 (QLR_ORTH_SCHOLQR3).  Gram products and Cholesky factors in FP64, the
 * triangular solves in the storage precision of Y.  Y, Q: m x l column-major, same dtype
 * (F32 or F64), must not alias.  R: device FP64 l x l x 4, upper triangular, real positive
 * diagonal (the unique thin QR for full-rank Y).  R may be NULL if not needed.
 */
int qlr_cholqr(qlr_ctx* ctx, const qlr_qmat* Y, qlr_qmat* Q, double* R, int orth);

/*
 * qlr_qtsvd -- core truncated QSVD (R, k) of a small l x l quaternion matrix (the
 * "Truncated SVD(R,k)" step of Algorithms 1, 2, 4; QSVD of Def. 1 eq. qsvd) through the
 * complex adjoint chi(R) with structure-preserving one-sided Jacobi.  R: device FP64 l x l x 4
 * column-major.  Outputs (device, FP64): L (l x k x 4), S (k, descending), Rt (l x k x 4) with
 * R ~= L diag(S) Rt^H.  prec: QLR_F64 runs the Jacobi in FP64; QLR_F32 runs it in FP32 and
 * re-evaluates S, L in FP64 from the FP32 right vectors.  QLR_ENOCONV if it did not converge.
 */
int qlr_qtsvd(qlr_ctx* ctx, int l, const double* R, int k, double* L, double* S, double* Rt, int prec);

/*
 * qlr_qrangefinder -- v passes of Algorithm 2 (range finder part): for i = 1..v, odd i:
 * [Q1, R1] = QR(X Q2), even i: [Q2, R2] = QR(X^H Q1), starting from Q2 = Omega.
 * A: m x n row-major.  omega: Gaussian test matrix (Def. 2), l = k + p columns, n rows (side X)
 * or m rows (side X^H), column-major, dtype F64 or F32.  Q1 (m x l) and Q2 (n x l): column-major,
 * F64 or F32 (F64 iff compute is F64); Q2 is left equal to omega's contents when v == 1 is not
 * allowed (v >= 2).  R: device FP64 l x l x 4 -- R^(2) for even v, R^(1) for odd v.  side_used
 * (host, may be NULL) receives QLR_SIDE_X or QLR_SIDE_XH.  With side X^H the roles of (m, n) and
 * of (Q1, Q2) are those of the algorithm run on A^H (Q1 is then n x l).
 * Errors: QLR_ESHAPE if k + p > min(m, n) or v < 2.
 */
int qlr_qrangefinder(qlr_ctx* ctx, const qlr_qmat* A, int k, int p, int passes, const qlr_qmat* omega,
                     const qlr_opts* opts, qlr_qmat* Q1, qlr_qmat* Q2, double* R, int* side_used);

/*
 * qlr_qsvd_lowrank -- rank-k approximation A ~= U diag(S) V^H by Algorithm 2 (algo = QLR_ALG2)
 * or Algorithm 4 (QLR_ALG4, with block width l = k + p) with exactly `passes` passes over A,
 * followed by the truncated QSVD of the last R and the lifts V = Q2 V_hat, U = Q1 U_hat.
 * QLR_ALG1 and QLR_ALG3 (the classical power scheme and block Krylov method with q power steps,
 * 2q + 2 passes; `passes` must be even, else QLR_ESHAPE) give, for the same Omega, the result of
 * Algorithm 2 and Algorithm 4 with that number of passes -- Section 3 shows Algorithm 2 with
 * v = 2q + 2 is Algorithm 1, and for even v Algorithm 4's stacked basis spans Algorithm 3's Krylov
 * matrix (Section 5) -- and run those schedules, with a QR after every product.
 * U: m x k, V: n x k, column-major, F32 or F64; S: device FP64 array of k values, descending.
 * The call leaves the result defined up to a right unit-quaternion factor per column pair.
 */
int qlr_qsvd_lowrank(qlr_ctx* ctx, const qlr_qmat* A, int k, int p, int passes, int algo,
                     const qlr_qmat* omega, const qlr_opts* opts, qlr_qmat* U, double* S, qlr_qmat* V);

/*
 * qlr_qbasis -- the orthonormal bases and the last R factor of a qlr_qsvd_lowrank call, before its
 * truncated QSVD: Algorithm 2 (and 1) return the last Q1, Q2 and R as qlr_qrangefinder does;
 * Algorithm 4 (and 3) return Q1 = QR(K1) (even v: the range basis of width L = (v/2) l) with
 * [Q2, R2] = QR(X^H Q1), or Q2 = QR(K2) (odd v: L = ((v-1)/2) l) with [Q1, R1] = QR(X Q2) (Section
 * 5, Algorithm 4).  These are the bases whose projection errors ||X - Q1 Q1^H X||_2 and
 * ||X - X Q2 Q2^H||_2 Lemma 1, Theorem 3, eqs. (mn11)/(mn12) and Theorem 6 bound (measure them with
 * qlr_residual_norm).  Arguments as qlr_qsvd_lowrank; Q1: rows_fwd x L and Q2: rows_bwd x L
 * column-major in the thin dtype (F64 for COMPUTE_F64, else F32), with rows_fwd = m, rows_bwd = n
 * on side X and swapped on side X^H; R: device FP64 L x L x 4 (R2 for even v, R1 for odd v);
 * side_used (host, may be NULL).  L = l for Algorithms 1 and 2.  Same errors as qlr_qsvd_lowrank.
 */
int qlr_qbasis(qlr_ctx* ctx, const qlr_qmat* A, int k, int p, int passes, int algo, const qlr_qmat* omega,
               const qlr_opts* opts, qlr_qmat* Q1, qlr_qmat* Q2, double* R, int* side_used);

/*
 * qlr_qblock_krylov -- Algorithm 4 (flexible block Krylov, Section 5) with block size b >= k:
 * the same as qlr_qsvd_lowrank(..., k, b - k, passes, QLR_ALG4, ...).
 */
int qlr_qblock_krylov(qlr_ctx* ctx, const qlr_qmat* A, int k, int b, int passes, const qlr_qmat* omega,
                      const qlr_opts* opts, qlr_qmat* U, double* S, qlr_qmat* V);

/*
 * qlr_qsvd_lowrank_batched -- `count` independent Algorithm 2 problems of uneven sizes (the
 * paper's patches / frames setting).  Arrays (host) of `count` descriptors / values; S[i] is a
 * device FP64 buffer of k[i] values; every problem runs on the side X.  When every A[i] is BF16
 * (or FP32 with a TF32 compute mode) with a 16-byte multiple row pitch and 16-byte aligned planes,
 * Omega[i], U[i], V[i] are FP32 and k[i] + p[i] <= 80, the call builds a batch plan (below) without tuning or graph,
 * runs it once and frees it; otherwise it loops over qlr_qsvd_lowrank.
 */
int qlr_qsvd_lowrank_batched(qlr_ctx* ctx, int count, const qlr_qmat* A, const int* k, const int* p,
                             int passes, const qlr_qmat* omega, const qlr_opts* opts, qlr_qmat* U,
                             double* const* S, qlr_qmat* V);

/*
 * Batch plans: the batched Algorithm 2 above, planned once and run many times.
 *
 * qlr_batch_create -- checks and plans `count` problems (conditions as above, and l = k + p <= 80
 * for every problem, else QLR_EUNSUPPORTED; compute AUTO means BF16 for BF16 A and 3xTF32 for
 * FP32 A; side must be AUTO or X).  Every step runs as one grouped launch over all the problems:
 * each sketch pass is one grouped tensor-core launch over every output tile (plus one grouped
 * staging launch); each CholeskyQR step is a grouped Gram (FP64-class on the tensor cores; FP32
 * in the last step of CholeskyQR2, whose input is already nearly orthonormal), a grouped Cholesky
 * (double-FP32, one CTA per problem, also forming R^{-1} and the running product of the R
 * factors in FP32) and a grouped thin x small product; the core QSVDs (FP32 one-sided Jacobi,
 * sigma from the converged column norms) and the lifts are one launch each.  At creation the plan allocates its
 * device memory (cudaMalloc), times the variants of the grouped sketch (tile order x one CTA per
 * tile or persistent CTAs x, for persistent CTAs, the tile shape: K elements per stage and the
 * widest column block) and keeps the fastest (the autotuner), runs the whole sequence once
 * (its results are valid), and captures it into a CUDA graph unless opts.flags has
 * QLR_FLAG_NO_GRAPH.  The pointers in A, omega, U, S, V are baked into the plan: later runs read
 * and write the same buffers.
 * qlr_batch_run -- enqueues one run on the context stream (asynchronous; errors of the device
 * side show in qlr_sync).  A plan made with QLR_FLAG_NO_GRAPH runs its launches eagerly; then,
 * with timing enabled on the context (qlr_set_timing), each kernel class of the run is counted
 * and timed in the context's statistics (a graph replay is not broken down).  qlr_batch_info -- plan facts.  qlr_batch_destroy -- synchronises and
 * frees the plan (b may be NULL).
 */
typedef struct qlr_batch qlr_batch;
typedef struct {
  int32_t lanes;           /* streams a run uses (1: every step is one grouped launch) */
  int32_t graph;           /* 1 when runs replay the captured CUDA graph               */
  int32_t tile_order;      /* grouped sketch variant chosen (0..15): bit 0 tiles with the longest
                              reduction first (else problem order), bit 1 persistent CTAs (else one
                              per tile), bit 2 128-byte stage rows (persistent, BF16/TF32 K-major
                              A), bit 3 column blocks of at most 64 (else 128)                   */
  int32_t sketch_launches; /* grouped launches per run (staging + sketch per pass)     */
  float tune_ms[16];       /* autotuner: N + H sketch time of each variant (ms; 0 when the variant
                              is not timed: tile shapes apply to the persistent form only) */
  int64_t launches_per_run;/* kernels launched per run (all streams)                  */
  int32_t stage_k;         /* chosen shape of the first pass's sketch: K elements per stage, */
  int32_t col_block_max;   /*   widest column block (MMA N; the MMA M is 128 rows),        */
  int32_t ring_stages;     /*   pipeline stages                                            */
  int32_t reserved;
} qlr_batch_stats;
int qlr_batch_create(qlr_ctx* ctx, int count, const qlr_qmat* A, const int* k, const int* p, int passes,
                     const qlr_qmat* omega, const qlr_opts* opts, qlr_qmat* U, double* const* S, qlr_qmat* V,
                     qlr_batch** out);
int qlr_batch_run(qlr_batch* b);
int qlr_batch_info(const qlr_batch* b, qlr_batch_stats* st);
int qlr_batch_destroy(qlr_batch* b);

/*
 * qlr_residual_norm -- measurement pass (not one of the method's passes): estimate
 * ||A - Q Q^H A||_2 (side == QLR_SIDE_X, Q m x l) or ||A - A Q Q^H||_2 (side == QLR_SIDE_XH,
 * Q n x l) -- the errors bounded by Lemma 1, Theorem 3 and eqs. (mn11)/(mn12) -- by `iters`
 * steps of block power iteration with `nvec` vectors started from `start` (column-major F32/F64,
 * n x nvec for side X, m x nvec for side X^H).  *out (host) receives the estimate: the largest,
 * over the steps, Rayleigh-Ritz value ||E x||_2 = sqrt(lambda_max(Y^H Y)) of the residual operator
 * E on the step's orthonormal block x (Y = E x), a lower bound that converges to the norm.
 * Synchronises the stream.
 */
int qlr_residual_norm(qlr_ctx* ctx, const qlr_qmat* A, const qlr_qmat* Q, int side, const qlr_qmat* start,
                      int iters, double* out);

/*
 * qlr_qcomplete_update -- the masked update of quaternion matrix completion (Section 7, eq. Step2):
 * C = mask .* M + (1 - mask) .* (U diag(S) V^H), mask the 0/1 pattern of observed entries.
 * M, C: m x n row-major, one dtype (F32 or F64); M may be pure (plane[0] == NULL: zero real part);
 * C needs all four planes and may be M itself (in place: only observed entries of M are read,
 * each by the thread that writes it).  mask: device uint8, m x n row-major with row stride
 * mask_ld >= n, non-zero = observed.  U: m x k and V: n x k column-major in the dtype of C (only
 * their first k columns are read); S: device FP64, k values.  k = 0 (U, S, V may be NULL) writes
 * the starting point P_Omega(M), zero at the unobserved entries.  The rank-k product is formed
 * tile by tile in registers (FP32 for F32, FP64 for F64) and never stored.
 * Errors: QLR_EINVAL (null pointers, layouts, dtypes), QLR_ESHAPE (sizes, k < 0),
 * QLR_EUNSUPPORTED (more than 65535 * 32 rows).
 */
int qlr_qcomplete_update(qlr_ctx* ctx, const qlr_qmat* M, const uint8_t* mask, int64_t mask_ld, const qlr_qmat* U,
                         const double* S, const qlr_qmat* V, int k, qlr_qmat* C);

/*
 * qlr_qcomplete -- quaternion matrix completion by alternating updates (Section 7, eqs. Step1 and
 * Step2): C = P_Omega(M), then `iters` times X = U diag(S) V^H, the rank-k approximation of C by
 * qlr_qsvd_lowrank(C, k, p, passes, algo, omega, opts), and C = mask .* M + (1 - mask) .* X.
 * Arguments as qlr_qcomplete_update and qlr_qsvd_lowrank, with C in the role of A (row-major; a
 * row pitch that is a multiple of 16 bytes lets the sketches run on the tensor cores) and U, V in
 * C's dtype.  The paper starts from no stated C; this call starts from P_Omega(M).  The same omega
 * serves every iteration.  On return C holds the last update and U, S, V the factors of the last
 * X.  The Gaussian smoothing the paper applies to images after each iteration is image
 * post-processing outside the operator and is not applied.
 * Errors: as the two calls; QLR_ESHAPE for iters < 1.
 */
int qlr_qcomplete(qlr_ctx* ctx, const qlr_qmat* M, const uint8_t* mask, int64_t mask_ld, int k, int p, int passes,
                  int algo, int iters, const qlr_qmat* omega, const qlr_opts* opts, qlr_qmat* C, qlr_qmat* U,
                  double* S, qlr_qmat* V);

/*
 * qlr_selftest_wait_timeout -- failure-detection self test (the paper has no counterpart):
 * launches one CTA that waits on an mbarrier nothing arrives at, through the bounded wait the
 * tensor-core pipelines use.  The wait gives up after its limit (1.5 s), records QLR_ETIMEOUT in
 * the context's device error word and the kernel returns: qlr_sync then returns QLR_ETIMEOUT
 * once, and later calls on the context run normally.  Nothing faults or traps.
 */
int qlr_selftest_wait_timeout(qlr_ctx* ctx);

/*
 * qlr_qsketch_noalloc -- the tensor-core sketch product of qlr_qsketch (same op, operands, layouts
 * and results, compute QLR_COMPUTE_TF32, QLR_COMPUTE_TF32X3 or QLR_COMPUTE_BF16) for callers that
 * cannot allocate device memory.  The paper has no counterpart; this is a deployment convenience.
 * Who cannot allocate: cudaMalloc may synchronise the whole device and takes a driver-wide lock,
 * so latency-critical serving loops keep it out of their steady state, and some host applications
 * give all device memory to their own pool allocator and forbid other allocations; neither can
 * create a qlr context (which allocates its error word and workspace).
 * No context: the call runs on `stream` (a cudaStream_t, NULL = legacy default stream) on that
 * stream's device (made current for the call, the caller's current device restored on return) and
 * takes all scratch memory from one fixed 128 MiB device array compiled into the library (every GPU
 * that loads it keeps those 128 MiB until the process exits; the size leaves room for the staged
 * operand and the stream-K partial tiles of every SM at l up to ~128 and K up to ~20000).  It calls no cudaMalloc / cudaFree.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress, with the
 * device current) and keeps it for the life of the process, so make the first call on each device
 * before any stream capture, and do not call this entry point on a device after a cudaDeviceReset
 * of it (the kept address would be stale).  The stream-K schedule uses as many CTAs as the array's
 * partial-tile space allows (up to one per SM).
 * The array is shared by all calls on a device and keeps the previous call's contents; each call
 * clears the parts that must start at zero.  Calls that overlap on the GPU (other streams or
 * threads) race on the array: serialise them.  `err` (device int, may be NULL) receives
 * QLR_ETIMEOUT if a bounded device wait gives up.
 * Degenerate sizes as qlr_qsketch: an empty Y launches nothing; an empty inner dimension writes Y = 0.
 * Errors: QLR_EINVAL / QLR_ESHAPE as qlr_qsketch; QLR_EUNSUPPORTED for a row pitch of A that is not
 * a multiple of 16 bytes; QLR_ENOMEM when the operands need more scratch than the 128 MiB array
 * (the staged thin operand alone needs 32 bytes per quaternion entry of X for TF32X3, 8 for BF16).
 */
int qlr_qsketch_noalloc(void* stream, int op, const qlr_qmat* A, const qlr_qmat* X, qlr_qmat* Y, int compute,
                        int* err);

#ifdef __cplusplus
}
#endif
#endif /* QLR_H */
