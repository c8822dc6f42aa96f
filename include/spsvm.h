/*
 * spsvm.h -- C ABI of libspsvm.so, a GB300 (sm_103a) implementation of the
 * sparse primal kernel SVM (SP-SVM) of "Parallel Support Vector Machines in
 * Practice" (Tyree, Gardner, Weinberger, Agrawal, Tran), Section 4,
 * "Sparse primal optimization", Eq. 4.
 *
 * Problem.  Given points x_1..x_n in R^d with labels y_i in {-1,+1}, an RBF
 * kernel k(x,z) = exp(-gamma ||x-z||^2) (Section 2) and lambda = 1/C, find a
 * basis J (indices of training points, grown greedily) and coefficients
 * beta minimising
 *     f(beta) = lambda/2 beta^T K_JJ beta + 1/2 sum_i max(0, 1 - y_i o_i)^2,
 *     o = K_nJ beta,
 * which is Eq. 4 divided by C with the bias dropped (Section 2 omits b).
 *
 * Conventions for every entry point below.
 *  - Pointers documented as "device" must be CUDA device (or managed)
 *    memory on the current device; "host" pointers are ordinary memory.
 *  - Matrices of points are row-major: element (i, k) of X is X[i*ldx + k],
 *    ldx >= d.  Float data are IEEE binary32 unless stated.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Step-level calls only enqueue work; they do not
 *    synchronise unless stated.
 *  - Every call returns SPSVM_OK (0) or a negative status code; no C++
 *    exception crosses the ABI.  spsvm_last_error() gives a message for the
 *    last failure on the calling thread.
 *  - Nothing here allocates device memory except spsvm_fit with a NULL
 *    workspace, spsvm_model_* (the model's own basis copy) and the
 *    batched / server entry points, which say so.
 */
#ifndef SPSVM_H
#define SPSVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SPSVM_OK               0
#define SPSVM_ERR_ARG         (-1)  /* invalid argument (shape, pointer, value) */
#define SPSVM_ERR_OOM         (-2)  /* workspace too small or allocation failed */
#define SPSVM_ERR_NOT_PD      (-3)  /* Newton matrix not positive definite even with jitter 1e-2 tr(H)/|J| */
#define SPSVM_ERR_NO_CONVERGE (-4)  /* max Newton steps reached; a model is still returned */
#define SPSVM_ERR_CUDA        (-5)  /* CUDA runtime or launch error */
#define SPSVM_ERR_TIMEOUT     (-6)  /* bounded device wait gave up */
#define SPSVM_ERR_BUSY        (-7)  /* server: request not admitted yet */

/* ---- arithmetic forms -------------------------------------------------- */
/* SPSVM_FP32: kernel block and Gram matrix in FP32 SIMT arithmetic.
 * SPSVM_BF16SPLIT: kernel block and Gram matrix on tcgen05 tensor cores
 *   with FP32 operands split into BF16 terms and FP32 accumulation.  The
 *   kernel block splits each point as x = hi + mid + lo (three BF16 terms,
 *   exact for FP32) and forms the six products hi hi, hi mid, mid hi,
 *   mid mid, hi lo, lo hi (the three dropped ones are below 2^-24 of |x z|):
 *   kernel values as accurate as FP32 arithmetic.  The Gram matrix reads the
 *   compact copy K_SJ split as hi + lo and forms all four products (the
 *   Newton matrix then carries 2^-17 relative rounding; the gradient, and
 *   with it the minimiser the Newton iteration converges to, come from the
 *   FP32 kernel values).
 * Both forms store the kernel matrix K_nJ in FP32.  In both the Newton
 * system is, by default, factored in FP32 and solved with FP64 iterative
 * refinement to normwise backward error 1e-11 (SPSVM_SOLVE_MIXED: the fit
 * takes the same Newton steps to the same minimiser as with an FP64 solve),
 * or factored in FP64
 * (SPSVM_SOLVE_FP64, and the fallback of the mixed solve when its FP32
 * factor breaks down or the refinement stalls). */
#define SPSVM_FP32    0
#define SPSVM_BF16SPLIT  1

/* Newton-system solvers (spsvm_options.newton_solver). */
#define SPSVM_SOLVE_MIXED 0
#define SPSVM_SOLVE_FP64  1

/* spsvm_options.score */
#define SPSVM_SCORE_HEURISTIC 0
#define SPSVM_SCORE_EXACT     1

/* The growth stop's epsilon in the paper's experiments (Section 5): pass it
 * as spsvm_options.growth_tol to stop growing J when the training error rate
 * falls by less than this per added basis vector (0 runs to the budget). */
#define SPSVM_GROWTH_EPS_PAPER 5e-6

/* ---- stored kernel matrix ---------------------------------------------- */
/* K_nJ stored basis-major: row j (one basis vector) holds k(x_i, x_{J_j})
 * for i = 0..n-1 contiguously.  format SPSVM_FP32: element (j, i) at
 * ((float*)data)[j*ld + i].  format SPSVM_BF16SPLIT (two BF16 planes): hi plane
 * at ((uint16_t*)data)[j*ld + i], lo plane at ((uint16_t*)data)[plane +
 * j*ld + i]; value = hi + lo.
 * ld and plane are in elements; ld >= n, ld % 8 == 0, data 16-byte aligned. */
typedef struct spsvm_kmat {
  void*   data;     /* device */
  int32_t format;   /* SPSVM_FP32 or SPSVM_BF16SPLIT */
  int32_t pad_;
  int64_t n;        /* points (columns of the stored matrix) */
  int64_t rows;     /* basis vectors stored */
  int64_t ld;       /* elements between consecutive rows */
  int64_t plane;    /* elements between hi and lo planes (BF16SPLIT only) */
} spsvm_kmat;

/* Points prepared once per X: squared norms and, for SPSVM_BF16SPLIT, the
 * three BF16 split planes (hi = bf16(x), mid = bf16(x - hi), lo = bf16(x -
 * hi - mid)), each n x ldh with the columns d..ldh-1 zero.  All pointers
 * device; X is borrowed. */
typedef struct spsvm_points {
  const float* X;   /* device, n x d row-major, leading dimension ldx */
  int64_t n, d, ldx;
  float*    norms;  /* device, n: ||x_i||^2 (FP64 accumulation, rounded) */
  uint16_t* hi;     /* device, n x ldh, or NULL for SPSVM_FP32 */
  uint16_t* lo;     /* device, n x ldh, or NULL */
  int64_t   ldh;    /* multiple of 64, >= d */
  uint16_t* mid;    /* device, n x ldh, or NULL */
} spsvm_points;

/* ======================================================================= */
/* Step-level entry points: one per step of the fit, in the order a Newton */
/* growth round runs them.  The fit below is built from exactly these.    */
/* ======================================================================= */

/* Row norms ||x_i||^2 of the RBF distance expansion
 * ||x - z||^2 = ||x||^2 + ||z||^2 - 2 x^T z (Section 2, RBF kernel); and for
 * precision == SPSVM_BF16SPLIT the hi / mid / lo planes.  Fills p->norms
 * (and p->hi, p->mid, p->lo), which the caller allocated.  Errors: ARG if a
 * pointer is NULL or n < 0, d < 1, ldx < d, ldh < d or ldh % 64 != 0. */
int spsvm_prepare_points(spsvm_points* p, int32_t precision, void* stream);

/* Kernel block (Section 2 RBF; Section 4: K_nJ, O(|J| n) memory):
 *   out row (row0 + c), column i  =  exp(-gamma * max(0, ||x_i||^2 +
 *   ||x_{idx[c]}||^2 - 2 x_i^T x_{idx[c]}))   for c < m, i < n.
 * idx: device, m indices into the points.  The dot products are formed in
 * `precision`; out->format selects the storage: FP32 (either form) or the
 * two BF16 planes (SPSVM_FP32 arithmetic only).  Requires row0 + m <=
 * out->rows.  scratch: device, at least
 * spsvm_kernel_block_scratch_bytes(m, d, precision) bytes (the BF16SPLIT form
 * gathers the m basis rows' three planes there; 0 bytes for SPSVM_FP32).
 * Errors: ARG, OOM (scratch too small). */
size_t spsvm_kernel_block_scratch_bytes(int64_t m, int64_t d, int32_t precision);
int spsvm_kernel_block(const spsvm_points* p, const int64_t* idx, int32_t m,
                       float gamma, int32_t precision, spsvm_kmat* out,
                       int64_t row0, void* scratch, size_t scratch_bytes, void* stream);

/* Basis-vector selection score (Section 4, "Basis vector selection": a
 * heuristic estimate of the loss reduction from adding each sampled
 * point).  For each candidate c = idx[k]:
 *   g_k = lambda * o[c] + sum_{i in S} (o_i - y_i) K_ic,
 *   h_k = lambda * 1   + sum_{i in S} K_ic^2,      (K_cc = 1 for RBF)
 *   delta_k = g_k^2 / (2 h_k),
 * with S = {i : y_i o_i < 1} and o = K_nJ beta (so o[c] = k_cJ beta).
 * This is the second-order estimate of the decrease of f from a new
 * coefficient beta_c started at 0.  Kernel values are computed in
 * `precision` and reduced without being stored.
 * y, o: device, n.  idx: device, kappa.  g, h, delta: device, kappa (FP64).
 * scratch: device, at least spsvm_score_scratch_bytes(n, d, kappa) bytes.
 * Errors: ARG, OOM (scratch too small). */
size_t spsvm_score_scratch_bytes(int64_t n, int64_t d, int32_t kappa);
int spsvm_score_candidates(const spsvm_points* p, const float* y, const float* o,
                           const int64_t* idx, int32_t kappa, float gamma,
                           double lambda, int32_t precision, double* g, double* h,
                           double* delta, void* scratch, size_t scratch_bytes,
                           void* stream);

/* Exact one-dimensional variant of the selection score (the variant the
 * paper's "estimate of the reduction" heuristic approximates): f restricted
 * to a new coefficient beta_c, every other coefficient fixed, is convex and
 * piecewise quadratic; for each candidate c = idx[k] its minimiser t[k]
 * (signed) is found exactly -- 33-point grid passes over the points counting
 * the margin crossings in each cell, as the line search does, until the
 * root's cell holds none -- and delta[k] = f(beta) - f(beta + t[k] e_c)
 * (FP64).  The candidates' kernel rows are computed once, in `precision`,
 * into scratch; then one cooperative launch (bounded grid barriers) runs
 * all candidates, in groups of the GPU's co-resident CTAs.  y, o: device, n;
 * idx: device, kappa; bias: device FP64, the model's b when o carries one
 * (the regulariser's term is lambda (o_c - b)), or NULL; delta, t: device
 * FP64, kappa (t may be NULL);
 * scratch: device, 256-byte aligned, spsvm_score_exact_scratch_bytes bytes.
 * A wait that gives up returns SPSVM_ERR_TIMEOUT. */
size_t spsvm_score_exact_scratch_bytes(int64_t n, int64_t d, int32_t kappa, int32_t precision);
int spsvm_score_candidates_exact(const spsvm_points* p, const float* y, const float* o,
                                 const int64_t* idx, int32_t kappa, float gamma, double lambda,
                                 int32_t precision, const double* bias, double* delta, double* t,
                                 void* scratch, size_t scratch_bytes, void* stream);

/* Candidate scores without any device allocation or caller scratch.  The
 * paper has no counterpart: this serves callers that must not allocate
 * device memory -- a serving loop whose HBM budget is owned by a pool it
 * does not control, a host framework whose allocator owns every device
 * byte, or code that may not call cudaMalloc because it would synchronise
 * the device.  Same arguments and results as spsvm_score_candidates, whose
 * per-tile partial sums go instead to a fixed 16 MiB array inside the
 * library (a file-scope __device__ array, held by every GPU that loads the
 * library until the process exits).  Limit:
 * spsvm_score_scratch_bytes(n, d, kappa) <= 16 MiB (e.g. n = 500,000,
 * d = 128, kappa = 256 needs 16.2 MB); larger sizes are rejected with SPSVM_ERR_ARG
 * before any work.  The first call on each device (made current) looks up the array's
 * device address (and so does the first call after the device's context was
 * made anew, e.g. after cudaDeviceReset); make that first call before any
 * stream capture.  Calls
 * share the array: calls whose work overlaps on the GPU (different streams
 * or devices' threads racing on one device) race on it, so serialise them.
 * Every call overwrites the partial sums it reads, so nothing needs
 * clearing between calls. */
int spsvm_score_candidates_noalloc(const spsvm_points* p, const float* y, const float* o,
                                   const int64_t* idx, int32_t kappa, float gamma,
                                   double lambda, int32_t precision, double* g, double* h,
                                   double* delta, void* stream);

/* Outputs and active set (Eq. 4): o = K_nJ beta (FP32 result, products in
 * FP32, sums of 32 terms promoted to FP64); active[i] = (y_i o_i < 1);
 * stats[0] = 1/2 sum_i max(0, 1 - y_i o_i)^2, stats[1] = #{y_i o_i <= 0},
 * stats[2] = |S|.  beta: device FP64, K->rows entries.  If beta is NULL, o
 * is taken as given (not recomputed) and only flags/stats are produced.
 * o, y: device n.  active: device n bytes.  stats: device 3 doubles.
 * scratch: device, spsvm_reduce_scratch_bytes(n) bytes. */
size_t spsvm_reduce_scratch_bytes(int64_t n);
int spsvm_outputs(const spsvm_kmat* K, const double* beta, const float* y,
                  float* o, uint8_t* active, double* stats, void* scratch,
                  size_t scratch_bytes, void* stream);

/* Forward product u = K_nJ v (Eq. 4's o = K_nJ beta for any v; used for
 * the line-search direction u = K_nJ d).  v: device FP64 (K->rows);
 * u: device FP32 (n).  If `accumulate`, u += K_nJ v instead. */
int spsvm_gemv(const spsvm_kmat* K, const double* v, float* u, int32_t accumulate,
               void* stream);

/* Active-set compaction and masked transposed products (gradient of
 * Eq. 4: grad f = lambda K_JJ beta + K_SJ^T (o_S - y_S); Newton right-hand
 * side r = K_SJ^T y_S):
 *   pos[i]  = number of active points before i (exclusive scan);
 *   Kc row j, column pos[i] = K row j, column i   for active i (if Kc != NULL),
 *             zero-filled up to Kc->n (a multiple of 128);
 *   w1out_j = sum_{i active} w1_i K_ji,  w2out_j = sum_{i active} w2_i K_ji
 *   (each optional: NULL skips it).
 * active: device n bytes; w1, w2: device FP32 n; outputs device FP64.
 * n_active: device int64, written with |S|.  Kc must have the format of K
 * (or, for an FP32 K, the two BF16 planes: each value is then split as
 * hi = bf16(v), lo = bf16(v - hi)), the same rows and Kc->n >= |S| rounded
 * up to 128 (Kc->n = round_up(n,128) is always enough).  scratch:
 * spsvm_compact_scratch_bytes(n, K->rows). */
size_t spsvm_compact_scratch_bytes(int64_t n, int64_t rows);
int spsvm_compact_active(const spsvm_kmat* K, const uint8_t* active,
                         const float* w1, const float* w2, double* w1out,
                         double* w2out, spsvm_kmat* Kc, int64_t* n_active,
                         int32_t* pos, void* scratch, size_t scratch_bytes,
                         void* stream);

/* Change of the active set (Section 4 reoptimisation: between Newton steps
 * the set S of points with y_i o_i < 1 changes by a few points, and the
 * Newton matrix by their kernel rows):
 *   D = {i : active[i] != ref[i]} in increasing i, *k_dev = |D|;
 * when |D| <= kmax also Wt[j*ldw + r] = K row j, column D_r (j < K->rows,
 * r < |D|; columns |D|..ldw-1 untouched) and sign[r] = +1 if D_r entered S
 * (active) and -1 if it left.  active, ref: device n bytes; Wt: device FP32,
 * K->rows x ldw, ldw >= kmax; sign: device FP32, kmax; k_dev: device int32.
 * scratch: spsvm_compact_scratch_bytes(n, 0) bytes. */
int spsvm_active_diff(const spsvm_kmat* K, const uint8_t* active, const uint8_t* ref, int32_t kmax,
                      float* Wt, int64_t ldw, float* sign, int32_t* k_dev, void* scratch,
                      size_t scratch_bytes, void* stream);

/* Masked Gram matrix (the generalised Hessian of Eq. 4 on the active set):
 *   H = lambda * K_JJ + Kc^T Kc,   Kc = K_SJ (compacted, rows = basis),
 * where K_JJ[a][b] = K row b at column J[a] (symmetrised).  The
 * contraction over the first ns columns of Kc runs in `precision` with FP32
 * partial sums per slice of 8192 points, combined in FP64.  H: device FP64,
 * m x m, leading dimension ldh, both triangles written.  J: device int64, m.
 * scratch: spsvm_gram_scratch_bytes(m, ns). */
size_t spsvm_gram_scratch_bytes(int64_t m, int64_t ns);
int spsvm_gram(const spsvm_kmat* Kc, const int64_t* ns_dev, int64_t ns_max,
               const spsvm_kmat* K, const int64_t* J, double lambda,
               int32_t precision, double* H, int64_t ldh, void* scratch,
               size_t scratch_bytes, void* stream);

/* FP64 Cholesky factorisation H = L L^T in place (lower triangle, read and
 * written), the direct solver of the Newton system of Section 4's
 * reoptimisation.  Blocked right-looking with 64 x 64 blocks.  On success
 * the strict upper triangle of each 64 x 64 diagonal block is overwritten
 * with the inverse of that block of L (transposed), which
 * spsvm_cholesky_solve uses; the rest of the upper triangle is not touched.
 * info: device int32, 0 on success, else k+1 for the first non-positive
 * pivot k (the factor is then incomplete).  Read info after a stream sync.
 * work: device, spsvm_cholesky_work_bytes(m) bytes, or NULL.  With work, the
 * trailing updates of the 64-column steps run on the tensor cores in an
 * FP64-faithful split form (each panel row scaled by a power of two and cut
 * into eight 7-bit integer slices, exact in BF16; the slice products are
 * exact integers in the FP32 accumulators and are recombined in FP64), so the
 * result matches the FP64 factorisation to within FP64 rounding; without
 * work every step runs in FP64 on the CUDA cores. */
size_t spsvm_cholesky_work_bytes(int64_t m);
int spsvm_cholesky(double* H, int64_t m, int64_t ldh, int32_t* info, void* work,
                   size_t work_bytes, void* stream);

/* Solves L L^T x = b in place (b overwritten by x), FP64: forward then
 * backward substitution over 64-row block rows, one launch each, one CTA
 * per block row; each CTA applies the solution blocks published before its
 * own (bounded flag waits; a wait that gives up leaves b incomplete and
 * spsvm_device_status reports TIMEOUT).  L from spsvm_cholesky (it uses the
 * diagonal-block inverses that spsvm_cholesky stores).  b: device FP64, m;
 * work: device, 16-byte aligned, spsvm_cholesky_solve_work_bytes(m) bytes
 * (overwritten); smaller work returns SPSVM_ERR_OOM.  The Newton direction
 * of Section 4's reoptimisation. */
size_t spsvm_cholesky_solve_work_bytes(int64_t m);
int spsvm_cholesky_solve(const double* L, int64_t m, int64_t ldh, double* b, void* work,
                         size_t work_bytes, void* stream);

/* Mixed-precision solve of the Newton system (H + shift I) x = b of
 * Section 4's reoptimisation: an FP32 Cholesky factor of H + shift I, then
 * iterative refinement with FP64 residuals until the normwise backward error
 * ||r||_inf / (||H + shift I||_inf ||x||_inf + ||b||_inf) is at most tol.
 * H: device FP64, m x m, full and symmetric, row pitch ldh, read only (not
 * overwritten, unlike spsvm_cholesky).  shift >= 0.
 * spsvm_cholesky_mixed converts and factors into work (device, 256-byte
 * aligned, spsvm_mixed_work_bytes(m) bytes); info: device int32, 0 on success,
 * else k+1 for the first non-positive FP32 pivot k.  The FP32 factor L is
 * the lower triangle of the first m rows x round_up(m, 4) floats of work
 * (row-major); the upper triangle of each 64 x 64 diagonal block holds that
 * block's inverse, transposed.  The factorisation is one launch over
 * 64 x 64 tiles whose bounded waits give up after about a second
 * (spsvm_device_status then reports TIMEOUT).  spsvm_solve_mixed then
 * solves for b (device FP64, m) into x (device FP64, m) with the factor in
 * work.  The first three refinement steps are queued at once (a step's
 * kernels return at once on the device when an earlier step reached tol),
 * then the stream is synchronised once, and once per further step; it
 * returns OK, or SPSVM_ERR_NO_CONVERGE when the residual stops shrinking (by
 * half per step, from the third step on) or max_iter steps do not reach tol
 * (x then holds the last iterate).  iters, backward_error: host, may be
 * NULL. */
size_t spsvm_mixed_work_bytes(int64_t m);
int spsvm_cholesky_mixed(const double* H, int64_t m, int64_t ldh, double shift, int32_t* info,
                         void* work, size_t work_bytes, void* stream);
int spsvm_solve_mixed(const double* H, int64_t m, int64_t ldh, double shift, const double* b,
                      double* x, int32_t max_iter, double tol, int32_t* iters,
                      double* backward_error, void* work, size_t work_bytes, void* stream);

/* Low-rank correction of the mixed solve's factor (Section 4
 * reoptimisation, the Newton system after the active set changed by k
 * points): H = H_a + W^T Sigma W, where H_a is the matrix whose FP32 factor
 * L (L L^T = H_a, no shift) spsvm_cholesky_mixed left in mixed_work, W
 * (k x m) holds the kernel rows of the k points and Sigma = diag(sign) (+1
 * entered, -1 left).  spsvm_lowrank_factor forms V = L^{-1} W^T (FP32, one
 * launch over 64 x 16 tiles with bounded flag waits), the capacitance
 * C = Sigma + V^T V and its inverse (FP32 Gauss-Jordan, partial pivoting)
 * in lr_work; info: device int32, 0, or p + 1 when pivot p of C is below
 * 1e-3 of its largest entry (C too ill-conditioned for its FP32 inverse:
 * factor H afresh).
 * spsvm_solve_lowrank then solves H x = b by iterative refinement with FP64
 * residuals of the given H (full, symmetric, FP64), each step applying
 * H^{-1} ~ L^{-T} (I - V C^{-1} V^T) L^{-1} (Sherman-Morrison-Woodbury), with
 * the stopping rules and results of spsvm_solve_mixed; it leaves the factor
 * and the correction intact, so later right-hand sides reuse them.
 * Wt: device FP32, m x ldw (ldw >= k); sign: device FP32, k;
 * 1 <= k <= SPSVM_LOWRANK_KMAX; lr_work: device, 256-byte aligned,
 * spsvm_lowrank_work_bytes(m, k) bytes (enough for every smaller m and k). */
#define SPSVM_LOWRANK_KMAX 128
size_t spsvm_lowrank_work_bytes(int64_t m, int32_t kmax);
int spsvm_lowrank_factor(void* mixed_work, size_t mixed_bytes, int64_t m, const float* Wt,
                         int64_t ldw, const float* sign, int32_t k, void* lr_work,
                         size_t lr_bytes, int32_t* info, void* stream);
int spsvm_solve_lowrank(const double* H, int64_t m, int64_t ldh, const double* b, double* x,
                        int32_t max_iter, double tol, int32_t* iters, double* backward_error,
                        void* mixed_work, size_t mixed_bytes, void* lr_work, size_t lr_bytes,
                        int32_t k, void* stream);

/* Exact line search along a Newton direction (f is convex and piecewise
 * quadratic along a line; Section 4's Newton reoptimisation):
 *   phi'(t) = a0 + a1 t - sum_i v_i max(0, m_i - t v_i),
 *   m_i = 1 - y_i o_i, v_i = y_i u_i, a0 = lambda d^T o_J, a1 = lambda d^T u_J,
 * where o_J, u_J are o, u at the basis points (K_JJ beta = o_J).  Returns in
 * *t_host (and t_dev if not NULL) the smallest t >= 0 with phi'(t) = 0,
 * found by bracketing on a 33-point grid and solving the linear piece
 * exactly once a grid cell holds no breakpoint m_i / v_i; t = 1 if
 * |phi'(1)| <= 1e-6 |phi'(0)|.  d: device FP64 (m); J: device int64 (m).
 * Synchronises the stream.  scratch: spsvm_line_scratch_bytes(n). */
size_t spsvm_line_scratch_bytes(int64_t n);
int spsvm_line_search(const float* o, const float* u, const float* y, int64_t n,
                      const double* d, const int64_t* J, int32_t m, double lambda,
                      double* t_host, double* t_dev, void* scratch,
                      size_t scratch_bytes, void* stream);

/* Decision values (Section 4, h(x) = w^T phi(x) restricted to the basis):
 *   out[i] = sum_{j<m} beta_j exp(-gamma ||q_i - b_j||^2)
 * for query rows q (nq x d, ldq) and basis rows b (m x d, ldb), computed
 * tile by tile without storing the kernel block.  beta FP64; out FP32.
 * SPSVM_FP32: FP32 SIMT dot products, beta_j k summed in FP64.
 * SPSVM_BF16SPLIT: the kernel block's tensor-core engine (basis rows and
 * queries split into three BF16 planes, six products: the dot products
 * carry FP32-level error), beta_j k summed in FP32 over groups of 32 basis
 * rows and the groups in FP64 in a fixed order (results do not depend on
 * the launch); queries go in passes of at most 32,768.
 * All device.  scratch: spsvm_decision_scratch_bytes(nq, m, d, precision)
 * bytes (SPSVM_BF16SPLIT: the basis planes, one pass of query planes and
 * the partial sums, about m d 6 + min(nq, 32768) (6 d + m / 8) bytes).
 * Errors: ARG, OOM (scratch too small). */
size_t spsvm_decision_scratch_bytes(int64_t nq, int64_t m, int64_t d, int32_t precision);
int spsvm_decision(const float* B, int64_t m, int64_t ldb, const double* beta,
                   const float* Q, int64_t nq, int64_t ldq, int64_t d, float gamma,
                   int32_t precision, float* out, void* scratch,
                   size_t scratch_bytes, void* stream);

/* ======================================================================= */
/* Whole fit and prediction                                                */
/* ======================================================================= */

typedef struct spsvm_model spsvm_model;   /* opaque, owned by the library */

/* Options; an all-zero struct selects every default. */
typedef struct spsvm_options {
  int32_t  candidates;     /* kappa, points sampled per selection round (0 -> 256) */
  int32_t  add_per_round;  /* q, basis vectors added per round (0 -> 64) */
  int32_t  max_newton;     /* Newton steps per reoptimisation (0 -> 50) */
  int32_t  precision;      /* SPSVM_FP32 (0) or SPSVM_BF16SPLIT */
  double   growth_tol;     /* Section 4 stop: (change in training error rate) /
                              (vectors added) < growth_tol; 0 -> run to budget.
                              Section 5 uses 5e-6. */
  double   rel_tol;        /* gradient level of the Newton stop (0 -> 1e-6): see spsvm_fit */
  uint64_t seed;           /* candidate draw: counter-based splitmix64 */
  const int64_t* initial_basis;  /* host, n_initial indices (fixed basis), or NULL */
  int32_t  n_initial;
  int32_t  fixed_basis;    /* nonzero: no growth rounds (J = initial_basis) */
  int32_t  refine;         /* refinement sweeps per Newton step against the exactly applied
                              H (two passes over K each); <= 0 -> none (default) */
  int32_t  record;         /* keep candidates / chosen per round for replay checks */
  void*    stream;         /* cudaStream_t for all work (NULL = default stream) */
  int32_t  newton_solver;  /* SPSVM_SOLVE_MIXED (0): FP32 factor + FP64 refinement to
                              normwise backward error 1e-11, FP64 factorisation when
                              that fails;
                              SPSVM_SOLVE_FP64: FP64 factorisation always */
  int32_t  score;          /* basis selection: SPSVM_SCORE_HEURISTIC (0), Section 4's
                              second-order estimate g^2 / (2h); SPSVM_SCORE_EXACT, the
                              exact one-dimensional decrease (spsvm_score_candidates_exact) */
  int32_t  bias;           /* nonzero: fit Eq. 4's bias b as an unregularised coordinate
                              (f(x) = k(x, X_J) beta + b; spsvm_model_bias reads it); 0: b = 0
                              as Section 2 does.  Not with refine > 0. */
  int32_t  lowrank;        /* nonzero: with SPSVM_SOLVE_MIXED and |J| >= 512, when the active
                              set changed by k <= min(64, |J| / 8) points since the unshifted
                              FP32 factor in hand was formed, correct that factor by their
                              low-rank term (spsvm_lowrank_factor) instead of factoring afresh
                              (a correction whose capacitance fails the pivot test, or whose
                              direction finds no descent, falls back to a fresh factor);
                              0 (default): factor afresh whenever the active set changes */
} spsvm_options;

/* Per-Newton-step record (kept for every fit). */
typedef struct spsvm_step {
  int32_t basis;           /* |J| during the step */
  int32_t active;          /* |S| before the step */
  double  gnorm;           /* ||grad f|| before the step */
  double  t;               /* line-search step taken (0 for the final check) */
  double  loss;            /* 1/2 sum max(0, 1 - y o)^2 after the step */
  int32_t errors;          /* #{y_i o_i <= 0} after the step */
  int32_t jitter;          /* diagonal jitter level l of the factorisation: H + 10^(l-10) tr(H)/|J| I
                              (-1: none); tried upwards from the fit's previous level */
  int32_t changed;         /* points whose active flag the step changed */
  int32_t solve;           /* how the Newton system was solved: SPSVM_NEWTON_* (0 when no
                              step was taken) */
} spsvm_step;

/* spsvm_step.solve */
#define SPSVM_NEWTON_NONE     0  /* no Newton system solved (final check) */
#define SPSVM_NEWTON_FACTOR   1  /* new factorisation of H (+ shift) */
#define SPSVM_NEWTON_REUSE    2  /* factor in hand, the active set unchanged */
#define SPSVM_NEWTON_LOWRANK  3  /* factor in hand plus the low-rank correction
                                    (spsvm_lowrank_factor) for the points that
                                    entered or left the active set */

/* Device bytes the fit needs for n points in d dimensions and the budget;
 * the fit lays out all its buffers inside one workspace of this size. */
size_t spsvm_fit_workspace_bytes(int64_t n, int64_t d, int32_t basis_budget,
                                 const spsvm_options* opt);

/* Trains SP-SVM (Section 4): cycles basis-vector selection (kappa random
 * candidates from the points not in J, scored as in
 * spsvm_score_candidates, the q best appended) and reoptimisation of Eq. 4
 * by Newton steps with exact line search, until |J| = basis_budget or the
 * growth stop fires.  X: device, n x d (ldx); y: device, n values +-1.
 * gamma > 0, lambda > 0, 1 <= basis_budget <= n.  The Newton iteration of a
 * round stops at ||grad|| <= tol; or, once ||grad|| <= rel_tol ||r|| (r =
 * K_SJ^T y_S), when the next Newton step is below 1e-5 ||beta|| (it is not
 * taken), or when a step that kept the active set
 * did not halve ||grad|| or found no descent (rounding level); once the
 * fit runs with a diagonal jitter (beta is then not determined beyond the
 * gradient), at ||grad|| <= max(rel_tol, 5e-6) ||r||; or at max_newton
 * (NO_CONVERGE).
 * workspace: device, spsvm_fit_workspace_bytes
 * bytes, or NULL to let the library allocate (and free) it.  On success
 * *out is a self-contained model (basis rows copied).  Returns OK,
 * NO_CONVERGE (model still returned), or an error (no model).
 * X and y are borrowed for the duration of the call only. */
int spsvm_fit(const float* X, int64_t n, int64_t d, int64_t ldx, const float* y,
              float gamma, double lambda, int32_t basis_budget, double tol,
              const spsvm_options* opt, void* workspace, size_t workspace_bytes,
              spsvm_model** out);

/* Decision values for nq query rows (device, nq x d, ldq) into decision
 * (device FP32, nq); label = +1 if decision >= 0 else -1.  Computed in the
 * model's precision form (spsvm_decision).  A model of the BF16SPLIT form
 * takes spsvm_predict_work_bytes(model, nq) bytes of device work memory per
 * call: spsvm_predict takes them stream-ordered (cudaMallocAsync /
 * cudaFreeAsync on `stream`, no device synchronisation); spsvm_predict_ws
 * uses the caller's `work` (device, work_bytes >= that size; NULL / 0 when
 * the size is 0).  Concurrent calls on one model are safe when each has its
 * own work memory.  Errors: ARG, OOM (work too small). */
size_t spsvm_predict_work_bytes(const spsvm_model* model, int64_t nq);
int spsvm_predict(const spsvm_model* model, const float* Xq, int64_t nq, int64_t ldq,
                  float* decision, void* stream);
int spsvm_predict_ws(const spsvm_model* model, const float* Xq, int64_t nq, int64_t ldq,
                     float* decision, void* work, size_t work_bytes, void* stream);

/* Model facts.  Any output pointer may be NULL. */
int spsvm_model_info(const spsvm_model* model, int32_t* n_basis, int64_t* d,
                     float* gamma, double* lambda, double* objective,
                     int32_t* newton_steps, int32_t* rounds, int32_t* status);
/* Device bytes the model holds (its basis rows, beta, prediction scratch). */
size_t spsvm_model_device_bytes(const spsvm_model* model);
/* Eq. 4's bias b of the model (0 unless fitted with spsvm_options.bias). */
int spsvm_model_bias(const spsvm_model* model, double* b);

/* Copies J (host int64, n_basis) and beta (host FP64, n_basis). */
int spsvm_model_get(const spsvm_model* model, int64_t* basis_idx, double* beta);
/* Per-step history: copies min(cap, steps) records; *count = steps. */
int spsvm_model_history(const spsvm_model* model, spsvm_step* out, int32_t cap,
                        int32_t* count);
/* Round r's candidate list and chosen list (record = 1 only). */
int spsvm_model_round(const spsvm_model* model, int32_t r, int64_t* candidates,
                      int32_t* n_candidates, int64_t* chosen, int32_t* n_chosen);
/* Final training outputs o = K_nJ beta (host FP32, n) as the fit left them. */
int spsvm_model_outputs(const spsvm_model* model, float* o, int64_t n);
void spsvm_free(spsvm_model* model);

/* Candidate draw used by the fit (exported so that checks can reproduce
 * it): the points not in J in increasing order, then a partial
 * Fisher-Yates shuffle whose k-th swap partner is k + R mod (m - k), with
 * R = splitmix64 finaliser of seed + (counter + 1) * 0x9E3779B97F4A7C15,
 * counter = round * 2^32 + k.  J, out: host.  Returns the count drawn. */
int32_t spsvm_draw_candidates(int64_t n, const int64_t* J, int32_t nJ, int32_t kappa,
                              uint64_t seed, uint32_t round, int64_t* out);

/* ======================================================================= */
/* Many fits at once (Section 5 trains one binary SP-SVM per class pair;    */
/* the grid of one-vs-rest classes x (gamma, lambda) and the request loop   */
/* below have no further counterpart in the paper).                          */
/* ======================================================================= */

/* One binary problem on rows of a shared X. */
typedef struct spsvm_problem {
  const int64_t* rows;     /* host, n_rows indices into X, or NULL for all rows */
  int64_t  n_rows;
  const float* y;          /* host, n_rows labels +-1 (for those rows, in order) */
  float    gamma;
  float    pad_;
  double   lambda;
  int32_t  basis_budget;
  int32_t  pad2_;
  double   tol;
  uint64_t seed;           /* candidate draw seed (0: the options' seed) */
} spsvm_problem;

/* Fits `count` problems on the shared device matrix X (n x d, ldx).  Work is
 * spread over `workers` host threads, each with its own CUDA stream and its
 * own device buffers (allocated here, freed on return), largest problem
 * first.  Each problem's result equals what spsvm_fit returns for it alone
 * (fixed reduction order; no cross-problem arithmetic).  outs[p] receives
 * the model (or NULL), status[p] the fit's status.  Returns OK, or the first
 * error with status[] telling which problems failed. */
int spsvm_fit_batched(const float* X, int64_t n, int64_t d, int64_t ldx,
                      const spsvm_problem* probs, int32_t count, const spsvm_options* opt,
                      int32_t workers, spsvm_model** outs, int32_t* status);

/* One-vs-one multiclass (Section 5 trains its multiclass sets one against
 * one).  labels: host int32, n entries in [0, classes), every class present;
 * 2 <= classes <= 64.  The C = classes (classes - 1) / 2 binary problems are
 * the pairs (a, b), a < b, in the order (0,1), (0,2), ..., (0,C-1), (1,2),
 * ...; problem (a, b) holds the rows of class a (y = +1) and class b
 * (y = -1) in X order, with the basis budget capped at its row count, and
 * all of them are fitted as one batch by spsvm_fit_batched (same options,
 * workers, ownership and status rules).  outs and status: host arrays of C
 * entries, in pair order. */
int spsvm_fit_ovo(const float* X, int64_t n, int64_t d, int64_t ldx, const int32_t* labels,
                  int32_t classes, float gamma, double lambda, int32_t basis_budget, double tol,
                  const spsvm_options* opt, int32_t workers, spsvm_model** outs,
                  int32_t* status);

/* Labels of nq queries (device, nq x d, row pitch ldq) by one-vs-one voting:
 * pair model p = (a, b) (pair order as above; models: host array of its C
 * models) votes a where its decision value is >= 0 and b otherwise; the
 * class with the most votes wins, a tie going to the smaller class.
 * labels: device int32, nq; votes: device int32 nq x classes (row-major) or
 * NULL; work: device, spsvm_predict_ovo_work_bytes(classes, nq) bytes (the
 * pair decision values).  Runs on `stream`. */
size_t spsvm_predict_ovo_work_bytes(int32_t classes, int64_t nq);
int spsvm_predict_ovo(const spsvm_model* const* models, int32_t classes, const float* Xq,
                      int64_t nq, int64_t ldq, int32_t* labels, int32_t* votes, void* work,
                      size_t work_bytes, void* stream);

/* Request loop.  Requests carry host data (copied at submission).  The
 * HBM budget counts the device bytes the server holds: every worker's
 * buffers (the fit's X, y and workspace; the predict's queries and results),
 * which a worker keeps and grows across requests, so that the loop
 * allocates no transient buffers and frees none; and every fitted model,
 * from the start of its fit until spsvm_server_release (or destroy).  A
 * request is admitted, in arrival order, when a worker is free and the bytes
 * that worker must add to run it (its buffers grown to the request's needs,
 * plus the model of a fit) fit in what is left of the budget; later
 * requests that fit run ahead of one that does not (continuous batching),
 * unless it has waited more than two seconds, when idle workers give their
 * buffers back until it fits.  A predict request is admitted once its fit
 * request has finished.  Workers own one CUDA stream each, so admitted
 * requests overlap on the device.  A request whose own needs exceed the
 * budget is refused at submission (SPSVM_ERR_OOM). */
typedef struct spsvm_server spsvm_server;
int spsvm_server_create(size_t hbm_budget_bytes, int32_t workers, spsvm_server** out);
int spsvm_server_submit_fit(spsvm_server* s, const float* X, int64_t n, int64_t d,
                            const float* y, float gamma, double lambda, int32_t basis_budget,
                            double tol, const spsvm_options* opt, int64_t* request_id);
int spsvm_server_submit_predict(spsvm_server* s, int64_t fit_request_id, const float* Xq,
                                int64_t nq, int64_t* request_id);
/* Waits up to timeout_s (negative: forever) for a request; TIMEOUT if it has
 * not finished.  latency_ms: submission to completion. */
int spsvm_server_wait(spsvm_server* s, int64_t request_id, double timeout_s, int32_t* status,
                      double* latency_ms);
/* Results of a finished request: decision values (host, cap >= nq) of a
 * predict, or the model of a fit (owned by the server until destroy). */
int spsvm_server_result(spsvm_server* s, int64_t request_id, float* decision, int64_t cap,
                        spsvm_model** model);
/* Frees the model of a finished fit request (predicts of it can no longer
 * be submitted; BUSY while some are pending) and returns its bytes to the
 * budget. */
int spsvm_server_release(spsvm_server* s, int64_t fit_request_id);
/* hbm_in_use / hbm_peak: the budget's current and largest count (bytes). */
int spsvm_server_stats(spsvm_server* s, int64_t* done, int64_t* queued, size_t* hbm_in_use,
                       size_t* hbm_peak);
void spsvm_server_destroy(spsvm_server* s);

/* ---- instrumentation (no paper counterpart: measurement support) ---- */
/* Number of CUDA kernel launches the library has issued in this process. */
uint64_t spsvm_launch_count(void);
/* Per-step kernel timing with CUDA events recorded on the launching stream
 * around each step's launches.  enable(1) clears the totals and starts
 * recording, enable(0) stops.  Slots: 0 kernel_block, 1 score, 2 outputs,
 * 3 gemv, 4 compact, 5 gram, 6 cholesky, 7 solve, 8 line_search,
 * 9 decision, 10 fit, 11 lowrank (spsvm_lowrank_factor).  read() waits for
 * the recorded events and returns the launch count, total milliseconds and
 * total algorithmic work (flops for kernel_block / score / gram / cholesky /
 * decision / lowrank, bytes for the HBM passes) of a slot.  `name` receives
 * a static string. */
int spsvm_profile_enable(int32_t on);
int spsvm_profile_read(int32_t slot, const char** name, int64_t* launches, double* ms,
                       double* work);

/* Status of the kernels that wait on the device (tensor-core kernel block,
 * score and Gram; the FP64 Cholesky update; the FP32 tile factorisation; the
 * triangular solves; the low-rank tile solve).  Every such wait is bounded;
 * a wait that gives up records a nonzero site code in the status word of
 * the stream its kernel runs on (one word per stream: work on other
 * streams never sees it), and the kernel returns without its result.
 * spsvm_stream_status waits for `stream`, then reads and clears its word;
 * returns OK, or TIMEOUT with *code set (site codes: 11-27 tensor-core
 * kernels, 101-102 the FP64 Cholesky update, 221-231 the factorisation and
 * solves).  spsvm_device_status is the same for the legacy default stream
 * (work enqueued with stream NULL).  The fits check their own stream.  The
 * library tracks up to 1024 streams; past that the least recently used
 * stream's word is reused. */
int spsvm_stream_status(void* stream, int32_t* code);
int spsvm_device_status(int32_t* code);
/* Poll limit of every bounded device wait launched from now on (0, the
 * default, restores each wait's own limit, about a second).  A small limit
 * makes waits give up early, for testing the timeout path: results of the
 * affected kernels are then incomplete and the status reports TIMEOUT. */
void spsvm_set_wait_limit(uint32_t polls);
/* Grid of every FP32 tile factorisation (spsvm_cholesky_mixed and the fits'
 * mixed Newton solves) launched from now on: at most `ctas` CTAs (0, the
 * default, one per SM).  One CTA completes the factorisation on its own (it
 * runs the chain of diagonal tiles and takes the other tiles' work while it
 * waits), so any grid gives the same factor; a small grid is slower and
 * serves to test that. */
void spsvm_set_factor_ctas(uint32_t ctas);

const char* spsvm_strerror(int code);
const char* spsvm_last_error(void);
/* Library version string and the SM architecture it was compiled for. */
const char* spsvm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPSVM_H */
