/*
 * tcprod.h -- C ABI of the GB300 (sm_103a) cosine-product Krylov library.
 *
 * The library solves min_X || M(X) - C ||_F with M(X) = A *c X or
 * M(X) = A *c X *c B (eq. (eq2), §1 of El Ichi, El Guide, Jbilou,
 * "Discrete cosine transform LSQR and GMRES methods for multidimensional
 * ill-posed problems", arXiv 2103.11847), by the tensor Golub-Kahan, LSQR and
 * GMRES methods of §3, regularised by Tikhonov with the GCV choice of lambda.
 *
 * Conventions for every call below.
 *  - Tensors are FP32 in device memory, owned by the caller, laid out
 *    slice-major: a tensor of size rows x cols x n3 is n3 consecutive frontal
 *    slices, each rows x cols row-major (element (i, j, k) at k*rows*cols +
 *    i*cols + j).
 *  - Sizes: A is n1 x n2 x n3, X is n2 x s x n3, C and Y are n1 x s x n3, B is
 *    s x s x n3 (two-sided only).
 *  - The c-product is Definition 2.1 (ten(mat(A) mat(X))), computed through
 *    the mode-3 transform M = W^{-1} C_{n3} (I + Z) of Remark 2.1: A~ = A x_3 M
 *    is formed once per plan and kept resident; each product transforms the
 *    operand, multiplies the n3 frontal slices and transforms back.
 *  - "Adjoint" means the adjoint for the inner product of Definition 2.2,
 *    X -> M^T [ A~_k^T (M^{-T} Y)_k (B~_k^T) ]; this is the A^T *c that
 *    Algorithms 4 and 6 use.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream) unless it says otherwise. Arguments are checked on
 *    the host before anything is launched.
 *  - Return value: TC_OK (0) or a negative tc_status. Device-side outcomes of a
 *    solve (convergence, breakdown, non-finite values) are reported in the
 *    tc_solve_info the solve writes to device memory.
 *  - A plan may be used from one host thread at a time; calls on one plan
 *    that overlap on the GPU (different streams) race on its workspaces.
 */
#ifndef TCPROD_H
#define TCPROD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-identical to cudaStream_t. */
typedef struct CUstream_st* tc_stream_t;

typedef struct tc_plan tc_plan;
typedef struct tc_mlp tc_mlp;

typedef enum {
  TC_OK = 0,
  TC_EINVAL = -1,      /* bad argument (null pointer, size, misaligned, ...) */
  TC_ECUDA = -2,       /* a CUDA runtime call failed (see tc_last_error) */
  TC_EBREAKDOWN = -3,  /* a Krylov process broke down (alpha, beta or h = 0) */
  TC_ENONFINITE = -4,  /* a norm or inner product was NaN or Inf */
  TC_ETIMEOUT = -5,    /* a bounded device wait gave up */
  TC_ENOMEM = -6,      /* device allocation failed */
  TC_EUNSUPPORTED = -7 /* valid request this build does not implement */
} tc_status;

typedef enum {
  TC_FP32 = 0, /* slice GEMMs in FP32 (FFMA)                         */
  TC_TF32 = 1, /* slice GEMMs on tensor cores, TF32 in, FP32 accumulate */
  TC_BF16 = 2, /* slice GEMMs on tensor cores, BF16 in, FP32 accumulate */
  TC_BF16X3 = 3 /* FP32-level on the tensor cores: each operand of the slice
                   GEMMs (and, for n3 > 32, of the tube transforms) is split into
                   three BF16 planes, x = x0 + x1 + x2 (x0 = bf16(x), x1 =
                   bf16(x - x0), x2 = bf16(x - x0 - x1)), and the six products
                   x_i y_j with i + j <= 2 accumulate in FP32. Products are
                   within the FP32 plans' 1e-5 bound (about 1e-6 relative, a few
                   times the FFMA path's, set by the tensor cores' accumulation) */
} tc_precision;

typedef enum {
  TC_GCV_PAPER = 0, /* eq. (gcv2) as printed (square-matrix form)           */
  TC_GCV_FULL = 1   /* GCV of the (k+1) x k projected least-squares problem */
} tc_gcv_variant;

typedef enum {
  TC_TH = 0,       /* A~ = A x_3 M, M = W^{-1} C (I + Z): Definition 2.1, Remark 2.1 */
  TC_ORTHODCT = 1  /* A~ = dct(A, [], 3): Algorithm 1 as printed (orthonormal DCT-II;
                      the slice transpose is then the adjoint) */
} tc_product;

/* Where c-LSQR keeps its Krylov vectors (results are the same up to rounding):
 *   TC_ROUTE_AUTO: ORTHODCT plans off the fused route iterate on dct(C)
 *     (Definition 2.2's norms are the DCT's); every other solve is spatial.
 *   TC_ROUTE_SPATIAL: every product transforms its operand in and its result
 *     out (Algorithm 1), and the iteration runs on spatial tensors. (With
 *     TC_STORE_BF16, c-LSQR solves that keep the basis form each product's
 *     BF16 operand in the pass back of the product before it.)
 *   TC_ROUTE_DUAL: as AUTO, except that solves that keep the basis (X_reg
 *     requested) on BF16 plans of the TH product, one-sided, 32 < n3 <= 64,
 *     iterate in the transform domains (the dual-domain route): V as
 *     V x_3 M^{-T}, U as U x_3 M, each product one tcgen05 GEMM with the
 *     Krylov update in its store plus one tube pass by G = M^{-T} M^{-1} (or
 *     G^{-1} = M M^T) that writes the next GEMM's BF16 operand and the norm of
 *     the spatial tensor; X and X_reg are transformed back once (by M^T) at
 *     the end. On the 512 x 512 x 64 video it measures as fast as the spatial
 *     route with FP32-stored products and slower than the spatial route with
 *     BF16-stored, chained products (tc_store), so AUTO keeps the spatial one. */
typedef enum { TC_ROUTE_AUTO = 0, TC_ROUTE_SPATIAL = 1, TC_ROUTE_DUAL = 2 } tc_route;

/* How the tensor-core slice products reach the transform back (Algorithm 1,
 * step 3) on the spatial route:
 *   TC_STORE_F32: in FP32, the accumulator as it is (default);
 *   TC_STORE_BF16: rounded once to BF16 (the accumulation stays FP32), and
 *     the pass back reads them by TMA straight into its tensor-core operand.
 *     Each product then moves a quarter less: the GEMM writes and the pass
 *     reads half the bytes. The error this adds (one BF16 rounding of each
 *     transformed product, next to the operand's) keeps the regularised
 *     reconstruction error within the precision form's 2% of FP32's.
 *     TC_BF16 plans only, one-sided, 32 < n3 <= 64; TC_EUNSUPPORTED else. */
typedef enum { TC_STORE_F32 = 0, TC_STORE_BF16 = 1 } tc_store;

typedef struct {
  int precision;   /* tc_precision */
  int gcv_variant; /* tc_gcv_variant */
  int use_graphs;  /* nonzero: solves replay a captured CUDA graph */
  int product;     /* tc_product (default TC_TH) */
  int route;       /* tc_route (default TC_ROUTE_AUTO) */
  int store;       /* tc_store (default TC_STORE_F32) */
  int reserved[2]; /* must be zero */
} tc_opts;

/* Outcome of a solve, written to DEVICE memory by the solve (copy it back
 * after the stream synchronises). */
typedef struct {
  int iters;     /* LSQR iterations / GMRES Arnoldi steps / GK steps done */
  int status;    /* 0 ran to itermax, 1 converged (residual < tol),
                    TC_EBREAKDOWN or TC_ENONFINITE */
  int cycles;    /* GMRES restart cycles */
  int fallback;  /* tc_lsqr_c_learned: 1 when GCV replaced the predicted lambda */
  double resid;  /* LSQR: |phibar_{k+1}| = ||C - M(X_k)||_F (§3.3);
                    GMRES: ||C - M(X)||_F at the last check */
  double lambda; /* Tikhonov parameter used (NaN if none) */
  double gcv;    /* GCV value at lambda (NaN if none) */
  double beta1;  /* ||C||_F */
  int kopt;      /* tc_lsqr_c_lcurve: the L-curve corner k_opt (0 otherwise) */
  int reserved;
} tc_solve_info;

/* Library version string, and the message of the last TC_ECUDA (or of a
 * TC_EINVAL whose reason is not obvious) on this thread. */
const char* tc_version(void);
const char* tc_last_error(void);

/* Plan: validates sizes, copies nothing back, forms A~ = A x_3 M (and B~)
 * once with its slice transposes, and keeps them with its workspaces in
 * device memory it allocates (freed by tc_plan_destroy).
 *   A: device, n1 x n2 x n3.   B: device s x s x n3, or NULL for A *c X.
 *   opts: may be NULL (FP32, paper GCV, graphs on, TH product).
 * Sizes must be >= 1; n3 <= 64. Synchronises `stream` before returning.
 * Source: Remark 2.1 and eqs. (dft9), (dft8), §2.2. */
int tc_plan_create(tc_plan** plan, int n1, int n2, int s, int n3,
                   const float* A, const float* B, const tc_opts* opts,
                   tc_stream_t stream);
int tc_plan_destroy(tc_plan* plan);

/* Y = A *c X [*c B] (Definition 2.1 via Algorithm 1 with M).
 *   X: device n2 x s x n3 (read).  Y: device n1 x s x n3 (written).
 * X and Y must not overlap. */
int tc_cprod(tc_plan* plan, const float* X, float* Y, tc_stream_t stream);

/* X = adjoint(Y) (the A^T *c of Algorithms 4 and 6).
 *   Y: device n1 x s x n3 (read).  X: device n2 x s x n3 (written). */
int tc_cprod_adjoint(tc_plan* plan, const float* Y, float* X, tc_stream_t stream);

/* Tensor Golub-Kahan bidiagonalisation, Algorithm 4 (§3.2), one step per call.
 *   U: device, (mmax+1) consecutive tensors n1 x s x n3 (U_1 .. U_{mmax+1}).
 *   V: device, (mmax+1) consecutive tensors n2 x s x n3 (V_1 .. V_{mmax+1}).
 *   alpha, beta: device double[mmax+1]; alpha[j-1] = alpha_j, beta[j-1] = beta_j.
 * tc_gkb_init writes beta_1 = ||C||_F, U_1 = C/beta_1, alpha_1, V_1.
 * tc_gkb_step(j), 1 <= j <= mmax, reads U_j, V_j, alpha_j, beta_j and writes
 * U_{j+1}, beta_{j+1}, V_{j+1}, alpha_{j+1}. A zero beta or alpha (breakdown)
 * leaves the new basis tensor zero; the caller sees it in beta/alpha. */
int tc_gkb_init(tc_plan* plan, const float* C, float* U, float* V,
                double* alpha, double* beta, int mmax, tc_stream_t stream);
int tc_gkb_step(tc_plan* plan, int j, float* U, float* V, double* alpha,
                double* beta, int mmax, tc_stream_t stream);

/* DC-LSQR, Algorithm 6 (§3.3), from X_0 = 0, then optionally Tikhonov/GCV on
 * the projected bidiagonal C~_k (§3.2, eqs. (normeq2), (gcv2), (xmlsqr)).
 *   C: device n1 x s x n3.   X: device n2 x s x n3, the LSQR iterate X_k.
 *   X_reg: device n2 x s x n3 or NULL. If given (then itermax <= 128), the
 *     basis V_1..V_k is kept in plan workspace and
 *     X_reg = V_k (*) y_lambda with lambda = `lambda` if it is >= 0, else the
 *     GCV minimiser (opts.gcv_variant).
 *   itermax: 1 .. 4096.  tol: stop when |phibar_{j+1}| < tol (0: never).
 *     |phibar_{j+1}| = ||C - M(X_j)||_F, so tol = eta ||N||_F with a known
 *     noise norm and eta slightly above 1 is the discrepancy principle named
 *     in §2 (reading R19): the first iterate whose residual reaches the noise.
 *   phibar_hist: device double[itermax] or NULL: |phibar_{j+1}| per iteration.
 *   info: device tc_solve_info (required). */
int tc_lsqr_c(tc_plan* plan, const float* C, float* X, float* X_reg,
              int itermax, double tol, double lambda, double* phibar_hist,
              tc_solve_info* info, tc_stream_t stream);

/* DC-LSQR stopped at the L-curve corner k_opt (§3.3, after Algorithm 6).
 * Runs up to kmax steps of Algorithm 6 from X_0 = 0 (tol as in tc_lsqr_c),
 * then takes the K steps done as the curve P_k = (log ||R_k||_F,
 * log ||X_k||_F), k = 1..K, and k_opt as the point of largest signed Menger
 * curvature (the curvature of the circle through P_{k-1}, P_k, P_{k+1},
 * positive for the L-curve's turn; smallest k on ties; k_opt = K when
 * K < 3). The norms come from LSQR's rotations: ||R_k||_F = |phibar_{k+1}|
 * and ||X_k||_F = ||y_k||_2 with R_k y_k = f_k, which equal the definitions
 * for the orthonormal basis of Algorithm 4.
 *   C: device n1 x s x n3.  X: device n2 x s x n3, the last iterate X_K.
 *   X_opt: device n2 x s x n3, X_{k_opt} = V_k (*) y_k (§3.1 eq. (xm)).
 *   kmax: 1 .. 128.  curve: device double[2 kmax] or NULL: ||R_k|| at
 *   [k-1] and ||X_k|| at [kmax + k - 1] for k <= K.
 *   info: device tc_solve_info (required): iters = K, kopt = k_opt,
 *   resid = ||R_{k_opt}||_F, lambda and gcv NaN.
 * Replayed as one captured CUDA graph like tc_lsqr_c when the plan allows. */
int tc_lsqr_c_lcurve(tc_plan* plan, const float* C, float* X, float* X_opt, int kmax,
                     double tol, double* curve, tc_solve_info* info, tc_stream_t stream);

/* Restarted DC-GMRES(m) with Tikhonov/GCV, Algorithms 2 and 3 (§3.1).
 * Needs a square operator: n1 == n2 (the input and output shapes agree).
 *   C: device n1 x s x n3.  X0: device or NULL (zero).  X: device, the result.
 *   m: restart length 1 .. 128.  itermax: total Arnoldi steps.
 *   lambda >= 0 fixes lambda; < 0 chooses it by GCV each cycle.
 *   info: device tc_solve_info (required). */
int tc_gmres_c(tc_plan* plan, const float* C, const float* X0, float* X,
               int m, int itermax, double tol, double lambda,
               tc_solve_info* info, tc_stream_t stream);

/* Batched c-LSQR over independent problems of uneven sizes. This is the batched
 * form of the solver of Algorithm 6 (§3.3) with the Tikhonov/GCV projection.
 * tc_batch_create makes one plan per problem (one-sided, shared n3 and opts):
 *   n1, n2, s: host arrays[count]; A: host array[count] of device pointers,
 *   A[i] of size n1[i] x n2[i] x n3. Synchronises `stream`.
 * tc_lsqr_c_batched solves problem i exactly as tc_lsqr_c would on plan i, with
 * the same itermax, tol and lambda for all:
 *   C, X: host arrays[count] of device pointers (C[i]: n1[i] x s[i] x n3,
 *   X[i]: n2[i] x s[i] x n3). X_reg: host array of device pointers or NULL.
 *   infos: device array of count tc_solve_info.
 * Two forms, both replayed as one CUDA graph cached while the pointers and
 * parameters stay the same:
 *  - grouped (FP32 plans, or BF16 plans of the default product, with
 *    n3 <= 4 and X_reg given; BF16 plans also need n1, n2, s multiples of 8
 *    and every C[i] 16-byte aligned):
 *    every phase of the solve is one launch over all problems (a (problem,
 *    tile) work table, each problem's own scalars, flags and deterministic
 *    reductions), about 3 itermax + 10 launches a batch. The products fuse
 *    both mode-3 transforms: FFMA tiles for FP32 plans, tcgen05 tiles (BF16
 *    operands, FP32 accumulation) for BF16 plans. The tile shape is chosen
 *    on the first call by timing each candidate on the batch's forward
 *    product. Results equal tc_lsqr_c's up to the order of FP32 additions
 *    (the single solve may split K over a cluster, or run the BF16 transform
 *    as its own pass);
 *  - otherwise every problem's solve is captured as one child graph, side by
 *    side in one parent graph, results bit for bit tc_lsqr_c's. */
typedef struct tc_batch tc_batch;
int tc_batch_create(tc_batch** batch, int count, const int* n1, const int* n2, const int* s,
                    int n3, const float* const* A, const tc_opts* opts, tc_stream_t stream);
int tc_batch_destroy(tc_batch* batch);
int tc_lsqr_c_batched(tc_batch* batch, const float* const* C, float* const* X,
                      float* const* X_reg, int itermax, double tol, double lambda,
                      tc_solve_info* infos, tc_stream_t stream);
/* mode 0: the grouped form where the plans allow it, tile shape autotuned (the
 * default); 1: child graphs always; 2 + t: the grouped form with tile shape t
 * (no autotuning; a t the plans do not have gives TC_EINVAL at the next
 * solve); -1: unchanged. Writes (host, each may be NULL) whether the last
 * solve ran grouped, the tile shape in use (-1 before the first grouped
 * solve) and the candidates' forward-product times in ms (tune_ms[3], zero
 * where not timed). Tile shapes: FP32 plans 0: 64 x 64 tiles of 4 x 4 a
 * thread, 1: 32 x 32 of 4 x 2, 2: 64 x 64 of 8 x 4; BF16 plans 0: 128 x 64,
 * 1: 128 x 128. */
int tc_batch_info(tc_batch* batch, int mode, int* grouped, int* tile, float* tune_ms);

/* ---- Learned lambda and stopping index --------------------------------------
 * None of this has a counterpart in the paper. A small network stands in for the
 * per-solve GCV search (§3.1, eq. (gcv2)) and for the choice of the stopping
 * index (§3.3, k_opt); GCV stays as the fallback. The network is
 *   36 -> 64 -> 64 -> 2, GELU, W row-major (in x out), parameters one FP32
 *   vector [W1 | b1 | W2 | b2 | W3 | b3] of TC_MLP_NPARAMS values; the forward
 *   pass uses BF16 copies of the weights with FP32 accumulation.
 * Inputs (36, from the first 12 c-LSQR steps): log(alpha_i / beta_1),
 *   log(beta_{i+1} / beta_1), log(|phibar_{i+1}| / beta_1), i = 1..12.
 * Outputs: (log lambda, stopping index). The normalisation vector `norm`
 *   (TC_MLP_NORM values: input means[36], input stds[36], output means[2],
 *   output stds[2]) maps raw features and targets to network units; the
 *   training calls take data already normalised. */
#define TC_MLP_NPARAMS 6658
#define TC_MLP_NORM 76
int tc_mlp_create(tc_mlp** mlp, unsigned long long seed, tc_stream_t stream);
int tc_mlp_destroy(tc_mlp* mlp);
/* theta: device FP32[TC_MLP_NPARAMS] or NULL; norm: device FP32[TC_MLP_NORM] or NULL.
 * Setting theta resets the Adam state. */
int tc_mlp_set_params(tc_mlp* mlp, const float* theta, const float* norm, tc_stream_t stream);
int tc_mlp_get_params(tc_mlp* mlp, float* theta, float* norm, tc_stream_t stream);
/* Y (device B x 2) = network(X (device B x 36)), normalised units. */
int tc_mlp_forward(tc_mlp* mlp, const float* X, int B, float* Y, tc_stream_t stream);
/* loss = (1/2B) sum (Y - T)^2 and its gradient for one batch (B <= 1024):
 * loss: device float or NULL, grad: device FP32[TC_MLP_NPARAMS]. */
int tc_mlp_loss_grad(tc_mlp* mlp, const float* X, const float* T, int B, float* loss,
                     float* grad, tc_stream_t stream);
/* Set the network's normalisation from raw training data (N rows): column means
 * and standard deviations of Xraw (N x 36) and Traw (N x 2); writes the
 * normalised copies Xn, Tn (device, same shapes). */
int tc_mlp_fit_norm(tc_mlp* mlp, const float* Xraw, const float* Traw, int N, float* Xn,
                    float* Tn, tc_stream_t stream);
/* `steps` Adam steps (beta 0.9, 0.999, eps 1e-8, rate lr) on consecutive
 * batches of X (N x 36), T (N x 2), wrapping around; loss_hist: device
 * float[steps] or NULL. */
int tc_mlp_train(tc_mlp* mlp, const float* X, const float* T, int N, int batch, int steps,
                 float lr, float* loss_hist, tc_stream_t stream);
/* Training data from one solve: kmax (13 .. 128) steps of c-LSQR on C, then
 * the features (device float[36]) and the target (device float[2]):
 *   k_opt  = the smallest k in {4, 6, .., kmax} whose best error over lambda
 *            is within 1% of the best over all k, and
 *   lambda = the lambda that minimises the error at k_opt.
 * The error is ||V_k y_k(lambda) - X_true||_F, taken exactly from the Gram
 * matrix of the kept basis V, with lambda on 48 log-spaced values in
 * [1e-6, 1] ||C~_kmax||_F. */
int tc_lsqr_label(tc_plan* plan, const float* C, const float* X_true, int kmax, float* feat,
                  float* target, tc_stream_t stream);
/* c-LSQR with the learned stop index and lambda, all on the device. It runs
 * 12 steps, predicts (lambda, k), continues to min(k, kmax) steps, then
 * forms X_reg = V_k (*) y_lambda. If GCV(lambda) exceeds gcv_factor times the
 * GCV minimum (opts.gcv_variant), the GCV lambda is used and info.fallback = 1.
 *   kmax: 13 .. 128. X: the LSQR iterate. X_reg: required. info: device. */
int tc_lsqr_c_learned(tc_plan* plan, const tc_mlp* mlp, const float* C, float* X, float* X_reg,
                      int kmax, double gcv_factor, tc_solve_info* info, tc_stream_t stream);

/* Step 2 of Algorithm 1 alone: the n3 frontal-slice products in the transform
 * domain, Y~_k = A~_k X~_k (adjoint = 0) or Y~_k = A~_k^T X~_k (adjoint = 1),
 * with A~ = A x_3 M held by the plan (eqs. (dft9), (dft8)). One-sided plans only.
 *   Xh: device, n3 slices of K x s (K = n2, or n1 for the adjoint), in the
 *       plan's GEMM input type: FP32 for TC_FP32 plans, BF16 for TC_BF16, FP32
 *       already rounded to TF32 for TC_TF32, and for TC_BF16X3 three BF16 planes
 *       of n3 K s values each (x0, x1, x2 as above, plane q at Xh + q n3 K s).
 *   Yh: device FP32, n3 slices of M x s (M = n1, or n2 for the adjoint).
 * On the tensor-core forms this is one tcgen05 GEMM launch. */
int tc_slice_gemm(tc_plan* plan, const void* Xh, float* Yh, int adjoint, tc_stream_t stream);

/* The same slice products with Algorithm 4's update in their store (one
 * Golub-Kahan half-step in the transform domain, normalisation deferred):
 *   Yh = (1/s0) (A~_k Xh_k) - (s0/s1) prev   (prev non-NULL), or
 *   Yh = (1/s0) (A~_k Xh_k)                  (prev NULL; s1 unused);
 * adjoint = 1 takes A~_k^T. s0, s1: device doubles (s0 = 0 gives a zero
 * product term, s1 = 0 a zero prev term). prev: device FP32 like Yh, may
 * alias Yh. sumsq: device double for ||Yh||_F^2 (the library's
 * deterministic reduction), or NULL. Xh: BF16 as for tc_slice_gemm. TC_BF16
 * one-sided plans only (TC_EUNSUPPORTED otherwise); one tcgen05 launch, the
 * GEMM the dual-domain c-LSQR route runs. */
int tc_slice_gemm_gk(tc_plan* plan, const void* Xh, float* Yh, int adjoint, const double* s0,
                     const double* s1, const float* prev, double* sumsq, tc_stream_t stream);

/* Steps 1 and 3 of Algorithm 1 alone: the mode-3 transform of Remark 2.1,
 * out = in x_3 T (+ prev), on the plan's transform matrices:
 *   which: TC_M (M, forward), TC_MINV (M^{-1}, inverse), TC_MINVT (M^{-T}, the
 *   adjoint's forward transform) or TC_MT (M^T, the adjoint's inverse).
 *   in, out: device FP32, n3 slices of P values each (slice k at k P).
 *   P: 1 .. max(n1, n2) s. prev: device, same layout, or NULL; when given,
 *   out = in x_3 T + prev. sumsq: device double or NULL: ||out||_F^2 by the
 *   library's deterministic reduction.
 * It runs the pass the plan's products run: the tcgen05 form (operands split
 * into BF16 planes) for TF32/BF16/BF16X3 plans with n3 > 32, the FP32 pass
 * otherwise. A bounded wait that gives up sets the plan's status to
 * TC_ETIMEOUT (tc_plan_status). `in` must not alias out or prev. */
typedef enum { TC_M = 0, TC_MINV = 1, TC_MINVT = 2, TC_MT = 3 } tc_transform_kind;
int tc_transform(tc_plan* plan, int which, const float* in, float* out, size_t P,
                 const float* prev, double* sumsq, tc_stream_t stream);

/* tc_transform from BF16 input, the pass back that plans with TC_STORE_BF16
 * run (Algorithm 1's step 3 on BF16-stored slice products): out = in x_3 T
 * (+ prev), sumsq as for tc_transform. in: device BF16, n3 slices of P
 * values, 16-byte aligned, P a multiple of 8; out, prev: device FP32, same
 * layout (prev may not alias out). One tcgen05 pass: the input lands by TMA
 * straight in the tensor-core operand (one BF16 plane times the transform's
 * two).
 * nxt (device BF16, same layout, or NULL): the same pass also writes
 * nxt = bf16(out x_3 T_next), T_next chosen by which_next (TC_M .. TC_MT),
 * from out's FP32 values split into two BF16 planes, as tc_transform's BF16
 * form would from out. This is the first step of the product that follows
 * (c-LSQR chains its products this way). nxt may not alias in, out or prev.
 * TC_STORE_BF16 plans only, else TC_EUNSUPPORTED. */
int tc_transform_bf16in(tc_plan* plan, int which, const void* in, float* out, size_t P,
                        const float* prev, double* sumsq, int which_next, void* nxt,
                        tc_stream_t stream);

/* The change of domain of the dual-domain c-LSQR route (tc_route): the
 * forward product's result lives in the M domain (U^ = U x_3 M) and the
 * adjoint's operand in the M^{-T} domain, so between them
 *   which = TC_DUAL_U: out = bf16(in x_3 G), G = M^{-T} M^{-1}, and
 *                      *sumsq = ||in x_3 M^{-1}||_F^2 = ||U||_F^2;
 *   which = TC_DUAL_V: out = bf16(in x_3 G^{-1}), G^{-1} = M M^T, and
 *                      *sumsq = ||in x_3 M^T||_F^2 = ||V||_F^2 (in = V x_3 M^{-T}).
 * Definition 2.2's norm is taken of the spatial tensor, which the pass forms
 * from the same split BF16 planes of `in` (two planes, error near 2^-16 a
 * term) and reduces without storing. One tcgen05 pass.
 *   in: device FP32, n3 slices of P values (slice k at k P); out: device
 *   BF16, same layout; both 16-byte aligned, P a multiple of 8,
 *   P n3 <= max(n1, n2) s n3. sumsq: device double.
 * Plans of the dual-domain route only (TC_TH, TC_BF16, one-sided,
 * 32 < n3 <= 64, route TC_ROUTE_DUAL); TC_EUNSUPPORTED otherwise. */
typedef enum { TC_DUAL_U = 0, TC_DUAL_V = 1 } tc_dual_kind;
int tc_transform_dual(tc_plan* plan, int which, const float* in, void* out, size_t P,
                      double* sumsq, tc_stream_t stream);

/* The plan's device status word (TC_OK, or TC_ETIMEOUT once a bounded wait of
 * its tensor-core kernels gave up), copied to the host *status. Synchronous. */
int tc_plan_status(tc_plan* plan, int* status);

/* Kernel launches in the plan's captured c-LSQR graph (tc_lsqr_c and
 * tc_lsqr_c_lcurve with opts.use_graphs): every replay launches all of them,
 * including those that return at once after an early stop. *count = 0 when no
 * graph is cached. Host int. */
int tc_lsqr_graph_kernels(tc_plan* plan, int* count);

/* Self-check of the FP64 reciprocal and inverse square root that the solvers
 * use for their step scalars and epilogue coefficients (Newton's method from
 * the hardware estimates inside [DBL_MIN, 2^1000], IEEE division and square
 * root outside it): rcp[i] = 1/x[i], rsqrt[i] = 1/sqrt(x[i]) for x[i] > 0
 * (0 otherwise). x, rcp, rsqrt: device double[n], 1 <= n <= 2^28. */
int tc_check_recip(const double* x, size_t n, double* rcp, double* rsqrt,
                   tc_stream_t stream);

/* Peak-rate probe (the paper has no counterpart): a fixed amount of
 * independent arithmetic for the caller to time with CUDA events, giving the
 * measured peaks that the roofline fractions of FFMA-bound and TF32 kernels
 * divide by.
 *   kind 0: FP32 FFMA, 8 CTAs x 256 threads a SM, each thread iters x 8
 *           independent FMAs (flops = 2 * 8 * iters * threads);
 *   kind 1: the same in FP64;
 *   kind 2: tcgen05.mma kind::tf32, one CTA a SM, iters x 4 MMAs of
 *           128 x 256 x 8 (flops = 2 * 128 * 256 * 32 * iters * SMs);
 *   kind 3: tcgen05.mma kind::f16 with BF16 inputs, iters x 4 MMAs of
 *           128 x 256 x 16 (flops = 2 * 128 * 256 * 64 * iters * SMs).
 *   iters: 1 .. 2^24.  status: device int, zero before the call; set to
 *   TC_ETIMEOUT if the bounded wait for the MMAs gave up. */
int tc_peak_probe(int kind, int iters, int* status, tc_stream_t stream);

/* Tikhonov solution of a projected problem with GCV (§3.1, eqs. (leastsq),
 * (tikho2), (gcv2)): y = argmin ||beta e_1 - H y||^2 + lambda^2 ||y||^2.
 *   H: device double, (k+1) x k row-major (Hessenberg or lower bidiagonal).
 *   k: 1 .. 128.   beta: device double scalar.
 *   lambda_in >= 0 fixes lambda; < 0 minimises GCV (variant tc_gcv_variant).
 *   lambda_out: device double.  y: device double[k].  gcv_out: device or NULL. */
int tc_tikhonov_gcv(const double* H, int k, const double* beta, int variant,
                    double lambda_in, double* lambda_out, double* y,
                    double* gcv_out, tc_stream_t stream);

/* Frobenius norm ||X||_F of n FP32 values, written to *out (device double),
 * without allocating any device memory. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as code
 * whose device memory belongs to another allocator that has reserved the
 * device, or code that cannot accept the device synchronisation that
 * cudaMalloc and cudaFree may imply.
 *   X: device, n floats (read).  out: device double (written).
 *   n: 1 .. 79691776 (4864 CTAs x 256 threads x 64 values); larger n returns
 *      TC_EINVAL and tc_last_error() says why.
 * It computes the same reduction as the norm that tc_gkb_init writes to
 * beta[0]: the same grid, per-thread FP32 sums, then an FP64 tree in a fixed
 * order. Its scratch is a 39 KB array in the library's static device memory,
 * held by every GPU that loads the library until the process exits.
 * The first call on each device looks up that array's address with that
 * device current; make this first call before any stream capture. All calls
 * on a device share the array, so calls that overlap on the GPU (different
 * streams, or other host threads) race and must be serialised by the caller.
 * Each call clears the array's arrival counter on `stream` before its kernel. */
int tc_fro_norm_noalloc(const float* X, size_t n, double* out, tc_stream_t stream);

/* Self-check of the bounded-wait path. Every wait in the tensor-core kernels
 * polls an mbarrier a bounded number of times and, if the copies or MMAs it
 * waits for never arrive, reports TC_ETIMEOUT (in the plan's error status or
 * tc_solve_info) instead of hanging the GPU. This call runs one such wait on a
 * barrier that nothing arrives on and writes the outcome to *status.
 *   spins: 1 .. 2^20 polls.  status: device int, written with TC_ETIMEOUT
 *   (TC_OK would mean the wait completed, which it cannot).
 * When a wait gives up, the kernel waits once more (bounded) for the copies
 * and MMAs it has already issued before it frees its tensor memory and returns
 * (the slice GEMM and the tensor-core transform pass alike).
 * No fault or trap is involved; the context stays usable. */
int tc_check_bounded_wait(int spins, int* status, tc_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TCPROD_H */
