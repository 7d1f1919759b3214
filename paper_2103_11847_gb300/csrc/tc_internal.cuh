// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "tcprod.h"

// Slices handled by one CTA when the mode-3 transform is fused into the slice
// GEMM (prologue on the operand, epilogue back to the spatial domain). Larger
// n3 takes the unfused route: a transform pass, per-slice GEMMs, a transform
// pass with the Krylov epilogue.
#define TC_MAX_FUSED 4
#define TC_MAX_N3 64
// TF32/BF16 plans run the mode-3 transforms on the tensor cores for n3 above
// this: the FP32 pass does 2 n3 FLOP per value it moves and is bound by FP32
// issue at large n3; at or below this both are bound by HBM, and the FP32
// pass has less fixed work per CTA.
#define TC_TUBE_MIN_N3 32
#define TC_MAX_PROJ 128  // largest projected problem (k) on the device

// ---------------------------------------------------------------- epilogue --
// Every product and transform pass ends in
//     out = ca * value + cp * prev
// where (ca, cp) follow `rule` from device scalars s0, s1 (one thread reads
// them and shares through shared memory), optionally followed by a reduction
// of out (sum of squares, or dot with `other`) into a deterministic two-level
// tree: one FP64 partial per CTA, summed in CTA order by the last CTA.
enum CoefRule : int {
  COEF_ONE = 0,    // ca = 1,       cp = 0
  COEF_RESID = 1,  // ca = -1,      cp = 1       (R = C - M(X))
  COEF_GK = 2,     // ca = 1/s0,    cp = -s0/s1  (Golub-Kahan with deferred normalisation)
  COEF_INV = 3,    // ca = 1/s0,    cp = 0
  COEF_NEG = 4,    // ca = -1,      cp = 0
  COEF_AXPY = 5,   // ca = 1,       cp = -s0
  COEF_ADD = 6     // ca = 1,       cp = 1
};

struct Coef {
  int rule = COEF_ONE;
  const double* s0 = nullptr;
  const double* s1 = nullptr;
};

struct Red {
  double* out = nullptr;          // nullptr: no reduction
  const float* other = nullptr;   // nullptr: sum of squares; else <out, other>
  int sqrt_out = 0;               // write sqrt of the sum
  double* partials = nullptr;     // >= gridDim.x*gridDim.y*gridDim.z doubles
  unsigned* ticket = nullptr;     // zero before the launch; reset by the last CTA
  int* status = nullptr;          // set to TC_ENONFINITE when the sum is not finite
};

struct Epi {
  Coef coef;
  const float* prev = nullptr;    // same layout as the output, may alias it
  Red red;
  const int* skip = nullptr;      // nonzero: the whole kernel returns at once
};

// One LSQR step (Algorithm 6 steps (c)-(g), iteration j, 0-based): the Givens
// recurrences on the device scalars and the X, W (and basis) updates. Run by
// its own kernel, or by the CTAs of the next forward product before their
// GEMM (n == 0: no step). done_in = done[j] gates it; done_out = done[j+1] is
// written by CTA 0. flags: [1] iterations, [2] status. With X null the step
// is its scalars alone: the solve keeps the basis and forms X_k = V_k y_k
// from it once at the end (launch_lsqr_scalars, launch_lsqr_coeffs).
struct LsqrStep {
  float* X = nullptr;
  float* W = nullptr;
  const float* V = nullptr;       // V~_{j+1} (unnormalised)
  float* basis_slot = nullptr;    // V_{j+1} is stored here when non-null
  size_t n = 0;
  const double* alpha = nullptr;
  const double* beta = nullptr;
  double* rhobar = nullptr;
  double* phibar = nullptr;
  double* phibar_hist = nullptr;
  double* rgiv = nullptr;
  int j = 0;
  double tol = 0.0;
  int* flags = nullptr;
  const int* done_in = nullptr;
  int* done_out = nullptr;
  const int* stop_at = nullptr;   // learned stop index, or null
};

// --------------------------------------------------------------- workspaces --
struct Scratch {
  double* partials = nullptr;
  unsigned* tickets = nullptr;    // a few independent tickets
  size_t npartials = 0;
};

struct UmmaMaps;
struct tc_mlp;

struct tc_plan {
  int n1, n2, s, n3;
  bool two_sided;
  tc_opts opts;
  int device;
  size_t Tx, Ty;                  // elements of X (n2 s n3) and of Y (n1 s n3)
  float *Ah = nullptr, *AhT = nullptr;     // A x_3 M and its slice transposes
  float *Bh = nullptr, *BhT = nullptr;
  float *dM = nullptr, *dMinv = nullptr, *dMinvT = nullptr, *dMT = nullptr;  // n3 x n3
  float *dG = nullptr, *dGi = nullptr;  // dual-domain route: M^{-T} M^{-1} and M M^T
  bool store_bf16 = false;  // opts.store TC_STORE_BF16: slice products stored in BF16 (tmp2)
  float hM[TC_MAX_FUSED * TC_MAX_FUSED], hMinv[TC_MAX_FUSED * TC_MAX_FUSED];
  float hMinvT[TC_MAX_FUSED * TC_MAX_FUSED], hMT[TC_MAX_FUSED * TC_MAX_FUSED];
  float *tmp1 = nullptr, *tmp2 = nullptr;  // transform-domain intermediates
  float* tmp3 = nullptr;                   // TF32 plans: per-slice transposed GEMM operand
  size_t tmp_elems = 0;
  Scratch scratch;
  // solver workspaces (grow-only)
  float* lsqr_U = nullptr; float* lsqr_V = nullptr; float* lsqr_W = nullptr;
  float* lsqr_Ct = nullptr; float* lsqr_Xt = nullptr;  // transform-domain route: C~ and X~
  float* basis = nullptr; size_t basis_elems = 0;
  double* dscal = nullptr; size_t dscal_elems = 0;
  int* iflags = nullptr;
  int* lsqr_done = nullptr; size_t lsqr_done_elems = 0;  // done[j]: step j's launches return
  float* gm_basis = nullptr; size_t gm_basis_elems = 0;    // GMRES basis V_1..V_{m+1}
  double* gm_dscal = nullptr; size_t gm_dscal_elems = 0;
  int* gm_flags = nullptr;
  // tensor-core precision forms (opts.precision TF32 / BF16)
  void* AhL = nullptr;            // A~ rounded to the GEMM input type
  void* AhTL = nullptr;           // its slice transposes
  UmmaMaps* umf = nullptr;        // forward:  A~_k (n1 x n2) times X~_k (n2 x s)
  UmmaMaps* uma = nullptr;        // adjoint:  A~_k^T (n2 x n1) times Y'_k (n1 x s)
  // two-sided tensor-core plans: the right factor in the GEMM input type and
  // the second GEMMs, T_k B~_k (forward) and T_k B~_k^T (adjoint), whose left
  // operand T is the first GEMM's result rounded into the operand buffer
  void* BfL = nullptr;            // B~ as the forward GEMM's B operand
  void* BaL = nullptr;            // B~^T as the adjoint GEMM's B operand
  UmmaMaps* umf2 = nullptr;       // T_k (n1 x s) times B~_k (s x s)
  UmmaMaps* uma2 = nullptr;       // T_k (n2 x s) times B~_k^T (s x s)
  void* lowX = nullptr;           // TC_BF16X3 plans: the GEMM operand as three BF16 planes
  void* lowV = nullptr;           // BF16/BF16X3 ORTHODCT plans: bf16(V~) and bf16(U~) (three planes for BF16X3), the operands
  void* lowU = nullptr;           // of the transform-domain GEMMs with fused epilogues
  UmmaMaps* umf_td = nullptr;     // A~ times lowV
  UmmaMaps* uma_td = nullptr;     // A~^T times lowU
  int* dev_err = nullptr;         // set by a tensor-core GEMM whose bounded wait gave up
  void* aux = nullptr;            // tc_lsqr_label workspace (grow-only)
  size_t aux_bytes = 0;
  cudaStream_t cap_stream = nullptr;
  // graph cache for tc_lsqr_c
  cudaGraphExec_t lsqr_graph = nullptr;
  uintptr_t lsqr_key[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  int lsqr_kernels = 0;           // kernel nodes of the captured solve (each replay launches them all)
};

// ----------------------------------------------------------- error helpers --
void tc_set_error(const char* what, cudaError_t e);
void tc_set_message(const char* msg);
#define TC_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      tc_set_error(#call, e_);                          \
      return TC_ECUDA;                                  \
    }                                                   \
  } while (0)
#define TC_CHECK(cond)                                  \
  do {                                                  \
    if (!(cond)) return TC_EINVAL;                      \
  } while (0)
#define TC_TRY(call)                                    \
  do {                                                  \
    int r_ = (call);                                    \
    if (r_ != TC_OK) return r_;                         \
  } while (0)

// ---------------------------------------------------------- kernel drivers --
// gemm.cu: C_k = A_k * (pro-transformed B)_k for nslices slices, epilogue.
// A: M x K per slice (row-major), B: K x N, C/prev: M x N; slice strides are
// the dense sizes. pro/epi: n3 x n3 row-major (host arrays, by value), used
// only when the CTA owns all n3 <= TC_MAX_FUSED slices.
int launch_slice_gemm(const float* A, const float* B, float* C, int M, int N, int K,
                      int nslices, const float* pro, const float* epi, const Epi& ep,
                      cudaStream_t st);
// gemm2.cu: the whole two-sided fused product Y = epi[ A_k (pro X)_k B_k ]
// in one launch of thread-block clusters, for N = s <= 256 (cprod2_fits).
// At: the left factor K-major (K x M per slice: A_k^T), X: K x N, B: N x N,
// Y/prev: M x N.
bool cprod2_fits(int s);
int cprod2_init();
// A non-empty `step` is run by the product's CTAs first (and decides the skip).
int launch_cprod2(const float* At, const float* X, const float* B, float* Y, int M, int K,
                  int N, int nslices, const float* pro, const float* epi, const Epi& ep,
                  const LsqrStep& step, cudaStream_t st);
// transform.cu: out[k][p] = ca * sum_l T[k][l] in[l][p] + cp * prev[k][p] over P pixels.
int launch_mode3(const float* in, float* out, const float* T_dev, int n3, size_t P,
                 const Epi& ep, cudaStream_t st);
// The same transform writing the operand of a tensor-core GEMM: BF16, or FP32
// rounded to TF32 (bf16 = 0). No epilogue.
int launch_mode3_lowp(const float* in, void* out, const float* T_dev, int n3, size_t P,
                      int bf16, const int* skip, cudaStream_t st);
// GEMM operand types of the tensor-core forms: TF32 (in FP32 storage), BF16,
// and three BF16 planes (plane q of n values at out + q n) for the
// FP32-level form.
enum RoundKind { ROUND_TF32 = 0, ROUND_BF16 = 1, ROUND_BF16X3 = 2 };
// Tensor-core forms of launch_mode3 / launch_mode3_lowp (tcgen05, operands
// split into BF16 planes: two, relative error near 2^-16 a term, for the TF32
// and BF16 forms; three (split3 / ROUND_BF16X3), near 2^-27, for the
// FP32-level form). *err is set to TC_ETIMEOUT if the bounded wait for the
// MMAs gives up.
// With `after` (a scalars-only LSQR step, X null, and a norm in ep.red), the
// step's scalars run once the pass's norm is in place: inside the TMA form,
// by the CTA that finishes the norm (a skipped pass sets after->done_out),
// else as their own launch after the pass.
int launch_mode3_tc(const float* in, float* out, const float* T_dev, int n3, size_t P,
                    const Epi& ep, int* err, cudaStream_t st, int split3 = 0,
                    const LsqrStep* after = nullptr);
// Dual-domain pass (BF16 plans, n3 <= 64, P % 8 == 0, 16-byte aligned
// tensors; else TC_EUNSUPPORTED): out = bf16(in x_3 T) and ep.red = the
// reduction of ||in x_3 N||_F^2, both from the same split planes of `in`.
// No prev, no coefficients. after: as for launch_mode3_tc.
int launch_mode3_tc_norm(const float* in, void* out, const float* T_dev, const float* N_dev,
                         int n3, size_t P, const Epi& ep, int* err, cudaStream_t st,
                         const LsqrStep* after);
int launch_mode3_tc_lowp(const float* in, void* out, const float* T_dev, int n3, size_t P,
                         int kind, const int* skip, int* err, cudaStream_t st);
// The pass back from BF16 slice products (plans with opts.store TC_STORE_BF16):
// out = in x_3 T with the Krylov epilogue (ep: coef, prev, red) as
// launch_mode3_tc, `in` BF16 loaded by TMA straight into the MMA operand.
// TC_EUNSUPPORTED for shapes tube_inb_ok rejects. after: as launch_mode3_tc.
int launch_mode3_tc_inb(const void* in, float* out, const float* T_dev, int n3, size_t P,
                        const Epi& ep, int* err, cudaStream_t st, const LsqrStep* after);
// launch_mode3_tc_inb that also writes nxt = bf16(out x_3 T2) (BF16, same
// layout): the first pass of the product that follows, done here.
int launch_mode3_tc_chain(const void* in, float* out, const float* T_dev, void* nxt,
                          const float* T2_dev, int n3, size_t P, const Epi& ep, int* err,
                          cudaStream_t st, const LsqrStep* after);
// Whether launch_mode3_tc_inb takes n3 slices of P values at buf (a device
// buffer of the plan, 16-byte aligned).
bool tube_inb_ok(const void* buf, int n3, size_t P);
// Elementwise rounding of n FP32 values to the operand type `kind` (RoundKind).
int transform_init();  // shared-memory limits of the transform passes
int launch_round(const float* in, void* out, size_t n, int kind, cudaStream_t st,
                 const int* skip = nullptr);
// vec.cu
int vec_init();  // carveout preference of the vector passes; the SM count for their grids
// out = ca * in + cp * prev and the fused reduction (the Krylov epilogue as a pass)
int launch_epi(const float* in, float* out, size_t n, const Epi& ep, cudaStream_t st);
int launch_reduce(const float* x, const float* other, size_t n, const Red& red,
                  const int* skip, cudaStream_t st);
int launch_scale(const float* in, float* out, size_t n, const Coef& c, const float* prev,
                 const int* skip, cudaStream_t st);
int launch_lsqr_update(const LsqrStep& step, cudaStream_t st);
// The scalars of an LSQR step alone (one thread): the Givens recurrences,
// the state, the flags and done_out.
int launch_lsqr_scalars(const LsqrStep& step, cudaStream_t st);
// y = R_k^{-1} f_k, the LSQR iterate's coordinates in the basis (§3.3: X_k =
// V_k y_k), from the rotations rg (rho, theta, phi interleaved) with k =
// min(*kdev, kmax); zero beyond k.
int launch_lsqr_coeffs(const double* rg, const int* kdev, int kmax, double* y, cudaStream_t st);
int launch_combine(float* X, const float* X0, const float* basis, size_t stride, int kmax,
                   const int* kdev, const double* y, size_t n, const int* skip,
                   cudaStream_t st);
// Two combinations of one basis in one pass: X = sum_i (y_i / d_i) B_i and
// X2 = sum_i (y2_i / d_i) B_i (d null: 1), B_i at basis + i * stride.
int launch_combine2(float* X, const double* y, float* X2, const double* y2, const double* d,
                    const float* basis, size_t stride, int kmax, const int* kdev, size_t n,
                    cudaStream_t st);
int launch_mgs_pass(float* W, const float* Vi, const double* h, const float* Vnext,
                    size_t n, const Red& red, const int* skip, cudaStream_t st);
// small.cu (FP64, one CTA)
int launch_tikhonov_gcv(const double* H, int ld, int kmax, const int* kdev,
                        const double* beta, int variant, double lambda_in,
                        double* lambda_out, double* y, double* gcv_out, const int* skip,
                        cudaStream_t st);
int launch_build_bidiag(const double* alpha, const double* beta, const int* kdev, int kmax,
                        double* H, cudaStream_t st);
// gcv_bidiag.cu: lambda, GCV and y from LSQR's rotations (rho, theta, phi
// interleaved in rgiv) without an SVD; work holds 1200 doubles.
int launch_gcv_bidiag(const double* rg, const double* phibar, const double* alpha,
                      const double* beta, const int* kdev, int kmax, int variant,
                      double lambda_in, double* work, double* lambda_out, double* y,
                      double* gcv_out, cudaStream_t st, const double* lam_pred = nullptr,
                      double factor = 0.0, int* fallback = nullptr);

// The same for `count` problems in one launch each: problem i's doubles are
// i ps and its ints (kdev) i fsi further on.
int launch_gcv_bidiag_group(const double* rg, const double* phibar, const double* alpha,
                            const double* beta, const int* kdev, int kmax, int variant,
                            double lambda_in, double* work, double* lambda_out, double* y,
                            double* gcv_out, int count, size_t ps, int fsi, cudaStream_t st);

// gcv_bidiag.cu: the L-curve corner k_opt from LSQR's rotations (rg as in
// launch_gcv_bidiag); writes *kopt, y_{k_opt} (kmax doubles, zero beyond
// k_opt) and, when curve is non-null, ||R_k|| at [k-1] and ||X_k|| at
// [kmax + k - 1].
int launch_lcurve(const double* rg, const double* phibar, const int* kdev, int kmax,
                  double* curve, double* y, int* kopt, cudaStream_t st);

// plan.cu helpers used by solvers
// Chaining consecutive products on plans with BF16-stored slice products
// (p->store_bf16): in_ready: the product's BF16 GEMM operand is already in
// the operand buffer, written by the pass back of the product before it;
// next_T: this product's pass back also writes the next product's operand,
// bf16(result x_3 next_T), into the operand buffer (after its GEMM read it).
struct Chain {
  bool in_ready = false;
  const float* next_T = nullptr;
};
// With a non-null `step`, the LSQR step runs before the product: inside the
// product kernel (two-sided fused route) or as its own launch; ep.skip must
// then be step->done_out.
int cprod_epi(tc_plan* p, const float* X, float* Y, const Epi& ep, cudaStream_t st,
              const LsqrStep* step = nullptr, const Chain* ch = nullptr);
// With `after`, a scalars-only LSQR step runs once the product's norm is in
// place (folded into the tensor-core transform pass where there is one).
int adjoint_epi(tc_plan* p, const float* Y, float* X, const Epi& ep, cudaStream_t st,
                const LsqrStep* after = nullptr, const Chain* ch = nullptr);
Red make_red(tc_plan* p, double* out, int sqrt_out, const float* other, int* status);
// Transform-domain products (ORTHODCT plans off the fused route; td_route):
// operand and result are transformed tensors, the epilogue applies to them.
bool td_route(const tc_plan* p);
// The dual-domain route of TH plans (BF16, one-sided, 32 < n3 <= 64).
bool thd_route(const tc_plan* p);
int cprod_td(tc_plan* p, const float* Xt, float* Yt, const Epi& ep, cudaStream_t st);
int adjoint_td(tc_plan* p, const float* Yt, float* Xt, const Epi& ep, cudaStream_t st);
// With a fused-epilogue BF16 plan (umf_td set): operands from lowV / lowU,
// and each product writes the other's operand (see plan.cu).
int cprod_tdf(tc_plan* p, float* Yt, const Epi& ep, cudaStream_t st);
// Dual-domain products (thd_route): the GEMM with the Krylov update, then the
// change of domain writing the other product's BF16 operand and the norm.
int cprod_thd(tc_plan* p, float* Yt, const Epi& ep, cudaStream_t st);
int adjoint_thd(tc_plan* p, float* Xt, const Epi& ep, cudaStream_t st, const LsqrStep* after);
int adjoint_tdf(tc_plan* p, float* Xt, const Epi& ep, cudaStream_t st);
int tc_kernels_init();

// ------------------------------------------------------------ grouped solve --
// group.cu: the batched c-LSQR of many FP32 or BF16 problems with n3 <= 4
// (one-sided, X_reg requested) as grouped launches: each phase of the solve is
// one launch over all problems. Per problem:
struct GroupProb {
  const float* Ah = nullptr;   // A~ (n1 x n2 a slice) and its slice transposes
  const float* AhT = nullptr;
  const void* AhL = nullptr;   // BF16 plans: the same rounded to BF16
  const void* AhTL = nullptr;
  const float* C = nullptr;
  float* X = nullptr;
  float* Xr = nullptr;
  float* U = nullptr;          // U~ (n1 x s)
  float* V = nullptr;          // the last adjoint's V~ (n2 x s)
  float* basis = nullptr;      // V~_1 .. V~_itermax, Tx apart
  double* partials = nullptr;  // this problem's reduction partials
  unsigned* ticket = nullptr;  // and arrival ticket
  size_t Tx = 0, Ty = 0;
  int n1 = 0, n2 = 0, s = 0;
  int tiles_f = 0, tiles_a = 0;  // CTAs of the forward (M = n1) / adjoint (M = n2) product
  int pad = 0;
};
// The state of one grouped launch: which product, the step, and the
// per-problem scalars (lsqr_enqueue's layout, sstride doubles a problem),
// flags (16 ints a problem) and done flags (lstride ints a problem).
enum GroupOpKind { GOP_INIT = 0, GOP_FWD = 1, GOP_ADJ = 2 };
struct GroupOp {
  int op = GOP_FWD;
  int j = 0;
  int itermax = 0;
  int lstride = 0;     // itermax + 2
  double* scal = nullptr;
  size_t sstride = 0;
  int* flags = nullptr;
  int* done = nullptr;
};
// The fused products of step g.j of every problem in one launch; work[i] =
// (problem, tile) for CTA i. Tile shape cfg (0 .. group_cfg_count - 1) is
// group_tile_shape's tm x tn output tile:
// * gemm.cu, FP32 plans: FFMA, three shapes;
// * group_tc.cu, BF16 plans: tcgen05 with the transforms in the operand load
//   and the epilogue, two shapes.
#define GROUP_CFGS 3
int group_cfg_count(int bf16);
void group_tile_shape(int bf16, int cfg, int* tm, int* tn);
int launch_group_gemm(const GroupProb* probs, const int2* work, int nwork, const GroupOp& g,
                      const float* pro, const float* epi, int n3, int cfg, cudaStream_t st);
int launch_group_umma(const GroupProb* probs, const int2* work, int nwork, const GroupOp& g,
                      const float* pro, const float* epi, int n3, int cfg, cudaStream_t st);
int group_tc_init();

// solvers.cu: the c-LSQR solve as a sequence of launches on one stream
// (capturable), and the workspaces it needs.
struct LsqrArgs {
  const float* C;
  float* X;
  float* X_reg;
  int itermax;
  double tol, lambda;
  double* hist;
  tc_solve_info* info;
  const tc_mlp* mlp = nullptr;  // learned stop index and lambda (learned.cu)
  double factor = 1.05;         // GCV fallback threshold for the learned lambda
  int lcurve = 0;               // X_reg = X_{k_opt} at the L-curve corner, no GCV
  int spatial_basis = 0;        // keep the basis in the spatial domain (no transform-domain route)
  double* curve = nullptr;      // L-curve norms (2 itermax doubles) or null
};
// learned.cu: after MLP_FEAT_STEPS steps, features -> network -> lam_pred and
// stop_at (the step count to stop after).
int launch_learned_predict(const tc_mlp* m, const double* alpha, const double* beta,
                           const double* phibar, int kmax, double* lam_pred, int* stop_at,
                           cudaStream_t st);
int ensure_lsqr(tc_plan* p, int itermax, bool keep_basis);
int lsqr_enqueue(tc_plan* p, const LsqrArgs& a, cudaStream_t st);
