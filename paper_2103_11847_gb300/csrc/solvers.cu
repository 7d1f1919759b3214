// Krylov drivers of §3 on the device: Golub-Kahan (Algorithm 4), DC-LSQR
// (Algorithm 6) with the optional Tikhonov/GCV projection (Algorithm 5,
// eqs. (normeq2), (xmlsqr)), restarted DC-GMRES(m) (Algorithms 2 and 3), and
// the projected Tikhonov/GCV solve. The host only enqueues work: every scalar
// (alpha, beta, rho, phi, h, lambda) lives in device memory and kernels read it
// there, so a whole solve runs without a host round trip and can be replayed
// as one CUDA graph. Early stops (convergence, breakdown) raise a device flag
// that makes the remaining launches of the solve return at once.
#include <cmath>
#include <cstring>
#include <vector>

#include "mlp.cuh"
#include "tc_device.cuh"

namespace {

// Grow-only device buffer; *moved is set when the buffer was reallocated.
template <class T>
int grow(T** p, size_t* have, size_t need, bool* moved = nullptr) {
  if (*p && *have >= need) return TC_OK;
  if (moved) *moved = true;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc((void**)p, (need ? need : 1) * sizeof(T));
  if (e != cudaSuccess) {
    tc_set_error("cudaMalloc", e);
    *p = nullptr;
    return TC_ENOMEM;
  }
  *have = need;
  return TC_OK;
}

}  // namespace

int ensure_lsqr(tc_plan* p, int itermax, bool keep_basis) {
  bool moved = false;
  if (!p->lsqr_U) {
    moved = true;
    if (cudaMalloc((void**)&p->lsqr_U, p->Ty * 4) != cudaSuccess) return TC_ENOMEM;
    if (cudaMalloc((void**)&p->lsqr_V, p->Tx * 4) != cudaSuccess) return TC_ENOMEM;
    if (cudaMalloc((void**)&p->lsqr_W, p->Tx * 4) != cudaSuccess) return TC_ENOMEM;
  }
  if ((td_route(p) || thd_route(p)) && !p->lsqr_Ct) {
    moved = true;
    if (cudaMalloc((void**)&p->lsqr_Ct, p->Ty * 4) != cudaSuccess) return TC_ENOMEM;
    if (cudaMalloc((void**)&p->lsqr_Xt, p->Tx * 4) != cudaSuccess) return TC_ENOMEM;
  }
  if (!p->iflags && cudaMalloc((void**)&p->iflags, 16 * sizeof(int)) != cudaSuccess)
    return TC_ENOMEM;
  const size_t L = (size_t)itermax + 2;
  const size_t kp = (size_t)(itermax < TC_MAX_PROJ ? itermax : TC_MAX_PROJ);
  TC_TRY(grow(&p->dscal, &p->dscal_elems, 7 * L + 1200 + kp + 16, &moved));
  TC_TRY(grow(&p->lsqr_done, &p->lsqr_done_elems, L, &moved));
  if (keep_basis) TC_TRY(grow(&p->basis, &p->basis_elems, (size_t)itermax * p->Tx, &moved));
  if (moved && p->lsqr_graph) {  // a captured solve holds the old addresses
    cudaGraphExecDestroy(p->lsqr_graph);
    p->lsqr_graph = nullptr;
  }
  return TC_OK;
}

namespace {

// alpha_1 = ||A^T U_1|| and beta_1 = ||C|| are in place: set W_1 = V_1 and the
// Givens state rhobar_1 = alpha_1, phibar_1 = beta_1 (Algorithm 6 step 2).
// done[0] gates the first step: set on a start-up breakdown or non-finite norm.
__global__ void k_lsqr_init(const double* alpha, const double* beta, double* rhobar,
                            double* phibar, int* flags, int* done) {
  rhobar[0] = alpha[0];
  phibar[0] = beta[0];
  flags[1] = 0;
  if (!isfinite(alpha[0]) || !isfinite(beta[0])) flags[2] = TC_ENONFINITE;
  else if (alpha[0] == 0.0 || beta[0] == 0.0) flags[2] = TC_EBREAKDOWN;
  done[0] = flags[2] != 0;
}

// kopt: the L-curve corner (then resid is ||R_{k_opt}||), or null.
__global__ void k_lsqr_info(tc_solve_info* info, const int* flags, const double* phibar,
                            const double* beta, const double* lam, const double* gcv,
                            const int* kopt) {
  const int it = flags[1];
  info->iters = it;
  info->status = flags[2];
  info->cycles = 0;
  info->fallback = flags[7];
  info->resid = fabs(phibar[kopt ? *kopt : it]);
  info->lambda = lam ? *lam : nan("");
  info->gcv = gcv ? *gcv : nan("");
  info->beta1 = beta[0];
  info->kopt = kopt ? *kopt : 0;
  info->reserved = 0;
}

// GMRES helpers. flags: [0] done, [1] total steps, [2] status, [3] steps in the
// current cycle, [4] Arnoldi stopped in this cycle (done or h_{j+1,j} = 0).
__global__ void k_gmres_check(const double* rnorm, double tol, int* flags, double* resid,
                              int cycle) {
  if (flags[0]) return;
  *resid = *rnorm;
  if (!isfinite(*rnorm)) {
    flags[2] = TC_ENONFINITE;
    flags[0] = 1;
  } else if (*rnorm < tol || *rnorm == 0.0) {
    flags[2] = 1;
    flags[0] = 1;
  }
  flags[3] = 0;
  flags[4] = flags[0];
  flags[5] = cycle;
}

__global__ void k_gmres_step_done(const double* hnext, int j, int* flags) {
  if (flags[4]) return;
  flags[3] = j + 1;
  flags[1] += 1;
  if (!(*hnext > 0.0)) flags[4] = 1;  // h_{j+1,j} = 0 (or NaN): stop this cycle
}

__global__ void k_gmres_cycle_done(int* flags) {
  if (!flags[0]) flags[5] += 1;
}

__global__ void k_gmres_info(tc_solve_info* info, const int* flags, const double* resid,
                             const double* lam, const double* gcv, const double* beta1) {
  info->iters = flags[1];
  info->status = flags[2];
  info->cycles = flags[5];
  info->fallback = 0;
  info->resid = *resid;
  info->lambda = *lam;
  info->gcv = *gcv;
  info->beta1 = *beta1;
  info->kopt = 0;
  info->reserved = 0;
}

}  // namespace

// ----------------------------------------------------------------- LSQR ----
int lsqr_enqueue(tc_plan* p, const LsqrArgs& a, cudaStream_t st) {
  const size_t L = (size_t)a.itermax + 2;
  const int kp = a.itermax < TC_MAX_PROJ ? a.itermax : TC_MAX_PROJ;
  double* alpha = p->dscal;
  double* beta = alpha + L;
  double* rhobar = beta + L;
  double* phibar = rhobar + L;
  double* rgiv = phibar + L;  // rho_j, theta_{j+1}, phi_j interleaved (3 L)
  double* gwork = rgiv + 3 * L;
  double* y = gwork + 1200;
  double* lam = y + kp;
  double* gcv = lam + 1;
  double* lam_pred = gcv + 1;
  int* flags = p->iflags;  // [1] iterations [2] status [6] stop_at [7] fallback
  // done[j] nonzero: every launch of step j returns at once (set by step j-1's update)
  int* done = p->lsqr_done;
  float *U = p->lsqr_U, *V = p->lsqr_V, *W = p->lsqr_W;
  const bool keep = a.X_reg != nullptr;
  // With the basis kept, the iterate is formed from it once at the end,
  // X_k = V_k R_k^{-1} f_k (§3.3), instead of by the per-step X, W updates:
  // the basis holds the unnormalised V~_1..V~_k that the adjoint products
  // write (slot j is both the forward product's operand and the next
  // adjoint's prev), each step runs its scalars alone, and the final pass
  // forms X and X_reg together with coefficients y_i / alpha_i. tc_lsqr_label
  // reads the basis as normalised vectors and keeps the per-step updates.
  const bool defer = keep && !a.spatial_basis;
  auto slot = [&](int i) { return p->basis + (size_t)i * p->Tx; };

  TC_CUDA(cudaMemsetAsync(flags, 0, 16 * sizeof(int), st));
  TC_CUDA(cudaMemsetAsync(done, 0, L * sizeof(int), st));
  // Transform-domain route (ORTHODCT off the fused route): iterate on C~ =
  // dct(C) and X~ with products of slice GEMMs only; X (and X_reg) are
  // transformed back once at the end. Norms are unchanged by the orthogonal
  // transform, so every scalar of the solve is the same.
  const bool td = td_route(p) && !a.spatial_basis;
  // Dual-domain route (TH plans, thd_route, with the basis kept): U^ = U x_3 M
  // and V' = V x_3 M^{-T} throughout; C^ = C x_3 M is the first forward
  // product's prev and bf16(C x_3 M^{-T}) the first adjoint's operand. The
  // basis holds V'_1..V'_k, so X and X_reg are formed there and transformed
  // back by M^T once. Every scalar is the spatial route's, up to rounding.
  const bool thd = thd_route(p) && defer;
  const float* Cin = a.C;
  float* Xw = a.X;
  // The tensor-core transform (split BF16, error near 2^-16) serves the TF32
  // and BF16 plans above TC_TUBE_MIN_N3; the rest keep the FP32 pass.
  const bool tct = p->opts.precision != TC_FP32 && p->n3 > TC_TUBE_MIN_N3;
  auto mode3 = [&](const float* in, float* out, const float* T, size_t P) -> int {
    Epi none;
    return tct ? launch_mode3_tc(in, out, T, p->n3, P, none, p->dev_err, st,
                                 p->opts.precision == TC_BF16X3)
               : launch_mode3(in, out, T, p->n3, P, none, st);
  };
  if (td) {
    TC_TRY(mode3(a.C, p->lsqr_Ct, p->dM, p->Ty / p->n3));
    Cin = p->lsqr_Ct;
    Xw = p->lsqr_Xt;
  }
  if (thd) {
    TC_TRY(mode3(a.C, p->lsqr_Ct, p->dM, p->Ty / p->n3));
    TC_TRY(launch_mode3_tc_lowp(a.C, p->lowU, p->dMinvT, p->n3, p->Ty / p->n3, ROUND_BF16,
                                nullptr, p->dev_err, st));
    Cin = p->lsqr_Ct;
    Xw = p->lsqr_Xt;
  }
  // BF16 plans with fused epilogues keep the GEMM operands as BF16 copies that
  // each product's store writes for the next one; the first is bf16(C~).
  const bool tdf = td && p->umf_td != nullptr;
  if (tdf)
    TC_TRY(launch_round(Cin, p->lowU, p->Ty,
                        p->opts.precision == TC_BF16X3 ? ROUND_BF16X3 : ROUND_BF16, st));
  // Chained products (BF16-stored slice products on the spatial route, basis
  // kept): each product's pass back also writes the next product's BF16 GEMM
  // operand, so only the start-up adjoint transforms its operand itself.
  const bool chain = p->store_bf16 && defer && !td && !thd;
  const Chain ch_first{false, p->dM}, ch_fwd{true, p->dMinvT}, ch_adj{true, p->dM};
  int nadj = 0;
  auto fwd = [&](const float* Xv, float* Yv, const Epi& ep, const LsqrStep* step) -> int {
    if (thd) return cprod_thd(p, Yv, ep, st);  // steps run in the adjoint's pass (fold)
    if (!td) return cprod_epi(p, Xv, Yv, ep, st, step, chain ? &ch_fwd : nullptr);
    if (step) TC_TRY(step->X ? launch_lsqr_update(*step, st) : launch_lsqr_scalars(*step, st));
    return tdf ? cprod_tdf(p, Yv, ep, st) : cprod_td(p, Xv, Yv, ep, st);
  };
  auto adj = [&](const float* Yv, float* Xv, const Epi& ep, const LsqrStep* after) -> int {
    if (thd) return adjoint_thd(p, Xv, ep, st, after);
    if (tdf) return adjoint_tdf(p, Xv, ep, st);
    const Chain* ch = chain ? (nadj++ == 0 ? &ch_first : &ch_adj) : nullptr;
    return td ? adjoint_td(p, Yv, Xv, ep, st) : adjoint_epi(p, Yv, Xv, ep, st, after, ch);
  };
  // Deferred schedule on the tensor-core transform route: step j's scalars
  // need alpha_{j+1}, which the adjoint product of step j finishes in its
  // trailing transform pass; the CTA that finishes that norm runs them, and
  // the forward product of step j + 1 starts without a launch before it.
  const bool fold = defer && !td && tct;
  // beta_1 = ||C||_F
  TC_TRY(launch_reduce(thd ? a.C : Cin, nullptr, p->Ty, make_red(p, beta, 1, nullptr, flags + 2),
                       nullptr, st));
  // V~_1 = A^T (C / beta_1), alpha_1 = ||V~_1||
  {
    Epi ep;
    ep.coef.rule = COEF_INV;
    ep.coef.s0 = beta;
    ep.red = make_red(p, alpha, 1, nullptr, flags + 2);
    TC_TRY(adj(Cin, defer ? slot(0) : V, ep, nullptr));
  }
  if (!defer) {  // W_1 = V_1 = V~_1 / alpha_1; X_0 = 0
    Coef c;
    c.rule = COEF_INV;
    c.s0 = alpha;
    TC_TRY(launch_scale(V, W, p->Tx, c, nullptr, nullptr, st));
    if (keep) TC_TRY(launch_scale(V, p->basis, p->Tx, c, nullptr, nullptr, st));
    TC_CUDA(cudaMemsetAsync(Xw, 0, p->Tx * sizeof(float), st));
  }
  k_lsqr_init<<<1, 1, 0, st>>>(alpha, beta, rhobar, phibar, flags, done);
  TC_CUDA(cudaGetLastError());

  // Step j's Givens recurrences and X, W updates ((c)-(g)) need alpha_{j+1}
  // from the adjoint of step j; the forward product of step j + 1 does not
  // need them, so step j runs at the start of that product (inside the
  // product kernel on the two-sided fused route), and the last step after
  // the loop.
  auto make_step = [&](int j) {
    LsqrStep u;
    u.X = defer ? nullptr : Xw;  // deferred: the step's scalars alone
    u.W = defer ? nullptr : W;
    u.V = defer ? nullptr : V;
    u.basis_slot = (!defer && keep && j + 1 < a.itermax) ? slot(j + 1) : nullptr;
    u.n = p->Tx;
    u.alpha = alpha;
    u.beta = beta;
    u.rhobar = rhobar;
    u.phibar = phibar;
    u.phibar_hist = a.hist;
    u.rgiv = keep ? rgiv : nullptr;
    u.j = j;
    u.tol = a.tol;
    u.flags = flags;
    u.done_in = done + j;
    u.done_out = done + j + 1;
    u.stop_at = a.mlp ? flags + 6 : nullptr;
    return u;
  };
  for (int j = 0; j < a.itermax; ++j) {
    // (a) U~_{j+1} = A V_j - alpha_j U_j = (1/alpha_j) A V~_j - (alpha_j/beta_j) U~_j,
    // preceded by step j - 1 (which decides done[j])
    {
      Epi ep;
      ep.coef.rule = COEF_GK;
      ep.coef.s0 = alpha + j;
      ep.coef.s1 = beta + j;
      ep.prev = (j == 0) ? Cin : U;
      ep.red = make_red(p, beta + j + 1, 1, nullptr, flags + 2);
      ep.skip = done + j;
      const LsqrStep prev = j > 0 ? make_step(j - 1) : LsqrStep{};
      TC_TRY(fwd(defer ? slot(j) : V, U, ep, (j > 0 && !fold) ? &prev : nullptr));
    }
    // the learned predictor reads the first MLP_FEAT_STEPS steps
    if (a.mlp && j == MLP_FEAT_STEPS)
      TC_TRY(launch_learned_predict(a.mlp, alpha, beta, phibar, a.itermax, lam_pred, flags + 6, st));
    // (b) V~_{j+1} = (1/beta_{j+1}) A^T U~_{j+1} - (beta_{j+1}/alpha_j) V~_j
    {
      Epi ep;
      ep.coef.rule = COEF_GK;
      ep.coef.s0 = beta + j + 1;
      ep.coef.s1 = alpha + j;
      ep.prev = defer ? slot(j) : V;
      ep.red = make_red(p, alpha + j + 1, 1, nullptr, flags + 2);
      ep.skip = done + j;
      // deferred: V~_{j+1} into basis slot j + 1 (the last one, never part of
      // the basis, into the workspace)
      const LsqrStep step = make_step(j);
      TC_TRY(adj(U, defer ? (j + 1 < a.itermax ? slot(j + 1) : V) : V, ep, fold ? &step : nullptr));
    }
  }
  if (fold) {
    // every step's scalars ran in its adjoint product
  } else if (defer)
    TC_TRY(launch_lsqr_scalars(make_step(a.itermax - 1), st));
  else
    TC_TRY(launch_lsqr_update(make_step(a.itermax - 1), st));
  if (a.mlp && a.itermax == MLP_FEAT_STEPS)
    TC_TRY(launch_learned_predict(a.mlp, alpha, beta, phibar, a.itermax, lam_pred, flags + 6, st));
  const bool gcv_on = keep && !a.lcurve;
  // the basis combination lands in X_reg, or in a workspace to transform back
  float* Xr_w = (td || thd) ? p->tmp2 : a.X_reg;
  if (keep && a.lcurve) {  // X_reg = X_{k_opt} at the L-curve corner (flags[8] = k_opt)
    TC_TRY(launch_lcurve(rgiv, phibar, flags + 1, kp, a.curve, y, flags + 8, st));
  } else if (keep) {
    TC_TRY(launch_gcv_bidiag(rgiv, phibar, alpha, beta, flags + 1, kp, p->opts.gcv_variant,
                             a.mlp ? -1.0 : a.lambda, gwork, lam, y, gcv, st,
                             a.mlp ? lam_pred : nullptr, a.factor, flags + 7));
  }
  if (defer) {
    // X_k = V_k R_k^{-1} f_k and X_reg = V_k y (y of k_opt's iterate for the
    // L-curve, zero beyond it) in one pass over the unnormalised basis:
    // coefficients divided by alpha_i
    double* ylsqr = gwork;  // the GCV search's work space is free again
    TC_TRY(launch_lsqr_coeffs(rgiv, flags + 1, kp, ylsqr, st));
    TC_TRY(launch_combine2(Xw, ylsqr, Xr_w, y, alpha, p->basis, p->Tx, kp, flags + 1, p->Tx,
                           st));
  } else if (keep) {
    TC_TRY(launch_combine(Xr_w, nullptr, p->basis, p->Tx, kp, a.lcurve ? flags + 8 : flags + 1,
                          y, p->Tx, nullptr, st));
  }
  if (td || thd) {  // back to the spatial domain: X = idct(X~) (X' x_3 M^T), X_reg likewise
    const float* back = thd ? p->dMT : p->dMinv;
    TC_TRY(mode3(Xw, a.X, back, p->Tx / p->n3));
    if (keep) TC_TRY(mode3(Xr_w, a.X_reg, back, p->Tx / p->n3));
  }
  k_lsqr_info<<<1, 1, 0, st>>>(a.info, flags, phibar, beta, gcv_on ? lam : nullptr,
                               gcv_on ? gcv : nullptr, (keep && a.lcurve) ? flags + 8 : nullptr);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

namespace {

// Run a c-LSQR solve: enqueue it directly, or replay the plan's captured
// graph, capturing it again when the solve's parameters (key) changed.
int run_lsqr(tc_plan* p, const LsqrArgs& a, const uintptr_t (&key)[10], cudaStream_t st) {
  if (!p->opts.use_graphs) return lsqr_enqueue(p, a, st);
  if (!p->lsqr_graph || std::memcmp(key, p->lsqr_key, sizeof(key)) != 0) {
    if (p->lsqr_graph) {
      cudaGraphExecDestroy(p->lsqr_graph);
      p->lsqr_graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    TC_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int r = lsqr_enqueue(p, a, p->cap_stream);
    const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    if (r != TC_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) {
      tc_set_error("cudaStreamEndCapture", e);
      return TC_ECUDA;
    }
    size_t nn = 0;
    p->lsqr_kernels = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
        for (size_t i = 0; i < nn; ++i) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            ++p->lsqr_kernels;
        }
    }
    const cudaError_t e2 = cudaGraphInstantiate(&p->lsqr_graph, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
      p->lsqr_graph = nullptr;
      tc_set_error("cudaGraphInstantiate", e2);
      return TC_ECUDA;
    }
    std::memcpy(p->lsqr_key, key, sizeof(key));
  }
  TC_CUDA(cudaGraphLaunch(p->lsqr_graph, st));
  return TC_OK;
}

}  // namespace

extern "C" int tc_lsqr_c(tc_plan* p, const float* C, float* X, float* X_reg, int itermax,
                         double tol, double lambda, double* phibar_hist, tc_solve_info* info,
                         tc_stream_t stream) {
  if (!p || !C || !X || !info) return TC_EINVAL;
  if (itermax < 1 || itermax > 4096 || !(tol >= 0.0)) return TC_EINVAL;
  if (X_reg && itermax > TC_MAX_PROJ) return TC_EINVAL;
  if ((const void*)C == (const void*)X || (X_reg && (X_reg == X))) return TC_EINVAL;
  TC_TRY(ensure_lsqr(p, itermax, X_reg != nullptr));
  LsqrArgs a{C, X, X_reg, itermax, tol, lambda, phibar_hist, info};
  uint64_t tb, lb;
  std::memcpy(&tb, &tol, 8);
  std::memcpy(&lb, &lambda, 8);
  const uintptr_t key[10] = {(uintptr_t)C, (uintptr_t)X, (uintptr_t)X_reg, (uintptr_t)itermax,
                             (uintptr_t)tb, (uintptr_t)lb, (uintptr_t)phibar_hist,
                             (uintptr_t)info, 0, 0};
  return run_lsqr(p, a, key, (cudaStream_t)stream);
}

extern "C" int tc_lsqr_graph_kernels(tc_plan* p, int* count) {
  if (!p || !count) return TC_EINVAL;
  *count = p->lsqr_graph ? p->lsqr_kernels : 0;
  return TC_OK;
}

extern "C" int tc_lsqr_c_lcurve(tc_plan* p, const float* C, float* X, float* X_opt, int kmax,
                                double tol, double* curve, tc_solve_info* info,
                                tc_stream_t stream) {
  if (!p || !C || !X || !X_opt || !info) return TC_EINVAL;
  if (kmax < 1 || kmax > TC_MAX_PROJ || !(tol >= 0.0)) return TC_EINVAL;
  if ((const void*)C == (const void*)X || (const void*)C == (const void*)X_opt || X_opt == X)
    return TC_EINVAL;
  TC_TRY(ensure_lsqr(p, kmax, true));
  LsqrArgs a{C, X, X_opt, kmax, tol, -1.0, nullptr, info};
  a.lcurve = 1;
  a.curve = curve;
  uint64_t tb;
  std::memcpy(&tb, &tol, 8);
  const uintptr_t key[10] = {(uintptr_t)C, (uintptr_t)X, (uintptr_t)X_opt, (uintptr_t)kmax,
                             (uintptr_t)tb, 0, 0, (uintptr_t)info, 1, (uintptr_t)curve};
  return run_lsqr(p, a, key, (cudaStream_t)stream);
}

// ------------------------------------------------------------ Golub-Kahan ----
extern "C" int tc_gkb_init(tc_plan* p, const float* C, float* U, float* V, double* alpha,
                           double* beta, int mmax, tc_stream_t stream) {
  if (!p || !C || !U || !V || !alpha || !beta || mmax < 1) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  TC_TRY(launch_reduce(C, nullptr, p->Ty, make_red(p, beta, 1, nullptr, nullptr), nullptr, st));
  Coef c;
  c.rule = COEF_INV;
  c.s0 = beta;
  TC_TRY(launch_scale(C, U, p->Ty, c, nullptr, nullptr, st));
  Epi ep;
  ep.red = make_red(p, alpha, 1, nullptr, nullptr);
  TC_TRY(adjoint_epi(p, U, V, ep, st));
  c.s0 = alpha;
  return launch_scale(V, V, p->Tx, c, nullptr, nullptr, st);
}

extern "C" int tc_gkb_step(tc_plan* p, int j, float* U, float* V, double* alpha, double* beta,
                           int mmax, tc_stream_t stream) {
  if (!p || !U || !V || !alpha || !beta || j < 1 || j > mmax) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const float* Uj = U + (size_t)(j - 1) * p->Ty;
  float* Uj1 = U + (size_t)j * p->Ty;
  const float* Vj = V + (size_t)(j - 1) * p->Tx;
  float* Vj1 = V + (size_t)j * p->Tx;
  Coef inv;
  inv.rule = COEF_INV;
  {  // U~ = A V_j - alpha_j U_j, beta_{j+1} = ||U~||, U_{j+1} = U~ / beta_{j+1}
    Epi ep;
    ep.coef.rule = COEF_AXPY;
    ep.coef.s0 = alpha + (j - 1);
    ep.prev = Uj;
    ep.red = make_red(p, beta + j, 1, nullptr, nullptr);
    TC_TRY(cprod_epi(p, Vj, Uj1, ep, st));
    inv.s0 = beta + j;
    TC_TRY(launch_scale(Uj1, Uj1, p->Ty, inv, nullptr, nullptr, st));
  }
  {  // V~ = A^T U_{j+1} - beta_{j+1} V_j, alpha_{j+1} = ||V~||, V_{j+1} = V~ / alpha_{j+1}
    Epi ep;
    ep.coef.rule = COEF_AXPY;
    ep.coef.s0 = beta + j;
    ep.prev = Vj;
    ep.red = make_red(p, alpha + j, 1, nullptr, nullptr);
    TC_TRY(adjoint_epi(p, Uj1, Vj1, ep, st));
    inv.s0 = alpha + j;
    TC_TRY(launch_scale(Vj1, Vj1, p->Tx, inv, nullptr, nullptr, st));
  }
  return TC_OK;
}

// ------------------------------------------------------------------ GMRES ----
extern "C" int tc_gmres_c(tc_plan* p, const float* C, const float* X0, float* X, int m,
                          int itermax, double tol, double lambda, tc_solve_info* info,
                          tc_stream_t stream) {
  if (!p || !C || !X || !info) return TC_EINVAL;
  if (p->n1 != p->n2 || m < 1 || m > TC_MAX_PROJ || itermax < 1 || !(tol >= 0.0))
    return TC_EINVAL;
  if ((const void*)C == (const void*)X) return TC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t T = p->Tx;  // == Ty for a square operator
  TC_TRY(grow(&p->gm_basis, &p->gm_basis_elems, (size_t)(m + 1) * T));
  TC_TRY(grow(&p->gm_dscal, &p->gm_dscal_elems, (size_t)(m + 1) * m + m + 16));
  if (!p->gm_flags && cudaMalloc((void**)&p->gm_flags, 16 * sizeof(int)) != cudaSuccess)
    return TC_ENOMEM;
  double* H = p->gm_dscal;
  double* y = H + (size_t)(m + 1) * m;
  double* rnorm = y + m;
  double* lam = rnorm + 1;
  double* gcv = lam + 1;
  double* resid = gcv + 1;
  double* beta1 = resid + 1;
  int* flags = p->gm_flags;
  float* Vb = p->gm_basis;

  TC_CUDA(cudaMemsetAsync(flags, 0, 16 * sizeof(int), st));
  TC_CUDA(cudaMemsetAsync(lam, 0xff, 2 * sizeof(double), st));  // NaN until a cycle runs
  TC_TRY(launch_reduce(C, nullptr, T, make_red(p, beta1, 1, nullptr, nullptr), nullptr, st));
  if (X0) {
    TC_CUDA(cudaMemcpyAsync(X, X0, T * sizeof(float), cudaMemcpyDeviceToDevice, st));
  } else {
    TC_CUDA(cudaMemsetAsync(X, 0, T * sizeof(float), st));
  }
  int done = 0, cycle = 0;
  while (true) {
    // R_0 = C - A X (Algorithm 3 step 3; recomputed on every restart)
    Epi er;
    er.coef.rule = COEF_RESID;
    er.prev = C;
    er.red = make_red(p, rnorm, 1, nullptr, flags + 2);
    er.skip = flags;
    TC_TRY(cprod_epi(p, X, Vb, er, st));
    k_gmres_check<<<1, 1, 0, st>>>(rnorm, tol, flags, resid, cycle);
    TC_CUDA(cudaGetLastError());
    if (done >= itermax) break;
    const int mj = (m < itermax - done) ? m : (itermax - done);
    TC_CUDA(cudaMemsetAsync(H, 0, (size_t)(m + 1) * m * sizeof(double), st));
    // Algorithm 2: V_1 = R_0 / beta
    Coef inv;
    inv.rule = COEF_INV;
    inv.s0 = rnorm;
    TC_TRY(launch_scale(Vb, Vb, T, inv, nullptr, flags + 4, st));
    for (int j = 0; j < mj; ++j) {
      float* Vj = Vb + (size_t)j * T;
      float* Wn = Vb + (size_t)(j + 1) * T;
      double* hcol = H + j;  // H(i, j) at H[i*m + j]
      Epi ea;  // W = A V_j, fused with h_{1,j} = <V_1, W>
      ea.red = make_red(p, hcol, 0, Vb, flags + 2);
      ea.skip = flags + 4;
      TC_TRY(cprod_epi(p, Vj, Wn, ea, st));
      for (int i = 0; i <= j; ++i) {  // MGS: W -= h_ij V_i, then the next product
        const bool last = (i == j);
        Red r = make_red(p, H + (size_t)(i + 1) * m + j, last ? 1 : 0,
                         last ? nullptr : Vb + (size_t)(i + 1) * T, flags + 2);
        TC_TRY(launch_mgs_pass(Wn, Vb + (size_t)i * T, H + (size_t)i * m + j,
                               last ? nullptr : Vb + (size_t)(i + 1) * T, T, r, flags + 4, st));
      }
      inv.s0 = H + (size_t)(j + 1) * m + j;  // V_{j+1} = W / h_{j+1,j}
      TC_TRY(launch_scale(Wn, Wn, T, inv, nullptr, flags + 4, st));
      k_gmres_step_done<<<1, 1, 0, st>>>(H + (size_t)(j + 1) * m + j, j, flags);
      TC_CUDA(cudaGetLastError());
    }
    // Algorithm 3 steps 5-6: lambda by GCV on H~, y, X = X_0 + V (*) y
    TC_TRY(launch_tikhonov_gcv(H, m, mj, flags + 3, rnorm, p->opts.gcv_variant, lambda, lam, y,
                               gcv, flags, st));
    TC_TRY(launch_combine(X, X, Vb, T, mj, flags + 3, y, T, flags, st));
    k_gmres_cycle_done<<<1, 1, 0, st>>>(flags);
    TC_CUDA(cudaGetLastError());
    done += mj;
    ++cycle;
  }
  k_gmres_info<<<1, 1, 0, st>>>(info, flags, resid, lam, gcv, beta1);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// --------------------------------------------------------- Tikhonov / GCV ----
extern "C" int tc_tikhonov_gcv(const double* H, int k, const double* beta, int variant,
                               double lambda_in, double* lambda_out, double* y, double* gcv_out,
                               tc_stream_t stream) {
  if (!H || !beta || !lambda_out || !y || k < 1 || k > TC_MAX_PROJ) return TC_EINVAL;
  if (variant != TC_GCV_PAPER && variant != TC_GCV_FULL) return TC_EINVAL;
  return launch_tikhonov_gcv(H, k, k, nullptr, beta, variant, lambda_in, lambda_out, y, gcv_out,
                             nullptr, (cudaStream_t)stream);
}
