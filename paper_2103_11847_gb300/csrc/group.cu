// The batched c-LSQR (Algorithm 6 with the Tikhonov/GCV projection) of many
// independent FP32 problems of uneven sizes as grouped launches: every phase
// of the solve (the norm of C, the first adjoint product, each step's
// scalars, forward and adjoint products, the GCV search, the combination of
// the basis, the info record) is one launch over all problems, so a batch of
// 128 problems and 40 steps is about 130 launches instead of one launch per
// problem and phase. Problem i keeps its own scalars, flags, reduction
// partials and ticket; each product CTA knows its problem and tile from a
// work table. The fused products' tile shape (three candidates, gemm.cu) is
// chosen per batch by timing each on the batch's own forward product (autotune),
// and the whole grouped solve is captured once as a CUDA graph.
//
// It serves batches of FP32 or BF16 plans with n3 <= 4 (the products fuse
// the mode-3 transforms: gemm.cu's FFMA tiles, group_tc.cu's tcgen05 tiles)
// that request X_reg: the iterate is then formed from the kept basis at
// the end (the deferred schedule of lsqr_enqueue), and every kernel here
// follows that schedule problem by problem.
#include <vector>

#include "group.cuh"

namespace {

constexpr int GRP_NT = 256;
constexpr int NORM_CTAS = 32;  // CTAs a problem for the norm of C

struct Layout {  // offsets of one problem's scalars (lsqr_enqueue's layout)
  size_t L, kp;
  __host__ __device__ size_t beta() const { return L; }
  __host__ __device__ size_t rhobar() const { return 2 * L; }
  __host__ __device__ size_t phibar() const { return 3 * L; }
  __host__ __device__ size_t rgiv() const { return 4 * L; }
  __host__ __device__ size_t gwork() const { return 7 * L; }
  __host__ __device__ size_t y() const { return 7 * L + 1200; }
  __host__ __device__ size_t lam() const { return 7 * L + 1200 + kp; }
  __host__ __device__ size_t gcv() const { return lam() + 1; }
  __host__ __device__ size_t stride() const { return 7 * L + 1200 + kp + 16; }
};

__global__ void k_group_reset(int* flags, int* done, unsigned* tickets, int L, int count) {
  const int p = blockIdx.x;
  if (p >= count) return;
  if (threadIdx.x == 0) tickets[p] = 0u;  // left set only by a product that gave up
  for (int i = threadIdx.x; i < 16; i += blockDim.x) flags[16 * p + i] = 0;
  for (int i = threadIdx.x; i < L; i += blockDim.x) done[(size_t)p * L + i] = 0;
}

// beta_1 = ||C_p||_F: NORM_CTAS CTAs a problem (grid.y = problems).
__global__ void __launch_bounds__(GRP_NT)
k_group_norm_c(const GroupProb* __restrict__ probs, double* scal, Layout lay, int* flags) {
  const int p = blockIdx.y;
  const GroupProb& P = probs[p];
  float s = 0.f;
  for (size_t i = (size_t)blockIdx.x * GRP_NT + threadIdx.x; i < P.Ty;
       i += (size_t)gridDim.x * GRP_NT) {
    const float v = P.C[i];
    s = fmaf(v, v, s);
  }
  Red red;
  red.out = scal + p * lay.stride() + lay.beta();
  red.sqrt_out = 1;
  red.partials = P.partials;
  red.ticket = P.ticket;
  red.status = flags + 16 * p + 2;
  reduce_finish_n(s, red, blockIdx.x, gridDim.x);
}

// Algorithm 6 step 2 for every problem (k_lsqr_init of solvers.cu).
__global__ void k_group_lsqr_init(double* scal, Layout lay, int* flags, int* done, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  double* b = scal + p * lay.stride();
  int* f = flags + 16 * p;
  const double a0 = b[0], b0 = b[lay.beta()];
  b[lay.rhobar()] = a0;
  b[lay.phibar()] = b0;
  f[1] = 0;
  if (!isfinite(a0) || !isfinite(b0)) f[2] = TC_ENONFINITE;
  else if (a0 == 0.0 || b0 == 0.0) f[2] = TC_EBREAKDOWN;
  done[(size_t)p * lay.L] = f[2] != 0;
}

// The scalars of step j of every problem (the deferred schedule: no vectors).
__global__ void k_group_scalars(double* scal, Layout lay, int* flags, int* done, int j,
                                double tol, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  double* b = scal + p * lay.stride();
  LsqrStep u;
  u.alpha = b;
  u.beta = b + lay.beta();
  u.rhobar = b + lay.rhobar();
  u.phibar = b + lay.phibar();
  u.rgiv = b + lay.rgiv();
  u.j = j;
  u.tol = tol;
  u.flags = flags + 16 * p;
  u.done_in = done + (size_t)p * lay.L + j;
  u.done_out = done + (size_t)p * lay.L + j + 1;
  if (*u.done_in) {
    *u.done_out = 1;
    return;
  }
  float sh[3];
  lsqr_step_scalars(u, sh, true);
}

// y = R_k^{-1} f_k of every problem into its GCV work space (k_lsqr_coeffs).
__global__ void k_group_coeffs(double* scal, Layout lay, const int* flags, int kmax, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const double* rg = scal + p * lay.stride() + lay.rgiv();
  double* y = scal + p * lay.stride() + lay.gwork();
  const int k = max(0, min(flags[16 * p + 1], kmax));
  for (int i = kmax - 1; i >= k; --i) y[i] = 0.0;
  double yi = 0.0;
  for (int i = k - 1; i >= 0; --i) {
    const double num = rg[3 * i + 2] - (i + 1 < k ? rg[3 * i + 1] * yi : 0.0);
    yi = num / rg[3 * i];
    y[i] = yi;
  }
}

// X_k = sum_i (ylsqr_i / alpha_i) V~_i and X_reg = sum_i (y_i / alpha_i) V~_i
// of problem blockIdx.y (k_combine2), four elements a thread.
__global__ void __launch_bounds__(GRP_NT)
k_group_combine2(const GroupProb* __restrict__ probs, const double* scal, Layout lay,
                 const int* flags, int kmax) {
  __shared__ float c1[TC_MAX_PROJ], c2[TC_MAX_PROJ];
  const int p = blockIdx.y;
  const GroupProb& P = probs[p];
  const size_t e0 = 4 * ((size_t)blockIdx.x * GRP_NT);
  if (e0 >= P.Tx) return;  // uniform over the CTA
  const double* b = scal + p * lay.stride();
  const int k = max(0, min(flags[16 * p + 1], kmax));
  for (int i = threadIdx.x; i < k; i += GRP_NT) {
    const double d = b[i];  // alpha_{i+1}
    c1[i] = (float)(b[lay.gwork() + i] / d);
    c2[i] = (float)(b[lay.y() + i] / d);
  }
  __syncthreads();
  const size_t e = e0 + 4 * threadIdx.x;
  if (e >= P.Tx) return;
  const bool vec = P.Tx % 4 == 0 && ((reinterpret_cast<uintptr_t>(P.basis) |
                                      reinterpret_cast<uintptr_t>(P.X) |
                                      reinterpret_cast<uintptr_t>(P.Xr)) & 15) == 0;
  if (vec) {  // e + 3 < Tx
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), r = a;
    for (int i = 0; i < k; ++i) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(P.basis + (size_t)i * P.Tx + e));
      a.x = fmaf(c1[i], v.x, a.x); a.y = fmaf(c1[i], v.y, a.y);
      a.z = fmaf(c1[i], v.z, a.z); a.w = fmaf(c1[i], v.w, a.w);
      r.x = fmaf(c2[i], v.x, r.x); r.y = fmaf(c2[i], v.y, r.y);
      r.z = fmaf(c2[i], v.z, r.z); r.w = fmaf(c2[i], v.w, r.w);
    }
    *reinterpret_cast<float4*>(P.X + e) = a;
    *reinterpret_cast<float4*>(P.Xr + e) = r;
    return;
  }
  for (size_t q = e; q < e + 4 && q < P.Tx; ++q) {
    float a = 0.f, r = 0.f;
    for (int i = 0; i < k; ++i) {
      const float v = __ldg(P.basis + (size_t)i * P.Tx + q);
      a = fmaf(c1[i], v, a);
      r = fmaf(c2[i], v, r);
    }
    P.X[q] = a;
    P.Xr[q] = r;
  }
}

__global__ void k_group_info(tc_solve_info* infos, const double* scal, Layout lay,
                             const int* flags, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const double* b = scal + p * lay.stride();
  const int* f = flags + 16 * p;
  tc_solve_info* info = infos + p;
  const int it = f[1];
  info->iters = it;
  info->status = f[2];
  info->cycles = 0;
  info->fallback = 0;
  info->resid = fabs(b[lay.phibar() + it]);
  info->lambda = b[lay.lam()];
  info->gcv = b[lay.gcv()];
  info->beta1 = b[lay.beta()];
  info->kopt = 0;
  info->reserved = 0;
}

template <class T>
int dgrow(T** p, size_t* have, size_t need) {
  if (*p && *have >= need) return TC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  const cudaError_t e = cudaMalloc((void**)p, (need ? need : 1) * sizeof(T));
  if (e != cudaSuccess) {
    tc_set_error("cudaMalloc", e);
    return TC_ENOMEM;
  }
  *have = need;
  return TC_OK;
}

}  // namespace

bool group_eligible(const std::vector<tc_plan*>& plans, const float* const* C, bool keep) {
  if (!keep || plans.empty()) return false;
  const int prec = plans[0]->opts.precision;
  if (prec != TC_FP32 && prec != TC_BF16) return false;
  // BF16 ORTHODCT plans iterate in the transform domain (BF16 operands written
  // by the previous product's epilogue, no transform passes); as child graphs
  // that form is the faster one (6.5k against 5.3k solves/s on 128 problems
  // of n in 64..512, x3)
  if (prec == TC_BF16 && plans[0]->opts.product == TC_ORTHODCT) return false;
  for (const tc_plan* p : plans) {
    if (p->opts.precision != prec || p->n3 > TC_MAX_FUSED || p->two_sided ||
        p->n3 != plans[0]->n3 || p->opts.product != plans[0]->opts.product ||
        p->opts.gcv_variant != plans[0]->opts.gcv_variant)
      return false;
    if (prec == TC_BF16 &&
        (!p->AhL || !p->AhTL || p->n1 % 8 != 0 || p->n2 % 8 != 0 || p->s % 8 != 0))
      return false;
  }
  if (prec == TC_BF16)  // C is read as float4
    for (size_t i = 0; i < plans.size(); ++i)
      if (reinterpret_cast<uintptr_t>(C[i]) & 15) return false;
  return true;
}

void group_free(GroupState* g) {
  void* ps[] = {g->probs, g->scal, g->flags, g->done, g->partials, g->tickets};
  for (void* q : ps)
    if (q) cudaFree(q);
  for (int c = 0; c < GROUP_CFGS; ++c)
    for (int d = 0; d < 2; ++d)
      if (g->work[c][d]) cudaFree(g->work[c][d]);
  *g = GroupState{};
}

// Tables of the batch for itermax steps: per-problem descriptors (host and
// device), scalars, flags, partials, tickets and both tile shapes' work tables.
int group_prepare(GroupState* g, const std::vector<tc_plan*>& plans, const float* const* C,
                  float* const* X, float* const* Xr, int itermax, cudaStream_t st) {
  const int count = (int)plans.size();
  const Layout lay{(size_t)itermax + 2, (size_t)(itermax < TC_MAX_PROJ ? itermax : TC_MAX_PROJ)};
  const int bf16 = plans[0]->opts.precision == TC_BF16, ncfg = group_cfg_count(bf16);
  std::vector<GroupProb> hp(count);
  std::vector<int2> wk[GROUP_CFGS][2];
  size_t npart = 0;
  for (int i = 0; i < count; ++i) {
    tc_plan* p = plans[i];
    GroupProb& q = hp[i];
    q.Ah = p->Ah;
    q.AhT = p->AhT;
    q.AhL = p->AhL;
    q.AhTL = p->AhTL;
    q.C = C[i];
    q.X = X[i];
    q.Xr = Xr[i];
    q.U = p->lsqr_U;
    q.V = p->lsqr_V;
    q.basis = p->basis;
    q.Tx = p->Tx;
    q.Ty = p->Ty;
    q.n1 = p->n1;
    q.n2 = p->n2;
    q.s = p->s;
    size_t most = NORM_CTAS;
    for (int c = 0; c < ncfg; ++c) {
      int TM, TN;
      group_tile_shape(bf16, c, &TM, &TN);
      const int tn = (q.s + TN - 1) / TN;
      const int tf = ((q.n1 + TM - 1) / TM) * tn, ta = ((q.n2 + TM - 1) / TM) * tn;
      for (int t = 0; t < tf; ++t) wk[c][0].push_back(make_int2(i, t));
      for (int t = 0; t < ta; ++t) wk[c][1].push_back(make_int2(i, t));
      if ((size_t)tf > most) most = tf;
      if ((size_t)ta > most) most = ta;
    }
    q.partials = reinterpret_cast<double*>(npart);  // offset, made a pointer below
    npart += most;
  }
  TC_TRY(dgrow(&g->probs, &g->probs_n, (size_t)count));
  TC_TRY(dgrow(&g->scal, &g->scal_n, (size_t)count * lay.stride()));
  TC_TRY(dgrow(&g->flags, &g->flags_n, (size_t)count * 16));
  TC_TRY(dgrow(&g->done, &g->done_n, (size_t)count * lay.L));
  TC_TRY(dgrow(&g->partials, &g->partials_n, npart));
  if (!g->tickets || g->tickets_n < (size_t)count) {
    TC_TRY(dgrow(&g->tickets, &g->tickets_n, (size_t)count));
    TC_CUDA(cudaMemsetAsync(g->tickets, 0, (size_t)count * sizeof(unsigned), st));
  }
  for (int c = 0; c < ncfg; ++c)
    for (int d = 0; d < 2; ++d) {
      TC_TRY(dgrow(&g->work[c][d], &g->work_n[c][d], wk[c][d].size()));
      TC_CUDA(cudaMemcpyAsync(g->work[c][d], wk[c][d].data(), wk[c][d].size() * sizeof(int2),
                              cudaMemcpyHostToDevice, st));
      g->nwork[c][d] = (int)wk[c][d].size();
    }
  for (int i = 0; i < count; ++i) {
    hp[i].partials = g->partials + reinterpret_cast<size_t>(hp[i].partials);
    hp[i].ticket = g->tickets + i;
  }
  g->host = hp;
  g->bf16 = bf16;
  g->ncfg = ncfg;
  g->count = count;
  g->itermax = itermax;
  g->stride = lay.stride();
  g->L = lay.L;
  g->kp = lay.kp;
  TC_CUDA(cudaMemcpyAsync(g->probs, hp.data(), hp.size() * sizeof(GroupProb),
                          cudaMemcpyHostToDevice, st));
  TC_CUDA(cudaStreamSynchronize(st));
  return TC_OK;
}

namespace {
int set_tiles(GroupState* g, int cfg) {
  int TM, TN;
  group_tile_shape(g->bf16, cfg, &TM, &TN);
  for (int i = 0; i < g->count; ++i) {
    GroupProb& q = g->host[i];
    const int tn = (q.s + TN - 1) / TN;
    q.tiles_f = ((q.n1 + TM - 1) / TM) * tn;
    q.tiles_a = ((q.n2 + TM - 1) / TM) * tn;
  }
  return TC_OK;
}

GroupOp make_op(const GroupState* g, int kind, int j) {
  GroupOp o;
  o.op = kind;
  o.j = j;
  o.itermax = g->itermax;
  o.lstride = (int)g->L;
  o.scal = g->scal;
  o.sstride = g->stride;
  o.flags = g->flags;
  o.done = g->done;
  return o;
}

// Product `kind` of step j of every problem with tile shape cfg: the forward
// product transforms with (M, M^-1), the adjoint and the first product with
// (M^-T, M^T).
int launch_op(const GroupState* g, const tc_plan* p0, int kind, int j, int cfg, cudaStream_t st) {
  const int d = kind == GOP_FWD ? 0 : 1;
  const float* pro = d == 0 ? p0->hM : p0->hMinvT;
  const float* epi = d == 0 ? p0->hMinv : p0->hMT;
  const GroupOp o = make_op(g, kind, j);
  return g->bf16 ? launch_group_umma(g->probs, g->work[cfg][d], g->nwork[cfg][d], o, pro, epi,
                                     p0->n3, cfg, st)
                 : launch_group_gemm(g->probs, g->work[cfg][d], g->nwork[cfg][d], o, pro, epi,
                                     p0->n3, cfg, st);
}
}  // namespace

// Time the forward product of the batch with each tile shape (a warm-up and
// three launches each, CUDA events on `st`, outside any capture) and keep the
// fastest.
int group_autotune(GroupState* g, const tc_plan* p0, cudaStream_t st) {
  k_group_reset<<<g->count, 128, 0, st>>>(g->flags, g->done, g->tickets, (int)g->L, g->count);
  TC_CUDA(cudaGetLastError());
  float best = 1e30f;
  int pick = 0;
  cudaEvent_t e0, e1;
  TC_CUDA(cudaEventCreate(&e0));
  TC_CUDA(cudaEventCreate(&e1));
  for (int c = 0; c < GROUP_CFGS; ++c) g->tune_ms[c] = 0.f;
  for (int c = 0; c < g->ncfg; ++c) {
    set_tiles(g, c);
    TC_CUDA(cudaMemcpyAsync(g->probs, g->host.data(), g->host.size() * sizeof(GroupProb),
                            cudaMemcpyHostToDevice, st));
    TC_TRY(launch_op(g, p0, GOP_FWD, 0, c, st));  // warm-up
    TC_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; ++r) TC_TRY(launch_op(g, p0, GOP_FWD, 0, c, st));
    TC_CUDA(cudaEventRecord(e1, st));
    TC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    TC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    g->tune_ms[c] = ms / 3.f;
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->cfg = pick;
  set_tiles(g, pick);
  TC_CUDA(cudaMemcpyAsync(g->probs, g->host.data(), g->host.size() * sizeof(GroupProb),
                          cudaMemcpyHostToDevice, st));
  TC_CUDA(cudaStreamSynchronize(st));
  return TC_OK;
}

// Tile shape cfg without timing (tc_batch_info's forced modes).
int group_fix_tile(GroupState* g, int cfg, cudaStream_t st) {
  TC_CHECK(cfg >= 0 && cfg < g->ncfg);
  for (int c = 0; c < GROUP_CFGS; ++c) g->tune_ms[c] = 0.f;
  g->cfg = cfg;
  set_tiles(g, cfg);
  TC_CUDA(cudaMemcpyAsync(g->probs, g->host.data(), g->host.size() * sizeof(GroupProb),
                          cudaMemcpyHostToDevice, st));
  TC_CUDA(cudaStreamSynchronize(st));
  return TC_OK;
}

// The grouped solve on `st` (capturable): the same steps as lsqr_enqueue with
// a kept basis, every launch over all problems.
int group_enqueue(GroupState* g, const tc_plan* p0, double tol, double lambda,
                  tc_solve_info* infos, cudaStream_t st) {
  const int count = g->count, itermax = g->itermax, c = g->cfg;
  const Layout lay{g->L, g->kp};
  const int tb = (count + 127) / 128;
  k_group_reset<<<count, 128, 0, st>>>(g->flags, g->done, g->tickets, (int)g->L, count);
  TC_CUDA(cudaGetLastError());
  k_group_norm_c<<<dim3(NORM_CTAS, count), GRP_NT, 0, st>>>(g->probs, g->scal, lay, g->flags);
  TC_CUDA(cudaGetLastError());
  TC_TRY(launch_op(g, p0, GOP_INIT, 0, c, st));
  k_group_lsqr_init<<<tb, 128, 0, st>>>(g->scal, lay, g->flags, g->done, count);
  TC_CUDA(cudaGetLastError());
  for (int j = 0; j < itermax; ++j) {
    if (j > 0) {
      k_group_scalars<<<tb, 128, 0, st>>>(g->scal, lay, g->flags, g->done, j - 1, tol, count);
      TC_CUDA(cudaGetLastError());
    }
    TC_TRY(launch_op(g, p0, GOP_FWD, j, c, st));
    TC_TRY(launch_op(g, p0, GOP_ADJ, j, c, st));
  }
  k_group_scalars<<<tb, 128, 0, st>>>(g->scal, lay, g->flags, g->done, itermax - 1, tol, count);
  TC_CUDA(cudaGetLastError());
  const int kp = (int)g->kp;
  TC_TRY(launch_gcv_bidiag_group(g->scal + lay.rgiv(), g->scal + lay.phibar(), g->scal,
                                 g->scal + lay.beta(), g->flags + 1, kp, p0->opts.gcv_variant,
                                 lambda, g->scal + lay.gwork(), g->scal + lay.lam(),
                                 g->scal + lay.y(), g->scal + lay.gcv(), count, lay.stride(), 16,
                                 st));
  k_group_coeffs<<<tb, 128, 0, st>>>(g->scal, lay, g->flags, kp, count);
  TC_CUDA(cudaGetLastError());
  size_t most = 0;
  for (const GroupProb& q : g->host)
    if (q.Tx > most) most = q.Tx;
  const unsigned blocks = (unsigned)((most + 4 * (size_t)GRP_NT - 1) / (4 * (size_t)GRP_NT));
  k_group_combine2<<<dim3(blocks, count), GRP_NT, 0, st>>>(g->probs, g->scal, lay, g->flags, kp);
  TC_CUDA(cudaGetLastError());
  k_group_info<<<tb, 128, 0, st>>>(infos, g->scal, lay, g->flags, count);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
