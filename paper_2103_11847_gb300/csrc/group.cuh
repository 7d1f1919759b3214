// The grouped batched solve (group.cu): its device tables and entry points.
#pragma once

#include <vector>

#include "tc_device.cuh"

// The operands of grouped product g.op of problem p (k_group_gemm in gemm.cu,
// k_group_umma in group_tc.cu): Algorithm 6's products with their Krylov
// epilogues (steps 2, 3(a) and 3(b)), the deferred schedule (no vector
// updates; V~_j kept in the basis).
struct GroupOperands {
  bool fwd;
  int M, N, K;         // output rows and columns, contraction length
  const float* B;      // K x N a slice
  float* C;            // M x N a slice
  const float* prev;   // M x N a slice, or null
  Coef coef;
  Red red;
};

__device__ __forceinline__ GroupOperands group_operands(const GroupProb& P, const GroupOp& g,
                                                        int p) {
  const size_t L = (size_t)g.lstride;
  double* alpha = g.scal + (size_t)p * g.sstride;
  double* beta = alpha + L;
  GroupOperands o;
  o.fwd = g.op == GOP_FWD;
  o.M = o.fwd ? P.n1 : P.n2;
  o.K = o.fwd ? P.n2 : P.n1;
  o.N = P.s;
  o.prev = nullptr;
  o.red.sqrt_out = 1;
  o.red.partials = P.partials;
  o.red.ticket = P.ticket;
  o.red.status = g.flags + 16 * p + 2;
  if (g.op == GOP_INIT) {  // V~_1 = A^T (C / beta_1), alpha_1 = ||V~_1||
    o.B = P.C;
    o.C = P.basis;
    o.coef.rule = COEF_INV;
    o.coef.s0 = beta;
    o.red.out = alpha;
  } else if (o.fwd) {  // U~ = (1/alpha_j) A V~_j - (alpha_j/beta_j) U~, beta_{j+1}
    o.B = P.basis + (size_t)g.j * P.Tx;
    o.C = P.U;
    o.prev = g.j == 0 ? P.C : P.U;
    o.coef.rule = COEF_GK;
    o.coef.s0 = alpha + g.j;
    o.coef.s1 = beta + g.j;
    o.red.out = beta + g.j + 1;
  } else {  // V~_{j+1} = (1/beta_{j+1}) A^T U~ - (beta_{j+1}/alpha_j) V~_j, alpha_{j+1}
    o.B = P.U;
    o.C = g.j + 1 < g.itermax ? P.basis + (size_t)(g.j + 1) * P.Tx : P.V;
    o.prev = P.basis + (size_t)g.j * P.Tx;
    o.coef.rule = COEF_GK;
    o.coef.s0 = beta + g.j + 1;
    o.coef.s1 = alpha + g.j;
    o.red.out = alpha + g.j + 1;
  }
  return o;
}

struct GroupState {
  int count = 0, itermax = 0;
  size_t stride = 0, L = 0, kp = 0;  // per-problem scalars: doubles, steps + 2, projection size
  GroupProb* probs = nullptr;        // device table
  std::vector<GroupProb> host;       // its host copy
  double* scal = nullptr;
  int* flags = nullptr;
  int* done = nullptr;
  double* partials = nullptr;
  unsigned* tickets = nullptr;
  int bf16 = 0;                      // 1: BF16 plans (group_tc.cu), 0: FP32 (gemm.cu)
  int ncfg = 0;                      // tile shapes the autotuner times
  int2* work[GROUP_CFGS][2] = {};    // [tile shape][forward, adjoint]
  int nwork[GROUP_CFGS][2] = {};
  size_t probs_n = 0, scal_n = 0, flags_n = 0, done_n = 0, partials_n = 0, tickets_n = 0;
  size_t work_n[GROUP_CFGS][2] = {};
  int cfg = -1;                      // tile shape chosen by group_autotune
  float tune_ms[GROUP_CFGS] = {};    // the forward product's time with each
};

// Plans that take the grouped path: n3 <= TC_MAX_FUSED, one-sided, sharing
// precision, n3, product and GCV variant, with X_reg requested; FP32, or BF16
// under the default product with n1, n2 and s multiples of 8 (whole 16-byte
// operand chunks) and every C 16-byte aligned.
bool group_eligible(const std::vector<tc_plan*>& plans, const float* const* C, bool keep);
int group_prepare(GroupState* g, const std::vector<tc_plan*>& plans, const float* const* C,
                  float* const* X, float* const* Xr, int itermax, cudaStream_t st);
int group_autotune(GroupState* g, const tc_plan* p0, cudaStream_t st);
int group_fix_tile(GroupState* g, int cfg, cudaStream_t st);
int group_enqueue(GroupState* g, const tc_plan* p0, double tol, double lambda,
                  tc_solve_info* infos, cudaStream_t st);
void group_free(GroupState* g);
