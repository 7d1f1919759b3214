// Batched c-LSQR: many independent problems of uneven sizes solved together.
//
// Each problem has its own plan: A~ resident, its own workspaces. Two forms:
// * grouped (group.cu): FP32 or BF16 plans with n3 <= 4 and X_reg requested.
//   Every phase of the solve is one launch over all problems, the tile shape
//   autotuned per batch, the whole sequence captured as one CUDA graph;
// * otherwise each problem's whole solve (Algorithm 6, then the
//   Tikhonov/GCV projection) is captured as a child graph, and the children
//   sit side by side in one parent graph with no edges between them, so one
//   cudaGraphLaunch submits the batch and the problems' kernels run
//   concurrently.
// Either graph is kept and relaunched while the pointers and parameters stay
// the same.
#include <cstring>
#include <new>
#include <vector>

#include "group.cuh"

struct tc_batch {
  int count = 0;
  std::vector<tc_plan*> plans;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> key;
  GroupState grp;
  int batch_mode = 0;  // 0: grouped where eligible, 1: child graphs always, 2 + t: tile shape t
};

extern "C" int tc_batch_destroy(tc_batch* b) {
  if (!b) return TC_EINVAL;
  group_free(&b->grp);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (tc_plan* p : b->plans)
    if (p) tc_plan_destroy(p);
  delete b;
  return TC_OK;
}

extern "C" int tc_batch_create(tc_batch** out, int count, const int* n1, const int* n2,
                               const int* s, int n3, const float* const* A, const tc_opts* opts,
                               tc_stream_t stream) {
  if (!out || count < 1 || !n1 || !n2 || !s || !A) return TC_EINVAL;
  *out = nullptr;
  tc_batch* b = new (std::nothrow) tc_batch();
  if (!b) return TC_ENOMEM;
  b->count = count;
  b->plans.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    const int r = tc_plan_create(&b->plans[i], n1[i], n2[i], s[i], n3, A[i], nullptr, opts, stream);
    if (r != TC_OK) {
      tc_batch_destroy(b);
      return r;
    }
  }
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    tc_batch_destroy(b);
    return TC_ECUDA;
  }
  *out = b;
  return TC_OK;
}

extern "C" int tc_lsqr_c_batched(tc_batch* b, const float* const* C, float* const* X,
                                 float* const* X_reg, int itermax, double tol, double lambda,
                                 tc_solve_info* infos, tc_stream_t stream) {
  if (!b || !C || !X || !infos) return TC_EINVAL;
  if (itermax < 1 || itermax > 4096 || !(tol >= 0.0)) return TC_EINVAL;
  if (X_reg && itermax > TC_MAX_PROJ) return TC_EINVAL;
  const int n = b->count;
  for (int i = 0; i < n; ++i) {
    if (!C[i] || !X[i] || (X_reg && !X_reg[i])) return TC_EINVAL;
    TC_TRY(ensure_lsqr(b->plans[i], itermax, X_reg != nullptr));
  }
  uint64_t tb, lb;
  std::memcpy(&tb, &tol, 8);
  std::memcpy(&lb, &lambda, 8);
  std::vector<uintptr_t> key = {(uintptr_t)itermax, (uintptr_t)tb, (uintptr_t)lb, (uintptr_t)infos,
                                (uintptr_t)(X_reg != nullptr), (uintptr_t)b->batch_mode};
  for (int i = 0; i < n; ++i) {
    key.push_back((uintptr_t)C[i]);
    key.push_back((uintptr_t)X[i]);
    key.push_back(X_reg ? (uintptr_t)X_reg[i] : 0);
    key.push_back((uintptr_t)b->plans[i]->dscal);  // workspaces a capture depends on
    key.push_back((uintptr_t)b->plans[i]->basis);
  }
  const bool grouped = b->batch_mode != 1 && group_eligible(b->plans, C, X_reg != nullptr);
  if (grouped && (!b->exec || key != b->key)) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaStream_t st = (cudaStream_t)stream;
    TC_TRY(group_prepare(&b->grp, b->plans, C, X, X_reg, itermax, st));
    if (b->batch_mode == 0) TC_TRY(group_autotune(&b->grp, b->plans[0], st));
    else TC_TRY(group_fix_tile(&b->grp, b->batch_mode - 2, st));
    cudaGraph_t g = nullptr;
    TC_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    const int rc = group_enqueue(&b->grp, b->plans[0], tol, lambda, infos, b->cap);
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (rc != TC_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (rc != TC_OK) return rc;
      tc_set_error("cudaStreamEndCapture", e);
      return TC_ECUDA;
    }
    const cudaError_t e2 = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
      b->exec = nullptr;
      tc_set_error("cudaGraphInstantiate", e2);
      return TC_ECUDA;
    }
    b->key = key;
  }
  if (!grouped && (!b->exec || key != b->key)) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t parent = nullptr;
    TC_CUDA(cudaGraphCreate(&parent, 0));
    int rc = TC_OK;
    for (int i = 0; i < n && rc == TC_OK; ++i) {
      LsqrArgs a{C[i], X[i], X_reg ? X_reg[i] : nullptr, itermax, tol, lambda, nullptr, infos + i};
      cudaGraph_t child = nullptr;
      cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        tc_set_error("cudaStreamBeginCapture", e);
        rc = TC_ECUDA;
        break;
      }
      rc = lsqr_enqueue(b->plans[i], a, b->cap);
      e = cudaStreamEndCapture(b->cap, &child);
      if (rc == TC_OK && e != cudaSuccess) {
        tc_set_error("cudaStreamEndCapture", e);
        rc = TC_ECUDA;
      }
      if (rc == TC_OK) {
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, child);
        if (e != cudaSuccess) {
          tc_set_error("cudaGraphAddChildGraphNode", e);
          rc = TC_ECUDA;
        }
      }
      if (child) cudaGraphDestroy(child);
    }
    if (rc == TC_OK) {
      const cudaError_t e = cudaGraphInstantiate(&b->exec, parent, 0);
      if (e != cudaSuccess) {
        tc_set_error("cudaGraphInstantiate", e);
        b->exec = nullptr;
        rc = TC_ECUDA;
      }
    }
    cudaGraphDestroy(parent);
    if (rc != TC_OK) return rc;
    b->key = key;
  }
  TC_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return TC_OK;
}

extern "C" int tc_batch_info(tc_batch* b, int mode, int* grouped, int* tile, float* tune_ms) {
  if (!b || mode < -1 || mode > 1 + GROUP_CFGS) return TC_EINVAL;
  if (mode >= 0 && mode != b->batch_mode) {
    b->batch_mode = mode;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  if (grouped) *grouped = b->batch_mode != 1 && b->grp.cfg >= 0;
  if (tile) *tile = b->grp.cfg >= 0 ? b->grp.cfg : -1;
  if (tune_ms)
    for (int c = 0; c < GROUP_CFGS; ++c) tune_ms[c] = b->grp.tune_ms[c];
  return TC_OK;
}

