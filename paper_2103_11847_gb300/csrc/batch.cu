// Batched c-LSQR: many independent problems of uneven sizes solved together.
//
// Each problem has its own plan: A~ resident, its own workspaces, reduction
// scratch and device-side scalars. Its whole solve (Algorithm 6, then the
// Tikhonov/GCV projection) is captured as a child graph. The children are
// placed side by side in one parent graph with no edges between them, so one
// cudaGraphLaunch submits the batch and the GPU runs the problems' kernels
// concurrently: small problems fill the SMs that large ones leave idle. The
// parent graph is kept and relaunched while the pointers and parameters
// stay the same.
#include <cstring>
#include <new>
#include <vector>

#include "tc_device.cuh"

struct tc_batch {
  int count = 0;
  std::vector<tc_plan*> plans;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> key;
};

extern "C" int tc_batch_destroy(tc_batch* b) {
  if (!b) return TC_EINVAL;
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
                                (uintptr_t)(X_reg != nullptr)};
  for (int i = 0; i < n; ++i) {
    key.push_back((uintptr_t)C[i]);
    key.push_back((uintptr_t)X[i]);
    key.push_back(X_reg ? (uintptr_t)X_reg[i] : 0);
    key.push_back((uintptr_t)b->plans[i]->dscal);  // workspaces a capture depends on
    key.push_back((uintptr_t)b->plans[i]->basis);
  }
  if (!b->exec || key != b->key) {
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
