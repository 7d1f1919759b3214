// The grouped batched solve (group.cu): its device tables and entry points.
#pragma once

#include <vector>

#include "tc_device.cuh"

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
  int2* work[GROUP_CFGS][2] = {};    // [tile shape][forward, adjoint]
  int nwork[GROUP_CFGS][2] = {};
  size_t probs_n = 0, scal_n = 0, flags_n = 0, done_n = 0, partials_n = 0, tickets_n = 0;
  size_t work_n[GROUP_CFGS][2] = {};
  int cfg = -1;                      // tile shape chosen by group_autotune
  float tune_ms[GROUP_CFGS] = {};    // the forward product's time with each
};

// Plans that take the grouped path: FP32, n3 <= TC_MAX_FUSED, one-sided,
// sharing n3, product and GCV variant, with X_reg requested.
bool group_eligible(const std::vector<tc_plan*>& plans, bool keep);
int group_prepare(GroupState* g, const std::vector<tc_plan*>& plans, const float* const* C,
                  float* const* X, float* const* Xr, int itermax, cudaStream_t st);
int group_autotune(GroupState* g, const tc_plan* p0, cudaStream_t st);
int group_enqueue(GroupState* g, const tc_plan* p0, double tol, double lambda,
                  tc_solve_info* infos, cudaStream_t st);
void group_free(GroupState* g);
