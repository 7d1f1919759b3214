// The learned-lambda network (mlp.cu) and its use by the learned solve.
#pragma once

#include <cuda_bf16.h>

#include "tc_internal.cuh"

#define MLP_IN 36
#define MLP_HID 64
#define MLP_OUT 2
#define MLP_NPARAMS (MLP_IN * MLP_HID + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID * MLP_OUT + MLP_OUT)
#define MLP_NORM (2 * MLP_IN + 2 * MLP_OUT)  // feature mean, std; target mean, std
#define MLP_FEAT_STEPS 12

const __nv_bfloat16* mlp_weights(const tc_mlp* m);
const float* mlp_theta(const tc_mlp* m);
const float* mlp_norm(const tc_mlp* m);
