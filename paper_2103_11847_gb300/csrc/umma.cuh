// tcgen05 slice GEMM interface (umma.cu).
#pragma once

#include <cuda.h>

#include "tc_internal.cuh"

struct UmmaMaps {
  CUtensorMap a;  // M x K per slice, K contiguous (K-major operand)
  CUtensorMap b;  // BF16: K x N per slice (MN-major); TF32: N x K per slice (K-major)
  int M = 0, N = 0, K = 0, slices = 0, kind = 0;  // kind 0: BF16, 1: TF32
};

int umma_init();
int make_umma_maps(UmmaMaps* m, int kind, const void* A, const void* B, int M, int N, int K,
                   int slices);
// D_z = A_z B_z in FP32 for every slice; *err is set to TC_ETIMEOUT if a
// bounded wait gives up.
int launch_umma(const UmmaMaps& m, float* D, int* err, const int* skip, cudaStream_t st);
