// tcgen05 slice GEMM interface (umma.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "tc_internal.cuh"

struct UmmaMaps {
  CUtensorMap a;  // M x K per slice, K contiguous (K-major operand)
  CUtensorMap b;  // BF16: K x N per slice (MN-major); TF32: N x K per slice (K-major)
  int M = 0, N = 0, K = 0, slices = 0, kind = 0;  // kind 0: BF16, 1: TF32
  int nsplit = 1;  // 3: each operand is three stacked BF16 planes (FP32-level products)
};

int umma_init();
// nsplit 3 (BF16 only): A and B hold three planes each, plane p of slice z at
// slice p * slices + z.
int make_umma_maps(UmmaMaps* m, int kind, const void* A, const void* B, int M, int N, int K,
                   int slices, int nsplit = 1);
// D_z = A_z B_z in FP32 for every slice (nsplit 3: the six split products);
// *err is set to TC_ETIMEOUT if a bounded wait gives up.
// out_bf16 (BF16 maps, one plane): D receives BF16 values, bf16(A_z B_z).
int launch_umma(const UmmaMaps& m, float* D, int* err, const int* skip, cudaStream_t st,
                bool out_bf16 = false);
// BF16 maps only: the same GEMM with the Krylov epilogue in its store
// (D = ca * acc + cp * ep.prev, the reduction ep.red of D, ep.skip) and, when
// dlow is non-null, a BF16 copy of D written beside it (nsplit 3: its three
// planes, plane q at dlow + q slices M N).
int launch_umma_epi(const UmmaMaps& m, float* D, __nv_bfloat16* dlow, const Epi& ep, int* err,
                    cudaStream_t st);
// 3-D tiled map over `slices` row-major rows x inner matrices (FP32, or BF16
// with bf16 = 1), box (box_inner, box_rows, 1), 128-byte swizzle, zero fill
// out of bounds. The base must be 16-byte aligned and a row a multiple of 16
// bytes.
int make_tmap(CUtensorMap* map, const void* base, int bf16, int inner, int rows, int slices,
              int box_inner, int box_rows);
// 2-D tiled map over a rows x inner row-major tensor (FP32, or BF16 with
// bf16 = 1), box (box_inner, box_rows), no swizzle, zero fill out of bounds.
// The base must be 16-byte aligned and a row a multiple of 16 bytes.
int make_tmap_2d(CUtensorMap* map, const void* base, int bf16, size_t inner, size_t rows,
                 int box_inner, int box_rows);

