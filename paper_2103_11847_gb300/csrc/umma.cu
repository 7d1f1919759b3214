// Frontal-slice GEMMs on the 5th-generation tensor cores (tcgen05), for the
// TF32 and BF16 precision forms of the c-product (Algorithm 1, step 2):
//   D_z = A_z B_z,  A_z: M x K (K contiguous), B_z: K x N (N contiguous),
//   D_z: M x N FP32, for every slice z of the grid.
//
// One CTA computes a 128 x 128 tile of one slice with a 128-lane x 128-column
// FP32 accumulator in tensor memory:
//   warp 0, one lane : TMA producer (cp.async.bulk.tensor.3d, 128B swizzle),
//                      STAGES-deep ring of (A, B) stages in shared memory;
//   warp 1, one lane : issues tcgen05.mma (kind::f16 with BF16 inputs, or
//                      kind::tf32) and tcgen05.commit to release each stage;
//   all four warps   : epilogue, tcgen05.ld of 32 lanes x 32 columns at a time.
// A is read K-major. B is read MN-major straight from the row-major K x N
// operand for BF16. For TF32 it is read K-major from a per-slice transposed
// copy (N x K): kind::tf32 with an MN-major B left the accumulator unchanged
// on this part. Each CTA fetches its own tiles (no cluster multicast).
//
// Every mbarrier wait is bounded. A wait that gives up raises *err, and the
// CTA skips the rest of its work, waits (bounded) for the copies it issued,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "tc_device.cuh"
#include "umma.cuh"

namespace {

constexpr int BM = 128, BN = 128, STAGES = 3, NT = 128;  // 97 KB smem: 2 CTAs per SM
constexpr uint32_t A_BYTES = BM * 128;   // 128 rows of one 128-byte K slab
constexpr uint32_t B_BYTES = 128 * BN;   // (128 / elem) K rows x BN columns
constexpr int kSpin = 1 << 22;           // try_wait polls before giving up

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kSpin; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(su32(bar))
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (16-byte units), version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                     uint32_t accum) {
  if (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
      "%29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// KIND 0: BF16 inputs (kind::f16), KIND 1: TF32 inputs (kind::tf32).
// BKMAJ: B given as N x K per slice (K contiguous) instead of K x N.
// EPI: the Krylov epilogue in the store: D = ca * acc + cp * prev (prev may
// alias D; each element is read and written by one thread), an optional BF16
// copy of D into dlow (the next GEMM's operand), and the fused reduction of D.
// Without EPI the accumulator is stored as is.
template <int KIND, int BKMAJ, bool EPI>
__global__ void __launch_bounds__(NT, 2)
k_umma_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            float* D, int M, int N, int K, int* err, const int* skip, Epi ep,
            __nv_bfloat16* dlow) {
  constexpr int ES = KIND == 0 ? 2 : 4;       // bytes per element
  constexpr int BKE = 128 / ES;               // K elements per stage
  constexpr int UK = KIND == 0 ? 16 : 8;      // K per MMA instruction
  constexpr int NATOM = 128 / ES;             // N elements per B swizzle atom column
  constexpr int NBOX = BN / NATOM;            // B boxes per stage
  constexpr uint32_t B_COL = BKE * 128;       // bytes of one B atom column
  constexpr uint32_t FMT = KIND == 0 ? 1u : 2u;  // BF16 : TF32
  constexpr uint32_t BMAJ = BKMAJ ? 0u : 1u;  // 0: K-major, 1: MN-major
  constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) | (0u << 15) | (BMAJ << 16) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  if (skip && *skip) return;
  extern __shared__ uint8_t dsm_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int sh_fail;
  __shared__ float sh_coef[2];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN, z = blockIdx.z;
  const int nk = (K + BKE - 1) / BKE;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh_fail = 0;
  }
  if (EPI && threadIdx.x == 64) {  // warp 2 is idle until the epilogue
    double ca = 1.0, cp = 0.0;
    const Coef& c = ep.coef;
    if (c.rule == COEF_GK) {
      const double s0 = *c.s0, s1 = *c.s1;
      ca = (s0 != 0.0) ? 1.0 / s0 : 0.0;
      cp = (s1 != 0.0) ? -s0 / s1 : 0.0;
    } else if (c.rule == COEF_INV) {
      const double s0 = *c.s0;
      ca = (s0 != 0.0) ? 1.0 / s0 : 0.0;
    } else if (c.rule == COEF_RESID) {
      ca = -1.0;
      cp = 1.0;
    } else if (c.rule == COEF_NEG) {
      ca = -1.0;
    } else if (c.rule == COEF_AXPY) {
      cp = -*c.s0;
    }
    sh_coef[0] = (float)ca;
    sh_coef[1] = (float)cp;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tslot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  int issued = 0;  // stages the producer armed (for the bounded drain on failure)
  // EPI: prev does not depend on the GEMM, so every thread loads its row's
  // BN values of prev now and the loads overlap the main loop (whole 32-column
  // chunks with N % 4 == 0; the edge chunks read prev in the epilogue).
  float4 pre[EPI ? BN / 4 : 1];
  if (EPI) {
    const int prow = m0 + warp * 32 + lane;
#pragma unroll
    for (int q = 0; q < BN / 4; ++q) {
      const int col = n0 + 4 * q;
      const bool whole = ep.prev && prow < M && (N & 3) == 0 && n0 + (q / 8) * 32 + 32 <= N;
      pre[q] = whole ? *reinterpret_cast<const float4*>(ep.prev + (size_t)z * M * N +
                                                         (size_t)prow * N + col)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }

  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(empty + s, ph ^ 1)) {
        sh_fail = 1;
        break;
      }
      mbar_expect_tx(full + s, A_BYTES + B_BYTES);
      tma_load_3d(sA + s * A_BYTES, &tmA, kb * BKE, m0, z, full + s);
      if (BKMAJ) {
        tma_load_3d(sB + s * B_BYTES, &tmB, kb * BKE, n0, z, full + s);
      } else {
#pragma unroll
        for (int b = 0; b < NBOX; ++b)
          tma_load_3d(sB + s * B_BYTES + b * B_COL, &tmB, n0 + b * NATOM, kb * BKE, z, full + s);
      }
      issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(full + s, ph)) {
        sh_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = su32(sA + s * A_BYTES), b0 = su32(sB + s * B_BYTES);
#pragma unroll
      for (int kk = 0; kk < BKE / UK; ++kk) {
        const uint64_t ad = smem_desc(a0 + kk * UK * ES, 16, 1024);  // K-major: advance in the row
        const uint64_t bd = BKMAJ ? smem_desc(b0 + kk * UK * ES, 16, 1024)
                                  : smem_desc(b0 + kk * UK * 128, B_COL, 1024);  // MN: UK rows
        umma<KIND>(tmem, ad, bd, IDESC, (kb | kk) != 0);
      }
      umma_commit(empty + s);
    }
    umma_commit(done);
  }
  __syncwarp();
  const bool ok = mbar_wait(done, 0) && !sh_fail;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float local = 0.f;  // EPI: this thread's share of the reduction
  if (ok) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll
    for (int c = 0; c < BN / 32; ++c) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c * 32, v);
      const int col0 = n0 + c * 32;
      if (row < M) {
        const size_t o = (size_t)z * M * N + (size_t)row * N + col0;
        float* dst = D + o;
        if (EPI) {
          const float ca = sh_coef[0], cp = sh_coef[1];
          const bool vec = col0 + 32 <= N && (N & 3) == 0;
          if (vec) {  // this thread's 32 contiguous values of prev, loaded above
            if (ep.prev) {
              float4 pv[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) pv[q] = pre[8 * c + q];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                v[4 * q] = fmaf(cp, pv[q].x, ca * v[4 * q]);
                v[4 * q + 1] = fmaf(cp, pv[q].y, ca * v[4 * q + 1]);
                v[4 * q + 2] = fmaf(cp, pv[q].z, ca * v[4 * q + 2]);
                v[4 * q + 3] = fmaf(cp, pv[q].w, ca * v[4 * q + 3]);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j) v[j] *= ca;
            }
          } else {
            for (int j = 0; j < 32 && col0 + j < N; ++j) {
              float y = ca * v[j];
              if (ep.prev) y = fmaf(cp, ep.prev[o + j], y);
              v[j] = y;
            }
          }
          if (vec) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            if (dlow) {
#pragma unroll
              for (int j = 0; j < 32; j += 4) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(v[j], v[j + 1]);
                __nv_bfloat162 hi = __floats2bfloat162_rn(v[j + 2], v[j + 3]);
                uint2 pk;
                pk.x = *reinterpret_cast<uint32_t*>(&lo);
                pk.y = *reinterpret_cast<uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(dlow + o + j) = pk;
              }
            }
          } else {
            for (int j = 0; j < 32 && col0 + j < N; ++j) {
              dst[j] = v[j];
              if (dlow) dlow[o + j] = __float2bfloat16_rn(v[j]);
            }
          }
          if (ep.red.out) {
            if (vec && ep.red.other) {
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const float4 ov = *reinterpret_cast<const float4*>(ep.red.other + o + 4 * q);
                local = fmaf(v[4 * q], ov.x, fmaf(v[4 * q + 1], ov.y,
                        fmaf(v[4 * q + 2], ov.z, fmaf(v[4 * q + 3], ov.w, local))));
              }
            } else if (vec) {
#pragma unroll
              for (int j = 0; j < 32; ++j) local = fmaf(v[j], v[j], local);
            } else {
              for (int j = 0; j < 32 && col0 + j < N; ++j)
                local = fmaf(v[j], ep.red.other ? ep.red.other[o + j] : v[j], local);
            }
          }
        } else if (col0 + 32 <= N && (N & 3) == 0) {
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
          for (int j = 0; j < 32 && col0 + j < N; ++j) dst[j] = v[j];
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, TC_ETIMEOUT);
  }
  if (!ok && warp == 0 && lane == 0) {  // let the copies this CTA issued land
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      mbar_wait(full + kb % STAGES, (kb / STAGES) & 1);
  }
  if (EPI && ep.red.out) reduce_finish(local, ep.red);  // every thread of every CTA
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN)
                 : "memory");
}

size_t smem_bytes() { return 1024 + STAGES * (A_BYTES + B_BYTES) + (2 * STAGES + 1) * 8 + 16; }

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

int umma_init() {
  TC_CUDA(cudaFuncSetAttribute(k_umma_gemm<0, 0, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes()));
  TC_CUDA(cudaFuncSetAttribute(k_umma_gemm<1, 1, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes()));
  TC_CUDA(cudaFuncSetAttribute(k_umma_gemm<0, 0, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes()));
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    TC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return TC_EUNSUPPORTED;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return TC_OK;
}

// 3-D tiled map over `slices` row-major matrices rows x inner, box
// (box_inner, box_rows, 1), 128-byte swizzle, zero fill out of bounds.
int make_tmap(CUtensorMap* map, const void* base, int bf16, int inner, int rows, int slices,
              int box_inner, int box_rows) {
  if (!g_encode) return TC_EUNSUPPORTED;
  const cuuint64_t es = bf16 ? 2 : 4;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || ((cuuint64_t)inner * es) % 16 != 0)
    return TC_EINVAL;
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)slices};
  cuuint64_t strides[2] = {(cuuint64_t)inner * es, (cuuint64_t)inner * rows * es};
  cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? TC_OK : TC_EINVAL;
}

// A operand: M x K per slice, K contiguous. B operand: K x N with N contiguous
// (BF16), or its transpose N x K with K contiguous (TF32).
int make_umma_maps(UmmaMaps* m, int kind, const void* A, const void* B, int M, int N, int K,
                   int slices) {
  const int bf16 = kind == 0;
  const int bke = bf16 ? 64 : 32;
  TC_TRY(make_tmap(&m->a, A, bf16, K, M, slices, bke, BM));
  if (bf16)
    TC_TRY(make_tmap(&m->b, B, bf16, N, K, slices, 64, bke));
  else
    TC_TRY(make_tmap(&m->b, B, bf16, K, N, slices, bke, BN));
  m->M = M;
  m->N = N;
  m->K = K;
  m->slices = slices;
  m->kind = kind;
  return TC_OK;
}

int launch_umma(const UmmaMaps& m, float* D, int* err, const int* skip, cudaStream_t st) {
  dim3 grid((m.N + BN - 1) / BN, (m.M + BM - 1) / BM, m.slices);
  Epi none;
  if (m.kind == 0)
    k_umma_gemm<0, 0, false><<<grid, NT, smem_bytes(), st>>>(m.a, m.b, D, m.M, m.N, m.K, err,
                                                              skip, none, nullptr);
  else
    k_umma_gemm<1, 1, false><<<grid, NT, smem_bytes(), st>>>(m.a, m.b, D, m.M, m.N, m.K, err,
                                                              skip, none, nullptr);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_umma_epi(const UmmaMaps& m, float* D, __nv_bfloat16* dlow, const Epi& ep, int* err,
                    cudaStream_t st) {
  TC_CHECK(m.kind == 0);
  dim3 grid((m.N + BN - 1) / BN, (m.M + BM - 1) / BM, m.slices);
  k_umma_gemm<0, 0, true><<<grid, NT, smem_bytes(), st>>>(m.a, m.b, D, m.M, m.N, m.K, err,
                                                           ep.skip, ep, dlow);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
