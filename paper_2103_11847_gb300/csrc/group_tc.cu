// The grouped products of the batched BF16 c-LSQR (group.cu) on the tensor
// cores: one launch runs every (problem, tile) pair of one product of one
// step, each CTA one 128 x BN output tile of its problem over all n3 <= 4
// slices. Per K block of 64:
// * A~_k (BF16, resident, K-major) is copied into shared memory with cp.async
//   (zero-filled past the problem's edges);
// * the FP32 vector operand is read, transformed along the tubes in FP32 (the
//   product's leading mode-3 transform, Definition 2.1), rounded to BF16 and
//   stored MN-major: the same rounding as the separate BF16 transform pass of
//   a single solve;
// * one thread issues the n3 slice MMAs (kind::f16, FP32 accumulators in
//   tensor memory, n3 x BN columns).
// The epilogue reads the n3 accumulators of its row, applies the trailing
// transform in FP32, then the Krylov epilogue of group_operands (ca acc +
// cp prev and the norm partial of the problem's two-level reduction).
// Every wait is bounded; a CTA whose wait gives up records TC_ETIMEOUT in its
// problem's status, still joins the reduction (with nothing added) and frees
// its tensor memory.
#include <cuda_bf16.h>

#include <type_traits>

#include "group.cuh"
#include "tcgen05.cuh"

namespace {

using namespace tc5;

constexpr int GT_BM = 128, GT_BK = 64, GT_NT = 128;
constexpr uint32_t GT_A = GT_BM * GT_BK * 2;  // one slice's A block: 16 KB
constexpr uint32_t GT_ATOM = GT_BK * 128;     // one 64-column atom of a B block: 8 KB

struct GroupXf {  // the two mode-3 transforms, n3 x n3 row-major
  float pro[TC_MAX_FUSED * TC_MAX_FUSED];
  float epi[TC_MAX_FUSED * TC_MAX_FUSED];
};

template <int NS, int BN>
struct GtCfg {
  static constexpr uint32_t B_BYTES = GT_BK * BN * 2;  // one slice's B block
  static constexpr uint32_t COLS = NS * BN <= 64 ? 64 : NS * BN <= 128 ? 128 : NS * BN <= 256 ? 256 : 512;
  static constexpr size_t USED = 1024 + NS * (GT_A + B_BYTES) + 64;
  // The shared-memory request bounds the CTAs a SM by the tensor memory they
  // allocate: two (<= 256 columns each) for BN = 64, one for BN = 128.
  static constexpr size_t FLOOR = BN == 64 ? 80 * 1024 : 116 * 1024;
  static constexpr size_t SMEM = USED > FLOOR ? USED : FLOOR;
};

__device__ __forceinline__ void gt_cp16(void* dst, const void* src, uint32_t n) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(n)
               : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <int NS, int BN>
__global__ void __launch_bounds__(GT_NT, 1)
k_group_umma(const GroupProb* __restrict__ probs, const int2* __restrict__ work, GroupOp g,
             GroupXf f) {
  using Cfg = GtCfg<NS, BN>;
  constexpr int NB = BN / 64;  // 64-column atoms of a B block
  // D F32, A and B BF16, A K-major, B MN-major, N = BN, M = 128
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(GT_BM >> 4) << 24);
  const int2 w = work[blockIdx.x];
  const GroupProb& P = probs[w.x];
  if (g.op != GOP_INIT && g.done[(size_t)w.x * g.lstride + g.j]) return;  // uniform over the problem's CTAs
  const GroupOperands o = group_operands(P, g, w.x);
  const int M = o.M, N = o.N, K = o.K;
  const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(o.fwd ? P.AhL : P.AhTL);
  const int tn = (N + BN - 1) / BN;
  const int m0 = (w.y / tn) * GT_BM, n0 = (w.y % tn) * BN;

  extern __shared__ uint8_t gt_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(gt_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;                  // NS slices: 128 rows of 128 bytes, 128-byte swizzle
  uint8_t* sB = base + NS * GT_A;      // NS slices: NB atoms of 64 K rows x 128 bytes
  uint64_t* done = reinterpret_cast<uint64_t*>(sB + NS * Cfg::B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ float sh_coef[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tslot)),
                 "r"(Cfg::COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  coef_compute(o.coef, sh_coef);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  const size_t sA_el = (size_t)M * K, sB_el = (size_t)K * N, sC_el = (size_t)M * N;
  const int nk = (K + GT_BK - 1) / GT_BK;
  // B of a K block: 512 NB units (K row kr, chunk c of 8 columns, every
  // slice), four a thread a group; the group's loads are all issued before
  // its values are used, and group 0 of block kb + 1 is in flight while the
  // MMAs of block kb run.
  float xb[4][NS][8];
  auto load_b = [&](int kb, int grp) {
    const int k0 = kb * GT_BK;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int u = tid + GT_NT * (4 * grp + i), kr = u / (8 * NB), c = u % (8 * NB);
      const int krow = k0 + kr, col = n0 + 8 * c;
      const bool in = krow < K && col < N;  // N % 8 == 0: whole chunks
#pragma unroll
      for (int l = 0; l < NS; ++l) {
        const float* src = o.B + l * sB_el + (size_t)krow * N + col;
        const float4 a = in ? __ldg(reinterpret_cast<const float4*>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = in ? __ldg(reinterpret_cast<const float4*>(src + 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
        xb[i][l][0] = a.x; xb[i][l][1] = a.y; xb[i][l][2] = a.z; xb[i][l][3] = a.w;
        xb[i][l][4] = b.x; xb[i][l][5] = b.y; xb[i][l][6] = b.z; xb[i][l][7] = b.w;
      }
    }
  };
  // transformed along the tube in FP32, rounded to BF16, stored MN-major
  auto store_b = [&](int grp) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int u = tid + GT_NT * (4 * grp + i), kr = u / (8 * NB), c = u % (8 * NB);
      const uint32_t off = (c >> 3) * GT_ATOM + kr * 128 + (((c & 7) ^ (kr & 7)) << 4);
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        float y[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float t = 0.f;
#pragma unroll
          for (int l = 0; l < NS; ++l) t = fmaf(f.pro[k * NS + l], xb[i][l][e], t);
          y[e] = t;
        }
        *reinterpret_cast<uint4*>(sB + k * Cfg::B_BYTES + off) =
            make_uint4(pack_bf16(y[0], y[1]), pack_bf16(y[2], y[3]), pack_bf16(y[4], y[5]),
                       pack_bf16(y[6], y[7]));
      }
    }
  };
  bool ok = true;
  int kb = 0;
  load_b(0, 0);
  for (; kb < nk; ++kb) {
    const int k0 = kb * GT_BK;
    // A: unit (slice l, row r, chunk j) = K values k0 + 8 j .. + 7 of row m0 + r
#pragma unroll 4
    for (int i = 0; i < NS * 8; ++i) {
      const int u = tid + GT_NT * i, l = u >> 10, r = (u >> 3) & 127, j = u & 7;
      const int row = m0 + r, kc = k0 + 8 * j;
      const bool in = row < M && kc < K;  // K % 8 == 0: whole chunks
      const __nv_bfloat16* src = in ? A + l * sA_el + (size_t)row * K + kc : A;
      gt_cp16(sA + l * GT_A + r * 128 + ((j ^ (r & 7)) << 4), src, in ? 16u : 0u);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    store_b(0);
#pragma unroll
    for (int grp = 1; grp < NB; ++grp) {
      load_b(kb, grp);
      store_b(grp);
    }
    if (kb + 1 < nk) load_b(kb + 1, 0);
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const uint32_t a0 = su32(sA + k * GT_A), b0 = su32(sB + k * Cfg::B_BYTES);
#pragma unroll
        for (int kk = 0; kk < GT_BK / 16; ++kk)
          umma<0>(tmem + (uint32_t)(k * BN), smem_desc(a0 + kk * 32, 16, 1024),
                  smem_desc(b0 + kk * 16 * 128, GT_ATOM, 1024), IDESC, (kb | kk) != 0);
      }
      umma_commit(done);
    }
    // the next block overwrites sA and sB: its MMAs must have read them
    const bool got = mbar_wait(done, (uint32_t)(kb & 1));
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
  }

  float local = 0.f;
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const float ca = sh_coef[0], cp = sh_coef[1];
    const int row = m0 + 32 * warp + lane;
    const bool live = row < M;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[NS][16];
#pragma unroll
      for (int l = 0; l < NS; ++l) tmem_ld16_issue(trow + (uint32_t)(l * BN + c0), v[l]);
      const int col = n0 + c0;
      float4 pv[NS][4];
#pragma unroll
      for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          pv[k][q] = (o.prev && live && col + 4 * q < N)
                         ? *reinterpret_cast<const float4*>(o.prev + k * sC_el + (size_t)row * N +
                                                            col + 4 * q)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int l = 0; l < NS; ++l) tmem_ld16_wait(v[l]);
      if (!live) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (col + 4 * q >= N) break;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          float y[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float t = 0.f;
#pragma unroll
            for (int l = 0; l < NS; ++l)
              t = fmaf(f.epi[k * NS + l], __uint_as_float(v[l][4 * q + e]), t);
            y[e] = ca * t;
          }
          if (o.prev) {
            y[0] = fmaf(cp, pv[k][q].x, y[0]);
            y[1] = fmaf(cp, pv[k][q].y, y[1]);
            y[2] = fmaf(cp, pv[k][q].z, y[2]);
            y[3] = fmaf(cp, pv[k][q].w, y[3]);
          }
          *reinterpret_cast<float4*>(o.C + k * sC_el + (size_t)row * N + col + 4 * q) =
              make_float4(y[0], y[1], y[2], y[3]);
          local = fmaf(y[0], y[0], fmaf(y[1], y[1], fmaf(y[2], y[2], fmaf(y[3], y[3], local))));
        }
      }
    }
  } else if (tid == 0) {
    mbar_wait(done, (uint32_t)(kb & 1));  // let the MMAs issued last finish with shared and tensor memory
    atomicExch(o.red.status, TC_ETIMEOUT);
  }
  reduce_finish_n(local, o.red, (unsigned)w.y, (unsigned)(o.fwd ? P.tiles_f : P.tiles_a));
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Cfg::COLS)
                 : "memory");
}

template <int NS, int BN>
int set_smem() {
  TC_CUDA(cudaFuncSetAttribute(k_group_umma<NS, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)GtCfg<NS, BN>::SMEM));
  return TC_OK;
}

template <int NS, int BN>
int run(const GroupProb* probs, const int2* work, int nwork, const GroupOp& g, const GroupXf& f,
        cudaStream_t st) {
  k_group_umma<NS, BN><<<nwork, GT_NT, GtCfg<NS, BN>::SMEM, st>>>(probs, work, g, f);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace

int group_tc_init() {
  TC_TRY((set_smem<1, 64>()));
  TC_TRY((set_smem<2, 64>()));
  TC_TRY((set_smem<3, 64>()));
  TC_TRY((set_smem<4, 64>()));
  TC_TRY((set_smem<1, 128>()));
  TC_TRY((set_smem<2, 128>()));
  TC_TRY((set_smem<3, 128>()));
  TC_TRY((set_smem<4, 128>()));
  return TC_OK;
}

int launch_group_umma(const GroupProb* probs, const int2* work, int nwork, const GroupOp& g,
                      const float* pro, const float* epi, int n3, int cfg, cudaStream_t st) {
  TC_CHECK(n3 >= 1 && n3 <= TC_MAX_FUSED && nwork >= 1 && cfg >= 0 && cfg < 2);
  GroupXf f{};
  for (int i = 0; i < n3 * n3; ++i) {
    f.pro[i] = pro[i];
    f.epi[i] = epi[i];
  }
  auto go = [&](auto ns) -> int {
    constexpr int NS = decltype(ns)::value;
    return cfg == 1 ? run<NS, 128>(probs, work, nwork, g, f, st)
                    : run<NS, 64>(probs, work, nwork, g, f, st);
  };
  switch (n3) {
    case 1: return go(std::integral_constant<int, 1>{});
    case 2: return go(std::integral_constant<int, 2>{});
    case 3: return go(std::integral_constant<int, 3>{});
    default: return go(std::integral_constant<int, 4>{});
  }
}
