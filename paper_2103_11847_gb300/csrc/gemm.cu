// Frontal-slice GEMMs of the c-product (Algorithm 1, step 2; eqs. (dft9),
// (dft8)), FP32 on the FFMA pipe.
//
// Fused form (n3 <= TC_MAX_FUSED): one output tile (i, j) for all n3 slices
// per CTA, with the mode-3 transform of Remark 2.1 fused in:
//   prologue  B~_k = sum_l pro[k][l] B_l        (the operand's transform)
//   epilogue  Y_l  = sum_k epi[l][k] (A_k B~_k)  (back to the spatial domain)
// then out = ca * Y + cp * prev and an optional fused reduction. Small slices
// (a 256 x 256 image has only 64 tiles of 32 x 32) are split along K over a
// thread-block cluster of KS CTAs: each CTA accumulates its K range, the
// partial tiles are summed through distributed shared memory in rank order,
// and each rank finishes BM/KS rows of the tile.
//
// Per-slice form (no transforms): one tile of one slice per CTA, used when
// n3 > TC_MAX_FUSED between separate transform passes.
#include <cooperative_groups.h>

#include <type_traits>

#include "group.cuh"

namespace cg = cooperative_groups;

namespace {

struct Fused {
  float pro[TC_MAX_FUSED * TC_MAX_FUSED];
  float epi[TC_MAX_FUSED * TC_MAX_FUSED];
};

template <int NS, int BM, int BN, int BK, bool SPLIT>
struct Smem {
  static constexpr int kMain = NS * BK * (BM + BN);
  static constexpr int kPart = SPLIT ? NS * BM * BN : 0;
  static constexpr int kFloats = kMain > kPart ? kMain : kPart;
};

// The main loop of one fused tile: acc[k] += A_k (pro B)_k over K range
// [kbeg, kend) for the BM x BN tile at (i0, j0), all NS slices, with register
// double buffering (the next K tile's global loads are issued before the
// current tile's FMAs). Fast path: one float4 per thread and slice for each of
// the A and B tiles (16-byte aligned rows). sm: the Smem<..> floats.
template <int NS, int BM, int BN, int BK, int TM, int TN, bool PRO>
__device__ __forceinline__ void fused_tile_mainloop(const float* __restrict__ A,
                                                    const float* __restrict__ B, int M, int N,
                                                    int K, int kbeg, int kend, int i0, int j0,
                                                    const Fused& f, float* sm,
                                                    float (&acc)[NS][TM][TN]) {
  constexpr int TX = BN / TN;
  constexpr int NT = (BM / TM) * (BN / TN);
  float(*As)[BK][BM] = reinterpret_cast<float(*)[BK][BM]>(sm);
  float(*Bs)[BK][BN] = reinterpret_cast<float(*)[BK][BN]>(sm + NS * BK * BM);
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const size_t sA = (size_t)M * K, sB = (size_t)K * N;
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[k][i][j] = 0.f;

  static_assert(BM * BK == 4 * NT && BK * BN == 4 * NT, "one float4 per thread per tile");
  const bool vec = ((K | N) % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) |
                                           reinterpret_cast<uintptr_t>(B)) & 15) == 0;
  const int ar = tid / (BK / 4), ac = (tid % (BK / 4)) * 4;  // A tile: row, first column
  const int br = tid / (BN / 4), bc = (tid % (BN / 4)) * 4;  // B tile: row, first column
  float4 ra[NS], rb[NS];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int gi = i0 + ar, gk = k0 + ac;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (vec) {
        if (gi < M && gk + 3 < kend) {
          v = __ldg(reinterpret_cast<const float4*>(A + k * sA + (size_t)gi * K + gk));
        } else if (gi < M) {
          const float* src = A + k * sA + (size_t)gi * K;
          v.x = gk < kend ? __ldg(src + gk) : 0.f;
          v.y = gk + 1 < kend ? __ldg(src + gk + 1) : 0.f;
          v.z = gk + 2 < kend ? __ldg(src + gk + 2) : 0.f;
          v.w = gk + 3 < kend ? __ldg(src + gk + 3) : 0.f;
        }
      } else if (gi < M) {
        const float* src = A + k * sA + (size_t)gi * K;
        v.x = gk < kend ? __ldg(src + gk) : 0.f;
        v.y = gk + 1 < kend ? __ldg(src + gk + 1) : 0.f;
        v.z = gk + 2 < kend ? __ldg(src + gk + 2) : 0.f;
        v.w = gk + 3 < kend ? __ldg(src + gk + 3) : 0.f;
      }
      ra[k] = v;
      const int gk2 = k0 + br, gj = j0 + bc;
      float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gk2 < kend) {
        const float* src = B + k * sB + (size_t)gk2 * N;
        if (vec && gj + 3 < N) {
          u = __ldg(reinterpret_cast<const float4*>(src + gj));
        } else {
          u.x = gj < N ? __ldg(src + gj) : 0.f;
          u.y = gj + 1 < N ? __ldg(src + gj + 1) : 0.f;
          u.z = gj + 2 < N ? __ldg(src + gj + 2) : 0.f;
          u.w = gj + 3 < N ? __ldg(src + gj + 3) : 0.f;
        }
      }
      rb[k] = u;
    }
  };
  if (kbeg < kend) fetch(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      As[k][ac + 0][ar] = ra[k].x;
      As[k][ac + 1][ar] = ra[k].y;
      As[k][ac + 2][ar] = ra[k].z;
      As[k][ac + 3][ar] = ra[k].w;
    }
    if (PRO) {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int l = 0; l < NS; ++l) {
          const float m = f.pro[k * NS + l];
          t.x = fmaf(m, rb[l].x, t.x);
          t.y = fmaf(m, rb[l].y, t.y);
          t.z = fmaf(m, rb[l].z, t.z);
          t.w = fmaf(m, rb[l].w, t.w);
        }
        *reinterpret_cast<float4*>(&Bs[k][br][bc]) = t;
      }
    } else {
#pragma unroll
      for (int l = 0; l < NS; ++l) *reinterpret_cast<float4*>(&Bs[l][br][bc]) = rb[l];
    }
    __syncthreads();
    if (k0 + BK < kend) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        float a[TM], b[TN];
        if constexpr (TM % 4 == 0) {  // float4 reads of the A column
#pragma unroll
          for (int q = 0; q < TM; q += 4) {
            const float4 av = *reinterpret_cast<const float4*>(&As[k][kk][ty * TM + q]);
            a[q] = av.x; a[q + 1] = av.y; a[q + 2] = av.z; a[q + 3] = av.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = As[k][kk][ty * TM + i];
        }
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[k][kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[k][i][j] = fmaf(a[i], b[j], acc[k][i][j]);
      }
    }
    __syncthreads();
  }
}

// The store of a whole tile from the registers: Y_l = sum_k epi[l][k] acc[k]
// (EPI) back to the spatial domain, out = ca Y + cp prev; returns this
// thread's share of the reduction (sum of squares, or dot with `other`).
template <int NS, int BM, int BN, int TM, int TN, bool EPI>
__device__ __forceinline__ float fused_tile_store(float* C, const float* prev, const float* other,
                                                  bool reduce, int M, int N, int i0, int j0,
                                                  const Fused& f, float ca, float cp,
                                                  const float (&acc)[NS][TM][TN]) {
  constexpr int TX = BN / TN;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const size_t sC = (size_t)M * N;
  float local = 0.f;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int row = i0 + ty * TM + i;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int col = j0 + tx * TN + j;
      if (row < M && col < N) {
#pragma unroll
        for (int l = 0; l < NS; ++l) {
          float y;
          if (EPI) {
            y = 0.f;
#pragma unroll
            for (int k = 0; k < NS; ++k) y = fmaf(f.epi[l * NS + k], acc[k][i][j], y);
          } else {
            y = acc[l][i][j];
          }
          const size_t o = (size_t)l * sC + (size_t)row * N + col;
          float out = ca * y;
          if (prev) out = fmaf(cp, prev[o], out);
          C[o] = out;
          if (reduce) local = fmaf(out, other ? other[o] : out, local);
        }
      }
    }
  }
  return local;
}

// SPLIT: K is split over the cluster and the epilogue runs from the summed
// partial tiles; otherwise (cluster of one) it runs from the registers.
template <int NS, int BM, int BN, int BK, int TM, int TN, bool PRO, bool EPI, bool SPLIT>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_fused_gemm(const float* __restrict__ A, const float* __restrict__ B, float* C, int M, int N,
             int K, int kchunk, Fused f, Epi ep) {
  constexpr int TX = BN / TN;
  constexpr int NT = (BM / TM) * (BN / TN);
  if (ep.skip && *ep.skip) return;
  __shared__ __align__(16) float sm[Smem<NS, BM, BN, BK, SPLIT>::kFloats];
  __shared__ float sh_coef[2];
  float* P = sm;  // partial tile [NS][BM][BN] after the main loop

  cg::cluster_group cluster = cg::this_cluster();
  const int KS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const size_t sC = (size_t)M * N;
  const int kbeg = rank * kchunk;
  const int kend = min(K, kbeg + kchunk);

  float acc[NS][TM][TN];
  fused_tile_mainloop<NS, BM, BN, BK, TM, TN, PRO>(A, B, M, N, K, kbeg, kend, i0, j0, f, sm, acc);

  if (!SPLIT) {
    coef_compute(ep.coef, sh_coef);
    __syncthreads();
    const float local = fused_tile_store<NS, BM, BN, TM, TN, EPI>(
        C, ep.prev, ep.red.other, ep.red.out != nullptr, M, N, i0, j0, f, sh_coef[0], sh_coef[1],
        acc);
    if (ep.red.out) reduce_finish(local, ep.red);
    return;
  }
  // partial tile to shared memory, then sum over the cluster's K ranges
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) P[(k * BM + ty * TM + i) * BN + tx * TN + j] = acc[k][i][j];
  coef_compute(ep.coef, sh_coef);
  cluster.sync();
  const float ca = sh_coef[0], cp = sh_coef[1];
  const int rows = BM / KS;  // this rank finishes rows [rank*rows, (rank+1)*rows)
  float local = 0.f;
  for (int idx = tid; idx < rows * BN; idx += NT) {
    const int lr = rank * rows + idx / BN, lc = idx % BN;
    const int row = i0 + lr, col = j0 + lc;
    float v[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) v[k] = 0.f;
    for (int q = 0; q < KS; ++q) {
      const float* Pq = cluster.map_shared_rank(P, q);
#pragma unroll
      for (int k = 0; k < NS; ++k) v[k] += Pq[(k * BM + lr) * BN + lc];
    }
    if (row < M && col < N) {
#pragma unroll
      for (int l = 0; l < NS; ++l) {
        float y;
        if (EPI) {
          y = 0.f;
#pragma unroll
          for (int k = 0; k < NS; ++k) y = fmaf(f.epi[l * NS + k], v[k], y);
        } else {
          y = v[l];
        }
        const size_t o = (size_t)l * sC + (size_t)row * N + col;
        float out = ca * y;
        if (ep.prev) out = fmaf(cp, ep.prev[o], out);
        C[o] = out;
        if (ep.red.out) local = fmaf(out, ep.red.other ? ep.red.other[o] : out, local);
      }
    }
  }
  cluster.sync();  // peers may still read this CTA's partial tile until here
  if (ep.red.out) reduce_finish(local, ep.red);
}

// Per-slice GEMM without transforms: C_z = A_z B_z for slice z = blockIdx.z.
template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_slice_gemm(const float* __restrict__ A, const float* __restrict__ B, float* C, int M, int N,
             int K, const int* skip) {
  constexpr int TX = BN / TN;
  constexpr int NT = (BM / TM) * (BN / TN);
  if (skip && *skip) return;
  __shared__ float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const float* Ab = A + (size_t)blockIdx.z * M * K;
  const float* Bb = B + (size_t)blockIdx.z * K * N;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int idx = tid; idx < BM * BK; idx += NT) {
      const int r = idx / BK, c = idx % BK;
      const int gi = i0 + r, gk = k0 + c;
      As[c][r] = (gi < M && gk < K) ? __ldg(Ab + (size_t)gi * K + gk) : 0.f;
    }
    for (int idx = tid; idx < BK * BN; idx += NT) {
      const int r = idx / BN, c = idx % BN;
      const int gk = k0 + r, gj = j0 + c;
      Bs[r][c] = (gk < K && gj < N) ? __ldg(Bb + (size_t)gk * N + gj) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* Cb = C + (size_t)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int row = i0 + ty * TM + i;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int col = j0 + tx * TN + j;
      if (row < M && col < N) Cb[(size_t)row * N + col] = acc[i][j];
    }
  }
}

// Grouped fused products: CTA i takes tile work[i].y of problem work[i].x,
// reads that problem's operands, epilogue scalars and done flag (g.op, g.j),
// and reduces into that problem's partials with its tile index, so each
// problem keeps its own deterministic reduction. The pointers follow the
// deferred-iterate schedule of lsqr_enqueue: the forward product of step j
// reads basis slot j and writes U (prev: C at j = 0, else U), the adjoint
// reads U and writes basis slot j + 1 (prev: slot j), the first adjoint
// writes slot 0 from C.
template <int NS, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_group_gemm(const GroupProb* __restrict__ probs, const int2* __restrict__ work, GroupOp g,
             Fused f) {
  const int2 w = work[blockIdx.x];
  const GroupProb& P = probs[w.x];
  if (g.op != GOP_INIT && g.done[(size_t)w.x * g.lstride + g.j]) return;  // uniform over the problem's CTAs
  __shared__ __align__(16) float sm[Smem<NS, BM, BN, BK, false>::kFloats];
  __shared__ float sh_coef[2];
  const GroupOperands o = group_operands(P, g, w.x);
  const bool fwd = o.fwd;
  const int M = o.M, K = o.K, N = o.N;
  const float* A = fwd ? P.Ah : P.AhT;
  const int tn = (N + BN - 1) / BN;
  const int i0 = (w.y / tn) * BM, j0 = (w.y % tn) * BN;
  float acc[NS][TM][TN];
  fused_tile_mainloop<NS, BM, BN, BK, TM, TN, true>(A, o.B, M, N, K, 0, K, i0, j0, f, sm, acc);
  coef_compute(o.coef, sh_coef);
  __syncthreads();
  const float local = fused_tile_store<NS, BM, BN, TM, TN, true>(
      o.C, o.prev, nullptr, true, M, N, i0, j0, f, sh_coef[0], sh_coef[1], acc);
  reduce_finish_n(local, o.red, (unsigned)w.y, (unsigned)(fwd ? P.tiles_f : P.tiles_a));
}

// Tile shapes the autotuner chooses from: cfg 0: 64 x 64, 4 x 4 a thread
// (256 threads); 1: 32 x 32, 4 x 2 (128); 2: 64 x 64, 8 x 4 (128, K blocks
// of 8): fewer shared-memory loads an FMA.
template <int NS, int CFG>
int run_group(const GroupProb* probs, const int2* work, int nwork, const GroupOp& g,
              const Fused& f, cudaStream_t st) {
  constexpr int T = CFG == 1 ? 32 : 64;
  constexpr int BK = CFG == 2 ? 8 : 16, TM = CFG == 2 ? 8 : 4, TN = CFG == 0 ? 4 : (CFG == 1 ? 2 : 4);
  k_group_gemm<NS, T, T, BK, TM, TN><<<nwork, (T / TM) * (T / TN), 0, st>>>(probs, work, g, f);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

template <int NS, int BM, int BN, int BK, int TM, int TN, bool PRO, bool EPI, bool SPLIT>
int run_fused(const float* A, const float* B, float* C, int M, int N, int K, const Fused& f,
              const Epi& ep, cudaStream_t st) {
  const long tiles = (long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  // split K over a cluster until the grid covers every SM, keeping >= 2 K tiles per CTA
  int KS = 1;
  while (SPLIT && KS < 8 && tiles * KS < 152 && K >= 2 * BK * (KS * 2)) KS *= 2;
  const int kchunk = (((K + KS - 1) / KS) + BK - 1) / BK * BK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((N + BN - 1) / BN, (M + BM - 1) / BM, KS);
  cfg.blockDim = dim3((BM / TM) * (BN / TN));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = KS;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TC_CUDA(cudaLaunchKernelEx(&cfg, k_fused_gemm<NS, BM, BN, BK, TM, TN, PRO, EPI, SPLIT>, A, B, C,
                             M, N, K, kchunk, f, ep));
  return TC_OK;
}

template <int NS, bool PRO, bool EPI>
int pick_tile(const float* A, const float* B, float* C, int M, int N, int K, const Fused& f,
              const Epi& ep, cudaStream_t st) {
  const long big = (long)((M + 63) / 64) * ((N + 63) / 64);
  if (big >= 152)
    return run_fused<NS, 64, 64, 16, 4, 4, PRO, EPI, false>(A, B, C, M, N, K, f, ep, st);
  return run_fused<NS, 32, 32, 16, 4, 2, PRO, EPI, true>(A, B, C, M, N, K, f, ep, st);
}

template <int NS>
int pick_flags(bool pro, bool epi, const float* A, const float* B, float* C, int M, int N,
               int K, const Fused& f, const Epi& ep, cudaStream_t st) {
  if (pro && epi) return pick_tile<NS, true, true>(A, B, C, M, N, K, f, ep, st);
  if (pro) return pick_tile<NS, true, false>(A, B, C, M, N, K, f, ep, st);
  if (epi) return pick_tile<NS, false, true>(A, B, C, M, N, K, f, ep, st);
  return pick_tile<NS, false, false>(A, B, C, M, N, K, f, ep, st);
}

}  // namespace

int group_cfg_count(int bf16) { return bf16 ? 2 : 3; }

void group_tile_shape(int bf16, int cfg, int* tm, int* tn) {
  if (bf16) {  // group_tc.cu: 128 x 64 or 128 x 128
    *tm = 128;
    *tn = cfg == 1 ? 128 : 64;
  } else {
    *tm = *tn = cfg == 1 ? 32 : 64;
  }
}

int launch_group_gemm(const GroupProb* probs, const int2* work, int nwork, const GroupOp& g,
                      const float* pro, const float* epi, int n3, int cfg, cudaStream_t st) {
  TC_CHECK(n3 >= 1 && n3 <= TC_MAX_FUSED && nwork >= 1 && cfg >= 0 && cfg < GROUP_CFGS);
  Fused f{};
  for (int i = 0; i < n3 * n3; ++i) {
    f.pro[i] = pro[i];
    f.epi[i] = epi[i];
  }
  auto go = [&](auto ns) -> int {
    constexpr int NS = decltype(ns)::value;
    return cfg == 0 ? run_group<NS, 0>(probs, work, nwork, g, f, st)
         : cfg == 1 ? run_group<NS, 1>(probs, work, nwork, g, f, st)
                    : run_group<NS, 2>(probs, work, nwork, g, f, st);
  };
  switch (n3) {
    case 1: return go(std::integral_constant<int, 1>{});
    case 2: return go(std::integral_constant<int, 2>{});
    case 3: return go(std::integral_constant<int, 3>{});
    default: return go(std::integral_constant<int, 4>{});
  }
}

int launch_slice_gemm(const float* A, const float* B, float* C, int M, int N, int K,
                      int nslices, const float* pro, const float* epi, const Epi& ep,
                      cudaStream_t st) {
  if (pro || epi) {
    TC_CHECK(nslices <= TC_MAX_FUSED);
    Fused f{};
    for (int i = 0; i < nslices * nslices; ++i) {
      f.pro[i] = pro ? pro[i] : 0.f;
      f.epi[i] = epi ? epi[i] : 0.f;
    }
    switch (nslices) {
      case 1: return pick_flags<1>(pro, epi, A, B, C, M, N, K, f, ep, st);
      case 2: return pick_flags<2>(pro, epi, A, B, C, M, N, K, f, ep, st);
      case 3: return pick_flags<3>(pro, epi, A, B, C, M, N, K, f, ep, st);
      case 4: return pick_flags<4>(pro, epi, A, B, C, M, N, K, f, ep, st);
      default: return TC_EINVAL;
    }
  }
  // per-slice GEMM between transform passes: no epilogue beyond the store
  TC_CHECK(ep.prev == nullptr && ep.red.out == nullptr && ep.coef.rule == COEF_ONE);
  const long big = (long)((M + 63) / 64) * ((N + 63) / 64) * nslices;
  if (big >= 2 * 152) {
    dim3 grid((N + 63) / 64, (M + 63) / 64, nslices);
    k_slice_gemm<64, 64, 16, 4, 4><<<grid, 256, 0, st>>>(A, B, C, M, N, K, ep.skip);
  } else {
    dim3 grid((N + 31) / 32, (M + 31) / 32, nslices);
    k_slice_gemm<32, 32, 16, 4, 2><<<grid, 128, 0, st>>>(A, B, C, M, N, K, ep.skip);
  }
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
