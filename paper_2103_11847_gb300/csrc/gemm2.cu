// Two-sided c-product in one launch (Algorithm 1 with a right factor, eqs.
// (dft9), (dft8); Remark 2.1), for n3 <= TC_MAX_FUSED and s <= 256, FP32:
//   X~_k = sum_l pro[k][l] X_l                (prologue transform)
//   T_k  = A~_k X~_k                          (stage 1, K = n2)
//   Z_k  = T_k B~_k                           (stage 2, K = s)
//   Y_l  = sum_k epi[l][k] Z_k                (epilogue transform)
// then out = ca * Y + cp * prev and an optional fused reduction.
//
// A thread-block cluster of CS = ceil(s / 64) <= 4 CTAs owns a panel of 8
// output rows; CTA q of the cluster owns columns [64q, 64q + 64). Stage 1
// gives each CTA its 8 x 64 block of T for every slice; the CTA stores that
// block into the shared memory of every CTA of the cluster, so after one
// cluster barrier each CTA holds the whole 8 x s panel of T as the left
// operand of stage 2. T never goes to HBM and the product is one launch.
// Clusters of four fit the GPU in one wave at one CTA per SM (a 256 x 256
// image is 32 clusters); clusters of eight would not.
//
// Operands stream through a ring of S shared-memory slots filled with
// cp.async, S - 1 chunks ahead of the FMAs. The left operand of stage 1 is
// read K-major from the slice transposes of A~ that the plan keeps, so it
// lands in the layout the FMAs read. Each thread applies the prologue
// transform in place to the X positions it copied itself (all slices of
// them), so a chunk needs one barrier.
//
// Inside a CTA the eight warps split every 32-deep K chunk (4 rows of K
// each) and each owns the whole 8 x 64 x n3 block: every lane holds all 8
// rows and two adjacent columns of every slice. The left operand is then the
// same for the whole warp (one broadcast shared-memory read per 4 values) and
// the right operand is one 64-bit read per lane: 4 shared-memory wavefronts
// per 16 FMAs. The partial blocks are summed through shared memory at the
// end of each stage. (Sixteen warps, a 6-slot ring or 64-deep chunks
// measured no faster: at 8 rows per panel the per-SM fill rate of the ring
// and the shared-memory operand reads bound the loop, not latency.)
#include <cooperative_groups.h>

#include "tc_device.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int BM = 8;    // rows of a cluster's panel
constexpr int BN = 64;   // columns per CTA
constexpr int BK = 32;   // K chunk
constexpr int NW = 8;    // warps per CTA
constexpr int NT = 32 * NW;
constexpr int S = 4;     // ring slots
constexpr int CS_MAX = 4;
constexpr int KW = BK / NW;     // K rows of a chunk per warp
constexpr int NPOS = BK * BN / 4 / NT;  // float4 positions of a B chunk per thread (2)

struct Mix {
  float pro[TC_MAX_FUSED * TC_MAX_FUSED];
  float epi[TC_MAX_FUSED * TC_MAX_FUSED];
};

template <int NS>
struct Lay {
  static constexpr int kA = NS * BK * BM;         // left operand of a chunk [NS][BK][BM]
  static constexpr int kB = NS * BK * BN;         // right operand of a chunk [NS][BK][BN]
  static constexpr int kSlot = kA + kB;
  static constexpr int kRing = S * kSlot;
  static constexpr int kRed = NW * NS * BM * BN;  // per-warp partial blocks
  static constexpr int kStage = kRing > kRed ? kRing : kRed;
  // followed by Tt[NS][K2p][BM]: the panel of T, K-major, K2p = CS * BN
  // rounded up to whole chunks (the rounding rows are zero)
  __host__ __device__ static constexpr int k2p(int cs) { return (cs * BN + BK - 1) / BK * BK; }
  static constexpr size_t bytes(int cs) { return (size_t)(kStage + NS * k2p(cs) * BM) * 4; }
};

__device__ __forceinline__ void cp16(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Four consecutive floats of row r, columns c..c+3, of a rows x cols
// row-major matrix into shared memory; zero outside the matrix. VEC: whole
// 16-byte groups (cols % 4 == 0, 16-byte aligned base).
template <bool VEC>
__device__ __forceinline__ void cp_row4(float* dst, const float* base, int rows, int cols, int r,
                                        int c) {
  if (VEC) {
    const bool ok = r < rows && c < cols;
    cp16(dst, ok ? base + (size_t)r * cols + c : base, ok);
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool ok = r < rows && c + e < cols;
      cp4(dst + e, ok ? base + (size_t)r * cols + c + e : base, ok);
    }
  }
}

// acc[k][r][j] += a[k][kk][r] * b[k][kk][2 lane + j] over this warp's KW rows
// kk of a chunk. a: K-major with row length BM (a warp-uniform read), slice
// stride aSl; b: row length BN, slice stride bSl.
template <int NS>
__device__ __forceinline__ void mma_chunk(float (&acc)[NS][BM][2], const float* a, int aSl,
                                          const float* b, int bSl, int w, int lane) {
#pragma unroll
  for (int i = 0; i < KW; ++i) {
    const int kk = w * KW + i;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(a + k * aSl + kk * BM);
      const float4 a1 = *reinterpret_cast<const float4*>(a + k * aSl + kk * BM + 4);
      const float2 bv = *reinterpret_cast<const float2*>(b + k * bSl + kk * BN + 2 * lane);
      const float ar[BM] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int r = 0; r < BM; ++r) {
        acc[k][r][0] = fmaf(ar[r], bv.x, acc[k][r][0]);
        acc[k][r][1] = fmaf(ar[r], bv.y, acc[k][r][1]);
      }
    }
  }
}

// this warp's partial block to red[w][k][r][c]
template <int NS>
__device__ __forceinline__ void acc_to_red(float* red, const float (&acc)[NS][BM][2], int w,
                                           int lane) {
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int r = 0; r < BM; ++r)
      *reinterpret_cast<float2*>(red + ((w * NS + k) * BM + r) * BN + 2 * lane) =
          make_float2(acc[k][r][0], acc[k][r][1]);
}

// At: the left factor K-major (NS x K x M, the slice transposes), X: NS x K x
// N, B: NS x N x N, Y / prev / other: NS x M x N.
//
// A non-empty `step` (the previous LSQR step, which the forward product does
// not depend on: it reads V~ and normalises it through its coefficient) is
// run by the CTAs of this launch first: every CTA computes the same scalars
// and updates its share of X and W while its first operand chunks are in
// flight; the step's stop decision replaces ep.skip.
template <int NS, bool VEC>
__global__ void __launch_bounds__(NT, 1)
k_cprod2(const float* __restrict__ At, const float* __restrict__ X,
         const float* __restrict__ B, float* Y, int M, int K, int N, Mix f, Epi ep,
         LsqrStep step) {
  pdl_wait();
  __shared__ float sh_step[3];
  __shared__ int sh_stop;
  if (step.n) {
    if (*step.done_in) {  // the solve stopped before this step
      if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *step.done_out = 1;
      return;
    }
    if (threadIdx.x == 0)
      sh_stop = lsqr_step_scalars(step, sh_step, blockIdx.x == 0 && blockIdx.y == 0);
    __syncthreads();
  } else if (ep.skip && *ep.skip) {
    return;  // uniform over the grid: no CTA reaches a barrier alone
  }
  extern __shared__ __align__(16) float smem[];
  __shared__ float sh_coef[2];
  float* ring = smem;
  float* red = smem;  // after a stage's main loop
  float* Tt = smem + Lay<NS>::kStage;
  constexpr int kA = Lay<NS>::kA, kSlot = Lay<NS>::kSlot;

  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const int K2 = CS * BN, K2p = Lay<NS>::k2p(CS);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int r0 = blockIdx.y * BM, c0 = q * BN;
  const size_t sA = (size_t)K * M, sX = (size_t)K * N, sB = (size_t)N * N, sY = (size_t)M * N;
  coef_compute(ep.coef, sh_coef);  // read after the barriers below

  // zero the rounding rows of this CTA's panel (no peer writes them)
  for (int i = tid; i < NS * (K2p - K2) * BM; i += NT) {
    const int k = i / ((K2p - K2) * BM), r = i % ((K2p - K2) * BM);
    Tt[((size_t)k * K2p + K2) * BM + r] = 0.f;
  }

  // Copy roles of a chunk. Left operand (NS x BK k x 8 rows, 2 BK NS groups
  // of 4 floats): group t is slice t/(2 BK), k (t%(2 BK))/2, rows
  // 4(t%2)..+3. Right operand (BK k x 64 columns): thread t owns positions
  // p = t + NT i (i < NPOS), k p/16, columns 4(p%16)..+3, for every slice.
  auto issue1 = [&](int c) {
    const int k0 = c * BK;
    float* slot = ring + (c % S) * kSlot;
    for (int t = tid; t < NS * BK * 2; t += NT) {
      const int k = t / (2 * BK), kk = (t % (2 * BK)) >> 1, h = t & 1;
      cp_row4<VEC>(slot + (k * BK + kk) * BM + 4 * h, At + k * sA, K, M, k0 + kk, r0 + 4 * h);
    }
    float* b = slot + kA;
#pragma unroll
    for (int i = 0; i < NPOS; ++i) {
      const int p = tid + NT * i, kk = p >> 4, cq = (p & 15) * 4;
#pragma unroll
      for (int k = 0; k < NS; ++k)
        cp_row4<VEC>(b + (k * BK + kk) * BN + cq, X + k * sX, K, N, k0 + kk, c0 + cq);
    }
  };
  // X~_k = sum_l pro[k][l] X_l on this thread's own positions of a landed chunk
  auto transform1 = [&](int c) {
    float* b = ring + (c % S) * kSlot + kA;
#pragma unroll
    for (int i = 0; i < NPOS; ++i) {
      const int p = tid + NT * i, kk = p >> 4, cq = (p & 15) * 4;
      float4 x[NS];
#pragma unroll
      for (int l = 0; l < NS; ++l) x[l] = *reinterpret_cast<const float4*>(b + (l * BK + kk) * BN + cq);
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int l = 0; l < NS; ++l) {
          const float m = f.pro[k * NS + l];
          t.x = fmaf(m, x[l].x, t.x);
          t.y = fmaf(m, x[l].y, t.y);
          t.z = fmaf(m, x[l].z, t.z);
          t.w = fmaf(m, x[l].w, t.w);
        }
        *reinterpret_cast<float4*>(b + (k * BK + kk) * BN + cq) = t;
      }
    }
  };
  auto issue2 = [&](int c) {
    const int k0 = c * BK;
    float* b = ring + (c % S) * kSlot + kA;
#pragma unroll
    for (int i = 0; i < NPOS; ++i) {
      const int p = tid + NT * i, kk = p >> 4, cq = (p & 15) * 4;
#pragma unroll
      for (int k = 0; k < NS; ++k)
        cp_row4<VEC>(b + (k * BK + kk) * BN + cq, B + k * sB, N, N, k0 + kk, c0 + cq);
    }
  };

  float acc[NS][BM][2];
  auto zero_acc = [&]() {
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int r = 0; r < BM; ++r) acc[k][r][0] = acc[k][r][1] = 0.f;
  };

  // ------------------------------------------------ stage 1: T = A~ (pro X)
  const int nk1 = (K + BK - 1) / BK;
  for (int s = 0; s < S - 1; ++s) {
    if (s < nk1) issue1(s);
    cp_commit();
  }
  if (step.n) {  // this CTA's share of the LSQR step, under the first copies
    const size_t nb = (size_t)gridDim.x * gridDim.y;
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    const size_t per = (step.n + nb - 1) / nb;
    const size_t beg = b * per < step.n ? b * per : step.n;
    const size_t end = beg + per < step.n ? beg + per : step.n;
    lsqr_step_vectors(step, beg, end, sh_step[0], sh_step[1], sh_step[2], sh_stop != 0, NT);
    if (sh_stop) {  // uniform: every CTA took the same decision
      cp_wait<0>();
      return;
    }
  }
  // Every CTA of the cluster must be running before a peer stores into its
  // shared memory: arrive now, wait just before the first remote store.
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  zero_acc();
  for (int c = 0; c < nk1; ++c) {
    cp_wait<S - 2>();  // this thread's copies of chunk c have landed
    transform1(c);
    __syncthreads();   // chunk c complete; every warp is done with chunk c - 1
    if (c + S - 1 < nk1) issue1(c + S - 1);
    cp_commit();
    const float* slot = ring + (c % S) * kSlot;
    mma_chunk<NS>(acc, slot, BK * BM, slot + kA, BK * BN, w, lane);
  }
  cp_wait<0>();
  __syncthreads();  // every warp is done with the ring
  acc_to_red<NS>(red, acc, w, lane);
  __syncthreads();

  // Item i < NS * 128: slice i/128, column i%64, rows 4((i%128)/64)..+3 of
  // the block, summed over the warps and stored K-major into the panel of
  // every CTA of the cluster.
  asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
  for (int it = tid; it < NS * 2 * BN; it += NT) {
    const int k = it / (2 * BN), col = it & (BN - 1), rr = ((it % (2 * BN)) / BN) * 4;
    float x[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float sum = 0.f;
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) sum += red[((ww * NS + k) * BM + rr + r) * BN + col];
      x[r] = sum;
    }
    const float4 v = make_float4(x[0], x[1], x[2], x[3]);
    for (int p = 0; p < CS; ++p) {
      float* Tp = cluster.map_shared_rank(Tt, p);
      *reinterpret_cast<float4*>(Tp + ((size_t)k * K2p + c0 + col) * BM + rr) = v;
    }
  }
  __syncthreads();  // red is no longer read: the ring may be refilled

  // ---------------------------------------------------- stage 2: Z = T B~
  const int nk2 = K2p / BK;
  for (int s = 0; s < S - 1; ++s) {  // in flight across the cluster barrier
    if (s < nk2) issue2(s);
    cp_commit();
  }
  cluster.sync();  // the whole panel of T is in this CTA's shared memory
  zero_acc();
  for (int c = 0; c < nk2; ++c) {
    cp_wait<S - 2>();
    __syncthreads();
    if (c + S - 1 < nk2) issue2(c + S - 1);
    cp_commit();
    const float* slot = ring + (c % S) * kSlot;
    mma_chunk<NS>(acc, Tt + c * BK * BM, K2p * BM, slot + kA, BK * BN, w, lane);
  }
  cp_wait<0>();
  pdl_trigger();
  __syncthreads();
  acc_to_red<NS>(red, acc, w, lane);
  __syncthreads();

  // ------------------------------------------------------------ epilogue
  // threads 0..127: row t/16, columns 4(t%16)..+3 of the block, every slice
  const float ca = sh_coef[0], cp = sh_coef[1];
  const int row = (tid >> 4) & (BM - 1), cq = (tid & 15) * 4;
  const int gr = r0 + row, gc = c0 + cq;
  float local = 0.f;
  if (tid < BM * BN / 4 && gr < M && gc < N) {
    float4 z[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) {
        const float4 v = *reinterpret_cast<const float4*>(red + ((ww * NS + k) * BM + row) * BN + cq);
        s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
      }
      z[k] = s;
    }
#pragma unroll
    for (int l = 0; l < NS; ++l) {
      float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const float m = f.epi[l * NS + k];
        y[0] = fmaf(m, z[k].x, y[0]);
        y[1] = fmaf(m, z[k].y, y[1]);
        y[2] = fmaf(m, z[k].z, y[2]);
        y[3] = fmaf(m, z[k].w, y[3]);
      }
      const size_t o = (size_t)l * sY + (size_t)gr * N + gc;
      if (VEC) {  // gc + 3 < N: N is a multiple of 4
        float4 out = make_float4(ca * y[0], ca * y[1], ca * y[2], ca * y[3]);
        if (ep.prev) {
          const float4 pv = *reinterpret_cast<const float4*>(ep.prev + o);
          out.x = fmaf(cp, pv.x, out.x); out.y = fmaf(cp, pv.y, out.y);
          out.z = fmaf(cp, pv.z, out.z); out.w = fmaf(cp, pv.w, out.w);
        }
        *reinterpret_cast<float4*>(Y + o) = out;
        if (ep.red.out) {
          const float4 ov = ep.red.other ? *reinterpret_cast<const float4*>(ep.red.other + o)
                                         : out;
          local = fmaf(out.x, ov.x, fmaf(out.y, ov.y, fmaf(out.z, ov.z, fmaf(out.w, ov.w, local))));
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (gc + e >= N) break;
          float out = ca * y[e];
          if (ep.prev) out = fmaf(cp, ep.prev[o + e], out);
          Y[o + e] = out;
          if (ep.red.out) local = fmaf(out, ep.red.other ? ep.red.other[o + e] : out, local);
        }
      }
    }
  }
  if (ep.red.out) reduce_finish(local, ep.red);
}

template <int NS, bool VEC>
int run2(const float* At, const float* X, const float* B, float* Y, int M, int K, int N,
         const Mix& f, const Epi& ep, const LsqrStep& step, cudaStream_t st) {
  const int CS = (N + BN - 1) / BN;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS, (M + BM - 1) / BM, 1);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = Lay<NS>::bytes(CS);
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  TC_CUDA(cudaLaunchKernelEx(&cfg, k_cprod2<NS, VEC>, At, X, B, Y, M, K, N, f, ep, step));
  return TC_OK;
}

template <int NS>
int run2v(bool vec, const float* At, const float* X, const float* B, float* Y, int M, int K,
          int N, const Mix& f, const Epi& ep, const LsqrStep& step, cudaStream_t st) {
  return vec ? run2<NS, true>(At, X, B, Y, M, K, N, f, ep, step, st)
             : run2<NS, false>(At, X, B, Y, M, K, N, f, ep, step, st);
}

template <int NS>
int init2() {
  const int c = cudaSharedmemCarveoutMaxShared;
  TC_CUDA(cudaFuncSetAttribute(k_cprod2<NS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Lay<NS>::bytes(CS_MAX)));
  TC_CUDA(cudaFuncSetAttribute(k_cprod2<NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Lay<NS>::bytes(CS_MAX)));
  TC_CUDA(cudaFuncSetAttribute(k_cprod2<NS, true>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  TC_CUDA(cudaFuncSetAttribute(k_cprod2<NS, false>, cudaFuncAttributePreferredSharedMemoryCarveout, c));
  return TC_OK;
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

bool cprod2_fits(int s) { return s >= 1 && s <= CS_MAX * BN; }

int cprod2_init() {
  TC_TRY(init2<1>());
  TC_TRY(init2<2>());
  TC_TRY(init2<3>());
  TC_TRY(init2<4>());
  return TC_OK;
}

int launch_cprod2(const float* At, const float* X, const float* B, float* Y, int M, int K,
                  int N, int nslices, const float* pro, const float* epi, const Epi& ep,
                  const LsqrStep& step, cudaStream_t st) {
  TC_CHECK(nslices >= 1 && nslices <= TC_MAX_FUSED && cprod2_fits(N) && M >= 1 && K >= 1);
  Mix f{};
  for (int i = 0; i < nslices * nslices; ++i) {
    f.pro[i] = pro[i];
    f.epi[i] = epi[i];
  }
  const bool vec = M % 4 == 0 && N % 4 == 0 && al16(At) && al16(X) && al16(B) && al16(Y) &&
                   (!ep.prev || al16(ep.prev)) && (!ep.red.other || al16(ep.red.other));
  switch (nslices) {
    case 1: return run2v<1>(vec, At, X, B, Y, M, K, N, f, ep, step, st);
    case 2: return run2v<2>(vec, At, X, B, Y, M, K, N, f, ep, step, st);
    case 3: return run2v<3>(vec, At, X, B, Y, M, K, N, f, ep, step, st);
    default: return run2v<4>(vec, At, X, B, Y, M, K, N, f, ep, step, st);
  }
}
