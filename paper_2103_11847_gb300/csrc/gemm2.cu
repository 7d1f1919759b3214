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
// Inside a CTA the eight warps split every 64-deep K chunk (8 rows of K
// each) and each owns the whole 8 x 64 x n3 block: every lane holds all 8
// rows and two adjacent columns of every slice. The left operand is then the
// same for the whole warp (one broadcast shared-memory read per 4 values) and
// the right operand is one 64-bit read per lane: 4 shared-memory wavefronts
// per 16 FMAs. The eight partial blocks are summed through shared memory at
// the end of each stage. Operands stream through two register-staged buffers.
#include <cooperative_groups.h>

#include "tc_device.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int BM = 8;    // rows of a cluster's panel
constexpr int BN = 64;   // columns per CTA
constexpr int BK = 64;   // K chunk
constexpr int NW = 8;    // warps per CTA
constexpr int NT = 32 * NW;
constexpr int CS_MAX = 4;
constexpr int KW = BK / NW;  // K rows of a chunk per warp

struct Mix {
  float pro[TC_MAX_FUSED * TC_MAX_FUSED];
  float epi[TC_MAX_FUSED * TC_MAX_FUSED];
};

template <int NS>
struct Lay {
  static constexpr int kA = 2 * NS * BK * BM;     // As[2][NS][BK][BM] (K-major A chunk)
  static constexpr int kB = 2 * NS * BK * BN;     // Bs[2][NS][BK][BN]
  static constexpr int kRed = NW * NS * BM * BN;  // per-warp partial blocks
  static constexpr int kStage = (kA + kB) > kRed ? (kA + kB) : kRed;
  // followed by Tt[NS][K2p][BM]: the panel of T, K-major, K2p = CS * BN
  // rounded up to whole chunks (the rounding rows are zero)
  __host__ __device__ static constexpr int k2p(int cs) { return (cs * BN + BK - 1) / BK * BK; }
  static constexpr size_t bytes(int cs) { return (size_t)(kStage + NS * k2p(cs) * BM) * 4; }
};

// 4 consecutive floats of row r at column c of a rows x cols row-major
// matrix, zero outside it.
__device__ __forceinline__ float4 ld4(const float* base, int rows, int cols, int r, int c,
                                      bool vec) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (r >= rows) return v;
  const float* p = base + (size_t)r * cols;
  if (vec && c + 3 < cols) return __ldg(reinterpret_cast<const float4*>(p + c));
  if (c < cols) v.x = __ldg(p + c);
  if (c + 1 < cols) v.y = __ldg(p + c + 1);
  if (c + 2 < cols) v.z = __ldg(p + c + 2);
  if (c + 3 < cols) v.w = __ldg(p + c + 3);
  return v;
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

template <int NS>
__global__ void __launch_bounds__(NT, 1)
k_cprod2(const float* __restrict__ A, const float* __restrict__ X,
         const float* __restrict__ B, float* Y, int M, int K, int N, Mix f, Epi ep) {
  if (ep.skip && *ep.skip) return;  // uniform over the grid: no CTA reaches a barrier alone
  extern __shared__ __align__(16) float smem[];
  __shared__ float sh_coef[2];
  float* As = smem;
  float* Bs = smem + Lay<NS>::kA;
  float* red = smem;
  float* Tt = smem + Lay<NS>::kStage;

  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const int K2 = CS * BN, K2p = Lay<NS>::k2p(CS);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int r0 = blockIdx.y * BM, c0 = q * BN;
  const size_t sA = (size_t)M * K, sX = (size_t)K * N, sB = (size_t)N * N, sY = (size_t)M * N;
  const bool vec = (K % 4 == 0) && (N % 4 == 0) &&
                   (((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(X) |
                      reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(Y)) & 15) == 0) &&
                   (!ep.prev || (reinterpret_cast<uintptr_t>(ep.prev) & 15) == 0) &&
                   (!ep.red.other || (reinterpret_cast<uintptr_t>(ep.red.other) & 15) == 0);
  coef_compute(ep.coef, sh_coef);  // read after the barriers below
  // Every CTA of the cluster must be running before a peer stores into its
  // shared memory: arrive now, wait just before the first remote store.
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");

  // zero the rounding rows of this CTA's panel (no peer writes them)
  for (int i = tid; i < NS * (K2p - K2) * BM; i += NT) {
    const int k = i / ((K2p - K2) * BM), r = i % ((K2p - K2) * BM);
    Tt[((size_t)k * K2p + K2) * BM + r] = 0.f;
  }

  // Loader roles. A chunk (8 rows x 64 k per slice, 128 float4): thread t
  // loads slices t/128, t/128 + 2 at row t%8, k 4((t%128)/8)..+3. X / B~
  // chunk (64 k x 64 columns per slice): four float4 per thread and slice,
  // k (t + 256 i)/16, columns 4(t%16)..+3.
  constexpr int NA = (NS + 1) / 2;
  const int la_s = tid >> 7, la_r = tid & 7, la_k = ((tid & 127) >> 3) * 4;
  const int lb_k = tid >> 4, lb_c = (tid & 15) * 4;  // i adds 16 to the k row

  float acc[NS][BM][2];
  float4 ra[NA], rb[4][NS];
  auto zero_acc = [&]() {
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int r = 0; r < BM; ++r) acc[k][r][0] = acc[k][r][1] = 0.f;
  };

  // ------------------------------------------------ stage 1: T = A~ (pro X)
  auto fetch1 = [&](int k0) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int k = la_s + 2 * j;
      ra[j] = (k < NS && k0 + la_k < K) ? ld4(A + k * sA, M, K, r0 + la_r, k0 + la_k, vec)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int i = 0; i < 4; ++i)
        rb[i][k] = ld4(X + k * sX, K, N, k0 + lb_k + 16 * i, c0 + lb_c, vec);
  };
  auto store1 = [&](int buf) {
    float* a = As + buf * NS * BK * BM;
    float* b = Bs + buf * NS * BK * BN;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int k = la_s + 2 * j;
      if (k < NS) {
        a[(k * BK + la_k + 0) * BM + la_r] = ra[j].x;
        a[(k * BK + la_k + 1) * BM + la_r] = ra[j].y;
        a[(k * BK + la_k + 2) * BM + la_r] = ra[j].z;
        a[(k * BK + la_k + 3) * BM + la_r] = ra[j].w;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int l = 0; l < NS; ++l) {
          const float m = f.pro[k * NS + l];
          t.x = fmaf(m, rb[i][l].x, t.x);
          t.y = fmaf(m, rb[i][l].y, t.y);
          t.z = fmaf(m, rb[i][l].z, t.z);
          t.w = fmaf(m, rb[i][l].w, t.w);
        }
        *reinterpret_cast<float4*>(b + (k * BK + lb_k + 16 * i) * BN + lb_c) = t;
      }
  };

  zero_acc();
  const int nk1 = (K + BK - 1) / BK;
  fetch1(0);
  for (int c = 0; c < nk1; ++c) {
    const int buf = c & 1;
    store1(buf);
    __syncthreads();
    if (c + 1 < nk1) fetch1((c + 1) * BK);
    mma_chunk<NS>(acc, As + buf * NS * BK * BM, BK * BM, Bs + buf * NS * BK * BN, BK * BN, w,
                  lane);
  }
  __syncthreads();  // every warp is done with the stage buffers
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
  // ---------------------------------------------------- stage 2: Z = T B~
  auto fetch2 = [&](int k0) {
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int i = 0; i < 4; ++i)
        rb[i][k] = ld4(B + k * sB, N, N, k0 + lb_k + 16 * i, c0 + lb_c, vec);
  };
  fetch2(0);       // in flight across the cluster barrier
  cluster.sync();  // the whole panel of T is in this CTA's shared memory
  zero_acc();
  const int nk2 = K2p / BK;
  for (int c = 0; c < nk2; ++c) {
    const int buf = c & 1;
    float* b = Bs + buf * NS * BK * BN;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < NS; ++k)
        *reinterpret_cast<float4*>(b + (k * BK + lb_k + 16 * i) * BN + lb_c) = rb[i][k];
    __syncthreads();
    if (c + 1 < nk2) fetch2((c + 1) * BK);
    mma_chunk<NS>(acc, Tt + c * BK * BM, K2p * BM, b, BK * BN, w, lane);
  }
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
      if (vec && gc + 3 < N) {
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
  if (ep.red.out) reduce_finish((double)local, ep.red);
}

template <int NS>
int run2(const float* A, const float* X, const float* B, float* Y, int M, int K, int N,
         const Mix& f, const Epi& ep, cudaStream_t st) {
  const int CS = (N + BN - 1) / BN;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS, (M + BM - 1) / BM, 1);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = Lay<NS>::bytes(CS);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TC_CUDA(cudaLaunchKernelEx(&cfg, k_cprod2<NS>, A, X, B, Y, M, K, N, f, ep));
  return TC_OK;
}

template <int NS>
int init2() {
  TC_CUDA(cudaFuncSetAttribute(k_cprod2<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Lay<NS>::bytes(CS_MAX)));
  TC_CUDA(cudaFuncSetAttribute(k_cprod2<NS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared));
  return TC_OK;
}

}  // namespace

bool cprod2_fits(int s) { return s >= 1 && s <= CS_MAX * BN; }

int cprod2_init() {
  TC_TRY(init2<1>());
  TC_TRY(init2<2>());
  TC_TRY(init2<3>());
  TC_TRY(init2<4>());
  return TC_OK;
}

int launch_cprod2(const float* A, const float* X, const float* B, float* Y, int M, int K,
                  int N, int nslices, const float* pro, const float* epi, const Epi& ep,
                  cudaStream_t st) {
  TC_CHECK(nslices >= 1 && nslices <= TC_MAX_FUSED && cprod2_fits(N) && M >= 1 && K >= 1);
  Mix f{};
  for (int i = 0; i < nslices * nslices; ++i) {
    f.pro[i] = pro[i];
    f.epi[i] = epi[i];
  }
  switch (nslices) {
    case 1: return run2<1>(A, X, B, Y, M, K, N, f, ep, st);
    case 2: return run2<2>(A, X, B, Y, M, K, N, f, ep, st);
    case 3: return run2<3>(A, X, B, Y, M, K, N, f, ep, st);
    default: return run2<4>(A, X, B, Y, M, K, N, f, ep, st);
  }
}
