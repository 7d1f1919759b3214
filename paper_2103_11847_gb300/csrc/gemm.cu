// Frontal-slice GEMMs of the c-product (Algorithm 1, step 2; eqs. (dft9),
// (dft8)), FP32 on the FFMA pipe, with the mode-3 transform of Remark 2.1
// fused in when n3 <= TC_MAX_FUSED:
//   prologue  B~_k = sum_l pro[k][l] B_l        (the operand's transform)
//   epilogue  Y_l  = sum_k epi[l][k] (A_k B~_k)  (back to the spatial domain)
// followed by out = ca * Y + cp * prev and an optional fused reduction.
// One CTA owns an (i, j) output tile for NS slices; with the transforms fused
// it owns all n3 slices, so the epilogue transform needs no other CTA.
#include "tc_device.cuh"

namespace {

struct Fused {
  float pro[TC_MAX_FUSED * TC_MAX_FUSED];
  float epi[TC_MAX_FUSED * TC_MAX_FUSED];
};

template <int NS, int BM, int BN, int BK, int TM, int TN, bool PRO, bool EPI>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_slice_gemm(const float* __restrict__ A, const float* __restrict__ B, float* C,
             int M, int N, int K, Fused f, Epi ep) {
  constexpr int TX = BN / TN;
  constexpr int NT = (BM / TM) * (BN / TN);
  if (ep.skip && *ep.skip) return;
  __shared__ float As[NS][BK][BM];
  __shared__ __align__(16) float Bs[NS][BK][BN];
  __shared__ float sh_coef[2];

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int z0 = blockIdx.z * NS;
  const size_t sA = (size_t)M * K, sB = (size_t)K * N, sC = (size_t)M * N;
  const float* Ab = A + z0 * sA;
  const float* Bb = B + z0 * sB;

  float acc[NS][TM][TN];
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[k][i][j] = 0.f;

  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int idx = tid; idx < BM * BK; idx += NT) {
      const int r = idx / BK, c = idx % BK;
      const int gi = i0 + r, gk = k0 + c;
      const bool ok = gi < M && gk < K;
#pragma unroll
      for (int k = 0; k < NS; ++k)
        As[k][c][r] = ok ? __ldg(Ab + k * sA + (size_t)gi * K + gk) : 0.f;
    }
    for (int idx = tid; idx < BK * BN; idx += NT) {
      const int r = idx / BN, c = idx % BN;
      const int gk = k0 + r, gj = j0 + c;
      const bool ok = gk < K && gj < N;
      float b[NS];
#pragma unroll
      for (int l = 0; l < NS; ++l) b[l] = ok ? __ldg(Bb + l * sB + (size_t)gk * N + gj) : 0.f;
      if (PRO) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          float t = 0.f;
#pragma unroll
          for (int l = 0; l < NS; ++l) t = fmaf(f.pro[k * NS + l], b[l], t);
          Bs[k][r][c] = t;
        }
      } else {
#pragma unroll
        for (int l = 0; l < NS; ++l) Bs[l][r][c] = b[l];
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        float a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[k][kk][ty * TM + i];
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

  coef_compute(ep.coef, sh_coef);
  __syncthreads();
  const float ca = sh_coef[0], cp = sh_coef[1];
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
          float v;
          if (EPI) {
            v = 0.f;
#pragma unroll
            for (int k = 0; k < NS; ++k) v = fmaf(f.epi[l * NS + k], acc[k][i][j], v);
          } else {
            v = acc[l][i][j];
          }
          const size_t idx = (size_t)(z0 + l) * sC + (size_t)row * N + col;
          float o = ca * v;
          if (ep.prev) o = fmaf(cp, ep.prev[idx], o);
          C[idx] = o;
          if (ep.red.out) local = fmaf(o, ep.red.other ? ep.red.other[idx] : o, local);
        }
      }
    }
  }
  if (ep.red.out) reduce_finish((double)local, ep.red);
}

template <int NS, int BM, int BN, int BK, int TM, int TN, bool PRO, bool EPI>
int run(const float* A, const float* B, float* C, int M, int N, int K, int nslices,
        const Fused& f, const Epi& ep, cudaStream_t st) {
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, nslices / NS);
  dim3 block((BM / TM) * (BN / TN));
  k_slice_gemm<NS, BM, BN, BK, TM, TN, PRO, EPI><<<grid, block, 0, st>>>(A, B, C, M, N, K, f, ep);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

template <int NS, bool PRO, bool EPI>
int pick_tile(const float* A, const float* B, float* C, int M, int N, int K, int nslices,
              const Fused& f, const Epi& ep, cudaStream_t st) {
  const long big = (long)((M + 63) / 64) * ((N + 63) / 64) * (nslices / NS);
  if (big >= 2 * 152)
    return run<NS, 64, 64, 16, 4, 4, PRO, EPI>(A, B, C, M, N, K, nslices, f, ep, st);
  return run<NS, 32, 32, 16, 2, 2, PRO, EPI>(A, B, C, M, N, K, nslices, f, ep, st);
}

template <int NS>
int pick_flags(bool pro, bool epi, const float* A, const float* B, float* C, int M, int N,
               int K, int nslices, const Fused& f, const Epi& ep, cudaStream_t st) {
  if (pro && epi) return pick_tile<NS, true, true>(A, B, C, M, N, K, nslices, f, ep, st);
  if (pro) return pick_tile<NS, true, false>(A, B, C, M, N, K, nslices, f, ep, st);
  if (epi) return pick_tile<NS, false, true>(A, B, C, M, N, K, nslices, f, ep, st);
  return pick_tile<NS, false, false>(A, B, C, M, N, K, nslices, f, ep, st);
}

}  // namespace

int launch_slice_gemm(const float* A, const float* B, float* C, int M, int N, int K,
                      int nslices, const float* pro, const float* epi, const Epi& ep,
                      cudaStream_t st) {
  Fused f{};
  const bool fused = (pro || epi);
  if (fused) {
    TC_CHECK(nslices <= TC_MAX_FUSED);
    for (int i = 0; i < nslices * nslices; ++i) {
      f.pro[i] = pro ? pro[i] : 0.f;
      f.epi[i] = epi ? epi[i] : 0.f;
    }
    switch (nslices) {
      case 1: return pick_flags<1>(pro, epi, A, B, C, M, N, K, 1, f, ep, st);
      case 2: return pick_flags<2>(pro, epi, A, B, C, M, N, K, 2, f, ep, st);
      case 3: return pick_flags<3>(pro, epi, A, B, C, M, N, K, 3, f, ep, st);
      case 4: return pick_flags<4>(pro, epi, A, B, C, M, N, K, 4, f, ep, st);
      default: return TC_EINVAL;
    }
  }
  return pick_tile<1, false, false>(A, B, C, M, N, K, nslices, f, ep, st);
}
