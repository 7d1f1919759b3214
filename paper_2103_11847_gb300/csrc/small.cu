// The projected problem in FP64 on one CTA (§3.1 eqs. (leastsq), (tikho2),
// (gcv2); §3.2 eqs. (normeq2), (leastsq0)):
//   1. one-sided Jacobi SVD of the (k+1) x k matrix H (Hestenes rotations,
//      round-robin pair order, warps rotate disjoint column pairs),
//      sigma_i = ||h_i||, g~_i = beta * (first row of H V)_i / sigma_i;
//   2. GCV(lambda) of eq. (gcv2) ("paper") or of the rectangular problem
//      ("full", with g~_{k+1}^2 = beta^2 - sum g~_i^2), minimised on three
//      nested log grids of 200 points: [1e-10 s, s] with s = ||H||_F, then
//      twice the bracket between the grid neighbours of the minimum (first
//      index on ties);
//   3. y from the normal equations (H^T H + lambda^2 I) y = beta H^T e_1 by
//      Cholesky.
// GB300 runs FP64 at a small fraction of its FP32 rate, so everything here is
// O(k^2)..O(k^3) work on k <= TC_MAX_PROJ numbers.
#include "tc_device.cuh"

namespace {

constexpr int NT = 1024;
constexpr int NW = NT / 32;
constexpr int NGRID = 200;
constexpr int NLEVEL = 3;
constexpr int MAX_SWEEPS = 40;

__device__ double gcv_eval(const double* sig, const double* g, int k, double gnull2,
                           double lam, int variant) {
  const double l2 = lam * lam;
  double num = 0.0, den = 0.0;
  if (variant == TC_GCV_FULL) {
    for (int i = 0; i < k; ++i) {
      const double d = sig[i] * sig[i] + l2;
      const double r = l2 * g[i] / d;
      num += r * r;
      den += l2 / d;
    }
    num += gnull2;
    den += 1.0;
    return num / (den * den);
  }
  for (int i = 0; i < k; ++i) {
    const double d = sig[i] * sig[i] + l2;
    const double r = g[i] / d;
    num += r * r;
    den += 1.0 / d;
  }
  return num / (den * den);
}

__device__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Dynamic shared memory: Hs[(k+1) * kk] (column-major working copy, kk = k
// rounded up to even), reused as the k x k normal matrix afterwards.
__global__ void __launch_bounds__(NT)
k_tikhonov_gcv(const double* __restrict__ H, int ld, int kmax, const int* kdev,
               const double* beta_p, int variant, double lambda_in, double* lambda_out,
               double* y, double* gcv_out, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ double dsm[];
  __shared__ double sig[TC_MAX_PROJ], g[TC_MAX_PROJ], dn[TC_MAX_PROJ];
  __shared__ double vals[NGRID];
  __shared__ double grid[NGRID];
  __shared__ int sh_rot;
  __shared__ double sh_misc[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = kdev ? min(*kdev, kmax) : kmax;
  const double beta = *beta_p;
  if (k <= 0) {
    if (tid == 0) {
      *lambda_out = nan("");
      if (gcv_out) *gcv_out = nan("");
    }
    return;
  }
  const int rows = k + 1;
  const int kk = k + (k & 1);
  double* Hs = dsm;  // column c at Hs + c*rows
  for (int idx = tid; idx < rows * kk; idx += NT) {
    const int c = idx / rows, r = idx % rows;
    Hs[idx] = (c < k) ? H[(size_t)r * ld + c] : 0.0;
  }
  __syncthreads();

  // ---- 1. one-sided Jacobi -------------------------------------------------
  // Rotate while |<h_p, h_q>| > rows * eps * ||h_p|| ||h_q||: below that the
  // inner product is rounding noise of the (rows)-term dot product. Each warp
  // rotates one column pair of the round; squared column norms d[] are
  // recomputed every sweep and updated by the exact rotation identities
  // d_p -= t gamma, d_q += t gamma in between.
  const double jtol = rows * 2.220446049250313e-16;
  const int npairs = kk / 2;
  for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
    if (tid == 0) sh_rot = 0;
    for (int c = warp; c < kk; c += NW) {
      const double* x = Hs + (size_t)c * rows;
      double s2 = 0.0;
      for (int r = lane; r < rows; r += 32) s2 += x[r] * x[r];
      s2 = warp_sum_d(s2);
      if (lane == 0) dn[c] = s2;
    }
    __syncthreads();
    for (int rnd = 0; rnd < kk - 1; ++rnd) {
      for (int pi = warp; pi < npairs; pi += NW) {
        // circle method: player 0 fixed, the others rotate by rnd
        const int a = (pi == 0) ? 0 : ((pi - 1 + rnd) % (kk - 1)) + 1;
        const int b = ((kk - 2 - pi + rnd) % (kk - 1)) + 1;
        double* xp = Hs + (size_t)a * rows;
        double* xq = Hs + (size_t)b * rows;
        double ga = 0.0;
        for (int r = lane; r < rows; r += 32) ga += xp[r] * xq[r];
        ga = warp_sum_d(ga);
        const double al = dn[a], be = dn[b];
        if (ga != 0.0 && fabs(ga) > jtol * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t);
          const double s = c * t;
          for (int r = lane; r < rows; r += 32) {
            const double u = xp[r], v = xq[r];
            xp[r] = c * u - s * v;
            xq[r] = s * u + c * v;
          }
          if (lane == 0) {
            dn[a] = al - t * ga;
            dn[b] = be + t * ga;
            sh_rot = 1;
          }
        }
      }
      __syncthreads();
    }
    const int any = sh_rot;
    __syncthreads();
    if (!any) break;
  }
  for (int c = warp; c < k; c += NW) {
    const double* x = Hs + (size_t)c * rows;
    double s2 = 0.0;
    for (int r = lane; r < rows; r += 32) s2 += x[r] * x[r];
    s2 = warp_sum_d(s2);
    if (lane == 0) {
      const double sv = sqrt(s2);
      sig[c] = sv;
      g[c] = (sv > 0.0) ? beta * x[0] / sv : 0.0;
    }
  }
  __syncthreads();
  if (tid == 0) {  // the part of beta e1 outside the range of H
    double gs = 0.0;
    for (int i = 0; i < k; ++i) gs += g[i] * g[i];
    sh_misc[2] = fmax(beta * beta - gs, 0.0);
  }
  __syncthreads();
  const double gnull2 = sh_misc[2];

  // ---- 2. lambda -------------------------------------------------------------
  double lam = lambda_in;
  if (!(lambda_in >= 0.0)) {
    double hs = 0.0;  // ||H||_F
    for (int idx = tid; idx < rows * k; idx += NT) {
      const double v = H[(size_t)(idx / k) * ld + idx % k];
      hs += v * v;
    }
    hs = warp_sum_d(hs);
    if (lane == 0) vals[warp] = hs;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NW; ++w) t += vals[w];
      sh_misc[5] = log(sqrt(t)) - 10.0 * log(10.0);
      sh_misc[6] = log(sqrt(t));
    }
    __syncthreads();
    for (int level = 0; level < NLEVEL; ++level) {
      const double lo = sh_misc[5], hi = sh_misc[6];
      const double step = (hi - lo) / (NGRID - 1);
      for (int i = tid; i < NGRID; i += NT) {
        grid[i] = exp(i == NGRID - 1 ? hi : lo + i * step);
        vals[i] = gcv_eval(sig, g, k, gnull2, grid[i], variant);
      }
      __syncthreads();
      if (tid == 0) {
        int bi = 0;
        for (int i = 1; i < NGRID; ++i)
          if (vals[i] < vals[bi]) bi = i;
        sh_misc[3] = grid[bi];
        sh_misc[4] = vals[bi];
        sh_misc[5] = log(grid[max(bi - 1, 0)]);
        sh_misc[6] = log(grid[min(bi + 1, NGRID - 1)]);
      }
      __syncthreads();
    }
    lam = sh_misc[3];
  } else if (tid == 0) {
    sh_misc[4] = gcv_eval(sig, g, k, gnull2, lam, variant);
  }
  __syncthreads();
  if (tid == 0) {
    *lambda_out = lam;
    if (gcv_out) *gcv_out = sh_misc[4];
  }

  // ---- 3. (H^T H + lambda^2 I) y = beta H^T e_1, Cholesky --------------------
  double* G = dsm;  // k x k row-major, overwrites the Jacobi copy
  __syncthreads();
  for (int idx = tid; idx < k * k; idx += NT) {
    const int i = idx / k, jj = idx % k;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += H[(size_t)r * ld + i] * H[(size_t)r * ld + jj];
    if (i == jj) s += lam * lam;
    G[idx] = s;
  }
  for (int i = tid; i < k; i += NT) g[i] = beta * H[i];  // rhs = beta * (row 1 of H)
  __syncthreads();
  for (int c = 0; c < k; ++c) {
    if (tid == 0) G[c * k + c] = sqrt(G[c * k + c]);
    __syncthreads();
    const double d = G[c * k + c];
    for (int r = c + 1 + tid; r < k; r += NT) G[r * k + c] /= d;
    __syncthreads();
    for (int idx = tid; idx < (k - c - 1) * (k - c - 1); idx += NT) {
      const int r = c + 1 + idx / (k - c - 1), q = c + 1 + idx % (k - c - 1);
      if (q <= r) G[r * k + q] -= G[r * k + c] * G[q * k + c];
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int r = 0; r < k; ++r) {  // L z = rhs
      double s = g[r];
      for (int q = 0; q < r; ++q) s -= G[r * k + q] * sig[q];
      sig[r] = s / G[r * k + r];
    }
    for (int r = k - 1; r >= 0; --r) {  // L^T y = z
      double s = sig[r];
      for (int q = r + 1; q < k; ++q) s -= G[q * k + r] * g[q];
      g[r] = s / G[r * k + r];
    }
  }
  __syncthreads();
  for (int i = tid; i < kmax; i += NT) y[i] = (i < k) ? g[i] : 0.0;
}

__global__ void k_build_bidiag(const double* alpha, const double* beta, const int* kdev,
                               int kmax, double* H) {
  const int k = kdev ? min(*kdev, kmax) : kmax;
  for (int idx = threadIdx.x; idx < (kmax + 1) * kmax; idx += blockDim.x) {
    const int r = idx / kmax, c = idx % kmax;
    double v = 0.0;
    if (c < k) {
      if (r == c) v = alpha[c];
      else if (r == c + 1) v = beta[c + 1];
    }
    H[idx] = v;
  }
}

}  // namespace

int launch_tikhonov_gcv(const double* H, int ld, int kmax, const int* kdev,
                        const double* beta, int variant, double lambda_in,
                        double* lambda_out, double* y, double* gcv_out, const int* skip,
                        cudaStream_t st) {
  TC_CHECK(kmax >= 1 && kmax <= TC_MAX_PROJ);
  const int kk = kmax + (kmax & 1);
  size_t smem = sizeof(double) * (size_t)(kmax + 1) * kk;
  const size_t gsz = sizeof(double) * (size_t)kmax * kmax;
  if (gsz > smem) smem = gsz;
  k_tikhonov_gcv<<<1, NT, smem, st>>>(H, ld, kmax, kdev, beta, variant, lambda_in, lambda_out,
                                      y, gcv_out, skip);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_build_bidiag(const double* alpha, const double* beta, const int* kdev, int kmax,
                        double* H, cudaStream_t st) {
  k_build_bidiag<<<1, 256, 0, st>>>(alpha, beta, kdev, kmax, H);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// Called once per process (from plan creation) so that no attribute call
// happens while a stream is being captured.
int tc_kernels_init() {
  TC_CUDA(cudaFuncSetAttribute(k_tikhonov_gcv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               200 * 1024));
  TC_TRY(cprod2_init());
  TC_TRY(vec_init());
  TC_TRY(transform_init());
  TC_TRY(group_tc_init());
  return TC_OK;
}
