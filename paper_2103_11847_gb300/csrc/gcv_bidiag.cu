// GCV and Tikhonov on the Golub-Kahan bidiagonal after c-LSQR, without an SVD
// (§3.2 eqs. (normeq2), (leastsq0), §3.1 eq. (gcv2)).
//
// LSQR's plane rotations already factor the (k+1) x k bidiagonal: Q C~_k = [R; 0]
// with R upper bidiagonal (diagonal rho_j, superdiagonal theta_{j+1}) and
// Q (beta_1 e_1) = (phi_1 .. phi_k, phibar_{k+1}) (§3.3). With C~_k = U S V^T,
// g~ = beta_1 U^T e_1 = (U_R^T f, phibar_{k+1}) where f = (phi_1 .. phi_k), so
//   sum_i 1 / (s_i^2 + l^2)              = trace((R R^T + l^2 I)^{-1}),
//   sum_i l^4 g~_i^2 / (s_i^2 + l^2)^2   = l^4 ||(R R^T + l^2 I)^{-1} f||^2,
// and y_l = argmin ||R y - f||^2 + l^2 ||y||^2, the Tikhonov solution of the
// projected problem, is R^T (R R^T + l^2 I)^{-1} f. For an upper bidiagonal
// matrix B, an O(k) sequence of plane rotations (two per column) reduces
// [B; l I] to an upper bidiagonal Rh (diagonal d, superdiagonal e) with
// B^T B + l^2 I = Rh^T Rh, and trace((Rh^T Rh)^{-1}) = ||Rh^{-1}||_F^2 =
// sum_j T_j / d_j^2 with T_1 = 1, T_{j+1} = 1 + (e_j / d_j)^2 T_j.
// This costs O(k) FP64 operations per lambda instead of an O(k^3) SVD; FP64
// is scarce on GB300.
//
// Search: the same three nested 200-point log grids as the general path
// (first level [1e-10 s, s] with s = ||C~_k||_F). Each lane of a warp runs one
// point's serial O(k) FP64 chain, 32 points a warp: the SM's narrow FP64 pipe
// takes a warp instruction at the same cost whether one lane or all 32 are
// active, so one point a warp (an earlier form) kept the pipe 87% busy on
// 1/32 of the work when the batched form's 128 problems filled the GPU.
#include "gcv_eval.cuh"

namespace {

constexpr int NGRID = 200;
constexpr int NLEVEL = 3;
constexpr int PPW = 32;  // grid points a warp (one a lane); one warp a CTA

// First index of the smallest of v[0..n) over one warp (ties to the lower index).
__device__ int warp_argmin(const double* v, int n) {
  const int lane = threadIdx.x & 31;
  double best = INFINITY;
  int bi = n;
  for (int t = lane; t < n; t += 32) {
    const double x = v[t];
    if (x < best) { best = x; bi = t; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  return bi < n ? bi : 0;
}

// One level of the search: lane l of CTA b evaluates grid point PPW b + l.
// Grouped launches (grid.y = problems): problem blockIdx.y's doubles are ps
// and its ints fsi further on (0 for a single problem).
__global__ void k_gcv_bd_level(const double* rg, const double* phibar, const double* alpha, const double* beta,
                               const int* kdev, int kmax, int variant, int level, double* lams,
                               double* vals, size_t ps = 0, int fsi = 0) {
  {
    const size_t od = (size_t)blockIdx.y * ps;
    rg += od; phibar += od; alpha += od; beta += od; lams += od; vals += od;
    if (kdev) kdev += (size_t)blockIdx.y * fsi;
  }
  const int k = kdev ? min(*kdev, kmax) : kmax;
  const int i = blockIdx.x * PPW + (int)threadIdx.x;
  if (k <= 0) {
    if (i < NGRID) {
      lams[level * NGRID + i] = nan("");
      vals[level * NGRID + i] = nan("");
    }
    return;
  }
  double lo, hi;
  if (level == 0) {
    // ||C~_k||_F^2: diagonal alpha_1..alpha_k, subdiagonal beta_2..beta_{k+1}
    double s2 = 0.0;
    for (int j = threadIdx.x & 31; j < k; j += 32) s2 += alpha[j] * alpha[j] + beta[j + 1] * beta[j + 1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    hi = log(sqrt(s2));
    lo = hi - 10.0 * log(10.0);
  } else {
    const double* pl = lams + (level - 1) * NGRID;
    const int b = warp_argmin(vals + (level - 1) * NGRID, NGRID);
    lo = log(pl[max(b - 1, 0)]);
    hi = log(pl[min(b + 1, NGRID - 1)]);
  }
  if (i >= NGRID) return;  // after the warp-wide bounds above
  const double step = (hi - lo) / (NGRID - 1);
  const double lam = exp(i == NGRID - 1 ? hi : lo + i * step);
  const double pb = phibar[k];
  lams[level * NGRID + i] = lam;
  vals[level * NGRID + i] = gcv_bd_eval(rg, k, pb * pb, lam, variant, nullptr);
}

// lambda (the last level's minimum, or lambda_in >= 0), GCV there, and y.
// With lam_pred (a predicted lambda): keep it unless its GCV exceeds factor
// times the last level's minimum, in which case the minimiser is used and
// *fallback is set to 1.
__global__ void k_gcv_bd_final(const double* rg, const double* phibar, const int* kdev, int kmax,
                               int variant, double lambda_in, const double* lams,
                               const double* vals, const double* lam_pred, double factor,
                               int* fallback, double* lambda_out, double* y, double* gcv_out,
                               size_t ps = 0, int fsi = 0) {
  {
    const size_t od = (size_t)blockIdx.x * ps, oi = (size_t)blockIdx.x * fsi;
    rg += od; phibar += od; lams += od; vals += od; lambda_out += od; y += od;
    if (gcv_out) gcv_out += od;
    if (lam_pred) lam_pred += od;
    if (kdev) kdev += oi;
    if (fallback) fallback += oi;
  }
  const int k = kdev ? min(*kdev, kmax) : kmax;
  for (int j = (k > 0 ? k : 0) + (int)threadIdx.x; j < kmax; j += 32) y[j] = 0.0;
  double lam = lambda_in;
  int b = 0;
  if (k > 0 && !(lambda_in >= 0.0)) {
    b = warp_argmin(vals + (NLEVEL - 1) * NGRID, NGRID);
    lam = lams[(NLEVEL - 1) * NGRID + b];
  }
  if (threadIdx.x != 0) return;
  if (k <= 0) {
    *lambda_out = nan("");
    if (gcv_out) *gcv_out = nan("");
    return;
  }
  const double pb = phibar[k];
  if (lam_pred) {
    const double lp = *lam_pred;
    const double gp = gcv_bd_eval(rg, k, pb * pb, lp, variant, nullptr);
    const double gmin = vals[(NLEVEL - 1) * NGRID + b];
    const bool use_pred = isfinite(gp) && lp > 0.0 && gp <= factor * gmin;
    if (fallback) *fallback = use_pred ? 0 : 1;
    if (use_pred) lam = lp;
  }
  const double gv = gcv_bd_eval(rg, k, pb * pb, lam, variant, y);
  *lambda_out = lam;
  if (gcv_out) *gcv_out = gv;
}

// L-curve corner (§3.3; reading: log-log curve, signed Menger curvature,
// smallest k on ties). Thread t takes k = t + 1 <= K:
//   ||R_k|| = |phibar_{k+1}|, ||X_k|| = ||y_k|| with R_k y_k = f_k solved
//   upward (y_{k-1} = phi_{k-1} / rho_{k-1}, y_i = (phi_i - theta_{i+1} y_{i+1}) / rho_i),
// then the curvature of the circle through P_{k-1}, P_k, P_{k+1} in log
// coordinates, 2 (-cross) / (|P_k - P_{k-1}| |P_{k+1} - P_k| |P_{k+1} - P_{k-1}|),
// and one warp takes the first maximum. Thread 0 writes y_{k_opt} (zero
// beyond k_opt) for the basis combination. One CTA of TC_MAX_PROJ threads.
__global__ void __launch_bounds__(TC_MAX_PROJ)
k_lcurve(const double* rg, const double* phibar, const int* kdev, int kmax, double* curve,
         double* y, int* kopt) {
  __shared__ double s_ir[TC_MAX_PROJ], s_lr[TC_MAX_PROJ], s_lx[TC_MAX_PROJ], s_kap[TC_MAX_PROJ];
  __shared__ int s_k;
  const int K = max(0, min(*kdev, kmax));
  const int t = threadIdx.x;
  if (t < K) s_ir[t] = 1.0 / rg[3 * t];
  __syncthreads();
  if (t < K) {
    const int k = t + 1;
    double yi = rg[3 * (k - 1) + 2] * s_ir[k - 1];
    double ss = yi * yi;
    for (int i = k - 2; i >= 0; --i) {
      yi = (rg[3 * i + 2] - rg[3 * i + 1] * yi) * s_ir[i];
      ss = fma(yi, yi, ss);
    }
    const double rn = fabs(phibar[k]), xn = sqrt(ss);
    if (curve) {
      curve[t] = rn;
      curve[kmax + t] = xn;
    }
    s_lr[t] = log(rn);
    s_lx[t] = log(xn);
  }
  __syncthreads();
  s_kap[t] = -INFINITY;
  if (t >= 1 && t + 1 < K) {
    const double ax = s_lr[t] - s_lr[t - 1], ay = s_lx[t] - s_lx[t - 1];
    const double bx = s_lr[t + 1] - s_lr[t], by = s_lx[t + 1] - s_lx[t];
    const double cx = s_lr[t + 1] - s_lr[t - 1], cy = s_lx[t + 1] - s_lx[t - 1];
    const double den = hypot(ax, ay) * hypot(bx, by) * hypot(cx, cy);
    const double cr = ax * by - ay * bx;
    s_kap[t] = den == 0.0 ? 0.0 : -2.0 * cr / den;
  }
  __syncthreads();
  if (t < 32) {
    double best = -INFINITY;
    int bi = TC_MAX_PROJ;
    for (int i = t; i < TC_MAX_PROJ; i += 32)
      if (s_kap[i] > best) { best = s_kap[i]; bi = i; }  // ascending i: first maximum kept
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (t == 0) s_k = (K < 3) ? K : bi + 1;
  }
  __syncthreads();
  const int ko = s_k;
  for (int i = t; i < kmax; i += blockDim.x)
    if (i >= ko) y[i] = 0.0;
  if (t == 0) {
    *kopt = ko;
    if (ko > 0) {
      double yi = rg[3 * (ko - 1) + 2] * s_ir[ko - 1];
      y[ko - 1] = yi;
      for (int i = ko - 2; i >= 0; --i) {
        yi = (rg[3 * i + 2] - rg[3 * i + 1] * yi) * s_ir[i];
        y[i] = yi;
      }
    }
  }
}

}  // namespace

int launch_lcurve(const double* rg, const double* phibar, const int* kdev, int kmax,
                  double* curve, double* y, int* kopt, cudaStream_t st) {
  TC_CHECK(kmax >= 1 && kmax <= TC_MAX_PROJ);
  k_lcurve<<<1, TC_MAX_PROJ, 0, st>>>(rg, phibar, kdev, kmax, curve, y, kopt);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_gcv_bidiag_group(const double* rg, const double* phibar, const double* alpha,
                            const double* beta, const int* kdev, int kmax, int variant,
                            double lambda_in, double* work, double* lambda_out, double* y,
                            double* gcv_out, int count, size_t ps, int fsi, cudaStream_t st) {
  TC_CHECK(kmax >= 1 && kmax <= TC_MAX_PROJ && count >= 1 && count <= 65535);
  double* lams = work;
  double* vals = work + NLEVEL * NGRID;
  if (!(lambda_in >= 0.0)) {
    for (int level = 0; level < NLEVEL; ++level) {
      k_gcv_bd_level<<<dim3((NGRID + PPW - 1) / PPW, count), PPW, 0, st>>>(
          rg, phibar, alpha, beta, kdev, kmax, variant, level, lams, vals, ps, fsi);
      TC_CUDA(cudaGetLastError());
    }
  }
  k_gcv_bd_final<<<count, 32, 0, st>>>(rg, phibar, kdev, kmax, variant, lambda_in, lams, vals,
                                       nullptr, 0.0, nullptr, lambda_out, y, gcv_out, ps, fsi);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int launch_gcv_bidiag(const double* rg, const double* phibar, const double* alpha,
                      const double* beta, const int* kdev, int kmax, int variant,
                      double lambda_in, double* work, double* lambda_out, double* y,
                      double* gcv_out, cudaStream_t st, const double* lam_pred, double factor,
                      int* fallback) {
  TC_CHECK(kmax >= 1 && kmax <= TC_MAX_PROJ);
  double* lams = work;
  double* vals = work + NLEVEL * NGRID;
  if (!(lambda_in >= 0.0)) {
    for (int level = 0; level < NLEVEL; ++level) {
      k_gcv_bd_level<<<(NGRID + PPW - 1) / PPW, PPW, 0, st>>>(
          rg, phibar, alpha, beta, kdev, kmax, variant, level, lams, vals);
      TC_CUDA(cudaGetLastError());
    }
  }
  k_gcv_bd_final<<<1, 32, 0, st>>>(rg, phibar, kdev, kmax, variant, lambda_in, lams, vals,
                                   lam_pred, factor, fallback, lambda_out, y, gcv_out);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
