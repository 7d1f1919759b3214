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
// (first level [1e-10 s, s] with s = ||C~_k||_F). Each point of a level runs on
// its own CTA, so the serial O(k) chains of the 200 points overlap across SMs.
#include "tc_device.cuh"

namespace {

constexpr int NGRID = 200;
constexpr int NLEVEL = 3;

// GCV at lambda (and y_lambda into y if given) from R (rho, theta), f (phi),
// interleaved as rg[3j] = rho_j, rg[3j+1] = theta_{j+1}, rg[3j+2] = phi_j,
// and pbar2 = phibar_{k+1}^2.
//
// The residual sum is formed as l^4 ||z||^2 with z = (R R^T + l^2 I)^{-1} f,
// never as f - R y: that difference cancels when l << sigma_min. R R^T is
// handled through R' = P R^T P (P reverses the order), which is upper
// bidiagonal: R R^T + l^2 I = P (R'^T R' + l^2 I) P = P Rh^T Rh P, where Rh
// comes from the rotations above applied to [R'; l I]. The trace is the same
// for R R^T and R^T R. y_l = R^T z.
__device__ double gcv_bd_eval(const double* rg, int k, double pbar2, double lam, int variant,
                              double* y) {
  double d[TC_MAX_PROJ], e[TC_MAX_PROJ], u[TC_MAX_PROJ];
  double mu = lam, T = 1.0, D = 0.0;
  for (int j = 0; j < k; ++j) {
    const int jr = k - 1 - j;  // R'_{jj} = rho_{jr}, R'_{j,j+1} = theta of column jr-1
    const double rj = rg[3 * jr];
    const double r = hypot(rj, mu);
    const double c = (r > 0.0) ? rj / r : 1.0, s = (r > 0.0) ? mu / r : 0.0;
    d[j] = r;
    D += T / (r * r);
    e[j] = 0.0;
    if (j + 1 < k) {
      const double th = rg[3 * (jr - 1) + 1];
      e[j] = c * th;
      const double fill = -s * th;  // row k+j, column j+1
      const double q = e[j] / r;
      T = 1.0 + q * q * T;
      mu = hypot(fill, lam);  // merge the fill into row k+j+1 (only l at column j+1)
    }
  }
  // Rh^T w = P f, Rh u = w; z = P u
  double wp = 0.0;
  for (int j = 0; j < k; ++j) {
    const double fj = rg[3 * (k - 1 - j) + 2];
    wp = (fj - (j > 0 ? e[j - 1] * wp : 0.0)) / d[j];
    u[j] = wp;
  }
  double uu = 0.0, un = 0.0;
  for (int j = k - 1; j >= 0; --j) {
    un = (u[j] - e[j] * un) / d[j];
    u[j] = un;
    uu += un * un;
  }
  if (y) {  // y_j = rho_j z_j + theta_j z_{j-1}, z_i = u_{k-1-i}
    for (int j = 0; j < k; ++j)
      y[j] = rg[3 * j] * u[k - 1 - j] + (j > 0 ? rg[3 * (j - 1) + 1] * u[k - j] : 0.0);
  }
  if (variant == TC_GCV_FULL) {
    const double l2 = lam * lam;
    const double den = 1.0 + l2 * D;
    return (l2 * l2 * uu + pbar2) / (den * den);
  }
  return uu / (D * D);
}

// One level of the search: CTA i evaluates grid point i of this level.
__global__ void k_gcv_bd_level(const double* rg, const double* phibar, const double* alpha, const double* beta,
                               const int* kdev, int kmax, int variant, int level, double* lams,
                               double* vals) {
  if (threadIdx.x != 0) return;
  const int k = kdev ? min(*kdev, kmax) : kmax;
  const int i = blockIdx.x;
  if (k <= 0) {
    lams[level * NGRID + i] = nan("");
    vals[level * NGRID + i] = nan("");
    return;
  }
  double lo, hi;
  if (level == 0) {
    double s2 = 0.0;  // ||C~_k||_F^2: diagonal alpha_1..alpha_k, subdiagonal beta_2..beta_{k+1}
    for (int j = 0; j < k; ++j) s2 += alpha[j] * alpha[j] + beta[j + 1] * beta[j + 1];
    hi = log(sqrt(s2));
    lo = hi - 10.0 * log(10.0);
  } else {
    const double* pl = lams + (level - 1) * NGRID;
    const double* pv = vals + (level - 1) * NGRID;
    int b = 0;
    for (int t = 1; t < NGRID; ++t)
      if (pv[t] < pv[b]) b = t;
    lo = log(pl[max(b - 1, 0)]);
    hi = log(pl[min(b + 1, NGRID - 1)]);
  }
  const double step = (hi - lo) / (NGRID - 1);
  const double lam = exp(i == NGRID - 1 ? hi : lo + i * step);
  const double pb = phibar[k];
  lams[level * NGRID + i] = lam;
  vals[level * NGRID + i] = gcv_bd_eval(rg, k, pb * pb, lam, variant, nullptr);
}

// lambda (the last level's minimum, or lambda_in >= 0), GCV there, and y.
__global__ void k_gcv_bd_final(const double* rg, const double* phibar, const int* kdev, int kmax, int variant,
                               double lambda_in, const double* lams, const double* vals,
                               double* lambda_out, double* y, double* gcv_out) {
  if (threadIdx.x != 0) return;
  const int k = kdev ? min(*kdev, kmax) : kmax;
  for (int j = (k > 0 ? k : 0); j < kmax; ++j) y[j] = 0.0;
  if (k <= 0) {
    *lambda_out = nan("");
    if (gcv_out) *gcv_out = nan("");
    return;
  }
  double lam = lambda_in;
  if (!(lambda_in >= 0.0)) {
    const double* pl = lams + (NLEVEL - 1) * NGRID;
    const double* pv = vals + (NLEVEL - 1) * NGRID;
    int b = 0;
    for (int t = 1; t < NGRID; ++t)
      if (pv[t] < pv[b]) b = t;
    lam = pl[b];
  }
  const double pb = phibar[k];
  const double gv = gcv_bd_eval(rg, k, pb * pb, lam, variant, y);
  *lambda_out = lam;
  if (gcv_out) *gcv_out = gv;
}

}  // namespace

int launch_gcv_bidiag(const double* rg, const double* phibar, const double* alpha, const double* beta,
                      const int* kdev, int kmax, int variant, double lambda_in, double* work,
                      double* lambda_out, double* y, double* gcv_out, cudaStream_t st) {
  TC_CHECK(kmax >= 1 && kmax <= TC_MAX_PROJ);
  double* lams = work;
  double* vals = work + NLEVEL * NGRID;
  if (!(lambda_in >= 0.0)) {
    for (int level = 0; level < NLEVEL; ++level) {
      k_gcv_bd_level<<<NGRID, 32, 0, st>>>(rg, phibar, alpha, beta, kdev, kmax,
                                           variant, level, lams, vals);
      TC_CUDA(cudaGetLastError());
    }
  }
  k_gcv_bd_final<<<1, 32, 0, st>>>(rg, phibar, kdev, kmax, variant, lambda_in, lams,
                                   vals, lambda_out, y, gcv_out);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}
