// Per-lambda GCV evaluation on LSQR's rotations (shared by gcv_bidiag.cu and
// learned.cu). See gcv_bidiag.cu for the derivation.
#pragma once

#include "tc_device.cuh"

// GCV at lambda (and y_lambda into y if given) from R (rho, theta), f (phi),
// interleaved as rg[3j] = rho_j, rg[3j+1] = theta_{j+1}, rg[3j+2] = phi_j,
// and pbar2 = phibar_{k+1}^2.
//
// The residual sum is formed as l^4 ||z||^2 with z = (R R^T + l^2 I)^{-1} f,
// never as f - R y, which cancels when l << sigma_min. R R^T is handled through
// R' = P R^T P (P reverses the order), which is upper bidiagonal (diagonal p_j,
// superdiagonal t_j): R R^T + l^2 I = P (R'^T R' + l^2 I) P = P Rh^T Rh P. Rh is
// the Cholesky factor given by the rotations that fold l I into R' column by
// column. In squared form it needs no square root and one division per
// column:
//   r2_j = p_j^2 + m2_j,  m2_0 = l^2,  m2_{j+1} = m2_j t_j^2 / r2_j + l^2
//   (r2_j = d_j^2; m2_j is the squared l-entry folded into column j),
//   g_j  = p_j t_j / r2_j = e_j / d_j,
//   trace = sum_j T_j / r2_j,  T_0 = 1,  T_{j+1} = 1 + g_j^2 T_j.
// With w~_j = d_j w_j, Rh^T w = P f and Rh u = w become
//   w~_j = f'_j - g_{j-1} w~_{j-1},   u_j = w~_j / r2_j - g_j u_{j+1}.
// y_l = R^T z, z = P u. FP64 throughout; GB300's FP64 latency is long, so the
// chain is kept to about ten dependent operations per column, and 1 / r2 is
// the hardware's approximate FP64 reciprocal refined by two Newton-Raphson
// steps (y <- y + y (1 - x y), quadratic convergence from the approximation's
// relative error, far below 2^-20, to the FP64 rounding level) instead of a
// full IEEE division with its special-case paths: r2 >= l^2 > 0 is finite
// and positive here.
// (rcp_newton of tc_device.cuh: the same two steps, and the IEEE division
// outside [DBL_MIN, 2^1000], e.g. for a subnormal r2 at a tiny lambda.)
__device__ __forceinline__ double recip_nr(double x) { return rcp_newton(x); }

__device__ __forceinline__ double gcv_bd_eval(const double* rg, int k, double pbar2, double lam, int variant,
                              double* y) {
  double inv[TC_MAX_PROJ], gg[TC_MAX_PROJ], wt[TC_MAX_PROJ];
  const double l2 = lam * lam;
  double m2 = l2, T = 1.0, D = 0.0, w = 0.0, gprev = 0.0;
  for (int j = 0; j < k; ++j) {
    const int jr = k - 1 - j;
    const double p = rg[3 * jr];
    const double t = (j + 1 < k) ? rg[3 * (jr - 1) + 1] : 0.0;
    const double r2 = fma(p, p, m2);
    const double iv = recip_nr(r2);
    const double g = p * t * iv;
    D = fma(T, iv, D);
    T = fma(g * g, T, 1.0);
    m2 = fma(m2 * t * t, iv, l2);
    w = rg[3 * jr + 2] - gprev * w;
    inv[j] = iv;
    gg[j] = g;
    wt[j] = w;
    gprev = g;
  }
  double uu = 0.0, un = 0.0;
  for (int j = k - 1; j >= 0; --j) {
    un = fma(wt[j], inv[j], -gg[j] * un);
    wt[j] = un;  // u_j
    uu = fma(un, un, uu);
  }
  if (y) {  // y_j = rho_j z_j + theta_j z_{j-1}, z_i = u_{k-1-i}
    for (int j = 0; j < k; ++j)
      y[j] = rg[3 * j] * wt[k - 1 - j] + (j > 0 ? rg[3 * (j - 1) + 1] * wt[k - j] : 0.0);
  }
  if (variant == TC_GCV_FULL) {
    const double den = fma(l2, D, 1.0);
    return fma(l2 * l2, uu, pbar2) / (den * den);
  }
  return uu / (D * D);
}

