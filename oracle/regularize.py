"""Projected Tikhonov problem and GCV choice of lambda, float64 (oracle).

Test infrastructure only: see the package docstring.

Paper references (arXiv 2103.11847):
  §3.1, eqs. (leastsq), (min) -- y = argmin ||beta e_1 - H y||^2 + lambda^2 ||y||^2
                                 for the (m+1) x m projected matrix H.
  §3.1, eq. (tikho2)          -- normal equations (H^T H + lambda^2 I) y = beta H^T e_1.
  §3.2, eqs. (normeq2), (leastsq0) -- the same for the Golub-Kahan bidiagonal.
  §3.1, eq. (gcv2)            -- GCV(lambda) from the SVD H = U Sigma V^T and
                                 g~ = beta U^T e_1.

Readings:
  * (tikho2) prints H~^T C~_m; (normeq2) prints alpha_1 = ||C||_F for the scale
    of e_1. Both are read as the standard problem above with beta_1 = ||C||_F.
  * (gcv2) as printed sums over i = 1..m with no g~_{m+1} term and no "+1" in
    the trace: it is the square-matrix GCV. That is the default ("paper"). The
    GCV of the rectangular (m+1) x m problem ("full") is
      (sum_i (lambda^2 g~_i / (s_i^2 + lambda^2))^2 + g~_{m+1}^2)
      / (1 + sum_i lambda^2 / (s_i^2 + lambda^2))^2.
  * The paper does not say how GCV is minimised. Here: three nested log grids
    of 200 points. Level 0 spans [1e-10 s, s] with s = ||H||_F (an upper
    bound of sigma_max that needs no SVD). Each later level spans the two
    grid neighbours of the previous level's minimum (first index on ties).
    The answer is the last level's minimum; its spacing is 1.2e-5 in
    log(lambda).
  * The Tikhonov weight is lambda^2 (eqs. (leastsq), (tikho2)), not the lambda of
    eq. (tr2); the reported parameter is lambda.
"""
import numpy as np

GRID_POINTS = 200
GRID_LEVELS = 3
GRID_DECADES = 10.0


def svd_projected(H, beta):
    """SVD of the projected matrix and g~ = beta U^T e_1 (below eq. (gcv2)).

    Returns (sigma[m], g[m+1]) with U the full (m+1) x (m+1) left factor."""
    U, sig, _ = np.linalg.svd(np.asarray(H, np.float64), full_matrices=True)
    g = beta * U[0, :]
    return sig, g


def gcv_value(sig, g, lam, variant="paper"):
    """GCV(lambda) of eq. (gcv2) ("paper") or of the rectangular problem ("full")."""
    m = sig.shape[0]
    d = sig ** 2 + lam ** 2
    if variant == "paper":
        num = np.sum((g[:m] / d) ** 2)
        den = np.sum(1.0 / d) ** 2
        return float(num / den)
    if variant == "full":
        r = lam ** 2 * g[:m] / d
        num = np.sum(r ** 2) + np.sum(g[m:] ** 2)
        den = (1.0 + np.sum(lam ** 2 / d)) ** 2
        return float(num / den)
    raise ValueError(variant)


def gcv_minimize(H, beta, variant="paper"):
    """lambda minimising GCV for the projected matrix H (m+1 x m) and beta,
    by the nested log grids described above."""
    sig, g = svd_projected(H, beta)
    s = float(np.linalg.norm(np.asarray(H, np.float64)))
    lo, hi = np.log(s) - GRID_DECADES * np.log(10.0), np.log(s)
    for _ in range(GRID_LEVELS):
        lams = np.exp(np.linspace(lo, hi, GRID_POINTS))
        vals = np.array([gcv_value(sig, g, t, variant) for t in lams])
        b = int(np.argmin(vals))
        lo = np.log(lams[max(b - 1, 0)])
        hi = np.log(lams[min(b + 1, GRID_POINTS - 1)])
    return float(lams[b]), float(vals[b])


def tikhonov_solve(H, beta, lam):
    """y solving the normal equations (H^T H + lambda^2 I) y = beta H^T e_1
    (eqs. (tikho2), (normeq2))."""
    H = np.asarray(H, np.float64)
    m = H.shape[1]
    rhs = beta * H[0, :]
    return np.linalg.solve(H.T @ H + lam ** 2 * np.eye(m), rhs)


def tikhonov_gcv(H, beta, variant="paper", lam=None):
    """Choose lambda by GCV (unless given) and solve the projected Tikhonov problem.

    Returns (lam, y, gcv_at_lam)."""
    if lam is None:
        lam, gv = gcv_minimize(H, beta, variant)
    else:
        sig, g = svd_projected(H, beta)
        gv = gcv_value(sig, g, lam, variant)
    return lam, tikhonov_solve(H, beta, lam), gv
