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
  * The paper does not say how GCV is minimised. Here: 200 log-spaced points
    on [lo, s_max] with lo = 1e-3 s_min (or 1e-12 s_max when s_min is 0), the
    smallest value taken (first index on ties), then 40 golden-section steps
    in log(lambda) on the bracket formed by the two grid neighbours.
  * The Tikhonov weight is lambda^2 (eqs. (leastsq), (tikho2)), not the lambda of
    eq. (tr2); the reported parameter is lambda.
"""
import numpy as np

GRID_POINTS = 200
GOLDEN_STEPS = 40
LO_FACTOR = 1e-3


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
    """lambda minimising GCV for the projected matrix H (m+1 x m) and beta.

    Log grid, then golden-section refinement in log(lambda) (reading above)."""
    sig, g = svd_projected(H, beta)
    smax = float(sig[0])
    smin = float(sig[-1])
    lo = LO_FACTOR * smin if smin > 0.0 else 1e-12 * smax
    grid = np.exp(np.linspace(np.log(lo), np.log(smax), GRID_POINTS))
    vals = np.array([gcv_value(sig, g, t, variant) for t in grid])
    i = int(np.argmin(vals))
    a = np.log(grid[max(i - 1, 0)])
    b = np.log(grid[min(i + 1, GRID_POINTS - 1)])
    invphi = (np.sqrt(5.0) - 1.0) / 2.0
    c = b - invphi * (b - a)
    d = a + invphi * (b - a)
    fc = gcv_value(sig, g, np.exp(c), variant)
    fd = gcv_value(sig, g, np.exp(d), variant)
    for _ in range(GOLDEN_STEPS):
        if fc <= fd:
            b, d, fd = d, c, fc
            c = b - invphi * (b - a)
            fc = gcv_value(sig, g, np.exp(c), variant)
        else:
            a, c, fc = c, d, fd
            d = a + invphi * (b - a)
            fd = gcv_value(sig, g, np.exp(d), variant)
    t = c if fc <= fd else d
    best = min(fc, fd)
    # keep the grid point if the refinement did not improve on it
    if vals[i] < best:
        return float(grid[i]), float(vals[i])
    return float(np.exp(t)), float(best)


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
