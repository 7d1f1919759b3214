"""FP64 oracle of the L-curve stopping index for DC-LSQR (test infrastructure only).

§3.3 (after Algorithm 6): for ill-posed problems the error of the LSQR
iterates falls and then rises, so the iteration is stopped at an optimal
index k_opt. The text proposes the L-curve criterion: plot the points
(||R_k||, ||X_k||) and take the point of maximum curvature, the corner.

The paper gives neither the scale nor a discrete curvature. Reading (R18):
  * the curve lives in log-log coordinates, P_k = (log ||R_k||_F, log ||X_k||_F),
    k = 1..K (the usual L-curve plot);
  * the curvature at P_k (1 < k < K) is the signed Menger curvature of
    (P_{k-1}, P_k, P_{k+1}): the reciprocal radius of the circle through the
    three points (Menger's discrete curvature; also the corner test of Cultrera
    and Callegaro's L-curve algorithm), taken positive when the curve turns
    the way an L-curve turns at its corner (from running towards smaller
    residual to running towards larger norm, a clockwise turn);
  * k_opt is the k of largest curvature, the smallest such k on ties; with
    K < 3 there is no interior point and k_opt = K.

Here X_k is the LSQR iterate after k steps and R_k = C - A *c X_k, both
computed from their definitions.
"""
import math

import numpy as np

from . import cproduct as cp
from . import krylov as kr


def menger_curvature(p0, p1, p2):
    """Signed curvature of the circle through three plane points: 4 * area /
    (product of the side lengths), positive for a clockwise turn at p1 (the
    L-curve's corner), zero for collinear points. Coincident points give 0."""
    ax, ay = p1[0] - p0[0], p1[1] - p0[1]
    bx, by = p2[0] - p1[0], p2[1] - p1[1]
    cross = ax * by - ay * bx  # twice the signed area; > 0 counter-clockwise
    a = math.hypot(ax, ay)
    b = math.hypot(bx, by)
    c = math.hypot(p2[0] - p0[0], p2[1] - p0[1])
    den = a * b * c
    if den == 0.0:
        return 0.0
    return -2.0 * cross / den


def corner(resnorm, solnorm):
    """k_opt (1-based) of the curve (log resnorm_k, log solnorm_k), k = 1..K."""
    K = len(resnorm)
    if K < 3:
        return K
    P = [(math.log(resnorm[k]), math.log(solnorm[k])) for k in range(K)]
    best, kbest = -math.inf, K
    for k in range(1, K - 1):
        kap = menger_curvature(P[k - 1], P[k], P[k + 1])
        if kap > best:
            best, kbest = kap, k + 1
    return kbest


def curvatures(resnorm, solnorm):
    """Curvature at every interior point (index k-1 for k = 2..K-1; NaN at the ends)."""
    K = len(resnorm)
    P = [(math.log(resnorm[k]), math.log(solnorm[k])) for k in range(K)]
    out = np.full(K, np.nan)
    for k in range(1, K - 1):
        out[k] = menger_curvature(P[k - 1], P[k], P[k + 1])
    return out


def lsqr_lcurve(op, adj, C, kmax):
    """DC-LSQR stopped at the L-curve corner: the iterates X_1..X_K, their
    residual and solution norms from the definitions, k_opt, and X_{k_opt}."""
    Xs = kr.lsqr(op, adj, C, itermax=kmax, keep_iterates=True)["Xs"]
    res = np.array([cp.fro(C - op(X)) for X in Xs])
    sol = np.array([cp.fro(X) for X in Xs])
    k = corner(res, sol)
    return dict(Xs=Xs, resnorm=res, solnorm=sol, kopt=k, X_opt=Xs[k - 1],
                curvature=curvatures(res, sol))
