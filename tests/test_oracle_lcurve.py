"""Pins of the L-curve oracle (oracle/lcurve.py, §3.3 and reading R18) to
geometry and to LSQR's own identities.

* Menger curvature: three points on a circle of radius R give exactly 1/R,
  signed by the turn; collinear and coincident points give 0.
* The corner of a polyline that runs left and then turns up is the bend, and
  it does not move when either norm is rescaled (a shift in log coordinates).
* The LSQR quantities the GPU uses for the curve equal the definitions:
  ||C - A *c X_k|| = |phibar_{k+1}| and ||X_k|| = ||R_k^{-1} f_k||, with R_k
  and f_k from a QR factorisation of the (k+1) x k bidiagonal and beta_1 e_1.
"""
import math

import numpy as np
import pytest

from oracle import cproduct as cp
from oracle import krylov as kr
from oracle import lcurve as lc
from paper_2103_11847_gb300 import inputs


@pytest.mark.parametrize("R,cx,cy,t0", [(1.0, 0.0, 0.0, 0.1), (0.25, 3.0, -2.0, 1.3),
                                        (17.5, -4.0, 8.0, 2.9)])
def test_menger_curvature_of_a_circle(R, cx, cy, t0):
    pts = [(cx + R * math.cos(t0 - d), cy + R * math.sin(t0 - d)) for d in (0.0, 0.4, 1.1)]
    # decreasing angle: a clockwise turn, positive
    assert abs(lc.menger_curvature(*pts) - 1.0 / R) < 1e-12 / R
    assert abs(lc.menger_curvature(*pts[::-1]) + 1.0 / R) < 1e-12 / R


def test_menger_curvature_degenerate():
    assert lc.menger_curvature((0, 0), (1, 2), (2, 4)) == 0.0
    assert lc.menger_curvature((1, 1), (1, 1), (3, 0)) == 0.0


def l_shape(bend=6, n_up=4):
    """Points running left along y = 0 to the origin (index `bend`), then up."""
    pts = [(float(bend - k), 0.0) for k in range(1, bend + 1)]
    pts += [(0.0, float(k)) for k in range(1, n_up + 1)]
    res = np.exp([p[0] for p in pts])
    sol = np.exp([p[1] for p in pts])
    return res, sol


def test_corner_of_an_l_is_the_bend():
    res, sol = l_shape(bend=6)
    assert lc.corner(res, sol) == 6
    kap = lc.curvatures(res, sol)
    assert abs(kap[5] - math.sqrt(2.0)) < 1e-12  # right angle, unit legs
    assert np.nanmax(np.abs(np.delete(kap, 5))) < 1e-12


def test_corner_is_scale_invariant_and_ties_go_low():
    res, sol = l_shape(bend=4, n_up=6)
    assert lc.corner(7.0 * res, 0.3 * sol) == lc.corner(res, sol) == 4
    # two equal bends: the first one wins
    x = [4, 3, 2, 2, 1, 1]
    y = [0, 0, 0, 1, 1, 2]
    assert lc.corner(np.exp(x), np.exp(y)) == 3
    assert lc.corner(np.array([2.0, 1.0]), np.array([1.0, 2.0])) == 2


def _problem(n=24, seed=5):
    p = inputs.random_problem(n, n, n, 3, seed=seed)
    A = p["A"].astype(np.float64)
    op = lambda X: cp.cprod(A, X)
    adj = lambda Y: cp.cprod_adjoint(A, Y)
    return op, adj, p["Y"].astype(np.float64)


def test_lsqr_norm_identities_behind_the_gpu_curve():
    op, adj, C = _problem()
    K = 8
    r = kr.lsqr(op, adj, C, itermax=K, keep_iterates=True)
    for k in range(1, K + 1):
        Xk = r["Xs"][k - 1]
        res = cp.fro(C - op(Xk))
        assert abs(res - r["phibar"][k - 1]) < 1e-9 * res
        B = kr.bidiagonal(r["alpha"], r["beta"], k)
        Q, Rk = np.linalg.qr(B, mode="complete")
        f = (Q.T @ (r["beta"][0] * np.eye(k + 1)[:, 0]))[:k]
        y = np.linalg.solve(Rk[:k, :k], f)
        assert abs(np.linalg.norm(y) - cp.fro(Xk)) < 1e-9 * cp.fro(Xk)


def test_lsqr_lcurve_returns_the_corner_iterate():
    op, adj, C = _problem(n=20, seed=8)
    out = lc.lsqr_lcurve(op, adj, C, kmax=10)
    k = out["kopt"]
    assert 1 <= k <= 10
    assert out["X_opt"] is out["Xs"][k - 1]
    assert k == lc.corner(out["resnorm"], out["solnorm"])
    # the residual never grows along LSQR's iterates
    assert np.all(np.diff(out["resnorm"]) <= 1e-12 * out["resnorm"][0])
