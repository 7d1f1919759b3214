"""Tensor cosine global Krylov methods, float64 (oracle).

Test infrastructure only: see the package docstring.

Every method takes the operator as functions so that the one-sided
A *c X and the two-sided A *c X *c B (eq. (eq2)) share the code:
  op(X)  -- X -> A *c X [*c B]
  adj(Y) -- its adjoint for <.,.> (the A^T *c of Algorithms 4 and 6).

Paper references (arXiv 2103.11847):
  §3.1, Algorithm 2 -- tensor discrete cosine (global) Arnoldi, modified
                       Gram-Schmidt, stop when h_{j+1,j} = 0.
  §3.1, Algorithm 3 -- restarted DC-GMRES(m) with Tikhonov/GCV, eq. (xm).
  §3.2, Algorithm 4 -- tensor discrete cosine Golub-Kahan bidiagonalisation.
  §3.2, Algorithm 5 -- DC-GK: Algorithm 4, GCV, y from (leastsq0), eq. (xmlsqr).
  §3.3, Algorithm 6 -- DC-LSQR, Givens recurrences below eq. (sollsqr).

Readings:
  * Algorithm 6 uses W_j both for the unnormalised U-direction (step (a)) and
    for the search direction (step (f)), and writes X_i for X_j. It is read as
    the standard LSQR recurrence: U_{j+1} from A *c V_j - alpha_j U_j, the
    search direction W with W_1 = V_1, X_j = X_{j-1} + (phi_j/rho_j) W_j.
  * Algorithm 3 step 7 says "go to Step 4" after X_0 = X_m; the residual of the
    new X_0 is recomputed first (step 3), otherwise the restart would run on
    the old residual.
  * Algorithm 3's iteration count: itermax counts Arnoldi steps (products) in
    total; a cycle runs min(m, itermax - done) steps.
  * Breakdown (alpha or beta = 0, tests left commented out in Algorithm 4;
    h_{j+1,j} = 0 in Algorithm 2): the process stops and reports the step.
    In LSQR a zero beta_{j+1} finishes step j with alpha_{j+1} = 0 (the Givens
    recurrences then give phibar_{j+1} = 0 and the exact solution) and stops.
  * The bidiagonal C~_m of §3.2 is printed lower bidiagonal (diagonal alpha_1..
    alpha_m, subdiagonal beta_2..beta_{m+1}) although the text says "upper";
    the printed matrix is used.
"""
import numpy as np

from .cproduct import fro, inner, circledast
from .regularize import tikhonov_gcv


def arnoldi(op, V, m):
    """Algorithm 2. Returns (basis [V_1..V_{k+1}], Hbar (k+1) x k, beta, k)
    with k <= m the number of completed steps (k < m on breakdown)."""
    beta = fro(V)
    basis = [V / beta]
    H = np.zeros((m + 1, m))
    k = 0
    for j in range(m):
        W = op(basis[j])
        for i in range(j + 1):
            H[i, j] = inner(basis[i], W)
            W = W - H[i, j] * basis[i]
        H[j + 1, j] = fro(W)
        k = j + 1
        if H[j + 1, j] == 0.0:
            basis.append(np.zeros_like(W))
            break
        basis.append(W / H[j + 1, j])
    return basis, H[:k + 1, :k], beta, k


def gmres(op, C, X0, m, itermax, tol=0.0, variant="paper", lam=None):
    """Algorithm 3, DC-GMRES(m) with Tikhonov regularisation.

    lam=None chooses lambda by GCV each cycle; a number fixes it.
    Returns dict(X, residuals (||R_0|| of every cycle plus the final one),
    lambdas, steps, cycles)."""
    X = np.array(X0, dtype=np.float64)
    done = 0
    residuals, lambdas = [], []
    while True:
        R = C - op(X)
        rn = fro(R)
        residuals.append(rn)
        if rn < tol or done >= itermax or rn == 0.0:
            break
        mj = min(m, itermax - done)
        basis, H, beta, k = arnoldi(op, R, mj)
        lam_j, y, _ = tikhonov_gcv(H, beta, variant, lam)
        lambdas.append(lam_j)
        X = X + circledast(basis[:k], y)
        done += mj
    return dict(X=X, residuals=residuals, lambdas=lambdas, steps=done,
                cycles=len(lambdas))


def gkb(op, adj, C, m):
    """Algorithm 4, m steps. Returns dict(U=[U_1..U_{m+1}], V=[V_1..V_{m+1}],
    alpha[m+1], beta[m+1] (beta[0] = beta_1), steps, breakdown)."""
    beta = [fro(C)]
    U = [C / beta[0]]
    t = adj(U[0])
    alpha = [fro(t)]
    V = [t / alpha[0]]
    steps = 0
    for j in range(m):
        Ut = op(V[j]) - alpha[j] * U[j]
        beta.append(fro(Ut))
        if beta[-1] == 0.0:
            return dict(U=U, V=V, alpha=np.array(alpha), beta=np.array(beta),
                        steps=steps, breakdown=True)
        U.append(Ut / beta[j + 1])
        Vt = adj(U[j + 1]) - beta[j + 1] * V[j]
        alpha.append(fro(Vt))
        steps = j + 1
        if alpha[-1] == 0.0:
            return dict(U=U, V=V, alpha=np.array(alpha), beta=np.array(beta),
                        steps=steps, breakdown=True)
        V.append(Vt / alpha[j + 1])
    return dict(U=U, V=V, alpha=np.array(alpha), beta=np.array(beta),
                steps=steps, breakdown=False)


def bidiagonal(alpha, beta, m):
    """C~_m of §3.2, (m+1) x m: diagonal alpha_1..alpha_m, subdiagonal
    beta_2..beta_{m+1} (alpha[0] = alpha_1, beta[0] = beta_1)."""
    Cm = np.zeros((m + 1, m))
    for j in range(m):
        Cm[j, j] = alpha[j]
        Cm[j + 1, j] = beta[j + 1]
    return Cm


def dc_gk(op, adj, C, m, variant="paper", lam=None):
    """Algorithm 5: m steps of Algorithm 4, lambda by GCV, y by (normeq2),
    X = V_m (*) y (eq. (xmlsqr)). Returns dict(X, lam, y, Cm)."""
    g = gkb(op, adj, C, m)
    k = g["steps"]
    Cm = bidiagonal(g["alpha"], g["beta"], k)
    lam_k, y, gv = tikhonov_gcv(Cm, g["beta"][0], variant, lam)
    return dict(X=circledast(g["V"][:k], y), lam=lam_k, y=y, Cm=Cm, gcv=gv,
                gkb=g)


def lsqr(op, adj, C, itermax, tol=0.0, keep_basis=False, keep_iterates=False):
    """Algorithm 6, DC-LSQR from X_0 = 0.

    Returns dict(X, phibar (|phibar_{j+1}| per iteration), alpha, beta, iters,
    V (the normalised V_1..V_iters when keep_basis), Xs (the iterates
    X_1..X_iters when keep_iterates), status)."""
    beta1 = fro(C)
    U = C / beta1
    t = adj(U)
    alpha1 = fro(t)
    V = t / alpha1
    W = V.copy()
    X = np.zeros_like(V)
    rhobar, phibar = alpha1, beta1
    alphas, betas, phis = [alpha1], [beta1], []
    basis = [V] if keep_basis else None
    iterates = [] if keep_iterates else None
    status = "maxiter"
    iters = 0
    for j in range(itermax):
        Ut = op(V) - alphas[j] * U
        b = fro(Ut)
        betas.append(b)
        if b > 0.0:
            U = Ut / b
            Vt = adj(U) - b * V
            a = fro(Vt)
        else:
            a = 0.0  # U_{j+1} undefined: finish this step with alpha_{j+1} = 0
        alphas.append(a)
        rho = np.hypot(rhobar, b)
        c = rhobar / rho
        s = b / rho
        theta = s * a
        rhobar = c * a
        phi = c * phibar
        phibar = -s * phibar
        X = X + (phi / rho) * W
        iters = j + 1
        phis.append(abs(phibar))
        if keep_iterates:
            iterates.append(X)
        if a == 0.0:  # beta_{j+1} = 0 or alpha_{j+1} = 0: X is the LS solution
            status = "breakdown"
            break
        V = Vt / a
        W = V - (theta / rho) * W
        if keep_basis:
            basis.append(V)
        if abs(phibar) < tol:
            status = "converged"
            break
    out = dict(X=X, phibar=np.array(phis), alpha=np.array(alphas),
               beta=np.array(betas), iters=iters, status=status)
    if keep_basis:
        out["V"] = basis[:iters]
    if keep_iterates:
        out["Xs"] = iterates
    return out


def lsqr_gcv(op, adj, C, itermax, variant="paper", lam=None):
    """c-LSQR followed by Tikhonov/GCV on the projected bidiagonal: itermax
    iterations of Algorithm 6 (keeping V_j and C~_k), lambda by GCV on C~_k,
    y from (normeq2), X_reg = V_k (*) y (eq. (xmlsqr)).

    Returns the LSQR result with X_reg, lam, y added."""
    r = lsqr(op, adj, C, itermax, tol=0.0, keep_basis=True)
    k = r["iters"]
    Cm = bidiagonal(r["alpha"], r["beta"], k)
    lam_k, y, gv = tikhonov_gcv(Cm, r["beta"][0], variant, lam)
    r.update(X_reg=circledast(r["V"][:k], y), lam=lam_k, y=y, Cm=Cm, gcv=gv)
    return r
