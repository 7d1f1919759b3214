"""Pins for the oracle's Krylov methods and regularisation (oracle/krylov.py,
oracle/regularize.py, oracle/metrics.py): Propositions 3.1 and 3.2, LSQR's
residual identity, dense least squares on the explicit operator matrix, exact
solves, GCV by brute force, Tikhonov by stacked least squares."""
import numpy as np
import pytest

from oracle import cproduct as cp
from oracle import krylov as kr
from oracle import regularize as rg
from oracle import metrics as mt
from paper_2103_11847_gb300 import inputs


def ops(A, B=None):
    return (lambda X: cp.cprod(A, X, B)), (lambda Y: cp.cprod_adjoint(A, Y, B))


def well_conditioned(n, n3, s, seed, two=False):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n3, n, n)) * 0.2
    A[0] += np.eye(n) * 2.0  # slice 1 carries the identity (M e_1 = 1)
    B = None
    if two:
        B = rng.standard_normal((n3, s, s)) * 0.2
        B[0] += np.eye(s) * 2.0
    C = rng.standard_normal((n3, n, s))
    return A, B, C


@pytest.mark.parametrize("two", [False, True])
def test_gkb_relations(two):
    # Proposition 3.2: A V_m = U_{m+1} (*) C~_m, A^T U_m = V_m (*) C_m^T,
    # U_{m+1} (*) (beta_1 e_1) = C, orthonormal bases.
    A, B, C = well_conditioned(5, 3, 4 if not two else 5, 1, two)
    op, adj = ops(A, B)
    m = 6
    g = kr.gkb(op, adj, C, m)
    U, V = g["U"], g["V"]
    Cm = kr.bidiagonal(g["alpha"], g["beta"], m)
    for j in range(m):
        assert np.allclose(op(V[j]), cp.circledast(U[:m + 1], Cm[:, j]), atol=1e-10)
        assert np.allclose(adj(U[j]), cp.circledast(V[:m], Cm[:m, :m].T[:, j]), atol=1e-10)
    assert np.allclose(cp.circledast(U, [g["beta"][0]] + [0.0] * m), C, atol=1e-12)
    assert np.allclose(cp.diamond(U[:m + 1], U[:m + 1]), np.eye(m + 1), atol=1e-10)
    assert np.allclose(cp.diamond(V[:m], V[:m]), np.eye(m), atol=1e-10)
    z = np.random.default_rng(2).standard_normal(m + 1)
    assert np.isclose(cp.fro(cp.circledast(U[:m + 1], z)), np.linalg.norm(z), rtol=1e-10)


def test_arnoldi_relations():
    # Proposition 3.1: A V_m = V_{m+1} (*) H~_m, V^T <> V = I, H_m = V_m^T <> A V_m.
    A, _, C = well_conditioned(5, 3, 3, 3)
    op, _ = ops(A)
    m = 7
    basis, H, beta, k = kr.arnoldi(op, C, m)
    assert k == m and np.isclose(beta, cp.fro(C))
    for j in range(m):
        assert np.allclose(op(basis[j]), cp.circledast(basis[:m + 1], H[:, j]), atol=1e-10)
    assert np.allclose(cp.diamond(basis, basis), np.eye(m + 1), atol=1e-10)
    AV = [op(v) for v in basis[:m]]
    assert np.allclose(cp.diamond(basis[:m], AV), H[:m, :], atol=1e-10)


def test_arnoldi_breakdown_on_invariant_subspace():
    # Algorithm 2 stops when h_{j+1,j} = 0. Slice 1 of A is D and the others are
    # zero, so A *c X = D X slice by slice (M e_1 = 1); C lies in a 2-dimensional
    # invariant subspace, so h_{3,2} vanishes to rounding.
    n3, n = 2, 3
    A = np.zeros((n3, n, n))
    A[0] = np.diag([1.0, 2.0, 3.0])
    C = np.zeros((n3, n, 1))
    C[0, 0, 0] = 1.0
    C[0, 1, 0] = 1.0
    basis, H, beta, k = kr.arnoldi(lambda X: cp.cprod(A, X), C, 2)
    assert abs(H[2, 1]) < 1e-14 * np.abs(H).max()
    # An exactly representable case stops at the first step: A = 2 I, n3 = 1.
    A1 = (2.0 * np.eye(n)).reshape(1, n, n)
    C1 = np.zeros((1, n, 1))
    C1[0, 0, 0] = 1.0
    basis, H, beta, k = kr.arnoldi(lambda X: cp.cprod(A1, X), C1, 5)
    assert k == 1 and H.shape == (2, 1) and H[1, 0] == 0.0 and H[0, 0] == 2.0


@pytest.mark.parametrize("two", [False, True])
def test_lsqr_residual_identity_and_dense_ls(two):
    # ||R_k||_F = |phibar_{k+1}| (§3.3), and LSQR reaches the dense least-squares
    # solution of the explicit operator matrix (Definition 2.1) after enough steps.
    n, n3, s = 4, 2, 2
    A, B, C = well_conditioned(n, n3, s, 4, two)
    op, adj = ops(A, B)
    r = kr.lsqr(op, adj, C, itermax=5)
    R = C - op(r["X"])
    assert np.isclose(cp.fro(R), r["phibar"][-1], rtol=1e-9)
    K = cp.operator_matrix(A, s, B)
    x_ls = np.linalg.lstsq(K, C.reshape(-1), rcond=None)[0]
    r = kr.lsqr(op, adj, C, itermax=K.shape[1])
    assert np.allclose(r["X"].reshape(-1), x_ls, atol=1e-8)


def test_lsqr_rectangular_overdetermined():
    # n1 > n2: a true least-squares problem; compare with numpy lstsq on K.
    rng = np.random.default_rng(5)
    n3, n1, n2, s = 2, 5, 3, 2
    A = rng.standard_normal((n3, n1, n2))
    C = rng.standard_normal((n3, n1, s))
    op, adj = ops(A)
    K = cp.operator_matrix(A, s)
    x_ls = np.linalg.lstsq(K, C.reshape(-1), rcond=None)[0]
    r = kr.lsqr(op, adj, C, itermax=3 * K.shape[1])
    assert np.allclose(r["X"].reshape(-1), x_ls, atol=1e-8)
    assert np.isclose(cp.fro(C - op(r["X"])), r["phibar"][-1], rtol=1e-6)


def test_lsqr_equals_dc_gk_at_lambda_zero():
    # DC-GK (Algorithm 5) with lambda = 0 minimises the same projected residual
    # as LSQR after the same number of steps (§3.3, eq. (sollsqr)).
    A, _, C = well_conditioned(6, 3, 3, 6)
    op, adj = ops(A)
    k = 5
    r = kr.lsqr(op, adj, C, itermax=k)
    g = kr.dc_gk(op, adj, C, k, lam=0.0)
    assert np.allclose(r["X"], g["X"], atol=1e-10)


def test_lsqr_gcv_uses_same_projection():
    A, _, C = well_conditioned(5, 3, 3, 7)
    op, adj = ops(A)
    r = kr.lsqr_gcv(op, adj, C, itermax=6, lam=0.0)
    assert np.allclose(r["X_reg"], r["X"], atol=1e-10)
    g = kr.dc_gk(op, adj, C, 6, lam=0.3)
    r2 = kr.lsqr_gcv(op, adj, C, itermax=6, lam=0.3)
    assert np.allclose(r2["X_reg"], g["X"], atol=1e-10)


def test_lsqr_breakdown_on_exact_solution():
    # C in the range after one step: beta_2 = 0 breaks the recurrence.
    n3, n = 1, 3
    A = np.eye(n).reshape(1, n, n) * 2.0
    C = np.ones((n3, n, 1))
    r = kr.lsqr(*ops(A), C, itermax=5)
    assert r["status"] == "breakdown"
    assert np.allclose(r["X"], C / 2.0, atol=1e-14)


def test_gmres_exact_on_small_invertible():
    # Algorithm 3 with m >= dimension and lambda = 0 solves the system exactly.
    n, n3, s = 3, 2, 1
    A, _, C = well_conditioned(n, n3, s, 8)
    op, _ = ops(A)
    K = cp.operator_matrix(A, s)
    x = np.linalg.solve(K, C.reshape(-1))
    r = kr.gmres(op, C, np.zeros_like(C), m=n * n3 * s, itermax=n * n3 * s, lam=0.0)
    assert np.allclose(r["X"].reshape(-1), x, atol=1e-9)


def test_gmres_restart_recomputes_residual():
    # Restarted cycles keep reducing the true residual ||C - A X|| (lambda = 0).
    A, _, C = well_conditioned(6, 3, 2, 9)
    op, _ = ops(A)
    r = kr.gmres(op, C, np.zeros_like(C), m=3, itermax=12, lam=0.0)
    res = r["residuals"]
    assert r["cycles"] == 4 and len(res) == 5
    assert all(res[i + 1] < res[i] for i in range(len(res) - 1))
    assert np.isclose(res[-1], cp.fro(C - op(r["X"])), rtol=1e-12)


def brute_gcv(H, beta, lam, variant):
    """GCV from the influence matrix, with no SVD (basis-independent)."""
    m = H.shape[1]
    b = np.zeros(H.shape[0])
    b[0] = beta
    infl = H @ np.linalg.solve(H.T @ H + lam ** 2 * np.eye(m), H.T)
    R = np.eye(H.shape[0]) - infl
    if variant == "full":
        return float(np.sum((R @ b) ** 2) / np.trace(R) ** 2)
    Q, _ = np.linalg.qr(H)  # orthonormal basis of range(H)
    return float(np.sum((Q.T @ R @ b) ** 2) / np.trace(Q.T @ R @ Q) ** 2)


@pytest.mark.parametrize("variant", ["paper", "full"])
def test_gcv_value_matches_influence_matrix(variant):
    rng = np.random.default_rng(12)
    H = kr.bidiagonal(np.abs(rng.standard_normal(7)) + 0.1, np.abs(rng.standard_normal(7)), 6)
    sig, g = rg.svd_projected(H, 2.5)
    for lam in [1e-3, 0.07, 0.5, 3.0]:
        assert np.isclose(rg.gcv_value(sig, g, lam, variant), brute_gcv(H, 2.5, lam, variant),
                          rtol=1e-9)


@pytest.mark.parametrize("variant", ["paper", "full"])
def test_gcv_minimiser_beats_dense_grid(variant):
    # The chosen lambda is no worse than a 20000-point brute-force grid.
    rng = np.random.default_rng(13)
    sv = np.logspace(0, -4, 9)
    H = np.zeros((10, 9))
    Q1, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    Q2, _ = np.linalg.qr(rng.standard_normal((9, 9)))
    H = Q1[:, :9] @ np.diag(sv) @ Q2.T
    beta = 1.7
    lam, gv = rg.gcv_minimize(H, beta, variant)
    grid = np.logspace(-9, 1, 20000)
    # the influence-matrix form loses accuracy for lambda << sigma_min (a trace
    # of near-cancelling terms), so it is only swept where it is well conditioned
    best = min(brute_gcv(H, beta, t, variant) for t in np.logspace(-6, 1, 400))
    sig, g = rg.svd_projected(H, beta)
    dense = min(rg.gcv_value(sig, g, t, variant) for t in grid)
    assert gv <= dense * (1 + 1e-6)
    assert gv <= best * (1 + 1e-6)
    assert np.isclose(gv, brute_gcv(H, beta, lam, variant), rtol=1e-8)


def test_tikhonov_matches_stacked_least_squares():
    # (tikho2)/(normeq2) normal equations == the stacked problem (min)/(leastsq0).
    rng = np.random.default_rng(14)
    H = rng.standard_normal((8, 7))
    beta, lam = 1.3, 0.21
    y = rg.tikhonov_solve(H, beta, lam)
    S = np.vstack([H, lam * np.eye(7)])
    rhs = np.zeros(15)
    rhs[0] = beta
    y_ls = np.linalg.lstsq(S, rhs, rcond=None)[0]
    assert np.allclose(y, y_ls, atol=1e-12)


def test_metrics_worked_example():
    """§4's relative error and SNR on a hand-worked 2-channel case
    (tests/golden/metrics_worked.txt): pins the global mean of reading R17,
    the squared norms and the base-10 dB scale."""
    from conftest import load_golden
    snr_ref, rel_ref = load_golden("metrics_worked.txt")[0]
    X_hat = np.array([[[0.0, 2.0]], [[10.0, 12.0]]])
    X = np.array([[[1.0, 2.0]], [[10.0, 14.0]]])
    assert abs(mt.snr_db(X_hat, X) - snr_ref) < 1e-6
    assert abs(mt.relative_error(X_hat, X) - rel_ref) < 1e-6


def test_metrics():
    X = np.random.default_rng(15).uniform(size=(3, 8, 8))
    assert mt.relative_error(X, X) == 0.0
    assert np.isclose(mt.relative_error(X, np.zeros_like(X)), 1.0)
    E = X + 0.01
    expect = 10 * np.log10(np.sum((X - X.mean()) ** 2) / (0.01 ** 2 * X.size))
    assert np.isclose(mt.snr_db(X, E), expect)


def test_deblur_workload_sanity():
    # End-to-end on the 64x64x3 colour deblur stand-in: LSQR reduces the error
    # well below that of X = 0 (relative error 1), and the residual identity
    # holds. The paper's Tables 1-4 (relative error 1.5e-2 .. 9.6e-2) are for
    # photographs that are not available; the stand-in has sharp rectangles,
    # so only a loose band is checked. Reconstruction quality is parity unpinned.
    p = inputs.colour_deblur(n=64, seed=0)
    op, adj = ops(p["A"])
    C = inputs.scale_noise(op(p["X_true"]), p["G"], p["nu"])
    r = kr.lsqr_gcv(op, adj, C, itermax=30)
    e_plain = mt.relative_error(p["X_true"], r["X"])
    e_reg = mt.relative_error(p["X_true"], r["X_reg"])
    assert e_plain < 0.3 and e_reg < 0.4
    assert np.isclose(cp.fro(C - op(r["X"])), r["phibar"][-1], rtol=1e-6)
    assert np.isclose(cp.fro(C - op(p["X_true"])) / cp.fro(op(p["X_true"])), p["nu"])
