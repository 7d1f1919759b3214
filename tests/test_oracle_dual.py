"""Pins for the dual-domain reading of c-LSQR under the TH product (the
transform-domain iteration that the library runs on BF16 plans with
32 < n3 <= 64), checked on the CPU in float64 against what the mathematics
fixes: the explicit operator matrix of Definition 2.1, the inner product of
Definition 2.2, and the oracle's own Algorithm 6.

The reading: with U^ = U x_3 M and V' = V x_3 M^{-T},
  * the forward product is facewise in the M domain,
      (A *c V) x_3 M = A~_k (V x_3 M)_k          (Definition 2.1, Algorithm 1);
  * the exact adjoint (the A^T *c of Algorithms 4 and 6, read as the adjoint
    for Definition 2.2's inner product) is facewise in the M^{-T} domain,
      (A^T *c U) x_3 M^{-T} = A~_k^T (U x_3 M^{-T})_k;
  * the change of domain between them is G = M^{-T} M^{-1} (its inverse M M^T),
    and ||U||_F = ||U^ x_3 M^{-1}||_F, ||V||_F = ||V' x_3 M^T||_F.
So Algorithm 6 run on U^ and V' computes the same scalars and iterates."""
import numpy as np
import pytest

from oracle import cproduct as cp
from oracle import krylov as kr
from paper_2103_11847_gb300 import inputs


def facewise(Ah, X, transpose=False):
    return np.einsum('kji,kjl->kil' if transpose else 'kij,kjl->kil', Ah, X)


@pytest.mark.parametrize("n3", [2, 3, 5, 9])
def test_norm_and_inner_product_in_the_two_domains(n3):
    # <U^, U'> = <U, U> elementwise (Definition 2.2), U' = U^ x_3 G, and the
    # norm of the spatial tensor from either representation.
    rng = np.random.default_rng(n3)
    U = rng.standard_normal((n3, 4, 3))
    M = cp.transform_matrix(n3)
    Mi = np.linalg.inv(M)
    Uh, Ud = cp.mode3(U, M), cp.mode3(U, Mi.T)
    G = Mi.T @ Mi
    assert np.isclose(np.sum(Uh * Ud), cp.inner(U, U), rtol=1e-12)
    assert np.allclose(cp.mode3(Uh, G), Ud, atol=1e-12 * np.abs(Ud).max())
    assert np.allclose(cp.mode3(Ud, M @ M.T), Uh, atol=1e-11 * np.abs(Uh).max())
    assert np.isclose(cp.fro(cp.mode3(Uh, Mi)), cp.fro(U), rtol=1e-12)
    assert np.isclose(cp.fro(cp.mode3(Ud, M.T)), cp.fro(U), rtol=1e-12)
    # G is not the identity under TH: the plain transform-domain norm differs
    assert abs(cp.fro(Uh) - cp.fro(U)) > 1e-3 * cp.fro(U)


@pytest.mark.parametrize("n3,n1,n2,s", [(3, 3, 2, 2), (4, 2, 3, 2)])
def test_products_facewise_in_their_domains(n3, n1, n2, s):
    # Against the explicit operator matrix K of Definition 2.1 (mat/ten) and
    # its transpose, the adjoint for Definition 2.2's inner product.
    rng = np.random.default_rng(100 + n3)
    A = rng.standard_normal((n3, n1, n2))
    X = rng.standard_normal((n3, n2, s))
    Y = rng.standard_normal((n3, n1, s))
    K = cp.operator_matrix(A, s)
    M = cp.transform_matrix(n3)
    Mit = np.linalg.inv(M).T
    Ah = cp.mode3(A, M)
    fwd = (K @ X.reshape(-1)).reshape(n3, n1, s)
    adj = (K.T @ Y.reshape(-1)).reshape(n3, n2, s)
    assert np.allclose(cp.mode3(fwd, M), facewise(Ah, cp.mode3(X, M)), atol=1e-10)
    assert np.allclose(cp.mode3(adj, Mit), facewise(Ah, cp.mode3(Y, Mit), transpose=True),
                       atol=1e-10)
    # the slice transpose in the M domain is not that adjoint under TH
    wrong = cp.mode3(facewise(Ah, cp.mode3(Y, M), transpose=True), np.linalg.inv(M))
    assert not np.allclose(wrong, adj, atol=1e-6)


def dual_lsqr_gcv(A, C, iters):
    """Algorithm 6 (with the Tikhonov/GCV projection) run on U^ = U x_3 M and
    V' = V x_3 M^{-T}, in the order the library's dual-domain route takes the
    steps: each forward product is the M-domain GEMM plus the change of domain
    by G, each adjoint the M^{-T}-domain GEMM plus G^{-1}; norms from the
    spatial tensors; X = X' x_3 M^T once at the end."""
    n3 = A.shape[0]
    M = cp.transform_matrix(n3)
    Mi = np.linalg.inv(M)
    G, Gi = Mi.T @ Mi, M @ M.T
    Ah = cp.mode3(A, M)
    beta = [cp.fro(C)]
    Uh = cp.mode3(C, M) / beta[0]
    Ud = cp.mode3(C, Mi.T) / beta[0]
    Vd = facewise(Ah, Ud, transpose=True)
    Vh = cp.mode3(Vd, Gi)
    alpha = [np.sqrt(np.sum(Vd * Vh))]
    Vd, Vh = Vd / alpha[0], Vh / alpha[0]
    basis = [Vd]
    for j in range(iters):
        Uh = facewise(Ah, Vh) - alpha[j] * Uh
        Ud = cp.mode3(Uh, G)
        beta.append(cp.fro(cp.mode3(Uh, Mi)))
        Uh, Ud = Uh / beta[-1], Ud / beta[-1]
        Vd = facewise(Ah, Ud, transpose=True) - beta[-1] * Vd
        Vh = cp.mode3(Vd, Gi)
        alpha.append(cp.fro(cp.mode3(Vd, M.T)))
        Vd, Vh = Vd / alpha[-1], Vh / alpha[-1]
        basis.append(Vd)
    Cm = kr.bidiagonal(np.array(alpha), np.array(beta), iters)
    from oracle.regularize import tikhonov_gcv
    lam, y, _ = tikhonov_gcv(Cm, beta[0])
    Xd = cp.circledast(basis[:iters], y)
    return np.array(alpha), np.array(beta), cp.mode3(Xd, M.T), lam


@pytest.mark.parametrize("frames", [9, 33])
def test_dual_route_reproduces_algorithm_6(frames):
    # Video deblur (per-frame Gaussian blurs), 24 x 24 frames: the dual-domain
    # iteration gives the oracle's alpha_j, beta_j, lambda and X_reg. (On
    # 12 x 12 frames the blur's spectrum is exhausted within 8 steps and both
    # FP64 recurrences run on rounding error from step 7 on.)
    w = inputs.video_deblur(n=24, frames=frames, seed=5)
    A = w["A"]
    op = lambda X: cp.cprod(A, X)
    adj = lambda Y: cp.cprod_adjoint(A, Y)
    C = inputs.scale_noise(op(w["X_true"]), w["G"], w["nu"])
    ref = kr.lsqr_gcv(op, adj, C, itermax=8)
    alpha, beta, Xr, lam = dual_lsqr_gcv(A, C, 8)
    assert np.allclose(alpha[:9], ref["alpha"][:9], rtol=1e-9)
    assert np.allclose(beta[:9], ref["beta"][:9], rtol=1e-9)
    assert np.isclose(lam, ref["lam"], rtol=1e-7)
    assert np.linalg.norm(Xr - ref["X_reg"]) < 1e-8 * np.linalg.norm(ref["X_reg"])


def test_dual_route_with_swapped_domains_fails():
    # A planted mistake: G and G^{-1} exchanged. The recurrence then runs on
    # another operator and leaves the oracle's scalars at the first step.
    w = inputs.video_deblur(n=10, frames=5, seed=6)
    A = w["A"]
    n3 = A.shape[0]
    M = cp.transform_matrix(n3)
    Mi = np.linalg.inv(M)
    Ah = cp.mode3(A, M)
    C = inputs.scale_noise(cp.cprod(A, w["X_true"]), w["G"], w["nu"])
    ref = kr.lsqr(lambda X: cp.cprod(A, X), lambda Y: cp.cprod_adjoint(A, Y), C, 2)
    b1 = cp.fro(C)
    Ud = cp.mode3(C, Mi.T) / b1
    Vd = facewise(Ah, Ud, transpose=True)
    Vh_wrong = cp.mode3(Vd, Mi.T @ Mi)
    a1_wrong = np.sqrt(np.sum(Vd * Vh_wrong))
    assert abs(a1_wrong - ref["alpha"][0]) > 1e-3 * ref["alpha"][0]
