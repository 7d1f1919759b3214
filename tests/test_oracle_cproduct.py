"""Pins for the FP64 oracle's c-product (oracle/cproduct.py) against what the
paper and the mathematics fix, independent of the oracle's own formulas."""
import numpy as np
import pytest
import scipy.fft

from oracle import cproduct as cp
from paper_2103_11847_gb300 import inputs
from tests.conftest import load_golden


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16])
def test_dct_orthogonal_and_matches_library(n):
    # eq. (dft1): C_n orthogonal; C_n v is SciPy's orthonormal DCT-II.
    C = cp.dct_matrix(n)
    assert np.allclose(C @ C.T, np.eye(n), atol=1e-14)
    v = np.random.default_rng(n).standard_normal(n)
    assert np.allclose(C @ v, scipy.fft.dct(v, type=2, norm="ortho"), atol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 4, 7, 12])
def test_th_diagonalised_by_dct(n):
    # eq. (dft5): C th(v) C^T is diagonal; Remark 2.1: the diagonal is M v.
    v = np.random.default_rng(10 + n).standard_normal(n)
    C = cp.dct_matrix(n)
    D = C @ cp.th(v) @ C.T
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-13
    assert np.allclose(np.diag(D), cp.transform_matrix(n) @ v, atol=1e-12)


def test_transform_matrix_golden_n3_3():
    # Hand-derived M for n3 = 3 (tests/golden/transform_n3_3.txt).
    M = load_golden("transform_n3_3.txt")
    assert np.allclose(cp.transform_matrix(3), M, atol=1e-14)
    assert np.allclose(cp.transform_matrix(3) @ [1, 0.7, 0.4], [3.2, 1.3, -0.1], atol=1e-14)


@pytest.mark.parametrize("n3", [1, 2, 3, 4, 9, 64])
def test_first_column_of_M_is_ones(n3):
    # Identity tensor (§2.2): M e_1 = 1 makes the spatial identity I in slice 1.
    M = cp.transform_matrix(n3)
    assert np.allclose(M[:, 0], 1.0, atol=1e-12)
    I = cp.identity_tensor(4, n3)
    expect = np.zeros((n3, 4, 4))
    expect[0] = np.eye(4)
    assert np.allclose(I, expect, atol=1e-12)


def test_tube_product_golden_n3_2():
    # Definition 2.1 worked by hand for 1x1x2 tubes (tests/golden/tube_product_n3_2.txt).
    for a1, a2, x1, x2, y1, y2 in load_golden("tube_product_n3_2.txt"):
        a = np.array([a1, a2]).reshape(2, 1, 1)
        x = np.array([x1, x2]).reshape(2, 1, 1)
        assert np.allclose(cp.cprod_def(a, x).ravel(), [y1, y2], atol=1e-12)
        assert np.allclose(cp.cprod(a, x).ravel(), [y1, y2], atol=1e-12)


@pytest.mark.parametrize("n1,n2,n3", [(2, 3, 1), (3, 2, 2), (4, 3, 3), (2, 2, 5)])
def test_ten_inverts_mat(n1, n2, n3):
    A = np.random.default_rng(n1 * 100 + n2 * 10 + n3).standard_normal((n3, n1, n2))
    assert np.allclose(cp.ten(cp.mat(A), n1, n2, n3), A, atol=1e-13)


@pytest.mark.parametrize("n1,n2,n3", [(3, 2, 2), (2, 4, 3), (3, 3, 4)])
def test_block_diagonalisation(n1, n2, n3):
    # eq. (dft8): (C (x) I) mat(A) (C^T (x) I) = blockdiag(A x_3 M).
    A = np.random.default_rng(7).standard_normal((n3, n1, n2))
    C = cp.dct_matrix(n3)
    L = np.kron(C, np.eye(n1))
    R = np.kron(C.T, np.eye(n2))
    D = L @ cp.mat(A) @ R
    Ah = cp.mode3(A, cp.transform_matrix(n3))
    expect = np.zeros_like(D)
    for k in range(n3):
        expect[k * n1:(k + 1) * n1, k * n2:(k + 1) * n2] = Ah[k]
    assert np.abs(D - expect).max() < 1e-12


@pytest.mark.parametrize("n1,n2,s,n3,two", [(3, 2, 2, 3, False), (2, 3, 4, 4, False),
                                            (3, 3, 2, 3, True), (2, 2, 3, 5, True),
                                            (4, 4, 1, 1, False)])
def test_transform_route_equals_definition(n1, n2, s, n3, two):
    # Algorithm 1 with M (Remark 2.1) == Definition 2.1 on explicit T+H matrices.
    p = inputs.random_problem(n1, n2, s, n3, two_sided=two, seed=3)
    ref = cp.cprod_def(p["A"], p["X"], p["B"])
    got = cp.cprod(p["A"], p["X"], p["B"])
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n1,n2,s,n3,two", [(3, 2, 2, 3, False), (2, 3, 2, 4, True),
                                            (3, 3, 3, 2, True)])
def test_adjoint_is_transpose_of_operator_matrix(n1, n2, s, n3, two):
    # The adjoint (A^T *c of Algorithms 4, 6) is K^T for the explicit operator K.
    p = inputs.random_problem(n1, n2, s, n3, two_sided=two, seed=4)
    K = cp.operator_matrix(p["A"], s, p["B"])
    got = cp.cprod_adjoint(p["A"], p["Y"], p["B"]).reshape(-1)
    assert np.allclose(got, K.T @ p["Y"].reshape(-1), atol=1e-11)


@pytest.mark.parametrize("two", [False, True])
def test_adjoint_identity_larger(two):
    # <A *c X, Y> = <X, A^T *c Y> at sizes beyond the explicit matrices.
    p = inputs.random_problem(17, 13, 11, 6, two_sided=two, seed=5)
    if two:
        p = inputs.random_problem(17, 13, 13, 6, two_sided=True, seed=5)
    lhs = cp.inner(cp.cprod(p["A"], p["X"], p["B"]), p["Y"])
    rhs = cp.inner(p["X"], cp.cprod_adjoint(p["A"], p["Y"], p["B"]))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_slice_transpose_is_not_the_adjoint():
    # Under Definition 2.1 the slice-transposed tensor is not the adjoint (n3 > 1).
    p = inputs.random_problem(3, 3, 2, 3, seed=6)
    At = np.transpose(p["A"], (0, 2, 1))
    lhs = cp.inner(cp.cprod(p["A"], p["X"]), p["Y"])
    rhs_slice_t = cp.inner(p["X"], cp.cprod(At, p["Y"]))
    assert abs(lhs - rhs_slice_t) > 1e-3 * abs(lhs)


def test_identity_and_associativity():
    rng = np.random.default_rng(8)
    n3 = 3
    A = rng.standard_normal((n3, 3, 3))
    Bt = rng.standard_normal((n3, 3, 3))
    X = rng.standard_normal((n3, 3, 2))
    I = cp.identity_tensor(3, n3)
    assert np.allclose(cp.cprod_def(I, X), X, atol=1e-13)
    lhs = cp.cprod_def(cp.cprod_def(A, Bt), X)
    rhs = cp.cprod_def(A, cp.cprod_def(Bt, X))
    assert np.allclose(lhs, rhs, atol=1e-11)


def test_right_factor_with_tube_e1_is_plain_right_multiplication():
    # §4, eq. (tensor_form): B with slices (A1^T, 0, 0) acts on every channel as
    # right multiplication by A1^T (its tube is e_1 and M e_1 = 1).
    rng = np.random.default_rng(9)
    A1 = rng.standard_normal((4, 4))
    B = np.zeros((3, 4, 4))
    B[0] = A1.T
    X = rng.standard_normal((3, 4, 4))
    I = cp.identity_tensor(4, 3)
    got = cp.cprod_def(I, X, B)
    assert np.allclose(got, X @ A1.T, atol=1e-12)


def test_inner_product_and_diamond():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((3, 4, 5))
    B = rng.standard_normal((3, 4, 5))
    assert np.isclose(cp.inner(A, B), float(A.ravel() @ B.ravel()), rtol=1e-14)
    assert np.isclose(cp.fro(A), np.linalg.norm(A.ravel()), rtol=1e-14)
    D = cp.diamond([A, B], [A, B, A + B])
    assert D.shape == (2, 3)
    assert np.isclose(D[1, 2], cp.inner(B, A) + cp.inner(B, B), rtol=1e-13)
    y = np.array([2.0, -1.0])
    assert np.allclose(cp.circledast([A, B], y), 2 * A - B)
