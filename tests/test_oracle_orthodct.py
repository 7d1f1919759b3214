"""Pins of the ORTHODCT product (Algorithm 1 taken literally, reading R20;
oracle/cproduct.py) to the paper's DCT matrix and to algebra.

* dct along mode 3 (the library routine) equals the mode-3 product with the
  C_n of eq. (dft1) written out in the oracle.
* The slice-transposed tensor gives the adjoint (dot-product test), unlike
  the TH product, and the adjoint routine equals that product.
* The identity tensor is neutral; the product is associative.
* n3 = 1: both products are the plain matrix product.
"""
import numpy as np
import pytest

from oracle import cproduct as cp


def rnd(*shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("n3", [1, 2, 3, 5, 8])
def test_library_dct_is_the_papers_matrix(n3):
    A = rnd(n3, 4, 3, seed=n3)
    assert np.allclose(cp.dct3(A), cp.mode3(A, cp.dct_matrix(n3)), atol=1e-13)
    assert np.allclose(cp.idct3(cp.dct3(A)), A, atol=1e-13)


@pytest.mark.parametrize("two", [False, True])
def test_slice_transpose_is_the_adjoint(two):
    n3, n1, n2, s = 4, 5, 3, 6
    A, X, Y = rnd(n3, n1, n2, seed=1), rnd(n3, n2, s, seed=2), rnd(n3, n1, s, seed=3)
    B = rnd(n3, s, s, seed=4) if two else None
    lhs = cp.inner(cp.cprod_orthodct(A, X, B), Y)
    rhs = cp.inner(X, cp.cprod_adjoint_orthodct(A, Y, B))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    At = np.transpose(A, (0, 2, 1))
    if two:
        Bt = np.transpose(B, (0, 2, 1))
        alt = cp.cprod_orthodct(At, Y, Bt)
    else:
        alt = cp.cprod_orthodct(At, Y)
    assert np.allclose(alt, cp.cprod_adjoint_orthodct(A, Y, B), atol=1e-12)
    # under the TH product the slice transpose is not the adjoint (reading R4)
    th = cp.inner(X, cp.cprod(At, Y))
    assert abs(th - cp.inner(cp.cprod(A, X), Y)) > 1e-3


def test_identity_and_associativity():
    n3, n = 5, 4
    I = cp.identity_tensor_orthodct(n, n3)
    X = rnd(n3, n, 3, seed=5)
    assert np.allclose(cp.cprod_orthodct(I, X), X, atol=1e-13)
    A, B = rnd(n3, 3, n, seed=6), rnd(n3, n, n, seed=7)
    lhs = cp.cprod_orthodct(cp.cprod_orthodct(A, B), X)
    rhs = cp.cprod_orthodct(A, cp.cprod_orthodct(B, X))
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_single_slice_is_the_matrix_product():
    A, X, B = rnd(1, 4, 3, seed=8), rnd(1, 3, 5, seed=9), rnd(1, 5, 5, seed=10)
    ref = A[0] @ X[0] @ B[0]
    assert np.allclose(cp.cprod_orthodct(A, X, B)[0], ref, atol=1e-13)
    assert np.allclose(cp.cprod(A, X, B)[0], ref, atol=1e-13)
