"""The cosine product (c-product) and its adjoint, in float64 (oracle).

Test infrastructure only: see the package docstring.

Paper references (arXiv 2103.11847):
  §2.1, eq. (dft1)  -- orthonormal DCT-II matrix C_n.
  §2.1, eq. (dft5)  -- C_n th(v) C_n^{-1} = Diag(C_n-transform of v); th(v) is
                       Toeplitz(v) + Hankel(v_2..v_n, 0, v_n..v_2).
  §2.2              -- mat(A): block Toeplitz-plus-Hankel unfolding; ten = its
                       inverse.
  §2.2, Remark 2.1  -- A~ = A x_3 M with M = W^{-1} C_{n3} (I + Z),
                       W = diag(C_{n3}(:, 1)), Z = ones on the superdiagonal.
  §2.2, eqs. (dft9), (dft8) -- (C (x) I) mat(A) (C^T (x) I) = blockdiag(A~_k).
  §2.2, Definition 2.1 -- A *c B = ten(mat(A) mat(B)).
  §2.2, Algorithm 1 -- the product through the transform: transform both
                       operands along mode 3, multiply frontal slices, invert.
  §2.2, Definition 2.2 -- <A, B> = sum of elementwise products, ||A||_F.
  §1, eq. (eq2)     -- the two-sided operator A *c X *c B.

Readings (where the text is ambiguous):
  * (dft1) prints "1 < i, j < n"; the matrix is n x n and orthogonal, so the
    index range is 1 <= i, j <= n.
  * Remark 2.1 calls Z "circulant" and reuses the letter W; the MATLAB command
    it prints, diag(ones(n3-1,1),1), is the nilpotent upshift. That is Z here.
  * Algorithm 1 writes dct(., [], 3); Definition 2.1, (dft8) and Remark 2.1 make
    the slice factors A x_3 M. The two disagree; Definition 2.1 is the product
    (the "TH" reading) and the transform used on both sides is M.
  * A^T *c is used by Algorithms 4 and 6 but never defined. Here it is the exact
    adjoint of X -> A *c X for <.,.> of Definition 2.2, which is
    M^T [ A~_k^T (M^{-T} Y)_k ] through the transform (and the transpose of the
    explicit operator matrix). The slice-transposed tensor is not that adjoint
    under the TH product.
"""
import numpy as np
import scipy.fft


# ----------------------------------------------------------------- §2.1 -----

def dct_matrix(n):
    """Orthonormal DCT-II matrix C_n of eq. (dft1), entries
    sqrt((2 - delta_{i1}) / n) cos((i - 1)(2j - 1) pi / (2n)), 1 <= i, j <= n."""
    C = np.empty((n, n))
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            C[i - 1, j - 1] = (np.sqrt((2.0 - (1.0 if i == 1 else 0.0)) / n)
                               * np.cos((i - 1) * (2 * j - 1) * np.pi / (2 * n)))
    return C


def th(v):
    """Toeplitz-plus-Hankel matrix th(v) of §2.1 (below eq. (dft5)).

    Toeplitz part: T_{ij} = v_{|i-j|+1}. Hankel part: H_{ij} = h_{i+j-1} with
    h = (v_2, ..., v_n, 0, v_n, ..., v_2) (1-based)."""
    v = np.asarray(v, dtype=np.float64)
    n = v.shape[0]
    T = np.empty((n, n))
    H = np.empty((n, n))
    h = np.concatenate([v[1:], [0.0], v[1:][::-1]])
    for i in range(n):
        for j in range(n):
            T[i, j] = v[abs(i - j)]
            H[i, j] = h[i + j]
    return T + H


# ----------------------------------------------------------------- §2.2 -----

def shift_matrix(n):
    """Z of Remark 2.1: ones on the first superdiagonal (diag(ones(n-1,1),1))."""
    return np.diag(np.ones(n - 1), 1)


def transform_matrix(n3):
    """M = W^{-1} C_{n3} (I + Z) of Remark 2.1, W = diag(C_{n3}(:, 1))."""
    C = dct_matrix(n3)
    W = np.diag(C[:, 0])
    return np.linalg.inv(W) @ C @ (np.eye(n3) + shift_matrix(n3))


def mode3(A, T):
    """Mode-3 product A x_3 T: slice k of the result is sum_l T[k, l] A[l]."""
    return np.einsum('kl,lij->kij', T, A)


def mat(A):
    """Block Toeplitz-plus-Hankel unfolding mat(A) of §2.2, size n1 n3 x n2 n3.

    Block (i, j) is sum_k th(e_k)[i, j] A_k, i.e. block Toeplitz in the frontal
    slices plus block Hankel built the same way as th(v)."""
    n3, n1, n2 = A.shape
    out = np.zeros((n1 * n3, n2 * n3))
    for k in range(n3):
        e = np.zeros(n3)
        e[k] = 1.0
        out += np.kron(th(e), A[k])
    return out


def ten(Mt, n1, n2, n3):
    """Inverse of mat: recover the tensor from a block Toeplitz-plus-Hankel matrix.

    The first block column of mat(A) is ((I + Z) (x) I) applied to the stacked
    slices (column 1 of th(v) is (I + Z) v), so the slices follow from one
    block-bidiagonal solve."""
    first = Mt[:, :n2].reshape(n3, n1, n2)
    return mode3(first, np.linalg.inv(np.eye(n3) + shift_matrix(n3)))


def cprod_def(A, X, B=None):
    """c-product by Definition 2.1, ten(mat(A) mat(X) [mat(B)]), on the explicit
    block Toeplitz-plus-Hankel matrices. Cost O((n n3)^3): tiny sizes only.

    A: (n3, n1, n2), X: (n3, n2, s), B: (n3, s, s) or None (eq. (eq2))."""
    n3, n1, _ = A.shape
    s = X.shape[2]
    P = mat(A) @ mat(X)
    if B is not None:
        P = P @ mat(B)
    return ten(P, n1, s, n3)


def operator_matrix(A, s, B=None):
    """Explicit matrix K of X -> A *c X [*c B] (Definition 2.1) acting on the
    stacked slices X.reshape(-1) of X with shape (n3, n2, s).

    Column q is cprod_def applied to the q-th unit tensor, so K is the
    definition itself written as a matrix. Tiny sizes only."""
    n3, n1, n2 = A.shape
    N = n3 * n2 * s
    K = np.empty((n3 * n1 * s, N))
    for q in range(N):
        E = np.zeros(N)
        E[q] = 1.0
        K[:, q] = cprod_def(A, E.reshape(n3, n2, s), B).reshape(-1)
    return K


def cprod(A, X, B=None):
    """c-product through the transform (Algorithm 1 with the mode-3 matrix M of
    Remark 2.1): X~ = X x_3 M, Y~_k = A~_k X~_k [B~_k], Y = Y~ x_3 M^{-1}.

    A: (n3, n1, n2), X: (n3, n2, s), B: (n3, s, s) or None."""
    n3 = A.shape[0]
    M = transform_matrix(n3)
    Ah = mode3(A, M)
    Xh = mode3(X, M)
    Yh = np.einsum('kij,kjl->kil', Ah, Xh)
    if B is not None:
        Yh = np.einsum('kij,kjl->kil', Yh, mode3(B, M))
    return mode3(Yh, np.linalg.inv(M))


def cprod_adjoint(A, Y, B=None):
    """Adjoint of X -> A *c X [*c B] for the inner product of Definition 2.2,
    through the transform: X = M^T [ A~_k^T (Y x_3 M^{-T})_k [B~_k^T] ].

    In vectorised form the product is (M^{-1} (x) I) blockdiag(A~_k) (M (x) I);
    its transpose is (M^T (x) I) blockdiag(A~_k^T) (M^{-T} (x) I)."""
    n3 = A.shape[0]
    M = transform_matrix(n3)
    Minv = np.linalg.inv(M)
    Ah = mode3(A, M)
    Yh = mode3(Y, Minv.T)
    Xh = np.einsum('kji,kjl->kil', Ah, Yh)
    if B is not None:
        Xh = np.einsum('kij,klj->kil', Xh, mode3(B, M))
    return mode3(Xh, M.T)


def identity_tensor(n, n3):
    """Identity tensor of §2.2 (Definition 2.2): every slice of I x_3 M is I_n.

    Formed from that definition, M^{-1} applied to tubes whose transformed
    slices are all I_n. The first column of M is the all-ones vector, so the
    result is I_n in slice 1 and zeros elsewhere (checked by the tests)."""
    Ih = np.broadcast_to(np.eye(n), (n3, n, n)).copy()
    return mode3(Ih, np.linalg.inv(transform_matrix(n3)))


def inner(A, B):
    """<A, B> of Definition 2.2: sum over all entries of a_{ijk} b_{ijk}."""
    return float(np.sum(np.asarray(A, np.float64) * np.asarray(B, np.float64)))


def fro(A):
    """||A||_F = sqrt(<A, A>) (Definition 2.2)."""
    return float(np.sqrt(inner(A, A)))


def diamond(AA, BB):
    """The diamond product of Definition 2.3: (AA^T <> BB)_{ij} = <A_i, B_j>
    for lists of equally shaped tensors."""
    return np.array([[inner(a, b) for b in BB] for a in AA])


def circledast(VV, y):
    """VV (*) y = sum_j y_j V_j (§3.1, below eq. (ev1))."""
    out = np.zeros_like(np.asarray(VV[0], np.float64))
    for v, c in zip(VV, y):
        out = out + c * np.asarray(v, np.float64)
    return out


# ----------------------------------------------- the ORTHODCT variant -----
# Algorithm 1 taken literally (reading R20): A~ = dct(A, [], 3), the
# orthonormal DCT-II of every tube (the library routine scipy.fft.dct, type 2,
# norm "ortho", stands for MATLAB's dct), then Y~_k = A~_k X~_k [B~_k] and
# Y = idct(Y~, [], 3). The transform is orthogonal, so the exact adjoint of
# X -> A *c X [*c B] applies A~_k^T (and B~_k^T) between dct and idct, which is
# the same product with the slice-transposed factors.

def dct3(A):
    """dct(A, [], 3): orthonormal DCT-II along mode 3 (axis 0 here)."""
    return scipy.fft.dct(np.asarray(A, np.float64), type=2, norm="ortho", axis=0)


def idct3(A):
    """idct(A, [], 3), the inverse of dct3."""
    return scipy.fft.idct(np.asarray(A, np.float64), type=2, norm="ortho", axis=0)


def cprod_orthodct(A, X, B=None):
    """Algorithm 1 with dct/idct: Y = idct(dct(A)_k dct(X)_k [dct(B)_k])."""
    Yh = np.einsum('kij,kjl->kil', dct3(A), dct3(X))
    if B is not None:
        Yh = np.einsum('kij,kjl->kil', Yh, dct3(B))
    return idct3(Yh)


def cprod_adjoint_orthodct(A, Y, B=None):
    """Exact adjoint of the ORTHODCT product: idct(dct(A)_k^T dct(Y)_k [dct(B)_k^T])."""
    Xh = np.einsum('kji,kjl->kil', dct3(A), dct3(Y))
    if B is not None:
        Xh = np.einsum('kij,klj->kil', Xh, dct3(B))
    return idct3(Xh)


def identity_tensor_orthodct(n, n3):
    """The tensor whose dct along mode 3 is I_n in every slice."""
    return idct3(np.broadcast_to(np.eye(n), (n3, n, n)).copy())

