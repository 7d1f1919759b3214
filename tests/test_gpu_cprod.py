"""GPU parity of tc_cprod / tc_cprod_adjoint (through the C ABI) against the
FP64 oracle on the same seeded FP32 inputs.

Tolerance: relative Frobenius error <= 1e-5 for the FP32 product (the bound
the c-product must meet in FP32). Sizes span several 32/64-wide tiles with
ragged tails, n3 in {1..5} (transform fused into the slice GEMM) and n3 > 4
(separate transform passes), one- and two-sided operators."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp
from paper_2103_11847_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11847_gb300 import tcprod
    tcprod.lib()
    return tcprod


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a, np.float64) - b).ravel()) / np.linalg.norm(b.ravel()))


def f32(x):
    return np.ascontiguousarray(np.asarray(x, np.float32))


def dev(x):
    return torch.from_numpy(f32(x)).cuda()


SHAPES = [  # n1, n2, s, n3, two_sided
    (64, 64, 64, 3, False), (97, 65, 33, 3, False), (1, 1, 1, 1, False), (40, 70, 17, 1, False),
    (33, 31, 29, 2, False), (50, 50, 50, 4, False), (37, 45, 23, 5, False), (64, 64, 48, 9, False),
    (30, 30, 30, 64, False), (70, 40, 20, 3, True), (32, 32, 32, 3, True), (29, 35, 31, 6, True),
    (130, 129, 131, 3, False), (200, 190, 70, 2, True),
    # two-sided, one launch per product: clusters of ceil(s / 32) CTAs, ragged
    # panels, odd widths (scalar loads), s = 256 (eight CTAs), and s = 257
    # (past the one-launch limit: two launches)
    (45, 61, 255, 4, True), (300, 96, 256, 1, True), (17, 250, 100, 3, True),
    (64, 48, 257, 3, True), (33, 200, 160, 2, True),
]


@pytest.mark.parametrize("n1,n2,s,n3,two", SHAPES)
def test_cprod_and_adjoint_match_oracle(tc, n1, n2, s, n3, two):
    p = inputs.random_problem(n1, n2, s, n3, two_sided=two, seed=n1 + n2 + s + n3)
    A, B, X, Y = (f32(p[k]) if p[k] is not None else None for k in ("A", "B", "X", "Y"))
    plan = tc.Plan(dev(A), dev(B) if two else None, s=s)
    Yg = plan.cprod(dev(X)).cpu().numpy()
    Xg = plan.adjoint(dev(Y)).cpu().numpy()
    Bd = B.astype(np.float64) if two else None
    assert rel(Yg, cp.cprod(A.astype(np.float64), X.astype(np.float64), Bd)) < TOL
    assert rel(Xg, cp.cprod_adjoint(A.astype(np.float64), Y.astype(np.float64), Bd)) < TOL
    plan.close()


def test_identity_tensor_and_adjoint_identity(tc):
    n, n3, s = 48, 3, 40
    I = cp.identity_tensor(n, n3)
    X = np.random.default_rng(1).standard_normal((n3, n, s))
    plan = tc.Plan(dev(I), s=s)
    assert rel(plan.cprod(dev(X)).cpu().numpy(), f32(X).astype(np.float64)) < 1e-6
    p = inputs.random_problem(60, 50, 30, 3, seed=2)
    plan = tc.Plan(dev(p["A"]), s=30)
    AX = plan.cprod(dev(p["X"])).double().cpu().numpy()
    AtY = plan.adjoint(dev(p["Y"])).double().cpu().numpy()
    lhs = float(np.sum(AX * f32(p["Y"])))
    rhs = float(np.sum(f32(p["X"]) * AtY))
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)


def test_two_sided_deblur_full_size(tc):
    # 256x256x3 two-sided Gaussian blur (the two-sided deblur workload) at full
    # size, compared entry by entry (the FP64 oracle is cheap at this size).
    w = inputs.two_sided_deblur(n=256, seed=1)
    A, B, X = f32(w["A"]), f32(w["B"]), f32(w["X_true"])
    plan = tc.Plan(dev(A), dev(B))
    Y = plan.cprod(dev(X)).cpu().numpy().astype(np.float64)
    ref = cp.cprod(A.astype(np.float64), X.astype(np.float64), B.astype(np.float64))
    assert rel(Y, ref) < TOL


