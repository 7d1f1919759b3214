"""GPU parity of the ORTHODCT product (tc_opts.product = TC_ORTHODCT,
Algorithm 1 as printed, reading R20) against the FP64 oracle
(oracle/cproduct.py: cprod_orthodct, cprod_adjoint_orthodct).

The plan swaps the transform pair (M, M^{-1}) for (C_{n3}, C_{n3}^T); every
route (fused n3 <= 4, one-launch two-sided, two-launch two-sided, transform
passes for n3 > 4, tcgen05 BF16) is exercised. Tolerances as for the TH
product: 1e-5 relative for FP32 products, 3e-2 for BF16 slice GEMMs; LSQR
iterates to 1e-3 at 15 steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp
from oracle import krylov as kr
from paper_2103_11847_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11847_gb300 import tcprod
    tcprod.lib()
    return tcprod


def f32(x):
    return np.ascontiguousarray(np.asarray(x, np.float32))


def dev(x):
    return torch.from_numpy(f32(x)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(np.asarray(a, np.float64) - b)) / np.linalg.norm(np.ravel(b)))


SHAPES = [  # n1, n2, s, n3, two_sided
    (64, 64, 64, 3, False), (37, 45, 23, 4, False), (30, 30, 30, 9, False), (64, 48, 40, 2, True),
    (45, 61, 255, 4, True), (64, 48, 257, 3, True), (29, 35, 31, 6, True), (1, 1, 1, 1, False),
]


@pytest.mark.parametrize("n1,n2,s,n3,two", SHAPES)
def test_orthodct_product_and_adjoint(tc, n1, n2, s, n3, two):
    p = inputs.random_problem(n1, n2, s, n3, two_sided=two, seed=n1 + 3 * n3)
    A, X, Y = f32(p["A"]), f32(p["X"]), f32(p["Y"])
    B = f32(p["B"]) if two else None
    plan = tc.Plan(dev(A), dev(B) if two else None, s=s, product=tc.TC_ORTHODCT)
    Bd = B.astype(np.float64) if two else None
    Yg = plan.cprod(dev(X)).cpu().numpy()
    Xg = plan.adjoint(dev(Y)).cpu().numpy()
    assert rel(Yg, cp.cprod_orthodct(A.astype(np.float64), X.astype(np.float64), Bd)) < 1e-5
    assert rel(Xg, cp.cprod_adjoint_orthodct(A.astype(np.float64), Y.astype(np.float64), Bd)) < 1e-5
    plan.close()


def test_orthodct_slice_transpose_is_the_adjoint(tc):
    # under ORTHODCT the plan of the slice-transposed tensor applies the adjoint
    p = inputs.random_problem(40, 56, 24, 5, seed=11)
    A, Y = f32(p["A"]), f32(p["Y"])
    At = np.ascontiguousarray(np.transpose(A, (0, 2, 1)))
    pa = tc.Plan(dev(A), s=24, product=tc.TC_ORTHODCT)
    pt = tc.Plan(dev(At), s=24, product=tc.TC_ORTHODCT)
    a1 = pa.adjoint(dev(Y)).cpu().numpy()
    a2 = pt.cprod(dev(Y)).cpu().numpy()
    assert rel(a1, a2.astype(np.float64)) < 1e-5
    pa.close()
    pt.close()


def test_orthodct_bf16_form(tc):
    p = inputs.random_problem(64, 64, 64, 8, seed=12)
    A, X = f32(p["A"]), f32(p["X"])
    plan = tc.Plan(dev(A), s=64, precision=tc.TC_BF16, product=tc.TC_ORTHODCT)
    Yg = plan.cprod(dev(X)).cpu().numpy()
    assert rel(Yg, cp.cprod_orthodct(A.astype(np.float64), X.astype(np.float64))) < 3e-2
    plan.close()


@pytest.mark.parametrize("two", [False, True])
def test_orthodct_lsqr_matches_oracle(tc, two):
    w = inputs.two_sided_deblur(n=48, seed=2) if two else inputs.colour_deblur(n=64, seed=2)
    A = f32(w["A"]).astype(np.float64)
    B = f32(w["B"]).astype(np.float64) if two else None
    op = lambda X: cp.cprod_orthodct(A, X, B)
    adj = lambda Y: cp.cprod_adjoint_orthodct(A, Y, B)
    C = f32(inputs.scale_noise(op(w["X_true"]), w["G"], 1e-2)).astype(np.float64)
    ref = kr.lsqr(op, adj, C, itermax=15)
    plan = tc.Plan(dev(A), dev(B) if two else None, s=C.shape[2], product=tc.TC_ORTHODCT)
    X, _, _, info = plan.lsqr(dev(C), 15)
    torch.cuda.synchronize()
    assert tc.read_info(info)["iters"] == ref["iters"]
    assert rel(X.cpu().numpy(), ref["X"]) < 1e-3
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16", "bf16x3"])
def test_transform_domain_lsqr(tc, precision):
    # ORTHODCT plans off the fused route (n3 > 4, or a tensor-core form)
    # iterate on dct(C) with slice GEMMs only and transform X, X_reg back at
    # the end (reading R21). FP32: the iterate to 1e-3 of the oracle's at 15
    # steps; every form: the regularised reconstruction error within 1% (FP32)
    # or 2% (TF32/BF16) of the oracle's.
    w = inputs.video_deblur(n=64, frames=9, seed=4)
    A = f32(w["A"]).astype(np.float64)
    op = lambda X: cp.cprod_orthodct(A, X)
    adj = lambda Y: cp.cprod_adjoint_orthodct(A, Y)
    Xt = w["X_true"]
    C = f32(inputs.scale_noise(op(Xt), w["G"], 1e-2)).astype(np.float64)
    ref = kr.lsqr_gcv(op, adj, C, itermax=15)
    prec = {"fp32": tc.TC_FP32, "tf32": tc.TC_TF32, "bf16": tc.TC_BF16,
            "bf16x3": tc.TC_BF16X3}[precision]
    plan = tc.Plan(dev(A), s=64, precision=prec, product=tc.TC_ORTHODCT)
    for _ in range(2):  # the second call replays the captured graph
        X, Xr, _, info = plan.lsqr(dev(C), 15, regularize=True)
        torch.cuda.synchronize()
        assert tc.read_info(info)["iters"] == 15
        e_ref = rel(ref["X_reg"], Xt)
        e_gpu = rel(Xr.cpu().numpy(), Xt)
        if precision in ("fp32", "bf16x3"):  # bf16x3: FP32-accurate products
            assert rel(X.cpu().numpy(), ref["X"]) < 1e-3
            assert abs(e_gpu - e_ref) <= 0.01 * e_ref
        else:
            assert abs(e_gpu - e_ref) <= 0.02 * e_ref
    plan.close()


def test_transform_domain_lcurve(tc):
    from oracle import lcurve as lc
    w = inputs.video_deblur(n=48, frames=6, seed=5)
    A = f32(w["A"]).astype(np.float64)
    op = lambda X: cp.cprod_orthodct(A, X)
    adj = lambda Y: cp.cprod_adjoint_orthodct(A, Y)
    C = f32(inputs.scale_noise(op(w["X_true"]), w["G"], 1e-2)).astype(np.float64)
    ref = lc.lsqr_lcurve(op, adj, C, 12)
    plan = tc.Plan(dev(A), s=48, product=tc.TC_ORTHODCT)
    X, Xo, curve, info = plan.lsqr_lcurve(dev(C), 12)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    cv = curve.cpu().numpy()
    assert np.max(np.abs(cv[:12] - ref["resnorm"]) / ref["resnorm"]) < 1e-4
    assert np.max(np.abs(cv[12:] - ref["solnorm"]) / ref["solnorm"]) < 1e-4
    k = inf["kopt"]
    kap = ref["curvature"]
    assert k == ref["kopt"] or kap[k - 1] >= np.nanmax(kap) * (1 - 1e-3)
    assert rel(Xo.cpu().numpy(), ref["Xs"][k - 1]) < 1e-3
    plan.close()
