"""The shapes of the paper's experiments (§4, Tables 1-4) against the FP64
oracle: the two-sided colour deblur A *c X *c B with the within-channel
Gaussian of §4 (sigma = 4, half-band 6) on both sides, on seeded stand-ins
for the missing photographs (inputs.paper_deblur).

* 256 x 256 x 3, noise 1e-3: DC-LSQR with the Table 1 iteration count (14),
  DC-GK (15 steps, Tikhonov/GCV on the projected bidiagonal) and
  DC-GMRES(10) (10 Arnoldi steps, GCV), each against the oracle's run of the
  same method: the iterate within 1e-3, the reconstruction error within 1%.
* 1024 x 1024 x 3: the product and its adjoint at full size (s > 256, where
  the FP32 two-sided product runs its two stages as separate launches)
  against the oracle, within the FP32 products' 1e-5, with the largest
  elementwise error reported.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp
from oracle import krylov as kr
from oracle import metrics as mt
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


def rel(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def paper256():
    w = inputs.paper_deblur(n=256, nu=1e-3)
    A, B = f32(w["A"]).astype(np.float64), f32(w["B"]).astype(np.float64)
    op = lambda X: cp.cprod(A, X, B)
    adj = lambda Y: cp.cprod_adjoint(A, Y, B)
    C = f32(inputs.scale_noise(op(w["X_true"]), w["G"], w["nu"])).astype(np.float64)
    return w, A, B, op, adj, C


def test_paper_256_dc_lsqr_and_dc_gk(tc, paper256):
    w, A, B, op, adj, C = paper256
    plan = tc.Plan(torch.from_numpy(f32(A)).cuda(), torch.from_numpy(f32(B)).cuda())
    Cd = torch.from_numpy(f32(C)).cuda()
    # DC-LSQR, Table 1's 14 iterations
    ref = kr.lsqr(op, adj, C, itermax=14)
    X, _, _, info = plan.lsqr(Cd, 14)
    torch.cuda.synchronize()
    assert tc.read_info(info)["iters"] == 14
    assert rel(X.cpu().numpy(), ref["X"]) < 1e-3
    e = mt.relative_error(w["X_true"], X.cpu().numpy())
    e_ref = mt.relative_error(w["X_true"], ref["X"])
    assert abs(e - e_ref) <= 0.01 * e_ref
    # DC-GK, Table 1's 15 steps: Tikhonov/GCV on the projected bidiagonal
    ref = kr.lsqr_gcv(op, adj, C, itermax=15)
    X, Xr, _, info = plan.lsqr(Cd, 15, regularize=True)
    torch.cuda.synchronize()
    e = mt.relative_error(w["X_true"], Xr.cpu().numpy())
    e_ref = mt.relative_error(w["X_true"], ref["X_reg"])
    print("DC-GK", e, e_ref)
    assert abs(e - e_ref) <= 0.01 * e_ref
    plan.close()


def test_paper_256_dc_gmres(tc, paper256):
    w, A, B, op, adj, C = paper256
    plan = tc.Plan(torch.from_numpy(f32(A)).cuda(), torch.from_numpy(f32(B)).cuda())
    ref = kr.gmres(op, C, np.zeros_like(C), m=10, itermax=10)
    X, info = plan.gmres(torch.from_numpy(f32(C)).cuda(), 10, 10)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["iters"] == 10 and inf["cycles"] == 1
    assert rel(X.cpu().numpy(), ref["X"]) < 1e-3
    e = mt.relative_error(w["X_true"], X.cpu().numpy())
    e_ref = mt.relative_error(w["X_true"], ref["X"])
    print("DC-GMRES(10)", e, e_ref)
    assert abs(e - e_ref) <= 0.01 * e_ref
    plan.close()


def test_paper_1024_product_full_size(tc):
    w = inputs.paper_deblur(n=1024, nu=1e-3)
    A, B, X = f32(w["A"]), f32(w["B"]), f32(w["X_true"])
    G = f32(w["G"])
    plan = tc.Plan(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    Y = plan.cprod(torch.from_numpy(X).cuda()).cpu().numpy()
    Z = plan.adjoint(torch.from_numpy(G).cuda()).cpu().numpy()
    plan.close()
    Ad, Bd = A.astype(np.float64), B.astype(np.float64)
    Yr = cp.cprod(Ad, X.astype(np.float64), Bd)
    Zr = cp.cprod_adjoint(Ad, G.astype(np.float64), Bd)
    for got, ref in ((Y, Yr), (Z, Zr)):
        fro = rel(got, ref)
        mx = float(np.abs(got - ref).max() / np.abs(ref).max())
        print("1024x1024x3", fro, mx)
        assert fro < 1e-5 and mx < 1e-5
