"""The dual-domain c-LSQR route of BF16 TH plans (32 < n3 <= 64) on the GPU,
through the C-ABI, against the FP64 oracle and against the spatial route of
the same plan (tc_route TC_ROUTE_SPATIAL).

Tolerances:
  * the change-of-domain pass: the BF16 output within BF16 rounding of
    in x_3 G (relative Frobenius error <= 4e-3: 2^-9 a value plus the split
    planes' 2^-16), the norm of the spatial tensor within 1e-4 (two BF16
    planes a term, FP32 accumulation);
  * the solve: regularised reconstruction error within 2% of the FP64
    oracle's (the precision form's matched-error rule) and within 0.5% of the
    spatial BF16 route's; the residual history |phibar_j| within 2% of the
    oracle's."""
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


def dev(x):
    return torch.from_numpy(f32(x)).cuda()


def rel(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("n3,P", [(64, 8192), (64, 1000), (37, 2056), (33, 8)])
def test_change_of_domain_pass(tc, n3, P):
    # P = 1000: seven full tiles of 128 pixels and a ragged tail of 104
    rng = np.random.default_rng(n3 + P)
    A = f32(rng.standard_normal((n3, 64, 64)))
    plan = tc.Plan(dev(A), s=128, precision=tc.TC_BF16, route=tc.TC_ROUTE_DUAL)
    M = cp.transform_matrix(n3)
    Mi = np.linalg.inv(M)
    X = f32(rng.standard_normal((n3, P)))
    for which, T, N in [(tc.TC_DUAL_U, Mi.T @ Mi, Mi), (tc.TC_DUAL_V, M @ M.T, M.T)]:
        Y = torch.empty((n3, P), dtype=torch.bfloat16, device="cuda")
        ss = torch.zeros(1, dtype=torch.float64, device="cuda")
        tc.tc_transform_dual(plan.handle, which, dev(X), Y, ss)
        torch.cuda.synchronize()
        ref = T @ X.astype(np.float64)
        e = rel(Y.float().cpu().numpy(), ref)
        nref = float(np.sum((N @ X.astype(np.float64)) ** 2))
        en = abs(float(ss.item()) - nref) / nref
        print(n3, P, which, e, en)
        assert e < 4e-3 and en < 1e-4
    assert tc.tc_plan_status(plan.handle) == tc.TC_OK
    plan.close()


def test_change_of_domain_pass_rejects_other_plans(tc):
    rng = np.random.default_rng(3)
    X = torch.zeros((64, 64), device="cuda")
    Y = torch.empty((64, 64), dtype=torch.bfloat16, device="cuda")
    ss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for kw in [dict(precision=tc.TC_FP32), dict(precision=tc.TC_TF32),
               dict(precision=tc.TC_BF16, product=tc.TC_ORTHODCT, route=tc.TC_ROUTE_DUAL),
               dict(precision=tc.TC_BF16, route=tc.TC_ROUTE_SPATIAL),
               dict(precision=tc.TC_BF16, route=tc.TC_ROUTE_AUTO)]:
        plan = tc.Plan(dev(rng.standard_normal((64, 64, 64))), s=64, **kw)
        with pytest.raises(tc.TcError) as e:
            tc.tc_transform_dual(plan.handle, tc.TC_DUAL_U, X, Y, ss)
        assert e.value.code == tc.TC_EUNSUPPORTED
        plan.close()
    plan = tc.Plan(dev(rng.standard_normal((16, 64, 64))), s=64, precision=tc.TC_BF16,
                   route=tc.TC_ROUTE_DUAL)
    with pytest.raises(tc.TcError):  # n3 = 16: no dual-domain route
        tc.tc_transform_dual(plan.handle, tc.TC_DUAL_U, X[:16], Y[:16], ss)
    plan.close()


@pytest.fixture(scope="module")
def video64():
    """128x128x64 video deblur: the observation and the FP64 oracle's c-LSQR
    (20 iterations) + Tikhonov/GCV."""
    w = inputs.video_deblur(n=128, frames=64, seed=11)
    A = f32(w["A"]).astype(np.float64)
    op = lambda X: cp.cprod(A, X)
    adj = lambda Y: cp.cprod_adjoint(A, Y)
    C = f32(inputs.scale_noise(op(w["X_true"]), w["G"], w["nu"])).astype(np.float64)
    ref = kr.lsqr_gcv(op, adj, C, itermax=20)
    return A, C, w["X_true"], ref


def test_dual_route_lsqr_against_oracle_and_spatial(tc, video64):
    A, C, Xt, ref = video64
    e_ref = mt.relative_error(Xt, ref["X_reg"])
    out = {}
    for route in (tc.TC_ROUTE_DUAL, tc.TC_ROUTE_SPATIAL):
        plan = tc.Plan(dev(A), s=128, precision=tc.TC_BF16, route=route)
        X, Xr, hist, info = plan.lsqr(dev(C), 20, regularize=True, history=True)
        torch.cuda.synchronize()
        inf = tc.read_info(info)
        assert inf["iters"] == 20 and inf["status"] == "maxiter", inf
        assert tc.tc_plan_status(plan.handle) == tc.TC_OK
        out[route] = (rel(Xr.cpu().numpy(), Xt), hist.cpu().numpy(), X.cpu().numpy(),
                      tc.tc_lsqr_graph_kernels(plan.handle))
        plan.close()
    e_d, h_d, X_d, k_d = out[tc.TC_ROUTE_DUAL]
    e_s, h_s, X_s, k_s = out[tc.TC_ROUTE_SPATIAL]
    print("oracle", e_ref, "dual", e_d, "spatial", e_s, "kernels", k_d, k_s)
    assert abs(e_d - e_ref) < 0.02 * e_ref
    assert abs(e_d - e_s) < 0.005 * e_s
    assert np.all(np.abs(h_d[:20] / ref["phibar"][:20] - 1) < 0.02)
    assert rel(X_d, ref["X"]) < 0.05 and rel(X_d, X_s) < 0.05
    assert k_d < k_s  # one change of domain a product instead of two transforms


@pytest.mark.parametrize("itermax", [1, 2])
def test_dual_route_short_solves(tc, video64, itermax):
    # The first steps alone (the start-up operands, the last adjoint into the
    # workspace): iterate and reconstruction against the oracle's.
    A, C, Xt, _ = video64
    op = lambda X: cp.cprod(A, X)
    adj = lambda Y: cp.cprod_adjoint(A, Y)
    ref = kr.lsqr_gcv(op, adj, C, itermax=itermax)
    plan = tc.Plan(dev(A), s=128, precision=tc.TC_BF16, route=tc.TC_ROUTE_DUAL)
    X, Xr, _, info = plan.lsqr(dev(C), itermax, regularize=True)
    torch.cuda.synchronize()
    assert tc.read_info(info)["iters"] == itermax
    assert rel(X.cpu().numpy(), ref["X"]) < 2e-2
    assert rel(Xr.cpu().numpy(), ref["X_reg"]) < 2e-2
    plan.close()


def test_dual_route_early_stop(tc, video64):
    # A tolerance met after a few steps: the remaining launches return at once
    # and the iterate is the oracle's at the same step.
    A, C, Xt, ref = video64
    tol = float(ref["phibar"][4]) * 1.0001
    op = lambda X: cp.cprod(A, X)
    adj = lambda Y: cp.cprod_adjoint(A, Y)
    r = kr.lsqr(op, adj, C, 20, tol=tol)
    plan = tc.Plan(dev(A), s=128, precision=tc.TC_BF16, route=tc.TC_ROUTE_DUAL)
    X, Xr, _, info = plan.lsqr(dev(C), 20, tol=tol, regularize=True)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    print(inf, r["iters"])
    assert inf["status"] == "converged" and abs(inf["iters"] - r["iters"]) <= 1
    assert rel(X.cpu().numpy(), r["X"]) < 3e-2
    plan.close()
