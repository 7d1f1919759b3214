"""GPU parity of tc_lsqr_c_lcurve (DC-LSQR stopped at the L-curve corner,
§3.3, reading R18) against the FP64 oracle (oracle/lcurve.py).

The oracle takes the norms from their definitions (||C - A *c X_k||,
||X_k|| of the iterates). The GPU takes them from LSQR's rotations
(|phibar_{k+1}|, ||R_k^{-1} f_k||), equal in exact arithmetic (pinned in
tests/test_oracle_lcurve.py). Tolerances follow from FP32 Krylov vectors
over at most 15 steps, where FP32 tracks the FP64 trajectory to about 1e-6:
norms to 1e-4 relative, X_{k_opt} to 1e-3. k_opt is an argmax decided from
those values: it must be the oracle's k_opt, or a k whose oracle curvature
is within 1e-3 of the largest (a near-tie)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp
from oracle import lcurve as lc
from paper_2103_11847_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11847_gb300 import tcprod
    tcprod.lib()
    return tcprod


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32))).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(np.asarray(a, np.float64) - b)) / np.linalg.norm(np.ravel(b)))


def problem(two_sided, nu, seed):
    w = inputs.two_sided_deblur(n=48, seed=seed) if two_sided else inputs.colour_deblur(n=64, seed=seed)
    A = w["A"].astype(np.float32).astype(np.float64)
    B = w["B"].astype(np.float32).astype(np.float64) if two_sided else None
    op = lambda X: cp.cprod(A, X, B)
    adj = lambda Y: cp.cprod_adjoint(A, Y, B)
    C = inputs.scale_noise(op(w["X_true"]), w["G"], nu).astype(np.float32).astype(np.float64)
    return A, B, C, op, adj


def check_kopt(k_gpu, ref):
    if k_gpu == ref["kopt"]:
        return
    kap = ref["curvature"]
    best = np.nanmax(kap)
    assert kap[k_gpu - 1] >= best - 1e-3 * abs(best), (k_gpu, ref["kopt"], kap)


@pytest.mark.parametrize("two_sided,nu,kmax", [(False, 1e-2, 15), (True, 1e-2, 12),
                                               (False, 1e-3, 15)])
def test_lcurve_matches_oracle(tc, two_sided, nu, kmax):
    A, B, C, op, adj = problem(two_sided, nu, seed=3)
    ref = lc.lsqr_lcurve(op, adj, C, kmax)
    plan = tc.Plan(dev(A), dev(B) if two_sided else None, s=C.shape[2])
    for _ in range(2):  # the second call replays the captured graph
        X, Xo, curve, info = plan.lsqr_lcurve(dev(C), kmax)
        torch.cuda.synchronize()
        inf = tc.read_info(info)
        K = inf["iters"]
        assert K == len(ref["resnorm"]) == kmax
        cv = curve.cpu().numpy()
        assert np.max(np.abs(cv[:K] - ref["resnorm"]) / ref["resnorm"]) < 1e-4
        assert np.max(np.abs(cv[kmax:kmax + K] - ref["solnorm"]) / ref["solnorm"]) < 1e-4
        check_kopt(inf["kopt"], ref)
        k = inf["kopt"]
        assert abs(inf["resid"] - cv[k - 1]) <= 1e-12 * cv[k - 1]
        assert rel(Xo.cpu().numpy(), ref["Xs"][k - 1]) < 1e-3
        assert rel(X.cpu().numpy(), ref["Xs"][-1]) < 1e-3
    plan.close()


def test_lcurve_short_runs(tc):
    # K < 3: no interior point, k_opt = K and X_opt is the last iterate
    A, B, C, op, adj = problem(False, 1e-2, seed=4)
    plan = tc.Plan(dev(A), s=C.shape[2])
    for kmax in (1, 2):
        X, Xo, curve, info = plan.lsqr_lcurve(dev(C), kmax)
        torch.cuda.synchronize()
        inf = tc.read_info(info)
        assert inf["iters"] == kmax and inf["kopt"] == kmax
        assert rel(Xo.cpu().numpy(), X.cpu().numpy().astype(np.float64)) < 1e-5
    plan.close()


def test_lcurve_after_early_stop(tc):
    # a tolerance that stops LSQR before kmax: the curve has K < kmax points
    A, B, C, op, adj = problem(False, 1e-2, seed=5)
    full = lc.lsqr_lcurve(op, adj, C, 15)
    tol = 0.5 * (full["resnorm"][7] + full["resnorm"][8])  # between steps 8 and 9
    plan = tc.Plan(dev(A), s=C.shape[2])
    X, Xo, curve, info = plan.lsqr_lcurve(dev(C), 15, tol=tol)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["status"] == "converged" and inf["iters"] == 9
    cv = curve.cpu().numpy()
    assert np.all(np.isnan(cv[9:15])) and np.all(np.isfinite(cv[:9]))
    ref = dict(kopt=lc.corner(full["resnorm"][:9], full["solnorm"][:9]),
               curvature=lc.curvatures(full["resnorm"][:9], full["solnorm"][:9]))
    check_kopt(inf["kopt"], ref)
    plan.close()


@pytest.mark.parametrize("two_sided,nu", [(False, 1e-2), (True, 1e-1), (False, 5e-2), (False, 2e-2)])
def test_discrepancy_principle_stop(tc, two_sided, nu):
    # Reading R19: stop at the first k with ||C - M(X_k)|| <= eta ||N||, eta =
    # 1.01. tc_lsqr_c's tol on |phibar_{k+1}| is that test. The index is an
    # integer decided from FP values: it must be the oracle's, or one away
    # when the oracle's residual there is within 1e-4 of the threshold.
    A, B, C, op, adj = problem(two_sided, nu, seed=6)
    Cc = op(inputs.two_sided_deblur(n=48, seed=6)["X_true"] if two_sided
            else inputs.colour_deblur(n=64, seed=6)["X_true"])
    delta = cp.fro(C - Cc)
    tol = 1.01 * delta
    from oracle import krylov as kr
    r = kr.lsqr(op, adj, C, itermax=60, tol=tol, keep_iterates=True)
    assert r["status"] == "converged"
    kd = r["iters"]
    res = np.array([cp.fro(C - op(X)) for X in r["Xs"]])
    assert res[kd - 1] <= tol and (kd == 1 or res[kd - 2] > tol)  # the definition
    plan = tc.Plan(dev(A), dev(B) if two_sided else None, s=C.shape[2])
    X, _, _, info = plan.lsqr(dev(C), 60, tol=tol)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["status"] == "converged"
    if inf["iters"] != kd:
        near = min(abs(res[kd - 1] - tol), abs(res[kd - 2] - tol)) / tol
        assert abs(inf["iters"] - kd) == 1 and near < 1e-4, (inf["iters"], kd, near)
    plan.close()
