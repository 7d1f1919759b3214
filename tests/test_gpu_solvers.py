"""GPU parity of the Krylov solvers (tc_lsqr_c, tc_gmres_c, tc_gkb_*,
tc_tikhonov_gcv) against the FP64 oracle on the same seeded FP32 inputs.

Tolerances: the iterate after a fixed number of iterations within 1e-3
relative (Frobenius) of the oracle's; the regularised reconstruction error
within 1% of the oracle's; lambda from GCV within 1e-3 relative (the
projected matrices themselves differ at FP32 rounding level); FP64 scalar
kernels (tc_tikhonov_gcv on a given matrix) within 1e-9."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp
from oracle import krylov as kr
from oracle import metrics as mt
from oracle import regularize as rg
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


def observe(w):
    """C = M(X_true) + N by the oracle, rounded to FP32 (the shared input)."""
    A = f32(w["A"]).astype(np.float64)
    B = f32(w["B"]).astype(np.float64) if w["B"] is not None else None
    C = inputs.scale_noise(cp.cprod(A, w["X_true"], B), w["G"], w["nu"])
    return A, B, f32(C).astype(np.float64)


def oracle_ops(A, B):
    return (lambda X: cp.cprod(A, X, B)), (lambda Y: cp.cprod_adjoint(A, Y, B))


def check_lambda(lam_gpu, ref, variant="paper", rtol=1e-3):
    """lambda parity. When GCV is flat where it is smallest (eq. (gcv2) can
    increase monotonically in lambda, leaving a plateau as lambda -> 0 whose
    values agree to rounding), every lambda on the plateau is a minimiser: then
    the oracle's GCV at the GPU's lambda must equal its minimum to 1e-9."""
    if abs(lam_gpu - ref["lam"]) <= rtol * ref["lam"]:
        return
    sig, g = rg.svd_projected(ref["Cm"], ref["beta"][0])
    g_at = rg.gcv_value(sig, g, lam_gpu, variant)
    assert abs(g_at - ref["gcv"]) <= 1e-9 * ref["gcv"], (lam_gpu, ref["lam"], g_at, ref["gcv"])


# FP32 envelope. The paper's Golub-Kahan process has no reorthogonalisation.
# On the 64x64x3 colour deblur, any FP32 execution of Algorithm 6 leaves the
# FP64 trajectory once Ritz values converge. A CPU emulation of the same
# recurrence in FP32 matches FP64 to 2.6e-7 at 15 iterations, but differs by
# 3.6e-3 at 20 and by 0.106 at 30. This holds with FP32 products and FP64
# vectors, and with FP64 products and FP32 vectors. Parity to 1e-3 is
# therefore checked at 15 iterations. At the full 30 the check is the
# envelope plus LSQR's own residual identity.
@pytest.mark.parametrize("use_graphs", [True, False])
def test_lsqr_gcv_colour_64(tc, use_graphs):
    # 64x64x3 colour deblur: 15 iterations of c-LSQR, then Tikhonov/GCV.
    w = inputs.colour_deblur(n=64, seed=0)
    A, B, C = observe(w)
    ref = kr.lsqr_gcv(*oracle_ops(A, B), C, itermax=15)
    plan = tc.Plan(dev(A), s=64, use_graphs=use_graphs)
    for _ in range(2):  # the second call replays the captured graph
        X, Xr, hist, info = plan.lsqr(dev(C), 15, regularize=True, history=True)
        torch.cuda.synchronize()
        inf = tc.read_info(info)
        assert inf["iters"] == 15 and inf["status"] == "maxiter"
        assert rel(X.cpu().numpy(), ref["X"]) < 1e-3
        assert np.allclose(hist.cpu().numpy(), ref["phibar"], rtol=1e-4)
        assert abs(inf["resid"] - ref["phibar"][-1]) < 1e-4 * ref["phibar"][-1]
        check_lambda(inf["lam"], ref)
        e_gpu = mt.relative_error(w["X_true"], Xr.cpu().numpy())
        e_ref = mt.relative_error(w["X_true"], ref["X_reg"])
        assert abs(e_gpu - e_ref) < 0.01 * e_ref
        assert rel(Xr.cpu().numpy(), ref["X_reg"]) < 1e-3
    plan.close()


def test_lsqr_gcv_full_variant_interior_minimum(tc):
    # The rectangular-problem GCV (TC_GCV_FULL) has an interior minimum on the
    # 64x64x3 deblur (lambda ~ 0.1 after 15 iterations): lambda to 1e-3.
    w = inputs.colour_deblur(n=64, seed=0)
    A, B, C = observe(w)
    ref = kr.lsqr_gcv(*oracle_ops(A, B), C, itermax=15, variant="full")
    assert 1e-3 < ref["lam"] < 10.0
    plan = tc.Plan(dev(A), s=64, gcv_variant=tc.TC_GCV_FULL)
    X, Xr, _, info = plan.lsqr(dev(C), 15, regularize=True)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert abs(inf["lam"] - ref["lam"]) < 1e-3 * ref["lam"]
    assert abs(inf["gcv"] - ref["gcv"]) < 1e-4 * ref["gcv"]
    assert rel(Xr.cpu().numpy(), ref["X_reg"]) < 1e-3
    plan.close()


@pytest.mark.parametrize("variant", ["paper", "full"])
def test_colour_64_thirty_iterations_gcv_reconstruction(tc, variant):
    # The 64x64x3 colour workload as stated: 30 c-LSQR iterations, then
    # Tikhonov/GCV on the projected bidiagonal (reading R14). FP32 loses the
    # basis's orthogonality after about 15 steps on this blur (no
    # reorthogonalisation, as in the paper), so at 30 steps the regularised
    # reconstructions differ by a few percent, in either direction: measured
    # 0.309 (GPU) vs 0.335 (oracle) with the printed GCV, whose flat minimum
    # leaves lambda to rounding, and 0.337 vs 0.331 with the full GCV. The
    # check is that the FP32 form loses no more than 2% of reconstruction
    # quality, and stays within 10% either way; the 1% parity holds at 15
    # steps (test_lsqr_gcv_colour_64).
    w = inputs.colour_deblur(n=64, seed=0)
    A, B, C = observe(w)
    ref = kr.lsqr_gcv(*oracle_ops(A, B), C, itermax=30, variant=variant)
    plan = tc.Plan(dev(A), s=64, gcv_variant=tc.TC_GCV_FULL if variant == "full" else tc.TC_GCV_PAPER)
    X, Xr, _, info = plan.lsqr(dev(C), 30, regularize=True)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["iters"] == 30
    e_gpu = mt.relative_error(w["X_true"], Xr.cpu().numpy())
    e_ref = mt.relative_error(w["X_true"], ref["X_reg"])
    print(variant, e_gpu, e_ref, inf["lam"], ref["lam"])
    assert e_gpu <= 1.02 * e_ref
    assert abs(e_gpu - e_ref) <= 0.1 * e_ref
    plan.close()


def test_lsqr_colour_64_full_length_envelope(tc):
    # 30 iterations: the FP32 envelope above (0.106 for a CPU FP32 run); the
    # GPU's residual |phibar| must equal ||C - A X|| recomputed by the oracle.
    w = inputs.colour_deblur(n=64, seed=0)
    A, B, C = observe(w)
    ref = kr.lsqr(*oracle_ops(A, B), C, itermax=30)
    plan = tc.Plan(dev(A), s=64)
    X, Xr, hist, info = plan.lsqr(dev(C), 30, regularize=True, history=True)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    Xg = X.cpu().numpy().astype(np.float64)
    assert inf["iters"] == 30
    assert rel(Xg, ref["X"]) < 0.2
    r_true = np.linalg.norm(C - cp.cprod(A, Xg, B))
    assert abs(inf["resid"] - r_true) < 2e-2 * r_true
    h = hist.cpu().numpy()
    assert np.all(np.diff(h) <= 1e-6 * h[0])  # |phibar| never increases


def test_lsqr_two_sided_256(tc):
    # Two-sided 256x256x3 deblur, 50 iterations (the benchmarked workload).
    w = inputs.two_sided_deblur(n=256, seed=1)
    A, B, C = observe(w)
    ref = kr.lsqr_gcv(*oracle_ops(A, B), C, itermax=50)
    plan = tc.Plan(dev(A), dev(B))
    X, Xr, hist, info = plan.lsqr(dev(C), 50, regularize=True, history=True)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["iters"] == 50
    assert rel(X.cpu().numpy(), ref["X"]) < 1e-3
    e_gpu = mt.relative_error(w["X_true"], Xr.cpu().numpy())
    e_ref = mt.relative_error(w["X_true"], ref["X_reg"])
    assert abs(e_gpu - e_ref) < 0.01 * e_ref
    check_lambda(inf["lam"], ref)


@pytest.mark.parametrize("n1,n2,s,n3", [(37, 29, 23, 3), (33, 33, 17, 7), (20, 20, 20, 1)])
def test_lsqr_ragged_and_unfused(tc, n1, n2, s, n3):
    rng = np.random.default_rng(n1 * n3)
    A = rng.standard_normal((n3, n1, n2)) * 0.3
    A[0, :min(n1, n2), :min(n1, n2)] += np.eye(min(n1, n2)) * 2
    C = f32(rng.standard_normal((n3, n1, s))).astype(np.float64)
    A = f32(A).astype(np.float64)
    ref = kr.lsqr(*oracle_ops(A, None), C, itermax=12)
    plan = tc.Plan(dev(A), s=s)
    X, _, _, info = plan.lsqr(dev(C), 12)
    torch.cuda.synchronize()
    assert rel(X.cpu().numpy(), ref["X"]) < 1e-4


def test_lsqr_tolerance_stop(tc):
    # Well-conditioned problem. tol is the geometric mean of two consecutive
    # oracle residuals with a wide gap, so FP32 and FP64 stop at the same step.
    rng = np.random.default_rng(4)
    n, n3, s = 24, 3, 8
    A = rng.standard_normal((n3, n, n)) * 0.01
    A[0] += np.eye(n) * 2.0
    A = f32(A).astype(np.float64)
    C = f32(rng.standard_normal((n3, n, s))).astype(np.float64)
    full = kr.lsqr(*oracle_ops(A, None), C, itermax=40)
    ph = full["phibar"]
    k = int(np.argmax(ph < 1e-4 * ph[0]))
    tol = float(np.sqrt(ph[k] * ph[k - 1]))
    ref = kr.lsqr(*oracle_ops(A, None), C, itermax=40, tol=tol)
    plan = tc.Plan(dev(A), s=s)
    X, _, _, info = plan.lsqr(dev(C), 40, tol=tol)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["status"] == "converged" and ref["status"] == "converged"
    assert inf["iters"] == ref["iters"] == k + 1
    assert rel(X.cpu().numpy(), ref["X"]) < 1e-4


def test_lsqr_breakdown_on_exact_solution(tc):
    # A = 2 I (n3 = 1), C = ones: beta_2 = 0 at the first step, X = C / 2.
    n = 16
    A = (2.0 * np.eye(n)).reshape(1, n, n)
    C = np.ones((1, n, 4))
    plan = tc.Plan(dev(A), s=4)
    X, _, _, info = plan.lsqr(dev(C), 5)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    ref = kr.lsqr(*oracle_ops(A, None), C, itermax=5)
    assert ref["status"] == "breakdown" and ref["iters"] == 1
    assert inf["status"] == "breakdown" and inf["iters"] == 1
    assert np.allclose(X.cpu().numpy(), 0.5, atol=1e-6)


def test_gkb_steps_match_oracle(tc):
    w = inputs.colour_deblur(n=48, seed=5)
    A, B, C = observe(w)
    m = 8
    g = kr.gkb(*oracle_ops(A, B), C, m)
    U = torch.zeros((m + 1, 3, 48, 48), device="cuda")
    V = torch.zeros((m + 1, 3, 48, 48), device="cuda")
    al = torch.zeros(m + 1, dtype=torch.float64, device="cuda")
    be = torch.zeros(m + 1, dtype=torch.float64, device="cuda")
    plan = tc.Plan(dev(A), s=48)
    tc.tc_gkb_init(plan.handle, dev(C), U, V, al, be, m)
    for j in range(1, m + 1):
        tc.tc_gkb_step(plan.handle, j, U, V, al, be, m)
    torch.cuda.synchronize()
    assert np.allclose(al.cpu().numpy(), g["alpha"], rtol=1e-4)
    assert np.allclose(be.cpu().numpy(), g["beta"], rtol=1e-4)
    Vg = V.cpu().numpy().astype(np.float64)
    Ug = U.cpu().numpy().astype(np.float64)
    a, b = al.cpu().numpy(), be.cpu().numpy()
    op, adj = oracle_ops(A, B)
    # Proposition 3.2's relations hold to FP32 rounding whatever the loss of
    # orthogonality, checked column by column with the oracle's operator on
    # the GPU's vectors: A V_j = alpha_j U_j + beta_{j+1} U_{j+1} and
    # A^T U_{j+1} = beta_{j+1} V_j + alpha_{j+1} V_{j+1}
    for j in range(m):
        AV = op(Vg[j])
        r1 = AV - a[j] * Ug[j] - b[j + 1] * Ug[j + 1]
        assert np.linalg.norm(r1) <= 1e-5 * np.linalg.norm(AV), j
        ATU = adj(Ug[j + 1])
        r2 = ATU - b[j + 1] * Vg[j] - a[j + 1] * Vg[j + 1]
        assert np.linalg.norm(r2) <= 1e-5 * np.linalg.norm(ATU), j
    # every basis tensor against the oracle's: FP32 rounding accumulates
    # step by step (measured 7.5e-8 for V_1 growing to 4.8e-6 for V_9 on a
    # GB300), bounded by 2e-6 (j + 1)
    dv = [rel(Vg[j], g["V"][j]) for j in range(m + 1)]
    print("basis differences", dv)
    for j in range(m + 1):
        assert dv[j] < 2e-6 * (j + 1), (j, dv[j])
    # orthonormality of U_1..U_9 and V_1..V_9 (Proposition 3.2) to FP32
    # rounding over these 8 steps: measured at most 1.2e-6
    for W in (Vg, Ug):
        G = np.array([[np.sum(W[i] * W[j]) for j in range(m + 1)] for i in range(m + 1)])
        dev_ = np.abs(G - np.eye(m + 1))
        print("orthogonality", [float(dev_[:k, :k].max()) for k in range(2, m + 2)])
        assert dev_[:4, :4].max() < 1e-6
        assert dev_.max() < 1e-5


def test_gmres_two_sided_256(tc):
    # DC-GMRES(10) with GCV on the two-sided 256x256x3 deblur, 50 Arnoldi steps.
    w = inputs.two_sided_deblur(n=256, seed=1)
    A, B, C = observe(w)
    op, _ = oracle_ops(A, B)
    ref = kr.gmres(op, C, np.zeros_like(C), m=10, itermax=50)
    plan = tc.Plan(dev(A), dev(B))
    X, info = plan.gmres(dev(C), 10, 50)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["iters"] == 50 and inf["cycles"] == 5
    e_gpu = mt.relative_error(w["X_true"], X.cpu().numpy())
    e_ref = mt.relative_error(w["X_true"], ref["X"])
    assert abs(e_gpu - e_ref) < 0.01 * e_ref
    assert rel(X.cpu().numpy(), ref["X"]) < 1e-3
    assert abs(inf["resid"] - ref["residuals"][-1]) < 1e-3 * ref["residuals"][-1]


def test_gmres_fixed_lambda_small(tc):
    rng = np.random.default_rng(6)
    n, n3, s = 20, 4, 6
    A = rng.standard_normal((n3, n, n)) * 0.2
    A[0] += np.eye(n) * 2
    A = f32(A).astype(np.float64)
    C = f32(rng.standard_normal((n3, n, s))).astype(np.float64)
    X0 = f32(rng.standard_normal((n3, n, s))).astype(np.float64)
    op, _ = oracle_ops(A, None)
    ref = kr.gmres(op, C, X0, m=4, itermax=10, lam=0.05)
    plan = tc.Plan(dev(A), s=s)
    X, info = plan.gmres(dev(C), 4, 10, lam=0.05, X0=dev(X0))
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["iters"] == 10 and inf["cycles"] == 3
    assert rel(X.cpu().numpy(), ref["X"]) < 1e-4


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("k", [1, 7, 30, 64])
def test_tikhonov_gcv_kernel(tc, variant, k):
    rng = np.random.default_rng(k + 10 * variant)
    alpha = np.abs(rng.standard_normal(k + 1)) + 0.05
    beta = np.abs(rng.standard_normal(k + 1)) * np.logspace(0, -3, k + 1)
    H = kr.bidiagonal(alpha, beta, k) if k % 2 == 0 else np.triu(rng.standard_normal((k + 1, k)), -1)
    b = 1.7
    name = "paper" if variant == 0 else "full"
    lam_ref, y_ref, g_ref = rg.tikhonov_gcv(H, b, name)
    dH = torch.from_numpy(np.ascontiguousarray(H)).cuda()
    db = torch.tensor([b], dtype=torch.float64, device="cuda")
    lo = torch.zeros(1, dtype=torch.float64, device="cuda")
    go = torch.zeros(1, dtype=torch.float64, device="cuda")
    y = torch.zeros(k, dtype=torch.float64, device="cuda")
    tc.tc_tikhonov_gcv(dH, k, db, variant, None, lo, y, go)
    torch.cuda.synchronize()
    assert abs(go.item() - g_ref) <= 1e-8 * abs(g_ref)
    if k == 1 and variant == 0:
        # eq. (gcv2) with one singular value is g~_1^2 for every lambda: any
        # lambda is a minimiser, so only the value is compared.
        sig, g = rg.svd_projected(H, b)
        assert abs(go.item() - g[0] ** 2) <= 1e-10 * g[0] ** 2
    else:
        assert abs(lo.item() - lam_ref) <= 1e-6 * lam_ref
        assert np.allclose(y.cpu().numpy(), y_ref, rtol=1e-6, atol=1e-9 * np.abs(y_ref).max())
    tc.tc_tikhonov_gcv(dH, k, db, variant, 0.3, lo, y, go)
    torch.cuda.synchronize()
    _, y_fix, g_fix = rg.tikhonov_gcv(H, b, name, lam=0.3)
    assert lo.item() == 0.3
    assert np.allclose(y.cpu().numpy(), y_fix, rtol=1e-9, atol=1e-12)
    assert abs(go.item() - g_fix) <= 1e-9 * abs(g_fix)
