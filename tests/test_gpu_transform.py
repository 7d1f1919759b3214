"""Steps 1 and 3 of Algorithm 1 alone (tc_transform), the FP64 reciprocal
helpers of the step scalars (tc_check_recip), and the kernel count of a
captured solve (tc_lsqr_graph_kernels), through the C ABI.

tc_transform runs the pass the plan's products run. Its error against the
FP64 oracle's mode-3 product (Remark 2.1 with M, M^-1, M^-T, M^T) is stated
per route:
  FP32 pass (k_mode3):               <= 1e-6 relative (FP32 sums of n3 terms)
  tcgen05 pass, two BF16 planes:     <= 1e-4 relative (each term near 2^-16;
                                      cond(M) = 16 at n3 = 64)
  tcgen05 pass, three BF16 planes:   <= 2e-6 relative (FP32-level)
The norm it reduces is compared with the norm of its own output (the
reduction, not the transform, is under test there): 1e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11847_gb300 import tcprod
    tcprod.lib()
    return tcprod


def rel(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def transform_matrices(n3):
    M = cp.transform_matrix(n3)
    Mi = np.linalg.inv(M)
    return {0: M, 1: Mi, 2: Mi.T, 3: M.T}


@pytest.mark.parametrize("prec,n3,tol", [("fp32", 9, 1e-6), ("fp32", 64, 1e-6),
                                         ("bf16", 64, 1e-4), ("tf32", 40, 1e-4),
                                         ("bf16x3", 64, 2e-6), ("bf16x3", 33, 2e-6)])
def test_transform_matches_oracle(tc, prec, n3, tol):
    code = {"fp32": tc.TC_FP32, "tf32": tc.TC_TF32, "bf16": tc.TC_BF16, "bf16x3": tc.TC_BF16X3}[prec]
    n, s = 48, 40  # P = 1920 pixels: 15 tiles of 128
    rng = np.random.default_rng(n3)
    A = rng.standard_normal((n3, n, n)).astype(np.float32)
    plan = tc.Plan(torch.from_numpy(A).cuda(), s=s, precision=code)
    X = rng.standard_normal((n3, n, s)).astype(np.float32)
    R = rng.standard_normal((n3, n, s)).astype(np.float32)
    Xd, Rd = torch.from_numpy(X).cuda(), torch.from_numpy(R).cuda()
    for which, T in transform_matrices(n3).items():
        Y = torch.empty_like(Xd)
        tc.tc_transform(plan.handle, which, Xd, Y)
        ref = cp.mode3(X.astype(np.float64), T)
        assert rel(Y.cpu().numpy(), ref) < tol, (which, rel(Y.cpu().numpy(), ref))
        # with prev and the fused norm
        Y2 = torch.empty_like(Xd)
        ss = torch.zeros(1, dtype=torch.float64, device="cuda")
        tc.tc_transform(plan.handle, which, Xd, Y2, prev=Rd, sumsq=ss)
        y2 = Y2.cpu().numpy()
        ref2 = ref + R.astype(np.float64)
        assert rel(y2, ref2) < tol, (which, rel(y2, ref2))
        own = float(np.sum(y2.astype(np.float64) ** 2))
        assert abs(float(ss.item()) - own) <= 1e-6 * own
    assert tc.tc_plan_status(plan.handle) == tc.TC_OK
    plan.close()


def test_transform_ragged_pixels(tc):
    """P = 525 pixels a slice: neither a multiple of the 128-pixel tile nor of
    4 (the element-by-element path)."""
    n3 = 64
    rng = np.random.default_rng(5)
    A = rng.standard_normal((n3, 32, 32)).astype(np.float32)
    X = rng.standard_normal((n3, 25, 21)).astype(np.float32)
    R = rng.standard_normal((n3, 25, 21)).astype(np.float32)
    T = transform_matrices(n3)[1]
    for code, tol in ((tc.TC_FP32, 1e-6), (tc.TC_BF16, 1e-4), (tc.TC_BF16X3, 2e-6)):
        plan = tc.Plan(torch.from_numpy(A).cuda(), s=32, precision=code)
        Xd, Rd = torch.from_numpy(X).cuda(), torch.from_numpy(R).cuda()
        Y = torch.empty_like(Xd)
        tc.tc_transform(plan.handle, tc.TC_MINV, Xd, Y, prev=Rd)
        ref = cp.mode3(X.astype(np.float64), T) + R
        assert rel(Y.cpu().numpy(), ref) < tol
        assert tc.tc_plan_status(plan.handle) == tc.TC_OK
        plan.close()


def test_transform_rejects_bad_arguments(tc):
    A = torch.randn(9, 16, 16, device="cuda")
    plan = tc.Plan(A, s=16)
    X = torch.randn(9, 16, 16, device="cuda")
    with pytest.raises(tc.TcError):
        tc.tc_transform(plan.handle, 4, X, torch.empty_like(X))
    big = torch.randn(9, 16, 40, device="cuda")  # P beyond max(n1, n2) s
    with pytest.raises(tc.TcError):
        tc.tc_transform(plan.handle, 0, big, torch.empty_like(big))
    with pytest.raises(tc.TcError):
        tc.tc_transform(plan.handle, 0, X, X)
    plan.close()


def ulps(a, b):
    """Distance in units in the last place of b (FP64)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_fp64_reciprocals_against_correct_rounding(tc):
    """rcp_newton / rsqrt_newton against correctly rounded host values over a
    log sweep of 1e-307 .. 1e300, random mantissas, and the ranges outside
    Newton's (subnormals, huge values) where the IEEE operations run."""
    rng = np.random.default_rng(11)
    sweep = 10.0 ** np.linspace(-307.5, 300.0, 20001)
    mant = rng.uniform(1.0, 2.0, 20000) * 2.0 ** rng.integers(-1000, 1000, 20000)
    sub = np.array([5e-324, 1e-320, 2.2e-310, 1e-308, 2.225073858507201e-308])
    huge = np.array([1.0715086071862673e301 * 1.5, 1e305, 1e308, 1.7976931348623157e308])
    x = np.concatenate([sweep, mant, sub, huge])
    x = np.concatenate([x, -x[: x.size // 4]])  # negative arguments of the reciprocal
    xd = torch.from_numpy(x).cuda()
    r = torch.empty_like(xd)
    q = torch.empty_like(xd)
    tc.tc_check_recip(xd, r, q)
    r, q = r.cpu().numpy(), q.cpu().numpy()
    with np.errstate(over="ignore", divide="ignore"):
        ref_r = 1.0 / x  # IEEE FP64 division: correctly rounded
    ax = np.abs(x)
    newton = (ax >= 2.2250738585072014e-308) & (ax <= 1.0715086071862673e301)
    assert np.all(np.isfinite(r[np.isfinite(ref_r)]))
    assert ulps(r[newton], ref_r[newton]).max() <= 2.0
    # outside Newton's range the device divides: 1/x of a subnormal overflows
    # to Inf exactly as on the host
    out = ~newton
    assert np.array_equal(r[out], ref_r[out])
    pos = x > 0
    # 1/sqrt in extended precision, rounded once to FP64
    ref_q = (1.0 / np.sqrt(x[pos].astype(np.longdouble))).astype(np.float64)
    qn = newton[pos]
    assert ulps(q[pos][qn], ref_q[qn]).max() <= 2.0
    # IEEE path: sqrt and division each rounded (half an ulp each, plus the
    # first rounding carried through the division)
    assert ulps(q[pos][~qn], ref_q[~qn]).max() <= 2.0
    assert np.all(q[~pos] == 0.0)


def test_graph_kernel_count_grows_by_a_fixed_count_per_iteration(tc):
    """Each replay of a captured solve launches every kernel node; the count
    grows linearly with the iteration count (a fixed set per iteration)."""
    n = 64
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, n, n)).astype(np.float32)
    C = rng.standard_normal((3, n, n)).astype(np.float32)
    plan = tc.Plan(torch.from_numpy(A).cuda(), s=n)
    Cd = torch.from_numpy(C).cuda()
    counts = []
    for it in (5, 10, 15):
        plan.lsqr(Cd, itermax=it, regularize=True)
        torch.cuda.synchronize()
        counts.append(tc.tc_lsqr_graph_kernels(plan.handle))
    assert counts[0] > 0
    assert counts[1] - counts[0] == counts[2] - counts[1] > 0
    plan.close()


@pytest.mark.parametrize("n3,P", [(64, 8192), (64, 1000), (37, 2056)])
def test_transform_from_bf16_input(tc, n3, P):
    # tc_transform_bf16in (TC_STORE_BF16 plans): out = in x_3 T + prev from a
    # BF16 input, against the FP64 transform of the same BF16 values; the
    # transform's two BF16 planes bound the error near 2^-16 a term.
    rng = np.random.default_rng(7 * n3 + P)
    A = torch.from_numpy(rng.standard_normal((n3, 64, 64)).astype(np.float32)).cuda()
    plan = tc.Plan(A, s=128, precision=tc.TC_BF16, store=tc.TC_STORE_BF16)
    M = cp.transform_matrix(n3)
    Mi = np.linalg.inv(M)
    Xb = torch.from_numpy(rng.standard_normal((n3, P)).astype(np.float32)).cuda().to(torch.bfloat16)
    Xd = Xb.float().cpu().numpy().astype(np.float64)
    prev = torch.from_numpy(rng.standard_normal((n3, P)).astype(np.float32)).cuda()
    for which, T in [(tc.TC_M, M), (tc.TC_MINV, Mi), (tc.TC_MINVT, Mi.T), (tc.TC_MT, M.T)]:
        Y = torch.empty((n3, P), device="cuda")
        ss = torch.zeros(1, dtype=torch.float64, device="cuda")
        tc.tc_transform_bf16in(plan.handle, which, Xb, Y, prev, ss)
        torch.cuda.synchronize()
        ref = T @ Xd + prev.cpu().numpy().astype(np.float64)
        e = np.linalg.norm(Y.cpu().numpy() - ref) / np.linalg.norm(ref)
        es = abs(float(ss.item()) - float(np.sum(ref ** 2))) / float(np.sum(ref ** 2))
        print(n3, P, which, e, es)
        assert e < 1e-4 and es < 1e-4
    assert tc.tc_plan_status(plan.handle) == tc.TC_OK
    plan.close()


@pytest.mark.parametrize("n3,P", [(64, 8192), (64, 1000), (37, 2056)])
def test_chained_transform_from_bf16_input(tc, n3, P):
    # The pass back that also writes the next product's operand:
    # out = in x_3 T + prev (FP32, 1e-4) and nxt = bf16(out x_3 T_next)
    # (within BF16 rounding of the FP64 chain, 4e-3), and out equal to the
    # unchained pass's to the bit.
    rng = np.random.default_rng(11 * n3 + P)
    A = torch.from_numpy(rng.standard_normal((n3, 64, 64)).astype(np.float32)).cuda()
    plan = tc.Plan(A, s=128, precision=tc.TC_BF16, store=tc.TC_STORE_BF16)
    M = cp.transform_matrix(n3)
    Mi = np.linalg.inv(M)
    mats = {tc.TC_M: M, tc.TC_MINV: Mi, tc.TC_MINVT: Mi.T, tc.TC_MT: M.T}
    Xb = torch.from_numpy(rng.standard_normal((n3, P)).astype(np.float32)).cuda().to(torch.bfloat16)
    Xd = Xb.float().cpu().numpy().astype(np.float64)
    prev = torch.from_numpy(rng.standard_normal((n3, P)).astype(np.float32)).cuda()
    for which, nxt_kind in [(tc.TC_MINV, tc.TC_MINVT), (tc.TC_MT, tc.TC_M)]:
        Y = torch.empty((n3, P), device="cuda")
        Y0 = torch.empty((n3, P), device="cuda")
        N = torch.empty((n3, P), dtype=torch.bfloat16, device="cuda")
        ss = torch.zeros(1, dtype=torch.float64, device="cuda")
        tc.tc_transform_bf16in(plan.handle, which, Xb, Y, prev, ss, which_next=nxt_kind, nxt=N)
        tc.tc_transform_bf16in(plan.handle, which, Xb, Y0, prev)
        torch.cuda.synchronize()
        ref = mats[which] @ Xd + prev.cpu().numpy().astype(np.float64)
        e = np.linalg.norm(Y.cpu().numpy() - ref) / np.linalg.norm(ref)
        nref = mats[nxt_kind] @ ref
        en = np.linalg.norm(N.float().cpu().numpy() - nref) / np.linalg.norm(nref)
        es = abs(float(ss.item()) - float(np.sum(ref ** 2))) / float(np.sum(ref ** 2))
        print(n3, P, which, e, en, es)
        assert e < 1e-4 and en < 4e-3 and es < 1e-4
        assert torch.equal(Y, Y0)
    assert tc.tc_plan_status(plan.handle) == tc.TC_OK
    plan.close()


def test_chained_lsqr_matches_unchained_products(tc):
    # c-LSQR on a BF16-stored plan chains its products (each pass back forms
    # the next GEMM operand). The operand it forms is the one the next
    # product's own transform would form from the same FP32 vector, so the
    # chained solve (X_reg requested) and a solve that transforms every
    # operand itself agree; the second is the same plan without X_reg, whose
    # iterate comes from the per-step updates, so the check is the iterate
    # to FP32 rounding of the recurrences.
    from paper_2103_11847_gb300 import inputs
    w = inputs.video_deblur(n=128, frames=64, seed=13)
    A = torch.from_numpy(w["A"].astype(np.float32)).cuda()
    Xt = torch.from_numpy(w["X_true"].astype(np.float32)).cuda()
    plan = tc.Plan(A, s=128, precision=tc.TC_BF16, store=tc.TC_STORE_BF16)
    C = plan.cprod(Xt)
    Xc, Xr, _, info = plan.lsqr(C, 10, regularize=True)
    Xu, _, _, info2 = plan.lsqr(C, 10, regularize=False)
    torch.cuda.synchronize()
    assert tc.read_info(info)["iters"] == 10 and tc.read_info(info2)["iters"] == 10
    d = float((Xc - Xu).norm() / Xu.norm())
    print("chained vs unchained iterate", d)
    assert d < 1e-4
    assert tc.tc_plan_status(plan.handle) == tc.TC_OK
    plan.close()
