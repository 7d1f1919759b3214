"""Precision forms of the slice GEMMs: TF32 and BF16 inputs with FP32
accumulation on the tcgen05 tensor cores (plans with precision TC_TF32 /
TC_BF16), against the FP64 oracle on the same seeded FP32 inputs.

Error is stated per result (relative Frobenius error of the c-product):
  TF32: <= 4e-3   (inputs rounded to 10 mantissa bits, 2^-11 = 4.9e-4 per value)
  BF16: <= 3e-2   (7 mantissa bits, 2^-8 = 3.9e-3 per value)
  BF16X3: <= 1e-5, the FP32 products' bound (three BF16 planes an operand, six
        products; measured 4e-7 .. 1.4e-6, where FP32 FFMA gives 1e-7 .. 3e-7:
        the tensor cores' FP32 accumulation, not the dropped split terms,
        sets it)
both including the growth by the mode-3 transform (cond(M) = 16 at n3 = 64).
Deblurring with the precision forms is checked at matched reconstruction
error: the relative error of the regularised solution against the clean image
within 2% of the FP32 GPU form's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp
from paper_2103_11847_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"tf32": 4e-3, "bf16": 3e-2, "bf16x3": 1e-5}  # bf16x3: the FP32 products' bound


@pytest.fixture(scope="module")
def tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11847_gb300 import tcprod
    tcprod.lib()
    return tcprod


def prec(tc, name):
    return {"fp32": tc.TC_FP32, "tf32": tc.TC_TF32, "bf16": tc.TC_BF16, "bf16x3": tc.TC_BF16X3}[name]


def f32(x):
    return np.ascontiguousarray(np.asarray(x, np.float32))


def dev(x):
    return torch.from_numpy(f32(x)).cuda()


def rel(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("name", ["tf32", "bf16", "bf16x3"])
@pytest.mark.parametrize("n1,n2,s,n3", [(64, 64, 64, 3), (136, 96, 40, 9), (128, 256, 200, 64),
                                        (200, 136, 72, 1), (72, 40, 56, 37), (24, 40, 24, 33)])
def test_lowp_cprod_and_adjoint(tc, name, n1, n2, s, n3):
    p = inputs.random_problem(n1, n2, s, n3, seed=n1 + s)
    A, X, Y = f32(p["A"]), f32(p["X"]), f32(p["Y"])
    plan = tc.Plan(dev(A), s=s, precision=prec(tc, name))
    Yg = plan.cprod(dev(X)).cpu().numpy()
    Xg = plan.adjoint(dev(Y)).cpu().numpy()
    e1 = rel(Yg, cp.cprod(A.astype(np.float64), X.astype(np.float64)))
    e2 = rel(Xg, cp.cprod_adjoint(A.astype(np.float64), Y.astype(np.float64)))
    print(name, (n1, n2, s, n3), e1, e2)
    assert e1 < TOL[name] and e2 < TOL[name]
    plan.close()


@pytest.mark.parametrize("name", ["tf32", "bf16", "bf16x3"])
def test_lowp_lsqr_matched_reconstruction(tc, name):
    # 128x128x16 video deblur: c-LSQR 20 iterations + Tikhonov/GCV in FP32 and
    # in the precision form; reconstruction errors within 2% of each other.
    w = inputs.video_deblur(n=128, frames=16, seed=7)
    A = f32(w["A"]).astype(np.float64)
    C = f32(inputs.scale_noise(cp.cprod(A, w["X_true"]), w["G"], w["nu"]))
    errs = {}
    for pr in ["fp32", name]:
        plan = tc.Plan(dev(A), s=128, precision=prec(tc, pr))
        X, Xr, _, info = plan.lsqr(dev(C), 20, regularize=True)
        torch.cuda.synchronize()
        inf = tc.read_info(info)
        assert inf["iters"] == 20 and inf["status"] == "maxiter", inf
        errs[pr] = rel(Xr.cpu().numpy(), w["X_true"])
        plan.close()
    print(name, errs)
    assert abs(errs[name] - errs["fp32"]) < 0.02 * errs["fp32"]


@pytest.fixture(scope="module")
def video_oracle_reg():
    """128x128x64 video deblur (n3 = 64: the tensor-core transform passes):
    the observation and the FP64 oracle's c-LSQR (20 iterations) + Tikhonov/GCV
    reconstruction error."""
    from oracle import krylov as kr
    from oracle import metrics as mt
    w = inputs.video_deblur(n=128, frames=64, seed=7)
    A = f32(w["A"]).astype(np.float64)
    op = lambda X: cp.cprod(A, X)
    adj = lambda Y: cp.cprod_adjoint(A, Y)
    C = f32(inputs.scale_noise(op(w["X_true"]), w["G"], w["nu"])).astype(np.float64)
    ref = kr.lsqr_gcv(op, adj, C, itermax=20)
    return A, C, w["X_true"], mt.relative_error(w["X_true"], ref["X_reg"])


@pytest.mark.parametrize("name", ["fp32", "tf32", "bf16", "bf16x3"])
def test_lowp_reconstruction_against_oracle(tc, video_oracle_reg, name):
    # Each form's regularised reconstruction error against the FP64 oracle's
    # on the same observation: within 1% for FP32 and the FP32-level BF16X3,
    # within 2% for TF32 and BF16 (the matched-error rule of the precision
    # form). Measured on a GB300: oracle 0.0952307; FP32 0.0952307, BF16X3
    # 0.0952307, TF32 0.0952313, BF16 0.0952505.
    A, C, Xt, e_ref = video_oracle_reg
    plan = tc.Plan(dev(A), s=128, precision=prec(tc, name))
    X, Xr, _, info = plan.lsqr(dev(C), 20, regularize=True)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["iters"] == 20 and inf["status"] == "maxiter", inf
    e = rel(Xr.cpu().numpy(), Xt)
    plan.close()
    print(name, e, e_ref)
    tol = 0.01 if name in ("fp32", "bf16x3") else 0.02
    assert abs(e - e_ref) < tol * e_ref


@pytest.mark.parametrize("frames", [40, 9])
def test_bf16x3_lsqr_matches_oracle(tc, frames):
    # The split form against the FP64 oracle: after 5 c-LSQR steps the iterate
    # is within 1e-5, where TF32 products leave 1e-4 (measured: 1e-6 here,
    # FP32 FFMA under 1e-6). Longer runs on this blur amplify every form's
    # rounding. frames = 40 runs the tube transforms on the tensor cores (three
    # planes), 9 the FP32 pass and the three-plane rounding.
    from oracle import krylov as kr
    w = inputs.video_deblur(n=64, frames=frames, seed=9)
    A = f32(w["A"]).astype(np.float64)
    op = lambda X: cp.cprod(A, X)
    adj = lambda Y: cp.cprod_adjoint(A, Y)
    C = f32(inputs.scale_noise(op(w["X_true"]), w["G"], 1e-2)).astype(np.float64)
    ref = kr.lsqr(op, adj, C, itermax=5)
    plan = tc.Plan(dev(A), s=64, precision=tc.TC_BF16X3)
    X, _, _, info = plan.lsqr(dev(C), 5)
    torch.cuda.synchronize()
    assert tc.read_info(info)["iters"] == ref["iters"]
    assert rel(X.cpu().numpy(), ref["X"]) < 1e-5
    plan.close()


def test_lowp_rejects_unsupported_shapes(tc):
    A = torch.zeros((3, 20, 20), device="cuda")
    with pytest.raises(tc.TcError):
        tc.Plan(A, s=20, precision=tc.TC_BF16)  # 20 is not a multiple of 8
    B = torch.zeros((3, 20, 20), device="cuda")
    with pytest.raises(tc.TcError):  # two-sided: s = 20 is not a multiple of 8 either
        tc.Plan(torch.zeros((3, 16, 16), device="cuda"), B, precision=tc.TC_TF32)


# Two-sided products A *c X *c B on the tensor cores: the first GEMM's T is
# rounded to the GEMM input type again before the second, so the TF32 and
# BF16 bounds double; BF16X3 stays at the FP32 products' bound.
TOL2 = {"tf32": 8e-3, "bf16": 6e-2, "bf16x3": 1e-5}


@pytest.mark.parametrize("name", ["tf32", "bf16", "bf16x3"])
@pytest.mark.parametrize("n1,n2,s,n3", [(64, 64, 64, 3), (256, 256, 256, 3), (136, 96, 40, 9),
                                        (72, 40, 56, 37), (24, 40, 24, 33), (128, 64, 200, 1)])
def test_lowp_two_sided_cprod_and_adjoint(tc, name, n1, n2, s, n3):
    p = inputs.random_problem(n1, n2, s, n3, two_sided=True, seed=n1 + 3 * s)
    A, X, Y, B = f32(p["A"]), f32(p["X"]), f32(p["Y"]), f32(p["B"])
    plan = tc.Plan(dev(A), dev(B), precision=prec(tc, name))
    Ad, Bd = A.astype(np.float64), B.astype(np.float64)
    yg = plan.cprod(dev(X)).cpu().numpy()
    xg = plan.adjoint(dev(Y)).cpu().numpy()
    assert tc.tc_plan_status(plan.handle) == tc.TC_OK
    plan.close()
    ey = rel(yg, cp.cprod(Ad, X.astype(np.float64), Bd))
    ex = rel(xg, cp.cprod_adjoint(Ad, Y.astype(np.float64), Bd))
    print(name, (n1, n2, s, n3), ey, ex)
    assert ey < TOL2[name] and ex < TOL2[name]


@pytest.mark.parametrize("name", ["bf16x3", "tf32"])
def test_lowp_two_sided_lsqr_256(tc, name):
    # The two-sided 256x256x3 workload (50 c-LSQR iterations + Tikhonov/GCV)
    # on the tensor cores against the FP64 oracle: BF16X3 (FP32-level
    # products) keeps the FP32 route's parity, the iterate within 1e-3 and the
    # reconstruction error within 1%; TF32 is held to the matched-error rule
    # (2%).
    from oracle import krylov as kr
    from oracle import metrics as mt
    w = inputs.two_sided_deblur(n=256, n3=3, seed=1)
    A, B = f32(w["A"]).astype(np.float64), f32(w["B"]).astype(np.float64)
    op = lambda X: cp.cprod(A, X, B)
    adj = lambda Y: cp.cprod_adjoint(A, Y, B)
    C = f32(inputs.scale_noise(op(w["X_true"]), w["G"], w["nu"])).astype(np.float64)
    ref = kr.lsqr_gcv(op, adj, C, itermax=50)
    plan = tc.Plan(dev(A), dev(B), precision=prec(tc, name))
    X, Xr, _, info = plan.lsqr(dev(C), 50, regularize=True)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["iters"] == 50
    e_gpu = mt.relative_error(w["X_true"], Xr.cpu().numpy())
    e_ref = mt.relative_error(w["X_true"], ref["X_reg"])
    d = rel(X.cpu().numpy(), ref["X"])
    print(name, d, e_gpu, e_ref)
    if name == "bf16x3":
        assert d < 1e-3
        assert abs(e_gpu - e_ref) < 0.01 * e_ref
    else:
        assert abs(e_gpu - e_ref) < 0.02 * e_ref
    plan.close()


def tf32_trunc(x):
    """FP32 values with the low 13 mantissa bits cleared: exact TF32 values."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


@pytest.mark.parametrize("name", ["tf32", "bf16", "bf16x3"])
def test_slice_scales_pass_through_exactly(tc, name):
    # Per-slice scaling (reading R22): BF16 and TF32 keep FP32's 8-bit
    # exponent and the slice GEMMs share no exponent between slices, so a
    # transformed slice 2^-60 or 2^60 times its neighbours gives exactly 2^e
    # times its unit-scale result: a per-slice power-of-two scale folded in
    # and divided out again would change no bit.
    n3, n, s = 3, 64, 48
    rng = np.random.default_rng(21)
    A = rng.standard_normal((n3, n, n)).astype(np.float32)
    plan = tc.Plan(dev(A), s=s, precision=prec(tc, name))
    Xh = rng.standard_normal((n3, n, s)).astype(np.float32)
    scale = np.array([2.0 ** -60, 1.0, 2.0 ** 60], np.float32)
    outs = []
    for sc in (np.ones(n3, np.float32), scale):
        Xs = Xh * sc[:, None, None]
        if name == "tf32":
            op = torch.from_numpy(tf32_trunc(Xs)).cuda()
        elif name == "bf16":
            op = torch.from_numpy(Xh).cuda().to(torch.bfloat16) * torch.from_numpy(sc).cuda().to(
                torch.bfloat16)[:, None, None]
        else:  # three planes of each slice, each plane scaled exactly
            x = torch.from_numpy(Xh).cuda()
            p0 = x.to(torch.bfloat16)
            r = x - p0.float()
            p1 = r.to(torch.bfloat16)
            p2 = (r - p1.float()).to(torch.bfloat16)
            f = torch.from_numpy(sc).cuda().to(torch.bfloat16)[:, None, None]
            op = torch.cat([p0 * f, p1 * f, p2 * f]).contiguous()
        Y = torch.empty((n3, n, s), device="cuda")
        tc.tc_slice_gemm(plan.handle, op.contiguous(), Y)
        outs.append(Y)
    torch.cuda.synchronize()
    for k in range(n3):
        assert torch.equal(outs[1][k], outs[0][k] * float(scale[k])), k
    # the whole product: A and the operand at 2^-60 and 2^60 (the transform
    # passes, the operand rounding, the GEMMs and the inverse all scale exactly)
    X = dev(rng.standard_normal((n3, n, s)))
    Y1 = plan.cprod(X)
    for e in (-60, 60):
        f = float(2.0 ** e)
        pf = tc.Plan(dev(A * np.float32(f)), s=s, precision=prec(tc, name))
        Yf = pf.cprod(X)
        Yg = plan.cprod((X * f).contiguous())
        torch.cuda.synchronize()
        assert torch.equal(Yf, Y1 * f) and torch.equal(Yg, Y1 * f), e
        pf.close()
    plan.close()



@pytest.mark.parametrize("n1,n2,s,n3", [(128, 256, 200, 64), (72, 40, 56, 37), (24, 40, 24, 33),
                                        (136, 96, 40, 64)])
def test_bf16_stored_products(tc, n1, n2, s, n3):
    # TC_STORE_BF16: the slice products rounded once to BF16 and read back by
    # the BF16-input pass; the product and adjoint within the BF16 bound.
    p = inputs.random_problem(n1, n2, s, n3, seed=n1 + 3 * s)
    A, X, Y = f32(p["A"]), f32(p["X"]), f32(p["Y"])
    plan = tc.Plan(dev(A), s=s, precision=tc.TC_BF16, store=tc.TC_STORE_BF16)
    Yg = plan.cprod(dev(X)).cpu().numpy()
    Xg = plan.adjoint(dev(Y)).cpu().numpy()
    e1 = rel(Yg, cp.cprod(A.astype(np.float64), X.astype(np.float64)))
    e2 = rel(Xg, cp.cprod_adjoint(A.astype(np.float64), Y.astype(np.float64)))
    print(n1, n2, s, n3, e1, e2)
    assert e1 < TOL["bf16"] and e2 < TOL["bf16"]
    assert tc.tc_plan_status(plan.handle) == tc.TC_OK
    plan.close()


def test_bf16_stored_products_reconstruction(tc, video_oracle_reg):
    # The 128x128x64 video, 20 c-LSQR iterations + GCV: the BF16-stored form
    # within the precision form's 2% of the FP64 oracle's reconstruction error.
    A, C, Xt, e_ref = video_oracle_reg
    plan = tc.Plan(dev(A), s=128, precision=tc.TC_BF16, store=tc.TC_STORE_BF16)
    X, Xr, _, info = plan.lsqr(dev(C), 20, regularize=True)
    torch.cuda.synchronize()
    inf = tc.read_info(info)
    assert inf["iters"] == 20 and inf["status"] == "maxiter", inf
    e = rel(Xr.cpu().numpy(), Xt)
    print("bf16 stored", e, e_ref)
    assert abs(e - e_ref) < 0.02 * e_ref
    plan.close()


def test_bf16_stored_products_rejected_elsewhere(tc):
    rng = np.random.default_rng(5)
    for kw, shape in [(dict(precision=tc.TC_FP32), (64, 64, 64)),
                      (dict(precision=tc.TC_TF32), (64, 64, 64)),
                      (dict(precision=tc.TC_BF16X3), (64, 64, 64)),
                      (dict(precision=tc.TC_BF16), (16, 64, 64))]:
        with pytest.raises(tc.TcError) as e:
            tc.Plan(dev(rng.standard_normal(shape)), s=64, store=tc.TC_STORE_BF16, **kw)
        assert e.value.code == tc.TC_EUNSUPPORTED
    Ad = dev(rng.standard_normal((64, 64, 64)))
    with pytest.raises(tc.TcError) as e:
        tc.Plan(Ad, B=Ad, precision=tc.TC_BF16, store=tc.TC_STORE_BF16)
    assert e.value.code == tc.TC_EUNSUPPORTED
