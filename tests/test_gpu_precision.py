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
def test_lowp_video_operator_full_size(tc, name):
    # 512x512x64 video operator: sampled output tubes against the oracle.
    w = inputs.video_deblur(n=512, frames=64, seed=2)
    A, X = f32(w["A"]), f32(w["X_true"])
    plan = tc.Plan(dev(A), s=512, precision=prec(tc, name))
    Y = plan.cprod(dev(X)).cpu().numpy()
    M = cp.transform_matrix(64)
    Minv = np.linalg.inv(M)
    rng = np.random.default_rng(5)
    num = den = 0.0
    for _ in range(16):
        i, j = int(rng.integers(0, 512)), int(rng.integers(0, 512))
        Ah_row = np.einsum("kl,lp->kp", M, A[:, i, :].astype(np.float64))
        Xh_col = np.einsum("kl,lp->kp", M, X[:, :, j].astype(np.float64))
        tube = Minv @ np.sum(Ah_row * Xh_col, axis=1)
        num += np.sum((Y[:, i, j] - tube) ** 2)
        den += np.sum(tube ** 2)
    assert np.sqrt(num / den) < TOL[name]


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
    B = torch.zeros((3, 16, 16), device="cuda")
    with pytest.raises(tc.TcError):
        tc.Plan(torch.zeros((3, 16, 16), device="cuda"), B, precision=tc.TC_TF32)
