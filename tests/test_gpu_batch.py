"""Batched c-LSQR (tc_batch_create / tc_lsqr_c_batched): independent problems of
uneven sizes in one graph launch. Each problem's result must equal, bit for bit,
what tc_lsqr_c gives on its own plan: the same kernels run in the same order
with deterministic reductions (checked at 15 iterations). Each result must
also match the FP64 oracle to 1e-3 at 8 iterations; the more ill-conditioned
problems of the batch leave the FP64 trajectory in FP32 before 15."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp
from oracle import krylov as kr
from paper_2103_11847_gb300 import inputs

pytestmark = pytest.mark.gpu
SIZES = [32, 64, 96, 40, 72, 128]


@pytest.fixture(scope="module")
def tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11847_gb300 import tcprod
    tcprod.lib()
    return tcprod


def problems():
    out = []
    for i, n in enumerate(SIZES):
        rng = np.random.default_rng(100 + i)
        sigma = 1.0 + 0.5 * i
        G = inputs.gaussian_blur(n, sigma, int(math.ceil(3 * sigma)))
        A = np.stack([w * G for w in (1.0, 0.7, 0.4)]).astype(np.float32).astype(np.float64)
        X = inputs.image(n, rng)
        C = inputs.scale_noise(cp.cprod(A, X), rng.standard_normal(X.shape), 1e-3)
        out.append((A, X, C.astype(np.float32).astype(np.float64)))
    return out


def test_batched_lsqr_matches_single_and_oracle(tc):
    probs = problems()
    As = [torch.from_numpy(p[0].astype(np.float32)).cuda() for p in probs]
    Cs = [torch.from_numpy(p[2].astype(np.float32)).cuda() for p in probs]
    Xs = [torch.empty_like(c) for c in Cs]
    Xr = [torch.empty_like(c) for c in Cs]
    infos = tc.new_infos(len(probs))
    h = tc.tc_batch_create(As, SIZES)
    for _ in range(2):  # the second call replays the cached parent graph
        for x in Xs + Xr:
            x.fill_(float("nan"))
        tc.tc_lsqr_c_batched(h, Cs, Xs, Xr, 15, 0.0, None, infos)
        torch.cuda.synchronize()
        for i, (A, X, C) in enumerate(probs):
            plan = tc.Plan(As[i], s=SIZES[i])
            x1, xr1, _, inf1 = plan.lsqr(Cs[i], 15, regularize=True)
            torch.cuda.synchronize()
            assert torch.equal(x1, Xs[i]) and torch.equal(xr1, Xr[i])
            plan.close()
    inf = tc.read_infos(infos, len(probs))
    assert all(d["iters"] == 15 and d["status"] == "maxiter" for d in inf)
    tc.tc_lsqr_c_batched(h, Cs, Xs, None, 8, 0.0, None, infos)
    torch.cuda.synchronize()
    for i, (A, X, C) in enumerate(probs):
        ref = kr.lsqr(lambda Z: cp.cprod(A, Z), lambda Y: cp.cprod_adjoint(A, Y), C, itermax=8)
        xg = Xs[i].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(xg - ref["X"]) < 1e-3 * np.linalg.norm(ref["X"]), i
    tc.tc_batch_destroy(h)
