"""Batched c-LSQR (tc_batch_create / tc_lsqr_c_batched): independent problems of
uneven sizes in one graph launch.

* Child-graph form: each problem's result equals, bit for bit, what
  tc_lsqr_c gives on its own plan (the same kernels in the same order with
  deterministic reductions), at 15 iterations.
* Grouped form (FP32 fused route with X_reg): every result matches the FP64
  oracle, the iterate within 1e-3 at 8 iterations (the more ill-conditioned
  problems leave the FP64 trajectory in FP32 before 15) and the regularised
  reconstruction error within 1%; it equals the child-graph form up to the
  order of FP32 additions (1e-5); repeated solves are bit-identical; the
  autotuner has picked a tile shape. The full 128-problem mix of the batched
  workload (n in 64..512) is checked against the child-graph form, and a
  spread of its sizes against the oracle.
* Grouped BF16 form (tcgen05 tiles with the transforms fused): on the same
  problems the regularised reconstruction error is within 2% of the FP64
  oracle's (the precision forms' matched-error bar), the iterate within 2e-3
  of the BF16 child-graph form (the same BF16 operands, summed in another
  order), repeated solves are bit-identical, and both tile shapes give the
  same result within 2e-3.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp
from oracle import krylov as kr
from oracle import metrics as mt
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


def rel(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_child_graph_form_equals_single_solves(tc):
    probs = problems()
    As = [torch.from_numpy(p[0].astype(np.float32)).cuda() for p in probs]
    Cs = [torch.from_numpy(p[2].astype(np.float32)).cuda() for p in probs]
    Xs = [torch.empty_like(c) for c in Cs]
    Xr = [torch.empty_like(c) for c in Cs]
    infos = tc.new_infos(len(probs))
    h = tc.tc_batch_create(As, SIZES)
    tc.tc_batch_info(h, mode=1)
    for _ in range(2):  # the second call replays the cached parent graph
        for x in Xs + Xr:
            x.fill_(float("nan"))
        tc.tc_lsqr_c_batched(h, Cs, Xs, Xr, 15, 0.0, None, infos)
        torch.cuda.synchronize()
        for i in range(len(probs)):
            plan = tc.Plan(As[i], s=SIZES[i])
            x1, xr1, _, inf1 = plan.lsqr(Cs[i], 15, regularize=True)
            torch.cuda.synchronize()
            assert torch.equal(x1, Xs[i]) and torch.equal(xr1, Xr[i])
            plan.close()
    assert tc.tc_batch_info(h)[0] is False
    inf = tc.read_infos(infos, len(probs))
    assert all(d["iters"] == 15 and d["status"] == "maxiter" for d in inf)
    tc.tc_batch_destroy(h)


def test_grouped_form_matches_oracle_and_child_graphs(tc):
    probs = problems()
    As = [torch.from_numpy(p[0].astype(np.float32)).cuda() for p in probs]
    Cs = [torch.from_numpy(p[2].astype(np.float32)).cuda() for p in probs]
    Xs = [torch.empty_like(c) for c in Cs]
    Xr = [torch.empty_like(c) for c in Cs]
    infos = tc.new_infos(len(probs))
    h = tc.tc_batch_create(As, SIZES)
    tc.tc_lsqr_c_batched(h, Cs, Xs, Xr, 8, 0.0, None, infos)
    torch.cuda.synchronize()
    grouped, tile, ms = tc.tc_batch_info(h)
    print("grouped", grouped, "tile", tile, "autotune ms", ms)
    assert grouped and tile in (0, 1, 2) and min(ms) > 0
    first = [x.clone() for x in Xs], [x.clone() for x in Xr]
    for x in Xs + Xr:
        x.fill_(float("nan"))
    tc.tc_lsqr_c_batched(h, Cs, Xs, Xr, 8, 0.0, None, infos)  # replay: bit-identical
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert torch.equal(first[0][i], Xs[i]) and torch.equal(first[1][i], Xr[i])
    inf = tc.read_infos(infos, len(probs))
    assert all(d["iters"] == 8 and d["status"] == "maxiter" for d in inf)
    for i, (A, X, C) in enumerate(probs):
        op = lambda Z: cp.cprod(A, Z)
        adj = lambda Y: cp.cprod_adjoint(A, Y)
        ref = kr.lsqr_gcv(op, adj, C, itermax=8)
        assert rel(Xs[i].cpu().numpy(), ref["X"]) < 1e-3, i
        e = mt.relative_error(X, Xr[i].cpu().numpy())
        e_ref = mt.relative_error(X, ref["X_reg"])
        assert abs(e - e_ref) <= 0.01 * e_ref, (i, e, e_ref)
    # the child-graph form of the same batch: the same up to FP32 addition order
    Xc = [torch.empty_like(c) for c in Cs]
    Xrc = [torch.empty_like(c) for c in Cs]
    tc.tc_batch_info(h, mode=1)
    tc.tc_lsqr_c_batched(h, Cs, Xc, Xrc, 8, 0.0, None, infos)
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert rel(Xs[i].cpu().numpy(), Xc[i].cpu().numpy().astype(np.float64)) < 1e-5
        assert rel(Xr[i].cpu().numpy(), Xrc[i].cpu().numpy().astype(np.float64)) < 1e-4
    tc.tc_batch_destroy(h)


def test_grouped_full_batch_mix(tc):
    # The batched workload's 128 problems (n in 64..512, x3): grouped against
    # the child-graph form for every problem, against the oracle for a spread
    # of sizes, at 8 iterations + GCV.
    sizes = inputs.batch_sizes(128)
    ws = [inputs.batch_problem(i, n) for i, n in enumerate(sizes)]
    As = [torch.from_numpy(w["A"].astype(np.float32)).cuda() for w in ws]
    Cs = []
    for w in ws:
        A = w["A"].astype(np.float32).astype(np.float64)
        C = inputs.scale_noise(cp.cprod(A, w["X_true"]), w["G"], w["nu"])
        Cs.append(torch.from_numpy(C.astype(np.float32)).cuda())
    Xg = [torch.empty_like(c) for c in Cs]
    Xrg = [torch.empty_like(c) for c in Cs]
    Xc = [torch.empty_like(c) for c in Cs]
    Xrc = [torch.empty_like(c) for c in Cs]
    infos = tc.new_infos(len(Cs))
    h = tc.tc_batch_create(As, sizes)
    tc.tc_lsqr_c_batched(h, Cs, Xg, Xrg, 8, 0.0, None, infos)
    torch.cuda.synchronize()
    assert tc.tc_batch_info(h)[0]
    tc.tc_batch_info(h, mode=1)
    tc.tc_lsqr_c_batched(h, Cs, Xc, Xrc, 8, 0.0, None, infos)
    torch.cuda.synchronize()
    worst = max(rel(Xg[i].cpu().numpy(), Xc[i].cpu().numpy().astype(np.float64))
                for i in range(len(Cs)))
    print("grouped vs child graphs, worst iterate difference", worst)
    assert worst < 1e-5
    picked = {}
    for i, n in enumerate(sizes):
        if n in (64, 160, 256, 352, 512) and n not in picked:
            picked[n] = i
    for n, i in picked.items():
        A = ws[i]["A"].astype(np.float32).astype(np.float64)
        ref = kr.lsqr(lambda Z: cp.cprod(A, Z), lambda Y: cp.cprod_adjoint(A, Y),
                      Cs[i].cpu().numpy().astype(np.float64), itermax=8)
        assert rel(Xg[i].cpu().numpy(), ref["X"]) < 1e-3, (n, i)
    tc.tc_batch_destroy(h)


def bf16_batch(tc, probs, sizes, iters, cfg_mode=0):
    As = [torch.from_numpy(p[0].astype(np.float32)).cuda() for p in probs]
    Cs = [torch.from_numpy(p[2].astype(np.float32)).cuda() for p in probs]
    h = tc.tc_batch_create(As, sizes, precision=tc.TC_BF16)
    tc.tc_batch_info(h, mode=cfg_mode)
    Xs = [torch.empty_like(c) for c in Cs]
    Xr = [torch.empty_like(c) for c in Cs]
    infos = tc.new_infos(len(probs))
    tc.tc_lsqr_c_batched(h, Cs, Xs, Xr, iters, 0.0, None, infos)
    torch.cuda.synchronize()
    return h, Cs, Xs, Xr, infos


def test_grouped_bf16_matches_oracle_and_child_graphs(tc):
    sizes = [64, 96, 40, 72, 128, 256]  # multiples of 8; two ragged against 128-row tiles
    probs = []
    for i, n in enumerate(sizes):
        rng = np.random.default_rng(300 + i)
        sigma = 1.0 + 0.5 * i
        G = inputs.gaussian_blur(n, sigma, int(math.ceil(3 * sigma)))
        A = np.stack([w * G for w in (1.0, 0.7, 0.4)]).astype(np.float32).astype(np.float64)
        X = inputs.image(n, rng)
        C = inputs.scale_noise(cp.cprod(A, X), rng.standard_normal(X.shape), 1e-3)
        probs.append((A, X, C.astype(np.float32).astype(np.float64)))
    iters = 8
    h, Cs, Xs, Xr, infos = bf16_batch(tc, probs, sizes, iters)
    grouped, tile, ms = tc.tc_batch_info(h)
    print("bf16 grouped", grouped, "tile", tile, "autotune ms", ms)
    assert grouped and tile in (0, 1) and ms[0] > 0 and ms[1] > 0
    inf = tc.read_infos(infos, len(probs))
    assert all(d["iters"] == iters and d["status"] == "maxiter" for d in inf), inf
    first = [x.clone() for x in Xs], [x.clone() for x in Xr]
    tc.tc_lsqr_c_batched(h, Cs, Xs, Xr, iters, 0.0, None, infos)  # replay: bit-identical
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert torch.equal(first[0][i], Xs[i]) and torch.equal(first[1][i], Xr[i])
    for i, (A, X, C) in enumerate(probs):
        ref = kr.lsqr_gcv(lambda Z: cp.cprod(A, Z), lambda Y: cp.cprod_adjoint(A, Y), C,
                          itermax=iters)
        e = mt.relative_error(X, Xr[i].cpu().numpy())
        e_ref = mt.relative_error(X, ref["X_reg"])
        print(sizes[i], "iterate vs oracle", rel(Xs[i].cpu().numpy(), ref["X"]), "errors", e, e_ref)
        assert abs(e - e_ref) <= 0.02 * e_ref, (i, e, e_ref)
    # the BF16 child-graph form: separate transform passes and GEMMs
    Xc = [torch.empty_like(c) for c in Cs]
    Xrc = [torch.empty_like(c) for c in Cs]
    tc.tc_batch_info(h, mode=1)
    tc.tc_lsqr_c_batched(h, Cs, Xc, Xrc, iters, 0.0, None, infos)
    torch.cuda.synchronize()
    assert tc.tc_batch_info(h)[0] is False
    for i in range(len(probs)):
        d = rel(Xs[i].cpu().numpy(), Xc[i].cpu().numpy().astype(np.float64))
        print(sizes[i], "grouped vs child graphs", d)
        assert d < 2e-3, (i, d)
    tc.tc_batch_destroy(h)


def test_grouped_bf16_tile_shapes_agree(tc):
    sizes = [64, 136, 200, 256]
    probs = []
    for i, n in enumerate(sizes):
        rng = np.random.default_rng(400 + i)
        G = inputs.gaussian_blur(n, 2.0, 6)
        A = np.stack([w * G for w in (1.0, 0.7, 0.4)]).astype(np.float32).astype(np.float64)
        X = inputs.image(n, rng)
        C = inputs.scale_noise(cp.cprod(A, X), rng.standard_normal(X.shape), 1e-3)
        probs.append((A, X, C.astype(np.float32).astype(np.float64)))
    out = []
    for tile in (0, 1):
        h, Cs, Xs, Xr, infos = bf16_batch(tc, probs, sizes, 6)
        tc.tc_batch_force_tile(h, tile)
        tc.tc_lsqr_c_batched(h, Cs, Xs, Xr, 6, 0.0, None, infos)
        torch.cuda.synchronize()
        assert tc.tc_batch_info(h)[1] == tile
        out.append([x.cpu().numpy().astype(np.float64) for x in Xs])
        tc.tc_batch_destroy(h)
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert rel(a, b) < 2e-3
