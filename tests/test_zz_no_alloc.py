"""tc_fro_norm_noalloc: the Frobenius norm without any device allocation.

This entry point is for callers that cannot call cudaMalloc. One example is
code whose device memory belongs to another allocator that has reserved the
device. Another is code that cannot accept the device synchronisation that
cudaMalloc and cudaFree may imply. Its scratch is a static array in the
library's device memory.

The test checks, through the C ABI, that two calls in a row agree with the
norm that tc_gkb_init writes to beta[0]. That norm is the allocating path's
result for the same reduction, and the tolerance is 1e-12 relative: both run
the same reduction tree in the same order. The test also checks that sizes
beyond the documented maximum are rejected on the host.

The file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
MAX_ELEMS = 152 * 32 * 256 * 64


@pytest.fixture(scope="module")
def tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11847_gb300 import tcprod
    tcprod.lib()
    return tcprod


@pytest.mark.parametrize("shape", [(3, 256, 256), (5, 131, 77), (1, 1, 3)])
def test_noalloc_norm_matches_allocating_path(tc, shape):
    n3, n1, s = shape
    rng = np.random.default_rng(sum(shape))
    C = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    A = torch.from_numpy(rng.standard_normal((n3, n1, n1)).astype(np.float32)).cuda()
    plan = tc.Plan(A, s=s)
    U = torch.zeros((2,) + shape, device="cuda")
    V = torch.zeros((2, n3, n1, s), device="cuda")
    al = torch.zeros(2, dtype=torch.float64, device="cuda")
    be = torch.zeros(2, dtype=torch.float64, device="cuda")
    tc.tc_gkb_init(plan.handle, C, U, V, al, be, 1)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    tc.tc_fro_norm_noalloc(C, out[0:1])
    tc.tc_fro_norm_noalloc(C, out[1:2])  # second call reuses the same scratch
    torch.cuda.synchronize()
    ref = be[0].item()
    got = out.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-12 * ref), (got, ref)
    exact = float(np.linalg.norm(C.cpu().numpy().astype(np.float64)))
    assert abs(got[0] - exact) <= 1e-6 * exact
    plan.close()


def test_noalloc_rejects_oversize_on_host(tc):
    lib = tc.lib()
    x = torch.zeros(4, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    r = lib.tc_fro_norm_noalloc(x.data_ptr(), MAX_ELEMS + 1, out.data_ptr(), None)
    assert r == tc.TC_EINVAL
    assert b"maximum" in lib.tc_last_error()
    torch.cuda.synchronize()
