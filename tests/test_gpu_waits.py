"""The bounded-wait path of the tensor-core kernels, exercised without a fault.

Every mbarrier wait in the tcgen05 kernels polls a bounded number of times and
reports TC_ETIMEOUT instead of hanging. tc_check_bounded_wait runs one such wait
on a barrier that nothing arrives on; the test reads the status, then checks
that the context still runs a tensor-core product correctly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cproduct as cp
from paper_2103_11847_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_11847_gb300 import tcprod
    tcprod.lib()
    return tcprod


def test_bounded_wait_reports_timeout_and_context_survives(tc):
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    tc.tc_check_bounded_wait(256, status)
    torch.cuda.synchronize()
    assert int(status.item()) == tc.TC_ETIMEOUT

    p = inputs.random_problem(64, 64, 64, 3, seed=3)
    A = np.ascontiguousarray(p["A"], np.float32)
    X = np.ascontiguousarray(p["X"], np.float32)
    plan = tc.Plan(torch.from_numpy(A).cuda(), s=64, precision=tc.TC_BF16)
    Y = plan.cprod(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    ref = cp.cprod(A.astype(np.float64), X.astype(np.float64))
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) < 3e-2
    plan.close()


def test_bounded_wait_rejects_bad_arguments(tc):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TcError):
        tc.tc_check_bounded_wait(0, status)
    with pytest.raises(tc.TcError):
        tc.tc_check_bounded_wait((1 << 20) + 1, status)
