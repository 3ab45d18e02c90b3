"""Failure detection on the GPU without a fault: a bounded wait runs out on a
condition that never becomes true, the kernel reports NLA_ERR_TIMEOUT through the
info word and returns, and the context stays usable for the next call."""
import numpy as np
import pytest

from paper_2608_21227_gb300 import inputs
import oracle

from _util import err_rel, tol_for

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nla():
    from paper_2608_21227_gb300 import nla as m

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


@pytest.mark.parametrize("mode", [0, 1])
def test_bounded_wait_reports_timeout_and_context_survives(nla, mode):
    info = nla.wait_selftest(mode, 50_000)  # 50 ms budget
    torch.cuda.synchronize()
    assert int(info.item()) == -5  # -NLA_ERR_TIMEOUT
    # the context is still usable: a full SVD right after
    A = inputs.gaussian(64, 48, 7)
    t = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    S, info2 = nla.gesvd_vals(t)
    torch.cuda.synchronize()
    assert int(info2.item()) == 0
    assert err_rel(S.cpu().numpy(), oracle.svdvals(A)) <= tol_for(0, 64)


def test_selftest_argument_errors(nla):
    with pytest.raises(nla.NLAError):
        nla.wait_selftest(2, 1000)
    with pytest.raises(nla.NLAError):
        nla.wait_selftest(0, 0)
