"""Failure handling on the GPU without a fault: every wait in the kernels is
bounded; a wait nothing satisfies (an mbarrier nobody arrives at, a counter
nobody raises) gives up after its limit, records NMF_ETIMEOUT for the host to
read, and the device stays usable for the next call."""
import numpy as np
import pytest

import oracle
from paper_2309_04623_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nmf():
    from paper_2309_04623_gb300 import build
    from paper_2309_04623_gb300 import nmf as _nmf

    build.build()
    _nmf.load()
    return _nmf


def test_bounded_waits_time_out_and_leave_the_device_usable(nmf):
    assert nmf.wait_selftest(1_000_000) == (nmf.NMF_ETIMEOUT, nmf.NMF_ETIMEOUT)
    assert nmf.wait_selftest(50_000) == (nmf.NMF_ETIMEOUT, nmf.NMF_ETIMEOUT)
    # the context is intact: a tensor-core fit right after agrees with the oracle as usual
    prob = synthetic.make_config(0, N=40, K=3, n_iter=30)
    W, H, chi2, done = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter, precision="bf16",
                                     polish_iters=5)
    torch.cuda.synchronize()
    ref = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter)
    np.testing.assert_allclose(chi2.cpu().numpy(), ref["chi2_hist"], rtol=1e-3)
