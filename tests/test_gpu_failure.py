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


def test_planted_timeout_inside_the_fit_kernels(nmf, monkeypatch):
    """A missing arrival inside the real tensor-core passes: at one iteration
    of the stage loop, block 0 of the W pass waits for an H-pass tile count
    that is never reached (nmf_debug_plant_timeout).  The wait gives up after
    200 us and records NMF_ETIMEOUT; the loop stops at that iteration instead
    of running the remaining ones (as a recorded graph's device-side loop and
    as direct launches); the block's copies and MMAs in flight complete before
    it leaves; and the next fit, with the plant removed, agrees with the
    oracle as usual."""
    prob = synthetic.make_config(0, N=200, K=4, n_iter=40)
    K, iters, t_fault = prob.K, 40, 7
    prm = nmf.make_params(prob.N, prob.P, K, iters, K - 1, False, 0.0, 1e-30, nmf.NMF_BF16_SPLIT, 0)
    assert nmf.nmf_debug_plant_timeout(t_fault, 200_000) == nmf.NMF_OK
    try:
        for graphs in (True, False):
            if not graphs:
                monkeypatch.setenv("NMF_NO_GRAPH", "1")
            ws = nmf.workspace(nmf.nmf_fit_workspace_bytes(prm))
            _, _, _, done = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, iters, k_start=K - 1,
                                          normalize=False, precision="bf16", check_status=False, ws=ws)
            assert nmf.nmf_workspace_status(nmf._ptr(ws), nmf._stream(None)) == nmf.NMF_ETIMEOUT
            # the state kept is the last one whose Eq. 2 was recorded: the
            # loop stopped at the planted iteration, not after all 40
            assert int(np_(done)[K - 1]) <= t_fault
            monkeypatch.delenv("NMF_NO_GRAPH", raising=False)
    finally:
        assert nmf.nmf_debug_plant_timeout(-1, 0) == nmf.NMF_OK
    assert nmf.nmf_debug_plant_timeout(3, 10) == nmf.NMF_EINVAL  # limit below 1 us
    # the context is intact and the plant is gone: a normal fit agrees with the oracle
    W, H, chi2, done = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, 30, precision="bf16", polish_iters=5)
    torch.cuda.synchronize()
    ref = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, 30)
    np.testing.assert_allclose(np_(chi2), ref["chi2_hist"], rtol=1e-3)
    assert np.all(np_(done) == 30)


def np_(t):
    return t.detach().cpu().numpy()
