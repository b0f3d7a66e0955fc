"""The vectorised NumPy CPU baseline (the paper's own CPU setup) against the
FP64 oracle: the float64 form follows the oracle's trajectory to rounding
order, the float32 form to single-precision accuracy."""
import numpy as np
import pytest

import oracle
from oracle import numpy_baseline as nb
from paper_2309_04623_gb300 import synthetic


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def prob():
    return synthetic.make_config(0, N=24, K=4, M=3, n_iter=40)


def test_fp64_fit_follows_oracle(prob):
    ref = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter)
    got = nb.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter)
    assert rel(got["W"], ref["W"]) <= 1e-10
    assert rel(got["H"], ref["H"]) <= 1e-10
    assert np.allclose(got["chi2_hist"], ref["chi2_hist"], rtol=1e-12, atol=0)
    assert np.array_equal(got["iters_done"], ref["iters_done"])


def test_fp64_iterate_trace_follows_oracle(prob):
    W, H = prob.W0[:, :3], prob.H0[:3]
    Wr, Hr, tr, _ = oracle.iterate(prob.V, prob.Wt, W, H, 7)
    Wg, Hg, tg = nb.iterate(prob.V, prob.Wt, W, H, 7)
    assert rel(Wg, Wr) <= 1e-12 and rel(Hg, Hr) <= 1e-12
    assert np.allclose(tg, tr, rtol=1e-12, atol=0)


def test_fp32_fit_close_to_oracle(prob):
    ref = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter)
    got = nb.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter, dtype=np.float32)
    assert got["W"].dtype == np.float32
    assert rel(got["H"], ref["H"]) <= 1e-4
    assert np.allclose(got["chi2_hist"], ref["chi2_hist"], rtol=1e-5, atol=0)


def test_stopping_rule_matches_oracle(prob):
    ref = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, 200, tol=1e-4)
    got = nb.fit(prob.V, prob.Wt, prob.W0, prob.H0, 200, tol=1e-4)
    assert np.array_equal(got["iters_done"], ref["iters_done"])
    assert np.any(ref["iters_done"] < 200)  # the rule fires


def test_zero_iterations_and_k_start(prob):
    ref = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, 0, k_start=2)
    got = nb.fit(prob.V, prob.Wt, prob.W0, prob.H0, 0, k_start=2)
    assert np.allclose(got["chi2_hist"][2:], ref["chi2_hist"][2:], rtol=1e-12, atol=0)
    assert np.array_equal(got["iters_done"], ref["iters_done"])


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
def test_projection_follows_oracle(prob, dtype, tol):
    H = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, 10)["H"]
    Cr = oracle.project(H, prob.T, prob.WtT, prob.C0, 30)
    Cg = nb.project(H, prob.T, prob.WtT, prob.C0, 30, dtype=dtype)
    assert rel(Cg, Cr) <= tol


def test_zero_entries_stay_zero(prob):
    W0 = prob.W0.copy()
    H0 = prob.H0.copy()
    W0[3, 1] = 0
    H0[2, 5] = 0
    got = nb.fit(prob.V, prob.Wt, W0, H0, 5, normalize=False)
    assert got["W"][3, 1] == 0 and got["H"][2, 5] == 0


def test_blas_threads_reports_a_count():
    n, how = nb.blas_threads()
    assert n >= 1 and how


def test_bench_numpy_sample_runs_on_cpu():
    """The benchmark's NumPy CPU-baseline leg on a small problem: both
    dtypes give a positive extrapolated rate and describe their sample."""
    import bench

    prob = synthetic.make_config(0, N=30, K=4, M=2, n_iter=20)
    for dt in (np.float64, np.float32):
        r = bench.cpu_numpy_sample(prob, prob.n_iter, prob.K, dt, seconds=0.2)
        assert r["value"] > 0 and r["threads"] >= 1
        assert r["dtype"] == np.dtype(dt).name and "NumPy iterations" in r["sample"]

