"""GPU parity: the CUDA path (through the C-ABI, via the ctypes binding)
against the FP64 oracle on the same seeded inputs and initial factors.

Tolerances (plain FP32 path): relative Frobenius error <= 1e-5 on W and H
after 20 iterations per stage; <= 1e-4 on the final cost Eq. 2 and on the
residual images after full-length runs.
"""
import zlib
from types import SimpleNamespace

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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def np_(t):
    return t.detach().cpu().numpy()


# (name, N, P, K, k_start, iters): every component-tile bucket (8/16/32/64/128),
# ragged N and P (not multiples of any tile), and tiny degenerate shapes.
FIT_CASES = [
    ("config0_20it", 50, 2712, 5, 0, 20),
    ("ragged_k3", 37, 1001, 3, 0, 20),
    ("k8_exact", 40, 777, 8, 6, 20),
    ("k9_bucket16", 45, 1537, 9, 7, 20),
    ("k17_bucket32", 61, 2049, 17, 15, 20),
    ("k33_bucket64", 70, 1111, 33, 31, 20),
    ("k65_bucket128", 97, 913, 65, 63, 20),
    ("k128_max", 130, 700, 128, 127, 10),
    ("N1_K1", 1, 333, 1, 0, 20),
    ("P1_K1", 9, 1, 1, 0, 20),
    ("rows_gt_chunk", 301, 640, 4, 2, 20),
]


def _problem(name, N, P, K):
    """Synthetic coronagraphic data for the case; uniform data when P is too
    small for an annular mask."""
    if name.startswith("config0"):
        return synthetic.make_config(0, N=N, K=K, n_iter=20)
    if P >= 64:
        return synthetic.make_problem(zlib.crc32(name.encode()), N, P, K, M=2, n_iter=20)
    rng = np.random.default_rng(N * 1000 + P)
    return SimpleNamespace(
        V=rng.uniform(0.0, 5.0, (N, P)).astype(np.float32),
        Wt=rng.uniform(0.2, 2.0, (N, P)).astype(np.float32),
        W0=rng.uniform(0.1, 1.0, (N, K)).astype(np.float32),
        H0=rng.uniform(0.1, 1.0, (K, P)).astype(np.float32),
    )


@pytest.mark.parametrize("case", FIT_CASES, ids=[c[0] for c in FIT_CASES])
def test_fit_matches_oracle(nmf, case):
    name, N, P, K, k_start, iters = case
    prob = _problem(name, N, P, K)
    W, H, chi2, done = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, iters, k_start=k_start)
    torch.cuda.synchronize()
    ref = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, iters, k_start=k_start)
    assert rel(np_(W), ref["W"]) <= 1e-5
    assert rel(np_(H), ref["H"]) <= 1e-5
    c = np_(chi2)[k_start:]
    # relative tolerance, with an absolute floor at FP32 resolution of the
    # cost scale sum Wt V^2 (an exact fit, e.g. N = K = 1, has cost ~0)
    scale = float((prob.Wt.astype(np.float64) * prob.V.astype(np.float64) ** 2).sum())
    np.testing.assert_allclose(c, ref["chi2_hist"][k_start:], rtol=1e-5, atol=1e-7 * scale)
    assert np.all(np_(done)[k_start:] == iters)
    # normalisation: unit rows for every fitted stage
    np.testing.assert_allclose(np.linalg.norm(np_(H)[:K].astype(np.float64), axis=1), 1.0, rtol=1e-5)


def test_fit_config0_full_length(nmf):
    """The oracle-size workload end to end: K=5 built sequentially, 200
    iterations each, then projection and subtraction of the science frame."""
    prob = synthetic.make_config(0)
    W, H, chi2, done = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter)
    C = nmf.project_target(H, prob.T, prob.WtT, prob.C0, prob.n_iter)
    R = nmf.subtract(prob.T, C, H)
    torch.cuda.synchronize()
    ref = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter)
    np.testing.assert_allclose(np_(chi2), ref["chi2_hist"], rtol=1e-4)
    assert np.all(np_(done) == prob.n_iter)
    Cref = oracle.project(ref["H"], prob.T, prob.WtT, prob.C0, prob.n_iter)
    Rref = oracle.subtract(prob.T, Cref, ref["H"])
    assert rel(np_(R), Rref) <= 1e-4
    # the same residual from the oracle projection of the GPU basis
    Hg = np_(H).astype(np.float64)
    Cg = oracle.project(Hg, prob.T, prob.WtT, prob.C0, prob.n_iter)
    assert rel(np_(C), Cg) <= 1e-5
    assert rel(np_(R), oracle.subtract(prob.T, Cg, Hg)) <= 1e-5


def test_stop_rule_matches_oracle(nmf):
    """Sec. 2 stopping rule evaluated on the device: the stage stops at the
    same iteration as the oracle.  tol is placed midway (geometrically)
    between two consecutive relative decreases so that FP32 rounding cannot
    flip the comparison."""
    prob = synthetic.make_config(0, N=30, K=2, n_iter=120)
    full = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter, k_start=1, trace=True)
    tr = full["chi2_trace"][1]
    dec = (tr[:-1] - tr[1:]) / tr[:-1]
    t0 = next(t for t in range(20, len(dec) - 1) if dec[t] > 0 and dec[t + 1] > 0 and dec[t] / dec[t + 1] > 1.02
              and np.all(dec[:t] > dec[t]))
    tol = float(np.sqrt(dec[t0] * dec[t0 + 1]))
    ref = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter, tol=tol, k_start=1)
    W, H, chi2, done = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter, tol=tol, k_start=1)
    torch.cuda.synchronize()
    # dec[i] is the relative decrease tested after iteration i + 2; dec[t0 + 1]
    # is the first one below tol
    assert int(ref["iters_done"][1]) == t0 + 3
    assert int(np_(done)[1]) == int(ref["iters_done"][1])
    assert rel(np_(W), ref["W"]) <= 1e-5 and rel(np_(H), ref["H"]) <= 1e-5
    np.testing.assert_allclose(np_(chi2)[1], ref["chi2_hist"][1], rtol=1e-5)


@pytest.mark.parametrize("K", [1, 5, 20, 40, 100])
def test_projection_matches_oracle(nmf, K):
    rng = np.random.default_rng(K)
    M, P = 7, 2049
    H = rng.uniform(0.0, 1.0, (K, P)).astype(np.float32)
    H[:, rng.random(P) < 0.05] = 0.0
    T = rng.uniform(0.0, 50.0, (M, P)).astype(np.float32)
    WtT = rng.uniform(0.01, 1.0, (M, P)).astype(np.float32)
    C0 = rng.uniform(0.1, 1.0, (M, K)).astype(np.float32)
    C0[0, 0] = 0.0  # an exact zero stays zero
    C = nmf.project_target(H, T, WtT, C0, 20)
    torch.cuda.synchronize()
    Cref = oracle.project(H.astype(np.float64), T, WtT, C0, 20)
    assert rel(np_(C), Cref) <= 1e-5
    assert np_(C)[0, 0] == 0.0


def test_projection_zero_iterations_is_identity(nmf):
    rng = np.random.default_rng(3)
    H = rng.uniform(0, 1, (4, 300)).astype(np.float32)
    T = rng.uniform(0, 1, (3, 300)).astype(np.float32)
    C0 = rng.uniform(0, 1, (3, 4)).astype(np.float32)
    C = nmf.project_target(H, T, np.ones_like(T), C0, 0)
    assert np.array_equal(np_(C), C0)


@pytest.mark.parametrize("with_factor", [False, True])
def test_subtract_and_scatter(nmf, with_factor):
    prob = synthetic.make_config(0, M=3)
    rng = np.random.default_rng(5)
    K = 6
    C = rng.uniform(0, 50, (prob.M, K)).astype(np.float32)
    H = rng.uniform(0, 1, (K, prob.P)).astype(np.float32)
    f = rng.uniform(0.5, 1.5, prob.M).astype(np.float32) if with_factor else None
    npix = prob.img_shape[0] * prob.img_shape[1]
    R, img = nmf.subtract(prob.T, C, H, factor=f, scatter_idx=prob.pix_idx, img_pixels=npix)
    torch.cuda.synchronize()
    Rref = oracle.subtract(prob.T, C.astype(np.float64), H.astype(np.float64),
                           factor=None if f is None else f.astype(np.float64))
    assert rel(np_(R), Rref) <= 1e-6
    im = np_(img)
    assert np.array_equal(im[:, prob.pix_idx], np_(R))
    mask = np.ones(npix, bool)
    mask[prob.pix_idx] = False
    assert np.all(im[:, mask] == 0.0)


def test_zero_entries_stay_zero(nmf):
    prob = synthetic.make_config(0, N=30, K=3, n_iter=15)
    W0, H0 = prob.W0.copy(), prob.H0.copy()
    W0[4, 1] = 0.0
    H0[2, 100:140] = 0.0
    W, H, _, _ = nmf.fit_basis(prob.V, prob.Wt, W0, H0, 15, normalize=False)
    assert np_(W)[4, 1] == 0.0
    assert np.all(np_(H)[2, 100:140] == 0.0)


@pytest.mark.parametrize("bad", ["negative_V", "nan_Wt", "inf_H0"])
def test_invalid_data_sets_device_status(nmf, bad):
    prob = synthetic.make_config(0, N=20, K=2, n_iter=3)
    V, Wt, H0 = prob.V.copy(), prob.Wt.copy(), prob.H0.copy()
    if bad == "negative_V":
        V[3, 7] = -1.0
    elif bad == "nan_Wt":
        Wt[1, 2] = np.nan
    else:
        H0[0, 5] = np.inf
    with pytest.raises(nmf.NmfError) as ei:
        nmf.fit_basis(V, Wt, prob.W0, H0, 3)
    assert ei.value.code == nmf.NMF_EDATA


def test_deterministic_and_host_entry_matches(nmf):
    """Fixed-order reductions: two runs are bit-identical, and the host-buffer
    entry point (copies inside) returns exactly the device path's result."""
    prob = synthetic.make_config(0, N=50, K=4, M=2, n_iter=30)
    a = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, 30)
    b = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, 30)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    C = nmf.project_target(a[1], prob.T, prob.WtT, prob.C0, 30)
    R = nmf.subtract(prob.T, C, a[1])
    out = nmf.reduce_host(prob.V, prob.Wt, prob.W0, prob.H0, prob.T, prob.WtT, prob.C0, 30, 30)
    assert np.array_equal(out["W"], np_(a[0]))
    assert np.array_equal(out["H"], np_(a[1]))
    assert np.array_equal(out["chi2_hist"], np_(a[2]))
    assert np.array_equal(out["C"], np_(C))
    assert np.array_equal(out["R"], np_(R))


# ---------------------------------------------------------------------------
# full-size STIS-shaped workload (N=300, P=49343, K=30), the benchmark's shape


@pytest.fixture(scope="module")
def config1():
    return synthetic.make_config(1)


def test_full_size_single_iteration(nmf, config1):
    """One iteration at the full size and k = K = 30 from the random start,
    element by element against the oracle."""
    prob = config1
    K = prob.K
    W, H, chi2, done = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, 1, k_start=K - 1, normalize=False)
    torch.cuda.synchronize()
    Wr, Hr, tr, _ = oracle.iterate(prob.V, prob.Wt, prob.W0, prob.H0, 1)
    assert rel(np_(W), Wr) <= 1e-5
    assert rel(np_(H), Hr) <= 1e-5
    np.testing.assert_allclose(np_(chi2)[K - 1], tr[0], rtol=1e-5)


def test_full_size_bench_configuration(nmf, config1):
    """The benchmarked launch configuration (K = 30 stages x 500 iterations,
    50 frames projected and subtracted), checked through properties the
    oracle can evaluate at this size: the reported costs equal Eq. 2
    recomputed in FP64 from the returned factors, costs fall with every added
    component, rows are unit norm, and sampled science frames match the
    oracle's projection on the same basis."""
    prob = config1
    W, H, chi2, done = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter)
    C = nmf.project_target(H, prob.T, prob.WtT, prob.C0, prob.n_iter)
    R = nmf.subtract(prob.T, C, H)
    torch.cuda.synchronize()
    Wg, Hg = np_(W).astype(np.float64), np_(H).astype(np.float64)
    assert np.all(np_(done) == prob.n_iter)
    c = np_(chi2)
    assert np.all(np.diff(c) < 0)
    np.testing.assert_allclose(c[-1], oracle.chi2(prob.V, prob.Wt, Wg, Hg), rtol=1e-5)
    np.testing.assert_allclose(np.linalg.norm(Hg, axis=1), 1.0, rtol=1e-5)
    sample = [0, 17, 49]
    Cs = oracle.project(Hg, prob.T[sample], prob.WtT[sample], prob.C0[sample], prob.n_iter)
    assert rel(np_(C)[sample], Cs) <= 1e-4
    Rs = oracle.subtract(prob.T[sample], Cs, Hg)
    assert rel(np_(R)[sample], Rs) <= 1e-4


@pytest.mark.parametrize("precision,tol,polish", [("fp32", 0.0, 0), ("fp32", 3e-4, 0), ("bf16", 0.0, 5),
                                                  ("bf16", 3e-4, 5)])
def test_graph_and_direct_launches_agree(nmf, monkeypatch, precision, tol, polish):
    """A call is recorded into a CUDA graph whose per-stage iteration loops are
    device-side WHILE nodes; with NMF_NO_GRAPH set the same kernels are
    launched one by one.  Both orders of the same kernels give identical
    results, with and without an early stop."""
    prob = synthetic.make_config(0, N=60, K=4, M=3, n_iter=40)
    kw = dict(tol=tol, precision=precision, polish_iters=polish)
    g = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, 40, **kw)
    g2 = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, 40, **kw)  # cached graph replay
    Cg = nmf.project_target(g[1], prob.T, prob.WtT, prob.C0, 30, precision=precision, polish_iters=polish)
    monkeypatch.setenv("NMF_NO_GRAPH", "1")
    d = nmf.fit_basis(prob.V, prob.Wt, prob.W0, prob.H0, 40, **kw)
    Cd = nmf.project_target(d[1], prob.T, prob.WtT, prob.C0, 30, precision=precision, polish_iters=polish)
    for x, y, z in zip(g, g2, d):
        assert torch.equal(x, y)
        assert torch.equal(x, z)
    assert torch.equal(Cg, Cd)
    if tol > 0:
        assert np.all(np_(g[3]) <= 40)
