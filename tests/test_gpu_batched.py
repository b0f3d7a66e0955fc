"""GPU checks of the batched form (nmf_fit_batched): many independent
reductions of uneven N, P, K, frame counts and precisions in one call, each
on its own concurrent branch.  Every problem's result must equal, bit for
bit, the separate nmf_fit_basis / nmf_project_target / nmf_subtract calls on
it (same kernels, same fixed-order reductions), with and without graph
recording; one FP32 member is also checked against the FP64 oracle at the
FP32 bar (<= 1e-5 relative Frobenius error)."""
import zlib

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


def np_(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# (name, N, P, K, M, iters, precision, polish): ragged sizes, the FP32 form
# and both tensor-core forms, a fit-only member, K above 64, K == N
MEMBERS = [
    ("fp32_small", 40, 1500, 3, 2, 12, "fp32", 0),
    ("bf16_k8", 70, 3001, 8, 3, 10, "bf16", 5),
    ("fp32_fit_only", 90, 2200, 70, 0, 2, "fp32", 0),
    ("bf16_k1", 33, 777, 1, 1, 6, "bf16", 2),
    ("fp32_k_eq_n", 5, 700, 5, 4, 8, "fp32", 0),
    ("bf16_two_tiles", 150, 5000, 20, 20, 4, "bf16", 3),
    ("bf16_wide", 120, 2000, 70, 2, 2, "bf16", 2),
    ("bf16w32_k20", 150, 5000, 20, 5, 4, "bf16w32", 3),
    ("bf16w32_wide", 120, 2000, 70, 2, 2, "bf16w32", 2),
]


def _batch():
    out = []
    for name, N, P, K, M, it, prec, pol in MEMBERS:
        pr = synthetic.make_problem(zlib.crc32(name.encode()), N, P, K, M=max(M, 1), n_iter=it)
        d = dict(V=pr.V, Wt=pr.Wt, W0=pr.W0, H0=pr.H0, iters_per_stage=it, proj_iters=it + 3, precision=prec,
                 polish_iters=pol)
        if M:
            d.update(T=pr.T, WtT=pr.WtT, C0=pr.C0)
        out.append(d)
    return out


def _separate(nmf, d):
    W, H, chi2, done = nmf.fit_basis(d["V"], d["Wt"], d["W0"], d["H0"], d["iters_per_stage"],
                                     precision=d["precision"], polish_iters=d["polish_iters"])
    r = dict(W=W, H=H, chi2_hist=chi2, iters_done=done)
    if "T" in d:
        C = nmf.project_target(H, d["T"], d["WtT"], d["C0"], d["proj_iters"], precision=d["precision"],
                               polish_iters=d["polish_iters"])
        r.update(C=C, R=nmf.subtract(d["T"], C, H))
    return r


def _assert_same(got, want, name):
    assert set(got) == set(want), name
    for key in want:
        assert torch.equal(got[key], want[key]), (name, key)


def test_batched_equals_separate_calls(nmf):
    batch = _batch()
    got = nmf.fit_batched(batch, 0, 0)
    torch.cuda.synchronize()
    for d, g, m in zip(batch, got, MEMBERS):
        _assert_same(g, _separate(nmf, d), m[0])
    # a second call (new buffers, so a second recording): the same results
    again = nmf.fit_batched(batch, 0, 0)
    torch.cuda.synchronize()
    for g, a, m in zip(got, again, MEMBERS):
        _assert_same(a, g, m[0])


def test_batched_direct_launches_match(nmf, monkeypatch):
    batch = _batch()
    with_graph = nmf.fit_batched(batch, 0, 0)
    torch.cuda.synchronize()
    monkeypatch.setenv("NMF_NO_GRAPH", "1")
    direct = nmf.fit_batched(batch, 0, 0)
    torch.cuda.synchronize()
    for a, b, m in zip(with_graph, direct, MEMBERS):
        _assert_same(b, a, m[0])


def test_batched_fp32_member_matches_oracle(nmf):
    batch = _batch()
    got = nmf.fit_batched(batch, 0, 0)
    torch.cuda.synchronize()
    d, g = batch[0], got[0]
    ref = oracle.fit(d["V"], d["Wt"], d["W0"], d["H0"], d["iters_per_stage"])
    assert rel(np_(g["W"]), ref["W"]) <= 1e-5
    assert rel(np_(g["H"]), ref["H"]) <= 1e-5
    assert np.all(np.abs(np_(g["chi2_hist"]) - ref["chi2_hist"]) <= 1e-4 * ref["chi2_hist"])
    Cref = oracle.project(ref["H"], d["T"], d["WtT"], d["C0"], d["proj_iters"])
    Rref = oracle.subtract(d["T"], Cref, ref["H"])
    assert rel(np_(g["C"]), Cref) <= 1e-5
    assert rel(np_(g["R"]), Rref) <= 1e-4


def test_batched_status_is_per_problem(nmf):
    """A non-finite input in one member is reported for that member only; the
    others complete with their normal results."""
    batch = _batch()[:3]
    V = batch[0]["V"].copy()
    V[3, 17] = np.nan
    batch[0]["V"] = V
    with pytest.raises(nmf.NmfError) as ei:
        nmf.fit_batched(batch, 0, 0)
    assert ei.value.code == nmf.NMF_EDATA
    assert ei.value.statuses == [nmf.NMF_EDATA, nmf.NMF_OK, nmf.NMF_OK]
    got = nmf.fit_batched(batch, 0, 0, check_status=False)
    torch.cuda.synchronize()
    for i in (1, 2):
        _assert_same(got[i], _separate(nmf, batch[i]), MEMBERS[i][0])
