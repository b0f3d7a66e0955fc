"""Pins for the FP64 oracle: each test checks the oracle against something
other than itself -- a closed form, a textbook special case, an invariance of
the update rule, a planted exact factorisation or a brute-force optimum -- so
that a dropped term, a wrong sign or index, or a transposed operand in
oracle/nmf_oracle.c fails at least one of them.

Paper: arXiv:2309.04623, Sec. 2 (Eq. 1-3) for the factorisation, Sec. 4.1 for
target modelling and subtraction.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2309_04623_gb300 import synthetic


def _rng(seed):
    return np.random.default_rng(seed)


def _pos(rng, shape, lo=0.2, hi=1.0):
    return rng.uniform(lo, hi, shape)


# ---------------------------------------------------------------------------
# Eq. 2


def test_chi2_brute_force_loops():
    rng = _rng(0)
    N, P, k = 4, 6, 2
    V = _pos(rng, (N, P)).astype(np.float32)
    Wt = _pos(rng, (N, P)).astype(np.float32)
    W, H = _pos(rng, (N, k)), _pos(rng, (k, P))
    s = 0.0
    for n in range(N):
        for p in range(P):
            r = sum(W[n, i] * H[i, p] for i in range(k))
            s += float(Wt[n, p]) * (float(V[n, p]) - r) ** 2
    assert oracle.chi2(V, Wt, W, H) == pytest.approx(s, rel=1e-14)


def test_chi2_zero_weight_is_missing_data():
    """Sec. 4.1: masked pixels are missing data -- a zero weight removes the
    pixel from the cost whatever its value."""
    rng = _rng(1)
    V = _pos(rng, (5, 7)).astype(np.float32)
    Wt = _pos(rng, (5, 7)).astype(np.float32)
    W, H = _pos(rng, (5, 2)), _pos(rng, (2, 7))
    Wt0 = Wt.copy()
    Wt0[:, 3] = 0.0
    V2 = V.copy()
    V2[:, 3] = 1e6
    assert oracle.chi2(V2, Wt0, W, H) == pytest.approx(oracle.chi2(V, Wt0, W, H), rel=1e-15)


# ---------------------------------------------------------------------------
# Eq. 3: closed forms and special cases


def test_rank1_iteration_is_alternating_weighted_least_squares():
    """For k = 1 the H rule reduces to the exact weighted least-squares
    solution for fixed W (the current H cancels), and the W rule to the one
    for fixed H; one iteration = one H solve then one W solve with the new H."""
    rng = _rng(2)
    N, P = 7, 11
    V = _pos(rng, (N, P)).astype(np.float32)
    Wt = _pos(rng, (N, P), 0.1, 3.0).astype(np.float32)
    W0, H0 = _pos(rng, (N, 1)), _pos(rng, (1, P))
    W, H, _, _ = oracle.iterate(V, Wt, W0, H0, 1)
    v, wt, w = V.astype(float), Wt.astype(float), W0[:, 0]
    h_ls = (wt * w[:, None] * v).sum(0) / (wt * w[:, None] ** 2).sum(0)
    w_ls = (wt * h_ls[None, :] * v).sum(1) / (wt * h_ls[None, :] ** 2).sum(1)
    np.testing.assert_allclose(H[0], h_ls, rtol=1e-14)
    np.testing.assert_allclose(W[:, 0], w_ls, rtol=1e-14)


def test_unit_weights_reduce_to_lee_seung_gram_form():
    """With Wt = 1 the weighted denominators W^T(WH) and (WH)H^T equal the Gram
    forms (W^T W) H and W (H H^T) of the unweighted Lee-Seung rules."""
    rng = _rng(3)
    N, P, k = 9, 13, 3
    V = _pos(rng, (N, P)).astype(np.float32)
    Wt = np.ones((N, P), np.float32)
    W0, H0 = _pos(rng, (N, k)), _pos(rng, (k, P))
    W, H, _, _ = oracle.iterate(V, Wt, W0, H0, 1)
    v = V.astype(float)
    H1 = H0 * (W0.T @ v) / ((W0.T @ W0) @ H0)
    W1 = W0 * (v @ H1.T) / (W0 @ (H1 @ H1.T))
    np.testing.assert_allclose(H, H1, rtol=1e-13)
    np.testing.assert_allclose(W, W1, rtol=1e-13)


def test_diagonal_weights_reweight_rows():
    """Weights constant along each row (Wt[n,p] = a_n) are the same as the
    unweighted problem on sqrt(a_n)-scaled rows for the H update."""
    rng = _rng(4)
    N, P, k = 6, 10, 2
    V = _pos(rng, (N, P)).astype(np.float32)
    a = rng.uniform(0.5, 2.0, N)
    Wt = np.repeat(a[:, None], P, 1).astype(np.float32)
    W0, H0 = _pos(rng, (N, k)), _pos(rng, (k, P))
    _, H, _, _ = oracle.iterate(V, Wt, W0, H0, 1)
    aw = Wt[:, 0].astype(float)
    Ws = W0 * np.sqrt(aw)[:, None]
    Vs = V.astype(float) * np.sqrt(aw)[:, None]
    H1 = H0 * (Ws.T @ Vs) / ((Ws.T @ Ws) @ H0)
    np.testing.assert_allclose(H, H1, rtol=1e-13)


# ---------------------------------------------------------------------------
# invariances


def test_weight_scale_invariance_is_bit_exact():
    """Eq. 3 is a ratio: Wt -> 4 Wt leaves every iterate bit-identical and
    multiplies the cost by exactly 4."""
    rng = _rng(5)
    N, P, k = 8, 15, 3
    V = _pos(rng, (N, P)).astype(np.float32)
    Wt = _pos(rng, (N, P), 0.1, 2.0).astype(np.float32)
    W0, H0 = _pos(rng, (N, k)), _pos(rng, (k, P))
    Wa, Ha, ta, _ = oracle.iterate(V, Wt, W0, H0, 6)
    Wb, Hb, tb, _ = oracle.iterate(V, (4 * Wt).astype(np.float32), W0, H0, 6)
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    assert np.array_equal(4 * ta, tb)


def test_permutation_equivariance():
    rng = _rng(6)
    N, P, k = 8, 14, 3
    V = _pos(rng, (N, P)).astype(np.float32)
    Wt = _pos(rng, (N, P), 0.1, 2.0).astype(np.float32)
    W0, H0 = _pos(rng, (N, k)), _pos(rng, (k, P))
    W, H, _, _ = oracle.iterate(V, Wt, W0, H0, 4)
    pr = rng.permutation(N)
    Wr, Hr, _, _ = oracle.iterate(V[pr], Wt[pr], W0[pr], H0, 4)
    np.testing.assert_allclose(Wr, W[pr], rtol=1e-12)
    np.testing.assert_allclose(Hr, H, rtol=1e-12)
    pc = rng.permutation(P)
    Wc, Hc, _, _ = oracle.iterate(V[:, pc], Wt[:, pc], W0, H0[:, pc], 4)
    np.testing.assert_allclose(Wc, W, rtol=1e-12)
    np.testing.assert_allclose(Hc, H[:, pc], rtol=1e-12)
    # swapping two components swaps the columns of W and the rows of H
    sw = [1, 0, 2]
    Ws, Hs, _, _ = oracle.iterate(V, Wt, W0[:, sw], H0[sw], 4)
    np.testing.assert_allclose(Ws, W[:, sw], rtol=1e-12)
    np.testing.assert_allclose(Hs, H[sw], rtol=1e-12)


def test_exact_zeros_stay_zero():
    rng = _rng(7)
    N, P, k = 10, 16, 3
    V = _pos(rng, (N, P)).astype(np.float32)
    Wt = _pos(rng, (N, P)).astype(np.float32)
    W0, H0 = _pos(rng, (N, k)), _pos(rng, (k, P))
    W0[2, 1] = W0[5, 0] = 0.0
    H0[0, 3] = H0[2, 9] = H0[1, 0] = 0.0
    W, H, _, _ = oracle.iterate(V, Wt, W0, H0, 25)
    assert W[2, 1] == 0.0 and W[5, 0] == 0.0
    assert H[0, 3] == 0.0 and H[2, 9] == 0.0 and H[1, 0] == 0.0
    assert np.all(W[W0 != 0] > 0) and np.all(H[H0 != 0] > 0)


def test_entries_below_the_single_precision_range_become_exact_zeros():
    """Reading (the paper is silent on underflow): an entry of W or H that an
    update leaves below 2^-126 becomes exactly 0 and stays 0.  On a problem
    where one H entry and one W entry decay geometrically (active
    non-negativity constraints at the optimum), the plain double-precision
    run (threshold 0) carries them down to ~1e-98; with the rule they are
    exact zeros, and every other entry equals the plain run's to 1e-12 (an
    entry below 2^-126 adds nothing visible to W H)."""
    rng = _rng(24)
    N, P, k = 10, 16, 3
    V = rng.uniform(0.2, 1.0, (N, P)).astype(np.float32)
    Wt = rng.uniform(0.2, 1.0, (N, P)).astype(np.float32)
    W0, H0 = rng.uniform(0.2, 1.0, (N, k)), rng.uniform(0.2, 1.0, (k, P))
    assert oracle.get_tiny() == 2.0**-126
    with oracle.tiny(0.0):
        Wp, Hp, trp, _ = oracle.iterate(V, Wt, W0, H0, 3000)
    Wf, Hf, trf, _ = oracle.iterate(V, Wt, W0, H0, 3000)
    tiny_h, tiny_w = Hp < 2.0**-126, Wp < 2.0**-126
    assert tiny_h.sum() >= 1 and tiny_w.sum() >= 1
    assert np.all(Hp[tiny_h] > 0) and np.all(Wp[tiny_w] > 0)  # the plain run keeps them positive
    assert np.all(Hf[tiny_h] == 0) and np.all(Wf[tiny_w] == 0)
    np.testing.assert_allclose(Hf[~tiny_h], Hp[~tiny_h], rtol=1e-12)
    np.testing.assert_allclose(Wf[~tiny_w], Wp[~tiny_w], rtol=1e-12)
    np.testing.assert_allclose(trf, trp, rtol=1e-12)
    # a zero reached this way stays zero when the iteration continues
    W2, H2, _, _ = oracle.iterate(V, Wt, Wf, Hf, 200)
    assert np.all(H2[tiny_h] == 0) and np.all(W2[tiny_w] == 0)


def test_epsilon_guards_zero_denominator():
    """A pixel with zero weight in every frame has a zero H denominator; the
    epsilon clamp keeps the update finite (it sends the entry to 0 because
    its numerator is 0 too)."""
    rng = _rng(8)
    N, P, k = 6, 9, 2
    V = _pos(rng, (N, P)).astype(np.float32)
    Wt = _pos(rng, (N, P)).astype(np.float32)
    Wt[:, 4] = 0.0
    W0, H0 = _pos(rng, (N, k)), _pos(rng, (k, P))
    W, H, tr, _ = oracle.iterate(V, Wt, W0, H0, 3)
    assert np.all(np.isfinite(W)) and np.all(np.isfinite(H))
    assert np.all(H[:, 4] == 0.0)


# ---------------------------------------------------------------------------
# convergence behaviour


def test_cost_is_monotone_on_config0():
    """Zhu's weighted multiplicative rules (Eq. 3) never increase Eq. 2."""
    prob = synthetic.make_config(0, n_iter=60, N=30)
    out = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter, trace=True)
    tr = out["chi2_trace"]
    assert np.all(np.isfinite(tr))
    rel_inc = np.diff(tr, axis=1) / tr[:, :-1]
    assert rel_inc.max() <= 1e-12
    # each added component lowers the final cost
    assert np.all(np.diff(out["chi2_hist"]) < 0)


def test_planted_exact_factorisation_is_recovered():
    """V = W* H* with identity sub-blocks (separable, unique up to scale and
    permutation).  Started from a perturbation that keeps the zero pattern,
    the iteration reaches the exact factorisation."""
    rng = _rng(9)
    N, P, k = 12, 20, 3
    Ws = rng.integers(2, 9, (N, k)) / 8.0
    Ws[:k] = np.eye(k)
    Hs = rng.integers(2, 9, (k, P)) / 8.0
    Hs[:, :k] = np.eye(k)
    V = Ws @ Hs
    assert np.array_equal(V.astype(np.float32).astype(float), V)  # exact in float32
    Wt = rng.uniform(0.5, 2.0, (N, P)).astype(np.float32)
    W0 = Ws * (1 + 0.2 * rng.uniform(-1, 1, Ws.shape))
    H0 = Hs * (1 + 0.2 * rng.uniform(-1, 1, Hs.shape))
    W, H, tr, _ = oracle.iterate(V.astype(np.float32), Wt, W0, H0, 20000)
    R = W @ H
    rel = np.sqrt((Wt * (V - R) ** 2).sum() / (Wt * V**2).sum())
    assert rel <= 1e-10
    # factors up to the scale ambiguity W -> W D, H -> D^-1 H
    d = W[:k].diagonal()
    np.testing.assert_allclose(W / d, Ws, atol=1e-8)
    np.testing.assert_allclose(H * d[:, None], Hs, atol=1e-8)


def test_stopping_rule_matches_trace():
    """Sec. 2: iterate until the change from one step to the next reaches a
    set value.  For each tolerance, the first stage stops at the first t >= 2
    whose relative decrease of Eq. 2 is at most tol in the full (tol = 0)
    trace, and keeps the state of that iteration."""
    prob = synthetic.make_config(0, N=20, K=3, n_iter=150)
    # one stage (k = 3) from the random start: a slowly decreasing cost
    fit = lambda tol: oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter, tol=tol, k_start=2, trace=True)
    full = fit(0.0)
    tr = full["chi2_trace"][2]
    dec = (tr[:-1] - tr[1:]) / tr[:-1]
    seen = set()
    for tol in np.geomspace(3e-3, 1e-6, 13):
        expect = next((t + 2 for t in range(len(dec)) if dec[t] <= tol), prob.n_iter)
        stop = fit(tol)
        t1 = int(stop["iters_done"][2])
        assert t1 == expect, tol
        np.testing.assert_array_equal(stop["chi2_trace"][2, :t1], tr[:t1])
        assert stop["chi2_hist"][2] == tr[t1 - 1]
        seen.add(t1)
    assert len(seen) >= 6  # the sweep really exercises different stop points


# ---------------------------------------------------------------------------
# sequential construction and normalisation


def test_first_stage_is_rank_one_fit_and_warm_start():
    rng = _rng(10)
    N, P, K, it = 9, 17, 3, 7
    V = _pos(rng, (N, P)).astype(np.float32)
    Wt = _pos(rng, (N, P)).astype(np.float32)
    W0, H0 = _pos(rng, (N, K)), _pos(rng, (K, P))
    out = oracle.fit(V, Wt, W0, H0, it, normalize=False)
    # stage 1 = `it` rank-1 iterations on the first column / row
    W1, H1, _, _ = oracle.iterate(V, Wt, W0[:, :1], H0[:1], it)
    # stage 2 warm-starts from stage 1 plus the second initial column / row
    W2, H2, _, _ = oracle.iterate(V, Wt, np.hstack([W1, W0[:, 1:2]]), np.vstack([H1, H0[1:2]]), it)
    W3, H3, _, _ = oracle.iterate(V, Wt, np.hstack([W2, W0[:, 2:3]]), np.vstack([H2, H0[2:3]]), it)
    np.testing.assert_allclose(out["W"], W3, rtol=1e-13)
    np.testing.assert_allclose(out["H"], H3, rtol=1e-13)


def test_normalisation_only_rescales():
    """Eq. 3 is equivariant under W -> W D, H -> D^-1 H, so unit-norm H rows
    change rounding only; W H and the costs are unchanged."""
    prob = synthetic.make_config(0, N=25, K=4, n_iter=30)
    a = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter, normalize=True)
    b = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter, normalize=False)
    np.testing.assert_allclose(np.linalg.norm(a["H"], axis=1), 1.0, rtol=1e-14)
    Ra, Rb = a["W"] @ a["H"], b["W"] @ b["H"]
    np.testing.assert_allclose(Ra, Rb, rtol=1e-9, atol=1e-9 * np.abs(Rb).max())
    np.testing.assert_allclose(a["chi2_hist"], b["chi2_hist"], rtol=1e-11)


def test_k_start_resumes():
    prob = synthetic.make_config(0, N=15, K=4, n_iter=10)
    full = oracle.fit(prob.V, prob.Wt, prob.W0, prob.H0, prob.n_iter)
    two = oracle.fit(prob.V, prob.Wt, prob.W0[:, :2], prob.H0[:2], prob.n_iter)
    W = np.hstack([two["W"], prob.W0[:, 2:]])
    H = np.vstack([two["H"], prob.H0[2:]])
    rest = oracle.fit(prob.V, prob.Wt, W, H, prob.n_iter, k_start=2)
    np.testing.assert_allclose(rest["W"], full["W"], rtol=1e-12)
    np.testing.assert_allclose(rest["H"], full["H"], rtol=1e-12)
    np.testing.assert_allclose(rest["chi2_hist"][2:], full["chi2_hist"][2:], rtol=1e-12)


# ---------------------------------------------------------------------------
# projection and subtraction (Sec. 4.1)


def _brute_wnnls(H, t, w):
    """min_c>=0 sum_p w_p (t_p - c.H_p)^2 by trying every support."""
    K = H.shape[0]
    sw = np.sqrt(w)
    best = (np.inf, None)
    for r in range(K + 1):
        for S in itertools.combinations(range(K), r):
            c = np.zeros(K)
            if S:
                cs, *_ = np.linalg.lstsq((H[list(S)] * sw).T, t * sw, rcond=None)
                if np.any(cs < 0):
                    continue
                c[list(S)] = cs
            f = float((w * (t - c @ H) ** 2).sum())
            if f < best[0]:
                best = (f, c)
    return best


@pytest.mark.parametrize("case", ["interior", "active"])
def test_projection_matches_bruteforce_nnls(case):
    rng = _rng(11)
    K, P = 5, 30
    H = rng.uniform(0.1, 1.0, (K, P))
    ct = rng.uniform(0.5, 2.0, K)
    t = ct @ H + 0.01 * rng.standard_normal(P)
    if case == "active":
        t = t - 1.5 * H[2] - 1.5 * H[4]
    t = np.maximum(t, 0).astype(np.float32)
    w = rng.uniform(0.5, 2.0, P).astype(np.float32)
    fb, cb = _brute_wnnls(H, t.astype(float), w.astype(float))
    C = oracle.project(H, t[None], w[None], np.ones((1, K)), 20000)
    c = C[0]
    f = float((w * (t - c @ H) ** 2).sum())
    assert abs(f - fb) <= 1e-10 * fb
    np.testing.assert_allclose(c, cb, atol=1e-8)
    # KKT: c >= 0, gradient >= 0 on the active set, c * grad = 0
    g = -2.0 * ((w * (t - c @ H)) @ H.T)
    assert np.all(c >= 0)
    assert np.all(g >= -1e-8)
    assert np.all(np.abs(c * g) <= 1e-8)
    if case == "active":
        assert (cb == 0).sum() >= 1


def test_projection_rows_independent():
    """Each science frame is modelled on its own (Sec. 4.1)."""
    rng = _rng(12)
    K, P, M = 3, 25, 4
    H = rng.uniform(0.1, 1.0, (K, P))
    T = rng.uniform(0.0, 2.0, (M, P)).astype(np.float32)
    WtT = rng.uniform(0.5, 2.0, (M, P)).astype(np.float32)
    C0 = rng.uniform(0.1, 1.0, (M, K))
    C = oracle.project(H, T, WtT, C0, 50)
    for m in range(M):
        cm = oracle.project(H, T[m:m + 1], WtT[m:m + 1], C0[m:m + 1], 50)
        np.testing.assert_array_equal(cm[0], C[m])


def test_projection_equals_w_step_of_the_fit():
    """Target modelling is Eq. 3's W rule with H held fixed: one projection
    iteration equals the W half of one fit iteration when H does not move
    (H-step numerator = denominator is forced by fitting V = W0 H0 exactly)."""
    rng = _rng(13)
    M, P, K = 5, 12, 2
    H = rng.uniform(0.1, 1.0, (K, P))
    T = rng.uniform(0.1, 2.0, (M, P)).astype(np.float32)
    WtT = rng.uniform(0.5, 2.0, (M, P)).astype(np.float32)
    C0 = rng.uniform(0.1, 1.0, (M, K))
    C = oracle.project(H, T, WtT, C0, 1)
    A = WtT.astype(float) * T.astype(float)
    D = WtT.astype(float) * (C0 @ H)
    expect = C0 * (A @ H.T) / (D @ H.T)
    np.testing.assert_allclose(C, expect, rtol=1e-14)


def test_subtract_is_target_minus_model():
    rng = _rng(14)
    M, P, K = 3, 40, 4
    T = rng.uniform(0, 10, (M, P)).astype(np.float32)
    C = rng.uniform(0, 1, (M, K))
    H = rng.uniform(0, 1, (K, P))
    R = oracle.subtract(T, C, H)
    model = C @ H
    np.testing.assert_allclose(R + model, T.astype(float), rtol=0, atol=4 * np.spacing(np.abs(T).max()))
    f = np.array([0.5, 1.0, 2.0])
    Rf = oracle.subtract(T, C, H, factor=f)
    np.testing.assert_allclose(Rf + f[:, None] * model, T.astype(float), rtol=0,
                               atol=4 * np.spacing(np.abs(T).max()))


def test_subtract_with_exact_model_is_zero():
    """A science frame that lies exactly in the span of H with non-negative
    coefficients is fully removed by projection + subtraction."""
    H = np.array([[1.0, 0.0, 0.5, 0.25], [0.0, 1.0, 0.5, 0.75]])
    c = np.array([[2.0, 3.0]])
    T = (c @ H).astype(np.float32)
    WtT = np.ones_like(T)
    C = oracle.project(H, T, WtT, np.ones((1, 2)), 5000)
    R = oracle.subtract(T, C, H)
    assert np.abs(R).max() <= 1e-10


# ---------------------------------------------------------------------------
# reference selection (Sec. 4.1): the closest library frames to each target


def _sel_inputs(seed, M=3, N=25, P=60):
    rng = _rng(seed)
    T = rng.uniform(0, 10, (M, P)).astype(np.float32)
    V = rng.uniform(0, 10, (N, P)).astype(np.float32)
    WtT = rng.uniform(0.1, 2.0, (M, P)).astype(np.float32)
    return T, WtT, V


def test_distances_with_unit_weights_are_squared_euclidean():
    """Unit weights reduce the distance to the squared Euclidean norm, which
    scipy computes independently."""
    scipy_dist = pytest.importorskip("scipy.spatial.distance")
    T, _, V = _sel_inputs(31)
    D = oracle.distances(T, np.ones_like(T), V)
    ref = scipy_dist.cdist(T.astype(np.float64), V.astype(np.float64), "sqeuclidean")
    np.testing.assert_allclose(D, ref, rtol=1e-12)


def test_distance_is_the_nmf_cost_of_one_frame():
    """D[m, n] is Eq. 2 for modelling target frame m by library frame n with
    coefficient 1 (the paper ranks frames by the norm that NMF minimises): the
    same number as the oracle's cost function."""
    T, WtT, V = _sel_inputs(32)
    D = oracle.distances(T, WtT, V)
    for m, n in ((0, 0), (1, 7), (2, 24)):
        c = oracle.chi2(T[m:m + 1], WtT[m:m + 1], np.ones((1, 1)), V[n:n + 1].astype(np.float64))
        assert abs(D[m, n] - c) <= 1e-12 * c


def test_distance_weight_scale_is_exact_and_masked_pixels_are_ignored():
    T, WtT, V = _sel_inputs(33)
    D = oracle.distances(T, WtT, V)
    assert np.array_equal(oracle.distances(T, 4 * WtT, V), 4 * D)
    W0 = WtT.copy()
    W0[:, 10:20] = 0.0
    V2 = V.copy()
    V2[:, 10:20] += 100.0  # changes only where every target weight is 0
    assert np.array_equal(oracle.distances(T, W0, V2), oracle.distances(T, W0, V))


def test_identical_library_frame_is_selected_first():
    T, WtT, V = _sel_inputs(34)
    V[7] = T[0]
    V[3] = T[2]
    D = oracle.distances(T, WtT, V)
    assert D[0, 7] == 0.0 and D[2, 3] == 0.0
    idx = oracle.select(D, 5)
    assert idx[0, 0] == 7 and idx[2, 0] == 3


def test_selection_is_the_stable_order_of_the_distances():
    """The n_keep closest frames, closest first, equal distances in library
    order: numpy's stable argsort gives the same list (ties planted)."""
    rng = _rng(35)
    D = rng.integers(0, 12, (4, 40)).astype(np.float64)  # many exact ties
    for n_keep in (1, 7, 40):
        ref = np.argsort(D, axis=1, kind="stable")[:, :n_keep]
        assert np.array_equal(oracle.select(D, n_keep), ref)


# ---------------------------------------------------------------------------
# North-up rotation and stacking of the subtracted frames (Sec. 4.1, 4.2)


def test_rotation_by_zero_is_the_identity_up_to_the_last_row_and_column():
    """Angle 0 copies every pixel, including the last row and column (whose
    right/lower neighbours carry zero weight and are not needed)."""
    rng = _rng(40)
    img = rng.normal(0, 1, (2, 23, 31)).astype(np.float32)
    img[0, 5, 7] = np.nan
    out = oracle.rotate(img, [0.0, 0.0], (15.0, 11.0))
    assert np.array_equal(np.isnan(out), np.isnan(img))
    assert np.array_equal(out[~np.isnan(out)], img[~np.isnan(img)].astype(np.float64))


@pytest.mark.parametrize("turns", [1, 2, 3])
def test_quarter_turns_are_numpy_rot90(turns):
    """About the centre pixel of an odd square frame, 90-degree multiples move
    pixels exactly: the content turns from +x towards +y (counter-clockwise
    with the first row drawn at the bottom), i.e. numpy's rot90 with k = -turns."""
    rng = _rng(41 + turns)
    img = rng.normal(0, 1, (1, 17, 17)).astype(np.float32)
    out = oracle.rotate(img, [90.0 * turns], (8.0, 8.0))
    assert np.array_equal(out[0], np.rot90(img[0], -turns).astype(np.float64))
    pt = np.zeros((1, 17, 17), np.float32)
    pt[0, 8, 8 + 5] = 1.0  # on the +x axis, 5 px from the centre
    moved = oracle.rotate(pt, [90.0], (8.0, 8.0))[0]
    assert moved[8 + 5, 8] == 1.0 and moved.sum() == 1.0  # now on the +y axis


def _exact_source(shape, theta_deg, cx, cy):
    ny, nx = shape
    th = np.deg2rad(theta_deg)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    xs = cx + np.cos(th) * (x - cx) + np.sin(th) * (y - cy)
    ys = cy + np.cos(th) * (y - cy) - np.sin(th) * (x - cx)
    return xs, ys


@pytest.mark.parametrize("theta", [17.0, -33.25, 123.4, 251.0])
def test_bilinear_rotation_is_exact_on_affine_images(theta):
    """Bilinear interpolation reproduces an affine function exactly, so the
    rotated frame of a + b x + e y is a + b xs + e ys at the exactly rotated
    position (up to the float rounding of that position); the frame is NaN
    exactly where that position leaves the frame (checked away from the edge)."""
    ny, nx, cx, cy = 40, 52, 24.3, 18.7
    a, b, e = 3.0, 0.75, -1.25
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    img = (a + b * x + e * y).astype(np.float32)
    out = oracle.rotate(img, [theta], (cx, cy))[0]
    xs, ys = _exact_source((ny, nx), theta, cx, cy)
    inside = (xs > 1e-3) & (xs < nx - 1 - 1e-3) & (ys > 1e-3) & (ys < ny - 1 - 1e-3)
    outside = (xs < -1e-3) | (xs > nx - 1 + 1e-3) | (ys < -1e-3) | (ys > ny - 1 + 1e-3)
    assert inside.sum() > 500 and outside.sum() > 100
    assert not np.isnan(out[inside]).any() and np.isnan(out[outside]).all()
    np.testing.assert_allclose(out[inside], (a + b * xs + e * ys)[inside], rtol=0, atol=2e-4)


@pytest.mark.parametrize("theta", [9.5, -71.0, 200.0])
def test_rotation_matches_scipy_linear_interpolation(theta):
    """scipy.ndimage.map_coordinates(order=1) is an independent bilinear
    interpolator: inside the frame the two agree (to the float rounding of
    the source position)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = _rng(45)
    ny, nx, cx, cy = 29, 37, 18.0, 14.5
    img = rng.uniform(0, 1, (ny, nx)).astype(np.float32)
    out = oracle.rotate(img, [theta], (cx, cy))[0]
    xs, ys = _exact_source((ny, nx), theta, cx, cy)
    ref = ndimage.map_coordinates(img.astype(np.float64), [ys, xs], order=1, mode="nearest")
    ok = ~np.isnan(out)
    assert ok.sum() > 300
    np.testing.assert_allclose(out[ok], ref[ok], rtol=0, atol=1e-4)


def test_missing_pixels_by_nan_or_by_mask_are_the_same():
    """A pixel flagged in `valid` and a NaN pixel are the same missing datum;
    an output that needs it (with nonzero weight) is NaN, the others are not
    affected."""
    rng = _rng(46)
    img = rng.uniform(0, 1, (3, 21, 25)).astype(np.float32)
    valid = np.ones((21, 25), np.uint8)
    valid[10:12, 4:9] = 0
    valid[0, :] = 0
    nan_img = img.copy()
    nan_img[:, valid == 0] = np.nan
    ang = [0.0, 31.0, -140.0]
    a = oracle.rotate(img, ang, (12.0, 10.0), valid=valid)
    b = oracle.rotate(nan_img, ang, (12.0, 10.0))
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])
    full = oracle.rotate(img, ang, (12.0, 10.0))
    keep = ~np.isnan(a)
    assert np.array_equal(a[keep], full[keep])
    assert np.isnan(a).sum() > np.isnan(full).sum()


@pytest.mark.parametrize("method", ["mean", "median"])
def test_combine_is_numpy_nanmean_nanmedian(method):
    """Stacking ignores missing frames per pixel; numpy's nanmean/nanmedian
    are the textbook definitions (even counts: mean of the two middle values).
    Pixels no frame covers are NaN with count 0."""
    import warnings
    rng = _rng(47)
    for F in (1, 2, 5, 8):
        fr = rng.normal(0, 1, (F, 13, 11))
        fr[rng.uniform(size=fr.shape) < 0.3] = np.nan
        fr[:, 0, 0] = np.nan
        out, cnt = oracle.combine(fr, method)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", RuntimeWarning)
            ref = np.nanmean(fr, axis=0) if method == "mean" else np.nanmedian(fr, axis=0)
        assert np.array_equal(cnt, (~np.isnan(fr)).sum(axis=0))
        assert np.array_equal(np.isnan(out), np.isnan(ref)) and np.isnan(out[0, 0]) and cnt[0, 0] == 0
        np.testing.assert_allclose(out[~np.isnan(out)], ref[~np.isnan(ref)], rtol=1e-15, atol=1e-15)
