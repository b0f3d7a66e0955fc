"""The seeded synthetic stand-ins for the paper's data (no method arithmetic):
the benchmark's workload shapes, determinism, and the value properties the
library validates (non-negative finite data, positive weights, U(0,1)
starts)."""
import numpy as np
import pytest

from paper_2309_04623_gb300 import synthetic


def _check_problem(p, N, P, K, M, shape):
    assert p.V.shape == (N, P) and p.Wt.shape == (N, P)
    assert p.T.shape == (M, P) and p.WtT.shape == (M, P)
    assert p.W0.shape == (N, K) and p.H0.shape == (K, P) and p.C0.shape == (M, K)
    assert p.img_shape == shape and p.pix_idx.shape == (P,)
    assert np.all(np.diff(p.pix_idx) > 0) and 0 <= p.pix_idx[0] and p.pix_idx[-1] < shape[0] * shape[1]
    for a in (p.V, p.Wt, p.T, p.WtT, p.W0, p.H0, p.C0):
        assert a.dtype == np.float32 and np.all(np.isfinite(a))
    assert p.V.min() >= 0 and p.T.min() >= 0
    assert p.Wt.min() > 0 and p.WtT.min() > 0
    for a in (p.W0, p.H0, p.C0):  # U(0,1) in float64 rounded to float32: (0, 1], no exact zero
        assert 0 < a.min() and a.max() <= 1


def test_oracle_size_workload():
    p = synthetic.make_config(0)
    _check_problem(p, 50, 2712, 5, 1, (64, 64))
    assert p.n_iter == 200


def test_stis_shaped_workload():
    p = synthetic.make_config(1)
    _check_problem(p, 300, 49343, 30, 50, (256, 256))
    assert p.n_iter == 500


def test_miri_shaped_mask_pixel_count():
    # the workload itself is large to build; its mask fixes P
    keep = synthetic.miri_4qpm_mask((224, 288), (112.0, 144.0))
    assert keep.shape == (224, 288) and int(keep.sum()) == 62961


def test_workloads_are_seeded():
    a, b = synthetic.make_config(0), synthetic.make_config(0)
    for x, y in ((a.V, b.V), (a.Wt, b.Wt), (a.W0, b.W0), (a.H0, b.H0), (a.T, b.T)):
        assert np.array_equal(x, y)
    c = synthetic.make_config(0, seed=123)
    assert not np.array_equal(a.V, c.V)


def test_batched_problem_shapes_follow_the_recipe():
    """Specs of the 64-problem batch (N, P, K, M ranges; K <= min(N, P)), on
    a few built members."""
    probs = synthetic.make_batched(count=3, n_iter=5)
    for p in probs:
        N, P, K, M = p.N, p.P, p.K, p.M
        assert 40 <= N <= 800 and 4000 <= P <= 80000 and 1 <= M <= 20
        assert 1 <= K <= min(N, P) and K <= 100
        _check_problem(p, N, P, K, M, p.img_shape)
    again = synthetic.make_batched(count=3, n_iter=5)
    assert all(np.array_equal(x.V, y.V) for x, y in zip(probs, again))


def test_roll_angles():
    ang = synthetic.roll_angles(50)
    assert ang.shape == (50,) and np.array_equal(ang, synthetic.roll_angles(50))
    centres = np.round(ang / 120.0) * 120.0
    assert set(np.unique(centres)) <= {0.0, 120.0, 240.0}
    assert np.all(np.abs(ang - centres) <= 30.0)
