"""Vectorised NumPy form of the weighted-NMF iteration: the analogue of the
paper's own CPU setup (Sec. 2: the method written as NumPy array arithmetic,
its matrix products going through the BLAS that NumPy links).

TEST AND BENCHMARK INFRASTRUCTURE ONLY.  The benchmark times this form as a
CPU baseline beside the oracle, and the test suite checks it against the
oracle.  It is not the oracle (that is `nmf_oracle.c`), and the product path
never imports it.  It computes in float64 or float32 (`dtype`).

It follows the same algorithm as the oracle, with whole-array operations:

  iterate   Eq. 3: the H-step, then the W-step with the new H.  Each update
            keeps exact zeros, clamps the denominator at eps, and sets
            entries below 2^-126 to zero (the underflow reading).  Eq. 2 of
            the updated pair follows each iteration.
  fit       Sec. 2 sequential construction k = 1..K: warm start from W0 and
            H0, the stopping rule on the relative decrease of Eq. 2, then
            the L2 normalisation of each H row, with W's column scaled back.
  project   Sec. 4.1 target modelling: Eq. 3's W-rule for the coefficients C
            of the science frames, with the basis H held fixed.
"""
from __future__ import annotations

import os

import numpy as np

TINY = 2.0 ** -126  # entries of W, H, C below this become exact zeros


def _mu(x, num, den, eps):
    """Eq. 3's multiplicative rule on whole arrays: 0 where x is 0, else
    x * num / max(den, eps), then entries below TINY set to 0."""
    out = x * num / np.maximum(den, x.dtype.type(eps))
    out[x == 0] = 0
    out[out < TINY] = 0
    return out


def chi2(V, Wt, W, H) -> float:
    """Eq. 2: sum of Wt * (V - W H)^2, accumulated in float64."""
    R = V - W @ H
    return float(np.sum(Wt * R * R, dtype=np.float64))


def iterate(V, Wt, W, H, n_iter: int, eps: float = 1e-30, dtype=np.float64, A=None):
    """n_iter iterations of Eq. 3 at the rank of H.  Returns (W, H, trace),
    trace holding Eq. 2 after each iteration."""
    V = np.asarray(V, dtype=dtype)
    Wt = np.asarray(Wt, dtype=dtype)
    A = Wt * V if A is None else A
    W = np.array(W, dtype=dtype)
    H = np.array(H, dtype=dtype)
    trace = np.empty(n_iter)
    for t in range(n_iter):
        # H-step: H <- H o [W^T (Wt o V)] / [W^T (Wt o (W H))]
        H = _mu(H, W.T @ A, W.T @ (Wt * (W @ H)), eps)
        # W-step with the new H: W <- W o [(Wt o V) H^T] / [(Wt o (W H)) H^T]
        W = _mu(W, A @ H.T, (Wt * (W @ H)) @ H.T, eps)
        trace[t] = chi2(V, Wt, W, H)
    return W, H, trace


def fit(V, Wt, W0, H0, n_iter: int, tol: float = 0.0, eps: float = 1e-30, normalize: bool = True,
        k_start: int = 0, dtype=np.float64):
    """Sequential weighted NMF (Sec. 2).  Returns dict(W, H, chi2_hist,
    iters_done) like the oracle's fit."""
    V = np.asarray(V, dtype=dtype)
    Wt = np.asarray(Wt, dtype=dtype)
    A = Wt * V
    W = np.array(W0, dtype=dtype)
    H = np.array(H0, dtype=dtype)
    K = H.shape[0]
    hist = np.zeros(K)
    done = np.zeros(K, dtype=np.int32)
    for k in range(k_start + 1, K + 1):
        Wk, Hk = W[:, :k], H[:k]
        prev, c, t_done = 0.0, chi2(V, Wt, Wk, Hk) if n_iter == 0 else float("nan"), 0
        for t in range(1, n_iter + 1):
            Wk, Hk, tr = iterate(V, Wt, Wk, Hk, 1, eps, dtype, A)
            c, t_done = float(tr[0]), t
            if tol > 0.0 and t >= 2 and (prev - c) <= tol * prev:
                break
            prev = c
        hist[k - 1], done[k - 1] = c, t_done
        if normalize:
            s = np.sqrt(np.sum(Hk.astype(np.float64) ** 2, axis=1))
            nz = s > 0
            Hn = Hk[nz] / s[nz, None].astype(dtype)
            Wn = Wk[:, nz] * s[nz].astype(dtype)
            Hn[Hn < TINY] = 0
            Wn[Wn < TINY] = 0
            Hk[nz], Wk[:, nz] = Hn, Wn
        W[:, :k], H[:k] = Wk, Hk
    return dict(W=W, H=H, chi2_hist=hist, iters_done=done)


def project(H, T, WtT, C0, n_iter: int, eps: float = 1e-30, dtype=np.float64):
    """Coefficients of the science frames on the fixed basis H (Sec. 4.1):
    C <- C o [(WtT o T) H^T] / [(WtT o (C H)) H^T], n_iter times."""
    H = np.asarray(H, dtype=dtype)
    T = np.asarray(T, dtype=dtype)
    WtT = np.asarray(WtT, dtype=dtype)
    C = np.array(C0, dtype=dtype)
    num = (WtT * T) @ H.T  # fixed while H is
    for _ in range(n_iter):
        C = _mu(C, num, (WtT * (C @ H)) @ H.T, eps)
    return C


def blas_threads():
    """(threads, how known) of the BLAS NumPy calls."""
    try:
        from threadpoolctl import threadpool_info
    except ImportError:
        threadpool_info = None
    if threadpool_info is not None:
        n = [d.get("num_threads", 0) for d in threadpool_info() if d.get("user_api") == "blas"]
        if n:
            return int(max(n)), "threadpoolctl"
    env = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
    if env and env.isdigit():
        return int(env), "OPENBLAS_NUM_THREADS/OMP_NUM_THREADS"
    return os.cpu_count() or 1, "BLAS default (one thread per core); elementwise NumPy operations run on one thread"
