"""FP64 CPU oracle for the weighted-NMF hot path of arXiv:2309.04623.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product path (the
CUDA library and its binding) never imports this package, and this package
never imports the product path.

The arithmetic lives in plain C (`nmf_oracle.c`, double precision, compiled
here with gcc); this module only marshals numpy arrays through ctypes.
Function-to-paper map:

  (reading)   entries of W, H, C that fall below 2^-126 become exact zeros
              (set_tiny / tiny change the threshold; 0 turns the rule off)
  chi2        Eq. 2   weighted Frobenius cost
  iterate     Eq. 3   H-step then W-step (new H), fixed rank
  fit         Sec. 2  sequential construction k = 1..K with warm start,
                      stopping rule, per-stage row normalisation
  project     Sec. 4.1 target modelling: Eq. 3 coefficient rule, H fixed
  subtract    Sec. 4.1 PSF subtraction
  distances,  Sec. 4.1 reference selection (closest library frames by the
  select               weighted Euclidean norm of Eq. 2)
  rotate      Sec. 4.1/4.2 North-up rotation of the subtracted frames
              (bilinear interpolation, missing data stay missing)
  combine     Sec. 4.1/4.2 stacking: per-pixel mean or median of the
              frames covering the pixel

Parity status: every function is pinned by the `-m "not gpu"` tests in
tests/test_oracle_pins.py (closed forms, special cases, invariants, planted
factorisations and brute-force NNLS).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nmf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile nmf_oracle.c into _liboracle.so (gcc, -O2, OpenMP, no -ffast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
               "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.oracle_set_tiny.restype = None
            lib.oracle_set_tiny.argtypes = [dbl]
            lib.oracle_get_tiny.restype = dbl
            lib.oracle_get_tiny.argtypes = []
            lib.oracle_num_threads.restype = i32
            lib.oracle_set_num_threads.argtypes = [i32]
            lib.oracle_chi2.restype = dbl
            lib.oracle_chi2.argtypes = [i64, i64, i32, _f32p, _f32p, _f64p, i32, _f64p]
            lib.oracle_iterate.restype = i32
            lib.oracle_iterate.argtypes = [i64, i64, i32, _f32p, _f32p, _f64p, i32, _f64p, i32, dbl, dbl,
                                           ctypes.c_void_p]
            lib.oracle_fit.restype = i32
            lib.oracle_fit.argtypes = [i64, i64, i32, _f32p, _f32p, _f64p, _f64p, i32, dbl, dbl, i32, i32,
                                       _f64p, _i32p, ctypes.c_void_p]
            lib.oracle_project.restype = i32
            lib.oracle_project.argtypes = [i64, i64, i32, _f64p, _f32p, _f32p, _f64p, i32, dbl]
            lib.oracle_subtract.restype = None
            lib.oracle_subtract.argtypes = [i64, i64, i32, _f32p, _f64p, _f64p, ctypes.c_void_p, _f64p]
            lib.oracle_distances.restype = None
            lib.oracle_distances.argtypes = [i64, i64, i64, _f32p, _f32p, _f32p, _f64p]
            lib.oracle_select.restype = None
            lib.oracle_select.argtypes = [i64, i64, _f64p, ctypes.c_int32, _i32p]
            lib.oracle_rotate.restype = None
            lib.oracle_rotate.argtypes = [i64, ctypes.c_int32, ctypes.c_int32, _f32p, ctypes.c_void_p, _f64p,
                                          ctypes.c_float, ctypes.c_float, _f64p]
            lib.oracle_combine.restype = None
            lib.oracle_combine.argtypes = [i64, i64, _f64p, ctypes.c_int32, _f64p, _i32p]
            _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


TINY = 2.0**-126  # default smallest magnitude a factor entry keeps


def set_tiny(t: float) -> None:
    """Entries of W, H, C that an update or the normalisation leaves below t
    become exact zeros (default 2^-126; 0 = plain double precision)."""
    _load().oracle_set_tiny(float(t))


def get_tiny() -> float:
    return float(_load().oracle_get_tiny())


class tiny:
    """Context manager: run the oracle with another tiny-entry threshold."""

    def __init__(self, t: float):
        self.t = float(t)

    def __enter__(self):
        self.prev = get_tiny()
        set_tiny(self.t)
        return self

    def __exit__(self, *exc):
        set_tiny(self.prev)
        return False


def chi2(V, Wt, W, H) -> float:
    """Eq. 2 for the pair (W, H); V, Wt float32 (N, P); W (N, k), H (k, P)."""
    V, Wt = _f32(V), _f32(Wt)
    W, H = _f64(W), _f64(H)
    N, P = V.shape
    k = H.shape[0]
    return float(_load().oracle_chi2(N, P, k, V, Wt, W, W.shape[1], H))


def iterate(V, Wt, W, H, n_iter: int, tol: float = 0.0, eps: float = 1e-30):
    """n_iter iterations of Eq. 3 at the rank of H.  Returns (W, H, trace, done)."""
    V, Wt = _f32(V), _f32(Wt)
    W, H = _f64(W).copy(), _f64(H).copy()
    N, P = V.shape
    k = H.shape[0]
    trace = np.full(max(n_iter, 1), np.nan)
    done = _load().oracle_iterate(N, P, k, V, Wt, W, W.shape[1], H, int(n_iter), float(tol), float(eps),
                                  trace.ctypes.data)
    if done < 0:
        raise MemoryError("oracle_iterate")
    return W, H, trace[:n_iter], int(done)


def fit(V, Wt, W0, H0, n_iter: int, tol: float = 0.0, eps: float = 1e-30, normalize: bool = True,
        k_start: int = 0, trace: bool = False):
    """Sequential weighted NMF (Sec. 2).  Returns dict(W, H, chi2_hist, iters_done[, chi2_trace])."""
    V, Wt = _f32(V), _f32(Wt)
    W, H = _f64(W0).copy(), _f64(H0).copy()
    N, P = V.shape
    K = H.shape[0]
    hist = np.zeros(K)
    done = np.zeros(K, dtype=np.int32)
    tr = np.full((K, max(n_iter, 1)), np.nan) if trace else None
    rc = _load().oracle_fit(N, P, K, V, Wt, W, H, int(n_iter), float(tol), float(eps), int(bool(normalize)),
                            int(k_start), hist, done, tr.ctypes.data if trace else None)
    if rc != 0:
        raise MemoryError("oracle_fit")
    out = dict(W=W, H=H, chi2_hist=hist, iters_done=done)
    if trace:
        out["chi2_trace"] = tr[:, :n_iter]
    return out


def project(H, T, WtT, C0, n_iter: int, eps: float = 1e-30):
    """Coefficients of the science frames on the fixed basis H (Sec. 4.1)."""
    H = _f64(H)
    T, WtT = _f32(T), _f32(WtT)
    C = _f64(C0).copy()
    M, P = T.shape
    K = H.shape[0]
    if _load().oracle_project(M, P, K, H, T, WtT, C, int(n_iter), float(eps)) != 0:
        raise MemoryError("oracle_project")
    return C


def subtract(T, C, H, factor=None):
    """Residual images T - f * (C H) in pixel space (Sec. 4.1)."""
    T = _f32(T)
    C, H = _f64(C), _f64(H)
    M, P = T.shape
    K = H.shape[0]
    out = np.empty((M, P))
    f = None if factor is None else _f64(factor)
    _load().oracle_subtract(M, P, K, T, C, H, None if f is None else f.ctypes.data, out)
    return out


def distances(T, WtT, V):
    """Reference selection (Sec. 4.1): D[m, n] = sum_p WtT[m, p] (T[m, p] - V[n, p])^2."""
    T, WtT, V = _f32(T), _f32(WtT), _f32(V)
    M, P = T.shape
    N = V.shape[0]
    D = np.empty((M, N))
    _load().oracle_distances(M, N, P, T, WtT, V, D)
    return D


def select(D, n_keep: int):
    """Indices of the n_keep closest library frames per target, closest first (ties by index)."""
    D = _f64(D)
    M, N = D.shape
    idx = np.empty((M, int(n_keep)), dtype=np.int32)
    _load().oracle_select(M, N, D, int(n_keep), idx)
    return idx


def rotate(img, angle_deg, center, valid=None):
    """Frames (F, ny, nx) rotated by angle_deg[f] degrees about center = (cx, cy)
    (Sec. 4.1/4.2 North-up step); float64, NaN where no value can be formed."""
    img = _f32(img)
    if img.ndim == 2:
        img = img[None]
    F, ny, nx = img.shape
    ang = _f64(np.broadcast_to(np.asarray(angle_deg, dtype=np.float64), (F,)))
    out = np.empty((F, ny, nx))
    v = None
    if valid is not None:
        v = np.ascontiguousarray(valid, dtype=np.uint8).reshape(ny, nx)
    cx, cy = center
    _load().oracle_rotate(F, ny, nx, img, None if v is None else v.ctypes.data, ang, float(cx), float(cy), out)
    return out


def combine(frames, method: str = "mean"):
    """Per-pixel mean or median over the frames that are not NaN (Sec. 4.1/4.2
    stacking).  Returns (image float64, count int32)."""
    frames = _f64(frames)
    F = frames.shape[0]
    shape = frames.shape[1:]
    npix = int(np.prod(shape)) if F else int(np.prod(shape))
    out = np.empty(npix)
    count = np.empty(npix, dtype=np.int32)
    m = {"mean": 0, "median": 1}[method]
    _load().oracle_combine(F, npix, frames.reshape(F, npix), m, out, count)
    return out.reshape(shape), count.reshape(shape)
