"""Thin Python binding of libnmfgb (include/nmf.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch is used for device memory, streams and the workspace
allocation.  There is no fallback: if libnmfgb.so is missing or cannot be
loaded, every call raises.

The low-level functions carry the C names (nmf_fit_basis, nmf_project_target,
nmf_subtract, ...) and take raw device pointers; the high-level helpers
(fit_basis, project_target, subtract, reduce_host) take torch tensors or
numpy arrays and allocate outputs and workspaces.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnmfgb.so")

NMF_OK, NMF_EINVAL, NMF_ENOMEM, NMF_ECUDA, NMF_ETIMEOUT, NMF_ENOTCONV, NMF_EDATA = range(7)
NMF_FP32, NMF_TF32_SPLIT, NMF_BF16_SPLIT, NMF_BF16_SPLIT_W32 = 0, 1, 2, 3
NMF_COMBINE_MEAN, NMF_COMBINE_MEDIAN = 0, 1
COMBINE = {"mean": NMF_COMBINE_MEAN, "median": NMF_COMBINE_MEDIAN}
PRECISIONS = {"fp32": NMF_FP32, "tf32": NMF_TF32_SPLIT, "bf16": NMF_BF16_SPLIT, "bf16w32": NMF_BF16_SPLIT_W32}

EXPORTED = (
    "nmf_version",
    "nmf_status_string",
    "nmf_fit_workspace_bytes",
    "nmf_fit_basis",
    "nmf_project_workspace_bytes",
    "nmf_project_target",
    "nmf_subtract",
    "nmf_workspace_status",
    "nmf_reduce_host",
    "nmf_launch_count",
    "nmf_last_cuda_error",
    "nmf_project_target_noalloc",
    "nmf_batched_workspace_bytes",
    "nmf_fit_batched",
    "nmf_batched_status",
    "nmf_select_references",
    "nmf_derotate_combine",
    "nmf_w_schedule",
    "nmf_wait_selftest",
    "nmf_debug_plant_timeout",
    "nmf_fp32_fma_rate",
)


class NmfError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {status_string(code)} ({code})"
        if code == NMF_ECUDA:
            msg += f" [{last_cuda_error()}]"
        super().__init__(msg)


class nmf_fit_params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64),
        ("P", ctypes.c_int64),
        ("K", ctypes.c_int32),
        ("iters_per_stage", ctypes.c_int32),
        ("k_start", ctypes.c_int32),
        ("normalize", ctypes.c_int32),
        ("tol", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("polish_iters", ctypes.c_int32),
    ]


class nmf_problem(ctypes.Structure):
    _fields_ = [
        ("V", ctypes.c_void_p),
        ("Wt", ctypes.c_void_p),
        ("W", ctypes.c_void_p),
        ("H", ctypes.c_void_p),
        ("chi2_hist", ctypes.c_void_p),
        ("iters_done", ctypes.c_void_p),
        ("prm", nmf_fit_params),
        ("T", ctypes.c_void_p),
        ("WtT", ctypes.c_void_p),
        ("C", ctypes.c_void_p),
        ("R", ctypes.c_void_p),
        ("M", ctypes.c_int64),
        ("proj_iters", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


_lib = None
_lock = threading.Lock()


def load(path: Optional[str] = None):
    """Load libnmfgb.so (built by paper_2309_04623_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libnmfgb.so not built ({p}); run paper_2309_04623_gb300.build.build()")
        lib = ctypes.CDLL(p)
        vp, sz, i32, i64, dbl = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        P_params = ctypes.POINTER(nmf_fit_params)
        lib.nmf_version.restype = i32
        lib.nmf_version.argtypes = []
        lib.nmf_status_string.restype = ctypes.c_char_p
        lib.nmf_status_string.argtypes = [ctypes.c_int]
        lib.nmf_fit_workspace_bytes.restype = sz
        lib.nmf_fit_workspace_bytes.argtypes = [P_params]
        lib.nmf_fit_basis.restype = ctypes.c_int
        lib.nmf_fit_basis.argtypes = [vp, vp, vp, vp, vp, vp, vp, sz, P_params, vp]
        lib.nmf_project_workspace_bytes.restype = sz
        lib.nmf_project_workspace_bytes.argtypes = [i64, i64, i32, i32]
        lib.nmf_project_target.restype = ctypes.c_int
        lib.nmf_project_target.argtypes = [vp, i32, i64, vp, vp, i64, vp, i32, dbl, dbl, i32, i32, vp, sz, vp]
        lib.nmf_project_target_noalloc.restype = ctypes.c_int
        lib.nmf_project_target_noalloc.argtypes = [vp, i32, i64, vp, vp, i64, vp, i32, dbl, vp]
        lib.nmf_subtract.restype = ctypes.c_int
        lib.nmf_subtract.argtypes = [vp, vp, vp, i64, i32, i64, vp, vp, vp, i64, vp, vp]
        lib.nmf_workspace_status.restype = ctypes.c_int
        lib.nmf_workspace_status.argtypes = [vp, vp]
        lib.nmf_last_cuda_error.restype = ctypes.c_char_p
        lib.nmf_last_cuda_error.argtypes = []
        lib.nmf_launch_count.restype = ctypes.c_uint64
        lib.nmf_launch_count.argtypes = []
        P_prob = ctypes.POINTER(nmf_problem)
        lib.nmf_batched_workspace_bytes.restype = sz
        lib.nmf_batched_workspace_bytes.argtypes = [P_prob, i32]
        lib.nmf_fit_batched.restype = ctypes.c_int
        lib.nmf_fit_batched.argtypes = [P_prob, i32, vp, sz, vp]
        lib.nmf_batched_status.restype = ctypes.c_int
        lib.nmf_batched_status.argtypes = [P_prob, i32, vp, vp, ctypes.POINTER(i32)]
        lib.nmf_select_references.restype = ctypes.c_int
        lib.nmf_select_references.argtypes = [vp, vp, i64, vp, i64, i64, i32, vp, vp, vp]
        lib.nmf_derotate_combine.restype = ctypes.c_int
        lib.nmf_derotate_combine.argtypes = [vp, i64, i32, i32, vp, vp, ctypes.c_float, ctypes.c_float, i32, vp,
                                             vp, vp, vp]
        lib.nmf_wait_selftest.restype = ctypes.c_int
        lib.nmf_wait_selftest.argtypes = [i64, vp, vp]
        lib.nmf_debug_plant_timeout.restype = ctypes.c_int
        lib.nmf_debug_plant_timeout.argtypes = [i32, i64]
        lib.nmf_fp32_fma_rate.restype = ctypes.c_int
        lib.nmf_fp32_fma_rate.argtypes = [i32, vp, vp]
        lib.nmf_w_schedule.restype = i32
        lib.nmf_w_schedule.argtypes = [i64, i64, i32, i32, vp, vp, vp, vp]
        lib.nmf_reduce_host.restype = ctypes.c_int
        lib.nmf_reduce_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, P_params, i32, vp, vp, vp, vp, vp, vp]
        _lib = lib
        return lib


def status_string(code: int) -> str:
    try:
        return load().nmf_status_string(int(code)).decode()
    except Exception:
        return f"status {code}"


def last_cuda_error() -> str:
    try:
        return load().nmf_last_cuda_error().decode()
    except Exception:
        return ""


def _check(code: int, what: str):
    if code != NMF_OK:
        raise NmfError(code, what)


# ---------------------------------------------------------------------------
# low-level: the C entry points, raw pointers (ints) and sizes


def make_params(N, P, K, iters_per_stage, k_start=0, normalize=True, tol=0.0, eps=1e-30, precision=NMF_FP32,
                polish_iters=0):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return nmf_fit_params(int(N), int(P), int(K), int(iters_per_stage), int(k_start), int(bool(normalize)),
                          float(tol), float(eps), int(precision), int(polish_iters))


def tc_max_k() -> int:
    """Largest K the tensor-core form (NMF_BF16_SPLIT) accepts."""
    for k in (128, 64, 32):
        if nmf_fit_workspace_bytes(make_params(1024, 4096, k, 1, precision=NMF_BF16_SPLIT)) > 0:
            return k
    return 0


def nmf_version() -> int:
    return int(load().nmf_version())


def nmf_launch_count() -> int:
    return int(load().nmf_launch_count())


def nmf_fit_workspace_bytes(params: nmf_fit_params) -> int:
    return int(load().nmf_fit_workspace_bytes(ctypes.byref(params)))


def nmf_fit_basis(V, Wt, W, H, chi2_hist, iters_done, ws, ws_bytes, params, stream) -> int:
    return int(load().nmf_fit_basis(V, Wt, W, H, chi2_hist, iters_done, ws, ws_bytes, ctypes.byref(params), stream))


def nmf_project_workspace_bytes(M, P, K, precision=NMF_FP32) -> int:
    return int(load().nmf_project_workspace_bytes(int(M), int(P), int(K), int(precision)))


def nmf_project_target(H, K, P, T, WtT, M, C, iters, tol, eps, precision, polish_iters, ws, ws_bytes,
                       stream) -> int:
    return int(load().nmf_project_target(H, K, P, T, WtT, M, C, iters, tol, eps, precision, polish_iters, ws,
                                         ws_bytes, stream))


def nmf_project_target_noalloc(H, K, P, T, WtT, M, C, iters, eps, stream) -> int:
    return int(load().nmf_project_target_noalloc(H, K, P, T, WtT, M, C, iters, eps, stream))


def nmf_subtract(T, C, H, M, K, P, factor, R, scatter_idx, img_pixels, img, stream) -> int:
    return int(load().nmf_subtract(T, C, H, M, K, P, factor, R, scatter_idx, img_pixels, img, stream))


def nmf_workspace_status(ws, stream) -> int:
    return int(load().nmf_workspace_status(ws, stream))


def nmf_batched_workspace_bytes(problems) -> int:
    arr = (nmf_problem * len(problems))(*problems)
    return int(load().nmf_batched_workspace_bytes(arr, len(problems)))


def nmf_fit_batched(problems, ws, ws_bytes, stream) -> int:
    arr = (nmf_problem * len(problems))(*problems)
    return int(load().nmf_fit_batched(arr, len(problems), ws, ws_bytes, stream))


def nmf_batched_status(problems, ws, stream):
    """Returns (first non-OK status or NMF_OK, list of per-problem statuses)."""
    arr = (nmf_problem * len(problems))(*problems)
    st = (ctypes.c_int32 * len(problems))()
    code = int(load().nmf_batched_status(arr, len(problems), ws, stream, st))
    return code, list(st)


def nmf_select_references(T, WtT, M, V, N, P, n_keep, dist, idx, stream) -> int:
    return int(load().nmf_select_references(T, WtT, M, V, N, P, n_keep, dist, idx, stream))


def nmf_reduce_host(V, Wt, W0, H0, T, WtT, C0, M, params, proj_iters, W, H, C, R, chi2_hist, iters_done) -> int:
    return int(load().nmf_reduce_host(V, Wt, W0, H0, T, WtT, C0, M, ctypes.byref(params), proj_iters, W, H, C, R,
                                      chi2_hist, iters_done))


# ---------------------------------------------------------------------------
# high-level helpers on torch tensors


def nmf_derotate_combine(img, F, ny, nx, valid, angle_deg, cx, cy, method, rot, out, count, stream) -> int:
    """angle_deg: host pointer (or ctypes array) of F doubles; the rest are device pointers."""
    return int(load().nmf_derotate_combine(img, F, ny, nx, valid, angle_deg, cx, cy, method, rot, out, count,
                                           stream))


def nmf_wait_selftest(limit_ns, status, stream) -> int:
    return int(load().nmf_wait_selftest(limit_ns, status, stream))


def nmf_debug_plant_timeout(t_fault, limit_ns) -> int:
    return int(load().nmf_debug_plant_timeout(int(t_fault), int(limit_ns)))


def fp32_fma_rate(iters: int = 1 << 16, *, stream=None) -> float:
    """nmf_fp32_fma_rate: the measured FP32 FMA rate of the CUDA cores (TFLOP/s)."""
    out = ctypes.c_double(0.0)
    _check(int(load().nmf_fp32_fma_rate(int(iters), ctypes.byref(out), _stream(stream))), "nmf_fp32_fma_rate")
    return float(out.value)


def nmf_w_schedule(rows, P, sms, max_blocks, tile, split, c0, c1) -> int:
    return int(load().nmf_w_schedule(rows, P, sms, max_blocks, tile, split, c0, c1))


def _torch():
    import torch

    return torch


def _dev(x, dtype=None, device=None):
    torch = _torch()
    if dtype is None:
        dtype = torch.float32
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    if device is None:
        device = x.device if x.is_cuda else torch.device("cuda")
    return x.to(device=device, dtype=dtype).contiguous()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def workspace(nbytes: int, device=None):
    """A caller-owned device workspace (torch allocations are 512-B aligned)."""
    torch = _torch()
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")


def fit_basis(V, Wt, W0, H0, iters_per_stage: int, *, tol: float = 0.0, eps: float = 1e-30, normalize=True,
              k_start: int = 0, precision="fp32", polish_iters: int = 0, stream=None, ws=None, check_status=True):
    """nmf_fit_basis on torch tensors.  Returns (W, H, chi2_hist, iters_done)."""
    torch = _torch()
    V = _dev(V)
    Wt = _dev(Wt, device=V.device)
    W = _dev(W0, device=V.device).clone()
    H = _dev(H0, device=V.device).clone()
    N, P = V.shape
    K = H.shape[0]
    prm = make_params(N, P, K, iters_per_stage, k_start, normalize, tol, eps, precision, polish_iters)
    need = nmf_fit_workspace_bytes(prm)
    if need == 0:
        raise NmfError(NMF_EINVAL, "nmf_fit_workspace_bytes")
    if ws is None or ws.numel() < need:
        ws = workspace(need, V.device)
    chi2 = torch.zeros(K, dtype=torch.float64, device=V.device)
    iters = torch.zeros(K, dtype=torch.int32, device=V.device)
    _check(nmf_fit_basis(_ptr(V), _ptr(Wt), _ptr(W), _ptr(H), _ptr(chi2), _ptr(iters), _ptr(ws), need, prm,
                         _stream(stream)), "nmf_fit_basis")
    if check_status:
        _check(nmf_workspace_status(_ptr(ws), _stream(stream)), "nmf_fit_basis (device status)")
    return W, H, chi2, iters


def project_target(H, T, WtT, C0, iters: int, *, eps: float = 1e-30, precision="fp32", polish_iters: int = 0,
                   stream=None, ws=None, check_status=True):
    """nmf_project_target on torch tensors.  Returns C."""
    H = _dev(H)
    T = _dev(T, device=H.device)
    WtT = _dev(WtT, device=H.device)
    C = _dev(C0, device=H.device).clone()
    M, P = T.shape
    K = H.shape[0]
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    need = nmf_project_workspace_bytes(M, P, K, prec)
    if need == 0:
        raise NmfError(NMF_EINVAL, "nmf_project_workspace_bytes")
    if ws is None or ws.numel() < need:
        ws = workspace(need, H.device)
    _check(nmf_project_target(_ptr(H), K, P, _ptr(T), _ptr(WtT), M, _ptr(C), int(iters), 0.0, float(eps), prec,
                              int(polish_iters), _ptr(ws), need, _stream(stream)), "nmf_project_target")
    if check_status:
        _check(nmf_workspace_status(_ptr(ws), _stream(stream)), "nmf_project_target (device status)")
    return C


def subtract(T, C, H, *, factor=None, scatter_idx=None, img_pixels: int = 0, stream=None):
    """nmf_subtract on torch tensors.  Returns R (M x P), or (R, img) with a scatter."""
    torch = _torch()
    T = _dev(T)
    C = _dev(C, device=T.device)
    H = _dev(H, device=T.device)
    M, P = T.shape
    K = H.shape[0]
    R = torch.empty_like(T)
    f = None if factor is None else _dev(factor, device=T.device)
    idx = img = None
    if scatter_idx is not None:
        idx = _dev(scatter_idx, dtype=torch.int32, device=T.device)
        img = torch.empty((M, int(img_pixels)), dtype=torch.float32, device=T.device)
    _check(nmf_subtract(_ptr(T), _ptr(C), _ptr(H), M, K, P, _ptr(f), _ptr(R), _ptr(idx), int(img_pixels), _ptr(img),
                        _stream(stream)), "nmf_subtract")
    return R if img is None else (R, img)


def _hptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def reduce_host(V, Wt, W0, H0, T, WtT, C0, iters_per_stage: int, proj_iters: int, *, tol=0.0, eps=1e-30,
                normalize=True, precision="fp32", polish_iters=0, out=None):
    """nmf_reduce_host: the whole path from host (numpy) buffers to host outputs."""
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    V, Wt, W0, H0 = f32(V), f32(Wt), f32(W0), f32(H0)
    N, P = V.shape
    K = H0.shape[0]
    M = 0 if T is None else T.shape[0]
    if M:
        T, WtT, C0 = f32(T), f32(WtT), f32(C0)
    if out is None:
        out = dict(W=np.empty((N, K), np.float32), H=np.empty((K, P), np.float32),
                   C=np.empty((max(M, 1), K), np.float32), R=np.empty((max(M, 1), P), np.float32),
                   chi2_hist=np.zeros(K), iters_done=np.zeros(K, np.int32))
    prm = make_params(N, P, K, iters_per_stage, 0, normalize, tol, eps, precision, polish_iters)
    _check(nmf_reduce_host(_hptr(V), _hptr(Wt), _hptr(W0), _hptr(H0), _hptr(T) if M else None,
                           _hptr(WtT) if M else None, _hptr(C0) if M else None, M, prm, int(proj_iters),
                           _hptr(out["W"]), _hptr(out["H"]), _hptr(out["C"]), _hptr(out["R"]),
                           _hptr(out["chi2_hist"]), _hptr(out["iters_done"])), "nmf_reduce_host")
    return out


def fit_batched(batch, iters_per_stage: int, proj_iters: int, *, tol: float = 0.0, eps: float = 1e-30,
                normalize=True, precision="fp32", polish_iters: int = 0, stream=None, ws=None, check_status=True):
    """nmf_fit_batched on torch tensors.

    `batch` is a sequence of dicts with keys V, Wt, W0, H0 and, optionally,
    T, WtT, C0 (science frames).  Per-problem overrides of iters_per_stage,
    proj_iters, precision and polish_iters may be given in the dict.  Returns
    a list of dicts with W, H, chi2_hist, iters_done and, with frames, C, R.
    """
    torch = _torch()
    out, probs, keep = [], [], []
    for b in batch:
        V = _dev(b["V"])
        Wt = _dev(b["Wt"], device=V.device)
        W = _dev(b["W0"], device=V.device).clone()
        H = _dev(b["H0"], device=V.device).clone()
        N, P = V.shape
        K = H.shape[0]
        prec = b.get("precision", precision)
        prm = make_params(N, P, K, b.get("iters_per_stage", iters_per_stage), 0, normalize, tol, eps, prec,
                          b.get("polish_iters", polish_iters))
        r = dict(W=W, H=H, chi2_hist=torch.zeros(K, dtype=torch.float64, device=V.device),
                 iters_done=torch.zeros(K, dtype=torch.int32, device=V.device))
        q = nmf_problem()
        q.V, q.Wt, q.W, q.H = V.data_ptr(), Wt.data_ptr(), W.data_ptr(), H.data_ptr()
        q.chi2_hist, q.iters_done = r["chi2_hist"].data_ptr(), r["iters_done"].data_ptr()
        q.prm = prm
        keep += [V, Wt]
        if b.get("T") is not None:
            T = _dev(b["T"], device=V.device)
            WtT = _dev(b["WtT"], device=V.device)
            C = _dev(b["C0"], device=V.device).clone()
            R = torch.empty_like(T)
            keep += [T, WtT]
            r.update(C=C, R=R)
            q.T, q.WtT, q.C, q.R = T.data_ptr(), WtT.data_ptr(), C.data_ptr(), R.data_ptr()
            q.M = T.shape[0]
            q.proj_iters = int(b.get("proj_iters", proj_iters))
        probs.append(q)
        out.append(r)
    need = nmf_batched_workspace_bytes(probs)
    if need == 0:
        raise NmfError(NMF_EINVAL, "nmf_batched_workspace_bytes")
    if ws is None or ws.numel() < need:
        ws = workspace(need)
    _check(nmf_fit_batched(probs, _ptr(ws), need, _stream(stream)), "nmf_fit_batched")
    if check_status:
        code, statuses = nmf_batched_status(probs, _ptr(ws), _stream(stream))
        if code != NMF_OK:
            err = NmfError(code, "nmf_fit_batched (device status)")
            err.statuses = statuses
            raise err
    return out


def select_references(T, WtT, V, n_keep: int, *, stream=None):
    """nmf_select_references on torch tensors.  Returns (dist M x N float64,
    idx M x n_keep int32): the n_keep closest library frames of every target."""
    torch = _torch()
    T = _dev(T)
    WtT = _dev(WtT, device=T.device)
    V = _dev(V, device=T.device)
    M, P = T.shape
    N = V.shape[0]
    dist = torch.empty((M, N), dtype=torch.float64, device=T.device)
    idx = torch.empty((M, int(n_keep)), dtype=torch.int32, device=T.device)
    _check(nmf_select_references(_ptr(T), _ptr(WtT), M, _ptr(V), N, P, int(n_keep), _ptr(dist), _ptr(idx),
                                 _stream(stream)), "nmf_select_references")
    return dist, idx


def derotate_combine(img, angle_deg, center, *, method: str = "mean", valid=None, rotated: bool = False,
                     stacked: bool = True, stream=None):
    """nmf_derotate_combine on torch tensors: frames (F, ny, nx) rotated by
    angle_deg[f] degrees about center = (cx, cy) and stacked per pixel.
    Returns (stacked ny x nx float32 or None, count ny x nx int32,
    rotated F x ny x nx float32 or None)."""
    torch = _torch()
    img = _dev(img)
    if img.dim() == 2:
        img = img.unsqueeze(0)
    F, ny, nx = img.shape
    ang = np.ascontiguousarray(np.broadcast_to(np.asarray(angle_deg, dtype=np.float64), (F,)))
    v = None if valid is None else _dev(valid, dtype=torch.uint8, device=img.device)
    out = torch.empty((ny, nx), dtype=torch.float32, device=img.device) if stacked else None
    count = torch.empty((ny, nx), dtype=torch.int32, device=img.device)
    rot = torch.empty((F, ny, nx), dtype=torch.float32, device=img.device) if rotated else None
    cx, cy = center
    _check(nmf_derotate_combine(_ptr(img), F, ny, nx, _ptr(v), ang.ctypes.data_as(ctypes.c_void_p), float(cx),
                                float(cy), COMBINE[method], _ptr(rot), _ptr(out), _ptr(count), _stream(stream)),
           "nmf_derotate_combine")
    return out, count, rot


def w_schedule(rows: int, P: int, sms: int, max_blocks: int = 256):
    """nmf_w_schedule: the W-pass block schedule (tile, split, c0, c1 as int32
    arrays, one entry per block), or None when the fit uses equal splits."""
    arrs = [np.zeros(max_blocks, dtype=np.int32) for _ in range(4)]
    n = int(load().nmf_w_schedule(int(rows), int(P), int(sms), int(max_blocks),
                                  *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs]))
    if n < 0:
        raise NmfError(NMF_EINVAL, "nmf_w_schedule")
    if n == 0:
        return None
    return tuple(a[:n].copy() for a in arrs)


def wait_selftest(limit_ns: int = 1_000_000, *, stream=None):
    """nmf_wait_selftest: the statuses recorded by a bounded mbarrier wait and
    a bounded counter wait that nothing satisfies (NMF_ETIMEOUT expected)."""
    st = np.zeros(2, dtype=np.int32)
    _check(int(load().nmf_wait_selftest(int(limit_ns), st.ctypes.data_as(ctypes.c_void_p), _stream(stream))),
           "nmf_wait_selftest")
    return int(st[0]), int(st[1])
