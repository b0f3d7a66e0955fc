"""Host-side checks of the C-ABI boundary (no GPU needed): the library builds,
loads, exports every entry point declared in include/nmf.h, and rejects bad
arguments synchronously before touching the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2309_04623_gb300 import build, nmf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return nmf.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"NMF_API[^;(]*?\b(nmf_\w+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("nmf_fit_basis", "nmf_project_target", "nmf_subtract", "nmf_fit_workspace_bytes",
                 "nmf_project_workspace_bytes", "nmf_status_string", "nmf_reduce_host", "nmf_workspace_status"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", nmf.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (nmf_\w+)", out))
    assert _declared() <= exported, _declared() - exported
    for name in _declared():
        assert hasattr(lib, name)
    assert set(nmf.EXPORTED) == _declared()


def test_version_and_status_strings(lib):
    assert nmf.nmf_version() >= 100
    for code in range(7):
        assert nmf.status_string(code).startswith("NMF_")
    assert "unknown" in nmf.status_string(99)


def test_workspace_query_validates(lib):
    ok = nmf.make_params(300, 49343, 30, 500)
    assert nmf.nmf_fit_workspace_bytes(ok) > 2 * 300 * 49343 * 4
    bad = [
        nmf.make_params(10, 100, 11, 5),  # K > N (components limited by the library size)
        nmf.make_params(10, 5, 6, 5),  # K > P
        nmf.make_params(300, 100, 129, 5),  # K above the kernel limit
        nmf.make_params(0, 100, 1, 5),
        nmf.make_params(10, 100, 3, -1),
        nmf.make_params(10, 100, 3, 5, k_start=4),
        nmf.make_params(10, 100, 3, 5, eps=0.0),
        nmf.make_params(10, 100, 3, 5, tol=-1.0),
        nmf.make_params(10, 100, 3, 5, precision=7),
        nmf.make_params(10, 100, 3, 5, precision="tf32"),  # reserved form
        nmf.make_params(200, 1000, 129, 5, precision="bf16"),  # tensor-core form: K <= 128
        nmf.make_params(10, 100, 3, 5, polish_iters=2),  # polish only for the split forms
        nmf.make_params(10, 100, 3, 5, precision="bf16", polish_iters=-1),
    ]
    for prm in bad:
        assert nmf.nmf_fit_workspace_bytes(prm) == 0
    assert nmf.nmf_project_workspace_bytes(50, 49343, 30) > 0
    assert nmf.nmf_project_workspace_bytes(50, 49343, 0) == 0
    assert nmf.nmf_project_workspace_bytes(50, 10, 11) == 0
    bf = nmf.make_params(300, 49343, 30, 500, precision="bf16", polish_iters=10)
    assert nmf.nmf_fit_workspace_bytes(bf) > nmf.nmf_fit_workspace_bytes(ok)
    assert nmf.nmf_project_workspace_bytes(50, 49343, 30, nmf.NMF_BF16_SPLIT) > 0
    assert nmf.nmf_project_workspace_bytes(50, 49343, 100, nmf.NMF_BF16_SPLIT) > 0
    assert nmf.nmf_project_workspace_bytes(50, 49343, 129, nmf.NMF_BF16_SPLIT) == 0
    # the FP32-weights form: the same component limit and the same workspace layout as the FP16-weights form
    assert nmf.nmf_project_workspace_bytes(50, 49343, 100, nmf.NMF_BF16_SPLIT_W32) > 0
    assert nmf.nmf_project_workspace_bytes(50, 49343, 129, nmf.NMF_BF16_SPLIT_W32) == 0
    assert (nmf.nmf_project_workspace_bytes(50, 49343, 100, nmf.NMF_BF16_SPLIT_W32)
            == nmf.nmf_project_workspace_bytes(50, 49343, 100, nmf.NMF_BF16_SPLIT))
    w32 = nmf.make_params(300, 49343, 30, 500, precision="bf16w32", polish_iters=10)
    assert nmf.nmf_fit_workspace_bytes(w32) == nmf.nmf_fit_workspace_bytes(bf)
    assert nmf.tc_max_k() == 128


def test_entry_points_reject_bad_arguments_without_device(lib):
    """Argument errors are returned before any CUDA call, so they work on a
    machine without a GPU."""
    p = ctypes.c_void_p(256)  # never dereferenced: the checks fail first
    prm = nmf.make_params(10, 100, 11, 5)
    assert nmf.nmf_fit_basis(p, p, p, p, p, p, p, 1 << 30, prm, None) == nmf.NMF_EINVAL
    good = nmf.make_params(10, 100, 3, 5)
    need = nmf.nmf_fit_workspace_bytes(good)
    assert nmf.nmf_fit_basis(None, p, p, p, p, p, p, need, good, None) == nmf.NMF_EINVAL
    assert nmf.nmf_fit_basis(p, p, p, p, p, p, p, need - 1, good, None) == nmf.NMF_EINVAL
    assert nmf.nmf_fit_basis(p, p, p, p, p, p, ctypes.c_void_p(257), need, good, None) == nmf.NMF_EINVAL
    assert nmf.nmf_project_target(p, 3, 100, p, p, 4, p, 5, 0.1, 1e-30, 0, 0, p, 1 << 30, None) == nmf.NMF_EINVAL
    assert nmf.nmf_project_target(p, 3, 100, p, p, 4, p, -1, 0.0, 1e-30, 0, 0, p, 1 << 30, None) == nmf.NMF_EINVAL
    assert nmf.nmf_subtract(p, p, p, 4, 0, 100, None, p, None, 0, None, None) == nmf.NMF_EINVAL
    assert nmf.nmf_subtract(p, p, p, 4, 3, 100, None, p, p, 0, None, None) == nmf.NMF_EINVAL
    assert nmf.nmf_subtract(p, p, p, 4, 3, 100, None, p, p, 50, p, None) == nmf.NMF_EINVAL
    assert nmf.nmf_workspace_status(None, None) == nmf.NMF_EINVAL
    assert nmf.nmf_reduce_host(p, p, p, p, None, None, None, 0, prm, 0, p, p, None, None, p, p) == nmf.NMF_EINVAL


def _problem(N, P, K, M=0, precision="fp32", polish=0, proj_iters=5):
    q = nmf.nmf_problem()
    q.V = q.Wt = q.W = q.H = q.chi2_hist = q.iters_done = 256
    q.prm = nmf.make_params(N, P, K, 5, precision=precision, polish_iters=polish)
    if M:
        q.T = q.WtT = q.C = q.R = 256
        q.M = M
        q.proj_iters = proj_iters
    return q


def test_batched_workspace_is_the_sum_of_fit_and_projection_slices(lib):
    a = _problem(40, 4000, 5)
    b = _problem(300, 20000, 30, M=7, precision="bf16", polish=3)
    c = _problem(800, 9000, 90, M=1)
    align = lambda x: (x + 255) // 256 * 256
    expect = 0
    for q in (a, b, c):
        expect += align(nmf.nmf_fit_workspace_bytes(q.prm))
        if q.M:
            expect += align(nmf.nmf_project_workspace_bytes(q.M, q.prm.P, q.prm.K, q.prm.precision))
    assert nmf.nmf_batched_workspace_bytes([a, b, c]) == expect
    assert nmf.nmf_batched_workspace_bytes([a]) == align(nmf.nmf_fit_workspace_bytes(a.prm))


def test_batched_rejects_bad_descriptors_without_device(lib):
    p = ctypes.c_void_p(256)
    good = _problem(40, 4000, 5, M=2)
    bad = []
    q = _problem(40, 4000, 5); q.reserved = 1; bad.append(q)
    q = _problem(40, 4000, 5); q.V = None; bad.append(q)
    q = _problem(40, 4000, 5, M=2); q.R = None; bad.append(q)
    q = _problem(40, 4000, 5, M=2); q.proj_iters = -1; bad.append(q)
    q = _problem(40, 4000, 5); q.M = -1; bad.append(q)
    bad.append(_problem(200, 4000, 129, precision="bf16"))  # above the component limit
    bad.append(_problem(10, 4000, 11))  # K > N
    for q in bad:
        assert nmf.nmf_batched_workspace_bytes([good, q]) == 0
        assert nmf.nmf_fit_batched([good, q], p, 1 << 40, None) == nmf.NMF_EINVAL
    need = nmf.nmf_batched_workspace_bytes([good])
    assert nmf.nmf_fit_batched([good], p, need - 1, None) == nmf.NMF_EINVAL
    assert nmf.nmf_fit_batched([good], ctypes.c_void_p(257), need, None) == nmf.NMF_EINVAL
    assert nmf.nmf_fit_batched([good], None, need, None) == nmf.NMF_EINVAL
    assert nmf.nmf_fit_batched([], p, need, None) == nmf.NMF_EINVAL
    assert nmf.nmf_batched_status([good], None, None)[0] == nmf.NMF_EINVAL


def test_reference_selection_rejects_bad_arguments_without_device(lib):
    p = ctypes.c_void_p(256)
    f = nmf.nmf_select_references
    assert f(None, p, 5, p, 300, 1000, 10, p, p, None) == nmf.NMF_EINVAL
    assert f(p, p, 0, p, 300, 1000, 10, p, p, None) == nmf.NMF_EINVAL
    assert f(p, p, 5, p, 300, 1000, 0, p, p, None) == nmf.NMF_EINVAL
    assert f(p, p, 5, p, 300, 1000, 301, p, p, None) == nmf.NMF_EINVAL
    assert f(p, p, 5, p, 8193, 1000, 10, p, p, None) == nmf.NMF_EINVAL
    assert f(p, p, 5, p, 300, 0, 10, p, p, None) == nmf.NMF_EINVAL
    assert f(p, p, 5, p, 300, 1000, 10, None, p, None) == nmf.NMF_EINVAL
    assert f(p, p, 262141, p, 300, 1000, 10, p, p, None) == nmf.NMF_EINVAL
    assert f(p, p, 5, p, 300, 1 << 28, 10, p, p, None) == nmf.NMF_EINVAL


def test_derotate_combine_rejects_bad_arguments_without_device(lib):
    p = ctypes.c_void_p(256)
    ang = (ctypes.c_double * 4)(0.0, 10.0, 20.0, 30.0)
    bad_ang = (ctypes.c_double * 4)(0.0, float("nan"), 20.0, 30.0)
    f = nmf.nmf_derotate_combine
    E = nmf.NMF_EINVAL
    assert f(None, 4, 64, 64, None, ang, 32.0, 32.0, 0, None, p, None, None) == E
    assert f(p, 4, 64, 64, None, None, 32.0, 32.0, 0, None, p, None, None) == E
    assert f(p, 4, 64, 64, None, ang, 32.0, 32.0, 0, None, None, None, None) == E  # no output at all
    assert f(p, 0, 64, 64, None, ang, 32.0, 32.0, 0, None, p, None, None) == E
    assert f(p, 1025, 64, 64, None, ang, 32.0, 32.0, 0, None, p, None, None) == E
    assert f(p, 4, 0, 64, None, ang, 32.0, 32.0, 0, None, p, None, None) == E
    assert f(p, 4, 64, 16385, None, ang, 32.0, 32.0, 0, None, p, None, None) == E
    assert f(p, 4, 64, 64, None, ang, 32.0, 32.0, 2, None, p, None, None) == E
    assert f(p, 4, 64, 64, None, ang, float("inf"), 32.0, 0, None, p, None, None) == E
    assert f(p, 4, 64, 64, None, ang, 32.0, float(2 ** 21), 0, None, p, None, None) == E
    assert f(p, 4, 64, 64, None, ang, float("nan"), 32.0, 0, None, p, None, None) == E
    assert f(p, 4, 64, 64, None, bad_ang, 32.0, 32.0, 0, None, p, None, None) == E


@pytest.mark.parametrize("rows,P,sms", [(300, 49343, 152), (1000, 62961, 152), (200, 25000, 152), (129, 40000, 148),
                                        (45, 30000, 132), (300, 4000, 152), (2100, 60000, 152), (640, 20000, 152)])
def test_w_schedule_covers_every_chunk_once(lib, rows, P, sms):
    """The tensor-core fit's W-pass schedule (host logic only): every 64-pixel
    chunk of every 128-row tile is streamed by exactly one block, each tile's
    partial slots are 0 .. n - 1, the blocks fit on the SMs at once, and the
    long first-wave blocks (launched first, onto the SMs the H pass frees a
    tile early) read only pixels the H pass writes before its last round."""
    Pp = -(-P // 128) * 128
    nch, ntr, ntiles = Pp // 64, -(-rows // 128), Pp // 128
    hb = min(ntiles, sms)
    r = nmf.w_schedule(rows, P, sms)
    if r is None:  # equal splits: tiles a multiple of the H blocks, or too many row tiles
        assert ntiles % hb == 0 or ntr > 16
        return
    tile, split, c0, c1 = r
    assert 0 < len(tile) <= sms
    for t in range(ntr):
        sel = np.flatnonzero(tile == t)
        assert sel.size >= 1
        ranges = sorted(zip(c0[sel].tolist(), c1[sel].tolist()))
        assert ranges[0][0] == 0 and ranges[-1][1] == nch
        assert all(a < b for a, b in ranges)
        assert all(ranges[i][1] == ranges[i + 1][0] for i in range(len(ranges) - 1))
        assert sorted(split[sel].tolist()) == list(range(sel.size))
    early_lim = (ntiles // hb) * hb * 128 // 64
    length = c1 - c0
    longest = np.flatnonzero(length == length.max())
    beyond = np.flatnonzero(c0 >= early_lim)
    assert length.max() > length.min()
    assert np.all(c1[longest] <= early_lim)
    if beyond.size:
        assert longest.max() < beyond.min()


def test_w_schedule_rejects_bad_arguments(lib):
    assert nmf.nmf_w_schedule(0, 100, 152, 0, None, None, None, None) == -1
    assert nmf.nmf_w_schedule(300, 49343, 0, 0, None, None, None, None) == -1
    assert nmf.nmf_w_schedule(300, 49343, 152, 4, None, None, None, None) == -1  # arrays missing
    with pytest.raises(nmf.NmfError):
        nmf.w_schedule(300, 49343, 152, max_blocks=8)  # more blocks than room


def test_wait_selftest_rejects_bad_arguments_without_device(lib):
    st = (ctypes.c_int32 * 2)()
    assert nmf.nmf_wait_selftest(1_000_000, None, None) == nmf.NMF_EINVAL
    assert nmf.nmf_wait_selftest(10, st, None) == nmf.NMF_EINVAL
    assert nmf.nmf_wait_selftest(10 ** 9, st, None) == nmf.NMF_EINVAL
