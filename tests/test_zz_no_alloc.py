"""The projection entry point that allocates nothing.

nmf_project_target_noalloc serves callers that cannot give the library a
workspace -- a program whose device memory is fixed at start-up or owned by
another framework, or a loop that must never reach cudaMalloc.  It keeps its
scratch in a fixed array compiled into the library, shared by all calls.
These checks call it through the C-ABI twice in a row (the shared scratch
keeps the previous call's contents) and compare each result with the
workspace-based nmf_project_target at the FP32 tolerance of the other parity
tests.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nmf():
    from paper_2309_04623_gb300 import build
    from paper_2309_04623_gb300 import nmf as _nmf

    build.build()
    _nmf.load()
    return _nmf


def _problem(seed, M, K, P):
    rng = np.random.default_rng(seed)
    H = rng.uniform(0.0, 1.0, (K, P)).astype(np.float32)
    T = (rng.uniform(0.2, 1.0, (M, K)) @ H + rng.normal(0.0, 0.05, (M, P))).clip(0.0).astype(np.float32)
    WtT = rng.uniform(0.5, 2.0, (M, P)).astype(np.float32)
    C0 = rng.uniform(0.1, 1.0, (M, K)).astype(np.float32)
    return H, T, WtT, C0


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_projection_matches_workspace_projection_twice(nmf):
    dev = torch.device("cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    # two different problems back to back: the second call must not be
    # affected by what the first one left in the shared scratch
    # (seed, M, K, P, iters): the narrow and the 33..64-component W-pass
    # layouts, and the two shapes that fill the scratch exactly (M = 64,
    # K = 64, 64 pixel splits of 128 and of 256 pixels)
    for seed, M, K, P, iters in ((1, 7, 12, 3001, 40), (2, 50, 30, 4999, 25), (3, 20, 40, 6007, 20),
                                 (4, 64, 64, 8192, 15), (5, 64, 64, 16384, 10)):
        H, T, WtT, C0 = _problem(seed, M, K, P)
        ref = nmf.project_target(H, T, WtT, C0, iters).cpu().numpy()
        Hd, Td, Wd = (torch.from_numpy(x).to(dev) for x in (H, T, WtT))
        Cd = torch.from_numpy(C0).to(dev)
        stream = torch.cuda.current_stream()
        rc = nmf.nmf_project_target_noalloc(p(Hd), K, P, p(Td), p(Wd), M, p(Cd), iters, 1e-30,
                                            ctypes.c_void_p(stream.cuda_stream))
        assert rc == nmf.NMF_OK, nmf.status_string(rc)
        torch.cuda.synchronize()
        got = Cd.cpu().numpy()
        assert _rel(got, ref) <= 1e-5


def test_noalloc_rejects_sizes_beyond_its_scratch(nmf):
    p = ctypes.c_void_p(256)  # never dereferenced: the size check fails first
    assert nmf.nmf_project_target_noalloc(p, 65, 1000, p, p, 4, p, 5, 1e-30, None) == nmf.NMF_EINVAL
    assert nmf.nmf_project_target_noalloc(p, 8, 1000, p, p, 65, p, 5, 1e-30, None) == nmf.NMF_EINVAL
    assert nmf.nmf_project_target_noalloc(p, 8, 4, p, p, 4, p, 5, 1e-30, None) == nmf.NMF_EINVAL
