"""GPU parity of the North-up rotation and stacking of the subtracted frames
(Sec. 4.1, 4.2) against the FP64 oracle.

Which source pixels a rotated pixel uses (and whether it is missing) is an
integer decision taken in float on both sides by the same rounded
operations, so the NaN pattern and the coverage counts must agree exactly.
The interpolated values are FP32 on the GPU: each is a weighted sum of at
most four pixels with weights in [0, 1] summing to 1, so its error is a few
float roundings of the largest neighbour; the mean (compensated FP32 sum)
and the median (1-Lipschitz in every value, final halving rounded once) add
one or two more.  Tolerance: 2e-6 of the frame's largest magnitude."""
import numpy as np
import pytest

import oracle
from paper_2309_04623_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REL = 2e-6


@pytest.fixture(scope="module")
def nmf():
    from paper_2309_04623_gb300 import build
    from paper_2309_04623_gb300 import nmf as _nmf

    build.build()
    _nmf.load()
    return _nmf


def _frames(seed, F, ny, nx, nan_frac=0.02, lo=-50.0, hi=50.0):
    rng = np.random.default_rng(seed)
    img = rng.uniform(lo, hi, (F, ny, nx)).astype(np.float32)
    img[rng.uniform(size=img.shape) < nan_frac] = np.nan
    return img


def _check(nmf, img, ang, center, valid=None, methods=("mean", "median")):
    scale = float(np.nanmax(np.abs(img))) if np.isfinite(img).any() else 1.0
    ref_rot = oracle.rotate(img, ang, center, valid=valid)
    for method in methods:
        out, cnt, rot = nmf.derotate_combine(img, ang, center, method=method, valid=valid, rotated=True)
        torch.cuda.synchronize()
        rot = rot.cpu().numpy()
        assert np.array_equal(np.isnan(rot), np.isnan(ref_rot))
        ok = ~np.isnan(ref_rot)
        np.testing.assert_allclose(rot[ok], ref_rot[ok], rtol=0, atol=REL * scale)
        ref_out, ref_cnt = oracle.combine(ref_rot, method)
        assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
        out = out.cpu().numpy()
        assert np.array_equal(np.isnan(out), np.isnan(ref_out))
        ok = ~np.isnan(ref_out)
        np.testing.assert_allclose(out[ok], ref_out[ok], rtol=0, atol=REL * scale)


@pytest.mark.parametrize("F,ny,nx", [(1, 1, 1), (3, 1, 40), (7, 37, 75), (12, 64, 96)])
def test_rotation_and_stacking_match_oracle(nmf, F, ny, nx):
    """Several 32 x 8 tiles with ragged right and bottom edges, NaN holes,
    angles including exact quarter turns and the identity."""
    img = _frames(F * 100 + ny, F, ny, nx)
    base = [0.0, 90.0, 180.0, -37.5, 12.25, 300.1, 45.0, 270.0, -0.3, 359.9, 1e-3, 91.7]
    ang = np.array(base[:F])
    _check(nmf, img, ang, ((nx - 1) / 2.0, (ny - 1) / 2.0))
    _check(nmf, img, ang, (nx * 0.37, ny * 0.61), methods=("median",))


def test_valid_mask_and_fully_missing_pixels(nmf):
    """Pixels flagged invalid are missing in every frame; a pixel that no
    frame covers stacks to NaN with count 0."""
    F, ny, nx = 5, 50, 70
    img = _frames(7, F, ny, nx, nan_frac=0.0)
    valid = np.ones((ny, nx), np.uint8)
    valid[20:30, 30:40] = 0  # the same hole in every frame stays uncovered at angle 0
    ang = np.zeros(F)
    _check(nmf, img, ang, (35.0, 25.0), valid=valid)
    out, cnt, _ = nmf.derotate_combine(img, ang, (35.0, 25.0), method="median", valid=valid)
    cnt = cnt.cpu().numpy()
    assert (cnt[20:30, 30:40] == 0).all() and np.isnan(out.cpu().numpy()[20:30, 30:40]).all()
    assert (cnt[valid == 1] == F).all()
    # rotations fill the hole from the other frames
    ang = np.array([0.0, 40.0, 80.0, 120.0, 160.0])
    _check(nmf, img, ang, (35.0, 25.0), valid=valid)


def test_identity_stacks_are_exact(nmf):
    """At angle 0 every rotated value is the input value itself, so the
    median equals numpy's nanmedian exactly (integer-valued frames, many
    ties, even and odd counts) and the coverage is the count of non-NaN."""
    rng = np.random.default_rng(11)
    F, ny, nx = 10, 19, 45
    img = rng.integers(-3, 4, (F, ny, nx)).astype(np.float32)
    img[rng.uniform(size=img.shape) < 0.3] = np.nan
    out, cnt, rot = nmf.derotate_combine(img, np.zeros(F), (22.0, 9.0), method="median", rotated=True)
    rot = rot.cpu().numpy()
    assert np.array_equal(np.isnan(rot), np.isnan(img)) and np.array_equal(rot[~np.isnan(img)], img[~np.isnan(img)])
    with np.errstate(all="ignore"):
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", RuntimeWarning)
            ref = np.nanmedian(img.astype(np.float64), axis=0)
    out = out.cpu().numpy()
    assert np.array_equal(np.isnan(out), np.isnan(ref))
    assert np.array_equal(out[~np.isnan(ref)], ref[~np.isnan(ref)].astype(np.float32))
    assert np.array_equal(cnt.cpu().numpy(), (~np.isnan(img)).sum(axis=0))


def test_many_frames_median(nmf):
    """F = 1024 (the limit): one row of 32 threads per block holds every
    frame's value for the selection."""
    F, ny, nx = 1024, 9, 40
    img = _frames(13, F, ny, nx, nan_frac=0.05)
    ang = np.random.default_rng(14).uniform(-180, 180, F)
    _check(nmf, img, ang, (19.5, 4.0), methods=("median",))


def test_rotation_only_and_count_only(nmf):
    F, ny, nx = 4, 33, 41
    img = _frames(15, F, ny, nx)
    ang = np.array([10.0, -20.0, 30.0, 200.0])
    _, cnt, rot = nmf.derotate_combine(img, ang, (20.0, 16.0), rotated=True, stacked=False)
    ref = oracle.rotate(img, ang, (20.0, 16.0))
    rot = rot.cpu().numpy()
    assert np.array_equal(np.isnan(rot), np.isnan(ref))
    assert np.array_equal(cnt.cpu().numpy(), (~np.isnan(ref)).sum(axis=0))


def test_stis_shaped_residual_stack(nmf):
    """The STIS-shaped grid (256 x 256, the wedge and spike mask as missing
    data), 50 subtracted-like frames at the synthetic roll angles (three
    orientations 120 degrees apart, +-30 degrees around each)."""
    F, ny, nx = 50, 256, 256
    keep = synthetic.stis_wedge_mask((ny, nx), (128.0, 128.0))
    rng = np.random.default_rng(16)
    img = rng.normal(0.0, 5.0, (F, ny, nx)).astype(np.float32)
    ang = synthetic.roll_angles(F)
    _check(nmf, img, ang, (128.0, 128.0), valid=keep.astype(np.uint8))
