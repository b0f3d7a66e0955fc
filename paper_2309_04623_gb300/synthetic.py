"""Seeded synthetic coronagraphic data: reference-PSF libraries, science frames
and the random initial factors.

This module is the one piece of code that both the CUDA path and the FP64
oracle consume.  It holds none of the method's arithmetic (no factorisation,
no projection, no subtraction): it only draws images, masks, weights and the
uniform random initial factors W0, H0, C0 that the method starts from (the
paper initialises H and W randomly, Sec. 2, after Eq. 3).

Data model (stand-in for the HST-STIS WedgeA1.0 and JWST-MIRI 4QPM frames of
Sec. 3 and Sec. 4, which are not available here):

* one reference frame = one row of V, holding the P pixels that survive the
  algorithmic mask (Sec. 4.1: masked regions are missing data); pixels are
  compacted and stored contiguously, row-major;
* weights Wt = 1 / sigma^2 on the surviving pixels (Eq. 2: the weighting term
  accounts for heteroscedastic errors; for HST it comes from the ERR
  extension, Sec. 2);
* PSF = amplitude * [Gaussian core (FWHM 3 px) + halo * (1 + (r/3)^2)^-1 *
  lognormal speckle field], speckles spatially correlated over 2 px and
  partially shared across references (correlation rho);
* photon noise is Poisson at a 1e4-count peak; MIRI-shaped frames add a
  thermal offset 50 +/- 5 counts and Gaussian read noise sigma 10, with
  negative values clamped to 0;
* a science frame = a Dirichlet(1)-weighted mixture of the noiseless
  references plus an inclined ring disk (peak 1% of the star), Poisson noise.

Every array is float32; every draw comes from numpy's PCG64 seeded per
workload (seed 2309046230 + workload index unless given).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

try:  # scipy is present on both machines; the fallback keeps the module importable
    from scipy.ndimage import gaussian_filter as _gaussian_filter
except Exception:  # pragma: no cover
    _gaussian_filter = None

SEED_BASE = 2309046230


@dataclasses.dataclass
class Problem:
    """One reduction: a reference library, its science frames and initial factors."""

    name: str
    V: np.ndarray  # (N, P) float32, reference library, non-negative
    Wt: np.ndarray  # (N, P) float32, weights 1/sigma^2 (0 = missing)
    T: np.ndarray  # (M, P) float32, science frames
    WtT: np.ndarray  # (M, P) float32, science-frame weights
    W0: np.ndarray  # (N, K) float32, U(0,1) initial coefficients
    H0: np.ndarray  # (K, P) float32, U(0,1) initial components
    C0: np.ndarray  # (M, K) float32, U(0,1) initial projection coefficients
    n_iter: int  # multiplicative-update iterations per stage (and per projection)
    pix_idx: np.ndarray  # (P,) int32, flat image index of each kept pixel
    img_shape: Tuple[int, int]
    meta: dict

    @property
    def N(self) -> int:
        return self.V.shape[0]

    @property
    def P(self) -> int:
        return self.V.shape[1]

    @property
    def K(self) -> int:
        return self.H0.shape[0]

    @property
    def M(self) -> int:
        return self.T.shape[0]


# ---------------------------------------------------------------------------
# masks


def _radius(shape, center):
    yy, xx = np.indices(shape, dtype=np.float64)
    return np.hypot(yy - center[0], xx - center[1]), yy - center[0], xx - center[1]


def annulus_mask(shape, center, r_in, r_out):
    r, _, _ = _radius(shape, center)
    return (r >= r_in) & (r <= r_out)


def stis_wedge_mask(shape, center, r_in=8.0, r_out=140.0, bar_width=20.0, spike_width=6.0):
    """Annulus minus a horizontal occulting bar and two diagonal spike bands
    (the WedgeA1.0 occulter and diffraction spikes treated as missing data)."""
    r, dy, dx = _radius(shape, center)
    keep = (r >= r_in) & (r <= r_out)
    keep &= np.abs(dy) > bar_width / 2.0
    # spikes along the two diagonals
    d1 = np.abs(dy - dx) / math.sqrt(2.0)
    d2 = np.abs(dy + dx) / math.sqrt(2.0)
    keep &= (d1 > spike_width / 2.0) & (d2 > spike_width / 2.0)
    return keep


def miri_4qpm_mask(shape, center, line_width=3, r_in=5.0):
    """Four-quadrant phase mask: the horizontal and vertical transition lines
    (line_width px) through the centre and a central disk r < r_in are zeroed."""
    r, dy, dx = _radius(shape, center)
    keep = r >= r_in
    half = line_width / 2.0
    keep &= np.abs(dy) > half - 0.5 + 1e-9
    keep &= np.abs(dx) > half - 0.5 + 1e-9
    return keep


def mask_with_count(side, P, bar_width, rng):
    """Square image of the given side with a random annulus / bar mask holding
    exactly P pixels (used for the uneven batched workload)."""
    c = (side / 2.0, side / 2.0)
    r, dy, dx = _radius((side, side), c)
    r_in = float(rng.uniform(3.0, 8.0))
    ok = (r >= r_in) & (np.abs(dy) > bar_width / 2.0)
    order = np.argsort(np.where(ok, r, np.inf).ravel(), kind="stable")
    keep = np.zeros(side * side, dtype=bool)
    if ok.sum() < P:
        raise ValueError("mask too small for requested P")
    keep[order[:P]] = True
    return keep.reshape(side, side)


# ---------------------------------------------------------------------------
# PSF model


def _smooth_unit_noise(rng, shape, sigma_px):
    g = rng.standard_normal(shape)
    if _gaussian_filter is not None:
        g = _gaussian_filter(g, sigma_px, mode="wrap")
    else:  # pragma: no cover - FFT smoothing
        ky = np.fft.fftfreq(shape[0])[:, None]
        kx = np.fft.fftfreq(shape[1])[None, :]
        g = np.fft.ifft2(np.fft.fft2(g) * np.exp(-2 * (math.pi * sigma_px) ** 2 * (kx**2 + ky**2))).real
    g -= g.mean()
    g /= g.std() + 1e-300
    return g


def _psf_stack(rng, n, shape, center, *, fwhm=3.0, halo=1e-2, sig_s=0.5, corr_px=2.0, rho=0.9, peak=1e4):
    """Noiseless PSFs lambda_n (n, H, W) in counts."""
    r, _, _ = _radius(shape, center)
    s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    core = np.exp(-(r**2) / (2.0 * s * s))
    halo_prof = halo / (1.0 + (r / 3.0) ** 2)
    g_common = _smooth_unit_noise(rng, shape, corr_px)
    out = np.empty((n,) + tuple(shape), dtype=np.float64)
    amps = rng.uniform(0.8, 1.2, size=n)
    for i in range(n):
        g = math.sqrt(rho) * g_common + math.sqrt(1.0 - rho) * _smooth_unit_noise(rng, shape, corr_px)
        speck = np.exp(sig_s * g - sig_s * sig_s / 2.0)
        out[i] = peak * amps[i] * (core + halo_prof * speck)
    return out


def _ring_disk(shape, center, radius, incl_deg, pa_deg, width, peak):
    _, dy, dx = _radius(shape, center)
    pa = math.radians(pa_deg)
    xp = dx * math.cos(pa) + dy * math.sin(pa)
    yp = (-dx * math.sin(pa) + dy * math.cos(pa)) / max(math.cos(math.radians(incl_deg)), 1e-6)
    rd = np.hypot(xp, yp)
    return peak * np.exp(-((rd - radius) ** 2) / (2.0 * width * width))


def _uniform_f32(rng, shape):
    # U(0,1) drawn in float64, rounded once to float32; exact zeros are
    # replaced so that no factor entry starts pinned at 0 by accident.
    x = rng.random(shape)
    x = np.where(x == 0.0, 0.5, x)
    return x.astype(np.float32)


def _build(
    name,
    rng,
    *,
    N,
    K,
    M,
    n_iter,
    shape,
    center,
    keep,
    disk_radius,
    miri=False,
    rho=0.9,
    halo=1e-2,
):
    lam = _psf_stack(rng, N, shape, center, rho=rho, halo=halo)
    pix_idx = np.flatnonzero(keep.ravel()).astype(np.int32)
    P = pix_idx.size
    lam_p = lam.reshape(N, -1)[:, pix_idx]
    if miri:
        offs = rng.normal(50.0, 5.0, size=(N, 1))
        lam_tot = lam_p + offs
        V = rng.poisson(lam_tot).astype(np.float64) + rng.normal(0.0, 10.0, size=lam_tot.shape)
        n_neg = int((V < 0).sum())
        V = np.maximum(V, 0.0)
        sig2 = np.maximum(lam_tot, 0.0) + 100.0
    else:
        lam_tot = lam_p
        V = rng.poisson(lam_tot).astype(np.float64)
        n_neg = 0
        sig2 = np.maximum(lam_tot, 1.0)
    Wt = 1.0 / sig2

    # science frames: Dirichlet(1) mixtures of the noiseless references + disk
    disk = _ring_disk(shape, center, disk_radius, 70.0, 30.0, 1.5, 0.01 * 1e4).ravel()[pix_idx]
    alpha = rng.dirichlet(np.ones(N), size=M)
    lamT = alpha @ lam_tot + disk[None, :]
    if miri:
        T = rng.poisson(lamT).astype(np.float64) + rng.normal(0.0, 10.0, size=lamT.shape)
        n_neg += int((T < 0).sum())
        T = np.maximum(T, 0.0)
        sig2T = np.maximum(lamT, 0.0) + 100.0
    else:
        T = rng.poisson(lamT).astype(np.float64)
        sig2T = np.maximum(lamT, 1.0)
    WtT = 1.0 / sig2T

    W0 = _uniform_f32(rng, (N, K))
    H0 = _uniform_f32(rng, (K, P))
    C0 = _uniform_f32(rng, (M, K))
    meta = dict(n_negative_clamped=n_neg, disk_radius=disk_radius, rho=rho, halo=halo, miri=miri)
    return Problem(
        name=name,
        V=np.ascontiguousarray(V, dtype=np.float32),
        Wt=np.ascontiguousarray(Wt, dtype=np.float32),
        T=np.ascontiguousarray(T, dtype=np.float32),
        WtT=np.ascontiguousarray(WtT, dtype=np.float32),
        W0=W0,
        H0=H0,
        C0=C0,
        n_iter=n_iter,
        pix_idx=pix_idx,
        img_shape=tuple(shape),
        meta=meta,
    )


# ---------------------------------------------------------------------------
# the five workloads

WORKLOADS = {
    0: "oracle-size: N=50 refs of 64x64, annulus 6<=r<=30 (P=2712), K=5 x 200 it",
    1: "STIS-shaped: N=300 refs of 256x256, annulus+wedge+spikes (P~49k), K=30 x 500 it, M=50",
    2: "STIS-shaped precision form: config-1 data, K up to 100",
    3: "MIRI-shaped: N=1000 refs of 224x288, 4QPM lines + r<5 (P~63k), K=50 x 500 it, M=50",
    4: "batched: 64 reductions, N~U[40,800], P~U[4k,80k], K~min(U[5,100],N), M~U[1,20]",
}


def make_config(idx: int, seed: Optional[int] = None, *, N=None, K=None, M=None, n_iter=None) -> Problem:
    """Build workload `idx` (0..3).  Keyword overrides shrink it for tests."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + idx if seed is None else seed))
    if idx == 0:
        shape, center = (64, 64), (32.0, 32.0)
        keep = annulus_mask(shape, center, 6.0, 30.0)
        return _build(
            "config0", rng, N=N or 50, K=K or 5, M=M or 1, n_iter=n_iter or 200,
            shape=shape, center=center, keep=keep, disk_radius=18.0,
        )
    if idx in (1, 2):
        shape, center = (256, 256), (128.0, 128.0)
        keep = stis_wedge_mask(shape, center)
        return _build(
            f"config{idx}", rng, N=N or 300, K=K or (30 if idx == 1 else 100), M=M or 50,
            n_iter=n_iter or 500, shape=shape, center=center, keep=keep, disk_radius=60.0,
        )
    if idx == 3:
        shape, center = (224, 288), (112.0, 144.0)
        keep = miri_4qpm_mask(shape, center)
        return _build(
            "config3", rng, N=N or 1000, K=K or 50, M=M or 50, n_iter=n_iter or 500,
            shape=shape, center=center, keep=keep, disk_radius=45.0, miri=True,
        )
    raise ValueError(f"unknown workload {idx}")


def make_problem(seed: int, N: int, P: int, K: int, M: int = 1, n_iter: int = 20, miri: bool = False) -> Problem:
    """A problem of arbitrary size on a square image holding exactly P pixels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    side = int(math.ceil(math.sqrt(P / 0.7))) + 4
    keep = mask_with_count(side, P, bar_width=float(rng.uniform(2.0, 8.0)), rng=rng)
    c = (side / 2.0, side / 2.0)
    return _build(
        f"problem_s{seed}", rng, N=N, K=K, M=M, n_iter=n_iter, shape=(side, side), center=c,
        keep=keep, disk_radius=side * 0.3, miri=miri,
    )


def _make_problem_spec(spec):
    sub, N, P, K, M, n_iter, name = spec
    pr = make_problem(sub, N, P, K, M, n_iter=n_iter)
    pr.name = name
    return pr


def make_batched(seed: Optional[int] = None, count: int = 64, *, n_iter: int = 100,
                 n_range=(40, 800), p_range=(4000, 80000), k_range=(5, 100), m_range=(1, 20),
                 workers: int = 1) -> List[Problem]:
    """The uneven batched workload: `count` independent reductions.

    Every problem has its own seed drawn from the batch's generator, so the
    result does not depend on `workers` (> 1 builds the problems in a pool
    of spawned processes)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4 if seed is None else seed))
    specs = []
    for b in range(count):
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        P = int(rng.integers(p_range[0], p_range[1] + 1))
        K = int(min(rng.integers(k_range[0], k_range[1] + 1), N, P))
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        sub = int(rng.integers(0, 2**31 - 1))
        specs.append((sub, N, P, K, M, n_iter, f"batch{b}"))
    if workers <= 1:
        return [_make_problem_spec(sp) for sp in specs]
    import concurrent.futures
    import multiprocessing

    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        return list(ex.map(_make_problem_spec, specs))


def roll_angles(F: int, seed: Optional[int] = None) -> np.ndarray:
    """Position angles (degrees) of F science frames for the North-up step:
    observations at three roll orientations 120 degrees apart, each frame
    within +-30 degrees of its orientation (HST-style roll dithers)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 77 if seed is None else seed))
    return (rng.integers(0, 3, F) * 120.0 + rng.uniform(-30.0, 30.0, F)).astype(np.float64)


def random_factors(seed: int, N: int, P: int, K: int):
    """Dense U(0,1) float32 W (N,K), H (K,P) for small self-contained tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _uniform_f32(rng, (N, K)), _uniform_f32(rng, (K, P))


def random_matrix(seed: int, shape, lo=0.0, hi=1.0, zero_frac=0.0):
    """U(lo,hi) float32 matrix with an optional fraction of exact zeros."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(lo, hi, size=shape)
    if zero_frac > 0:
        x[rng.random(shape) < zero_frac] = 0.0
    return x.astype(np.float32)
