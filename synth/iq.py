"""Seeded synthetic ultrasound IQ packets shaped like the paper's acquisitions.

Shared by the tests, the oracle runs and ``bench.py``.  This module holds
none of the clutter filter's arithmetic: it only draws inputs.

Recipe (the paper's phantom / kidney / liver data are not available, so
these stand in for them; sizes follow the workloads the library is timed on):

* tissue: complex white Gaussian noise on a padded grid, smoothed by an
  isotropic Gaussian kernel so that the field's autocorrelation has a FWHM of
  3 px (speckle), normalised to unit mean power over the image; every frame
  is the same field shifted axially by d(t) pixels with an exact Fourier
  sub-pixel shift, then cropped (the padding keeps the shift from wrapping);
  optionally each column x moves by d(t) g(x) with g a lateral ramp (motion
  that differs across the field of view, as in vivo);
* blood: straight vessels (pixels within width/2 of a line at a random angle
  and offset); per pixel a unit-variance complex AR(1) process
  b_t = rho*b_{t-1} + sqrt(1-rho^2)*n_t (rho = 0.99, scatterer decorrelation)
  times a Doppler phase ramp exp(i*phi*t), scaled to 10^(-TBR/10) power;
* noise: complex white Gaussian at ``noise_db`` dB below the tissue power.

Output: complex64 array [nt][nz][nx] (x fastest), the library's layout.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SPECKLE_FWHM_PX = 3.0


@dataclass(frozen=True)
class Recipe:
    nz: int
    nx: int
    nt: int
    n_vessels: int | tuple = 2
    width_px: float | tuple = 4.0
    phi_rad: float | tuple = 0.3          # Doppler step per frame (range -> uniform draw)
    tbr_db: float | tuple = 40.0          # tissue-to-blood power ratio
    noise_db: float = -60.0               # noise power relative to tissue
    motion_amp_px: float | tuple = 0.2    # axial sinusoid amplitude
    motion_period: float | None = None    # frames; None -> nt
    jitter_px: float = 0.0                # per-frame N(0, jitter^2) axial jitter
    rho: float = 0.99
    # lateral heterogeneity of the motion: column x moves by d(t) * g(x), g rising linearly from
    # motion_lateral_gain[0] at x = 0 to [1] at x = nx - 1 (None: every column moves by d(t))
    motion_lateral_gain: tuple | None = None


# Workloads, named by what they are.
SMALL_96x64x32 = Recipe(96, 64, 32, n_vessels=2, width_px=4.0, phi_rad=0.3, tbr_db=40.0,
                        noise_db=-60.0, motion_amp_px=0.2)
REALTIME_256x128x100 = Recipe(256, 128, 100, n_vessels=8, width_px=(2.0, 10.0),
                              phi_rad=(0.05, 1.0), tbr_db=50.0, noise_db=-65.0, motion_amp_px=0.2)
STREAM_512x256x200 = Recipe(512, 256, 200, n_vessels=8, width_px=(2.0, 10.0),
                            phi_rad=(0.05, 1.0), tbr_db=50.0, noise_db=-65.0, motion_amp_px=0.2)
STRESS_256x192x300 = Recipe(256, 192, 300, n_vessels=8, width_px=(2.0, 10.0),
                            phi_rad=(0.05, 1.0), tbr_db=60.0, noise_db=-75.0,
                            motion_amp_px=1.5, motion_period=200.0, jitter_px=0.5)
LEARNED_384x256x128 = Recipe(384, 256, 128, n_vessels=(2, 12), width_px=(2.0, 10.0),
                             phi_rad=(0.05, 1.0), tbr_db=(40.0, 60.0), noise_db=-65.0,
                             motion_amp_px=(0.0, 2.0))


def _draw(rng, v):
    if isinstance(v, tuple):
        lo, hi = v
        if isinstance(lo, int) and isinstance(hi, int):
            return int(rng.integers(lo, hi + 1))
        return float(rng.uniform(lo, hi))
    return v


def _speckle_field(rng, zp, xp):
    """Complex Gaussian field whose autocorrelation FWHM is SPECKLE_FWHM_PX."""
    # smoothing kernel std s: autocorrelation = kernel (x) kernel -> std sqrt(2)*s
    s = SPECKLE_FWHM_PX / (2.0 * np.sqrt(2.0 * np.log(2.0)) * np.sqrt(2.0))
    w = (rng.standard_normal((zp, xp)) + 1j * rng.standard_normal((zp, xp))) / np.sqrt(2.0)
    fz = np.fft.fftfreq(zp)[:, None]
    fx = np.fft.fftfreq(xp)[None, :]
    H = np.exp(-2.0 * np.pi ** 2 * s ** 2 * (fz ** 2 + fx ** 2))
    return np.fft.ifft2(np.fft.fft2(w) * H)


def vessel_masks(rng, nz, nx, n_vessels, width_px):
    masks = []
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    for _ in range(n_vessels):
        w = _draw(rng, width_px)
        th = rng.uniform(0.0, np.pi)
        z0, x0 = rng.uniform(0, nz), rng.uniform(0, nx)
        # distance to the line through (z0, x0) with direction (cos th, sin th)
        d = np.abs(-(zz - z0) * np.sin(th) + (xx - x0) * np.cos(th))
        masks.append(d <= 0.5 * w)
    return masks


def generate_frames(recipe: Recipe, n_frames: int, seed: int = 0, return_truth: bool = False):
    """A continuous sequence of ``n_frames`` frames [n_frames][nz][nx] complex64."""
    rng = np.random.default_rng(seed)
    nz, nx = recipe.nz, recipe.nx
    amp = _draw(rng, recipe.motion_amp_px)
    period = recipe.motion_period or recipe.nt
    t = np.arange(n_frames)
    d = amp * np.sin(2.0 * np.pi * t / period)
    if recipe.jitter_px > 0:
        d = d + rng.normal(0.0, recipe.jitter_px, n_frames)
    pad_z = int(np.ceil(np.max(np.abs(d)))) + 16
    pad_x = 8
    zp, xp = nz + 2 * pad_z, nx + 2 * pad_x
    field = _speckle_field(rng, zp, xp)
    crop = field[pad_z:pad_z + nz, pad_x:pad_x + nx]
    field /= np.sqrt(np.mean(np.abs(crop) ** 2))
    Fz = np.fft.fft(field, axis=0)
    kz = np.fft.fftfreq(zp)[:, None]

    n_v = _draw(rng, recipe.n_vessels)
    masks = vessel_masks(rng, nz, nx, n_v, recipe.width_px)
    tbr = _draw(rng, recipe.tbr_db)
    b_amp = np.sqrt(10.0 ** (-tbr / 10.0))
    phis = [(_draw(rng, recipe.phi_rad)) * (1 if rng.random() < 0.5 else -1) for _ in masks]
    idx = [np.nonzero(m.ravel())[0] for m in masks]
    states = [(rng.standard_normal(i.size) + 1j * rng.standard_normal(i.size)) / np.sqrt(2.0)
              for i in idx]
    n_amp = np.sqrt(10.0 ** (recipe.noise_db / 10.0))
    rho = recipe.rho
    inn = np.sqrt(1.0 - rho * rho)

    out = np.empty((n_frames, nz, nx), np.complex64)
    if recipe.motion_lateral_gain is not None:   # per-column gain over the padded width
        g0, g1 = recipe.motion_lateral_gain
        gx = g0 + (g1 - g0) * np.clip((np.arange(xp) - pad_x) / max(nx - 1, 1), 0.0, 1.0)
    else:
        gx = np.ones(xp)
    for f in range(n_frames):
        shifted = np.fft.ifft(Fz * np.exp(-2j * np.pi * kz * d[f] * gx[None, :]), axis=0)
        frame = shifted[pad_z:pad_z + nz, pad_x:pad_x + nx].copy()
        flat = frame.reshape(-1)
        for v in range(len(masks)):
            if f > 0:
                states[v] = rho * states[v] + inn * (
                    rng.standard_normal(idx[v].size) + 1j * rng.standard_normal(idx[v].size)
                ) / np.sqrt(2.0)
            flat[idx[v]] += b_amp * states[v] * np.exp(1j * phis[v] * f)
        frame += n_amp * (rng.standard_normal((nz, nx)) + 1j * rng.standard_normal((nz, nx))) / np.sqrt(2.0)
        out[f] = frame
    if return_truth:
        blood = np.zeros((nz, nx), bool)
        for m in masks:
            blood |= m
        return out, {"blood_mask": blood, "motion_px": d, "tbr_db": tbr, "n_vessels": n_v}
    return out


def generate_packet(recipe: Recipe, seed: int = 0, return_truth: bool = False):
    """One packet [nt][nz][nx] complex64."""
    return generate_frames(recipe, recipe.nt, seed=seed, return_truth=return_truth)


def packet_ring(recipe: Recipe, n_packets: int, seed: int = 0) -> np.ndarray:
    """``n_packets`` independent packets [n][nt][nz][nx] (seeds seed..seed+n-1)."""
    return np.stack([generate_packet(recipe, seed=seed + i) for i in range(n_packets)])
