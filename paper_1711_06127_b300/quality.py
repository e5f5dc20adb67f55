"""Image-quality measures used to judge the learned apodization against the
exact minimum-variance beamformer and delay-and-sum (evaluation only, host
NumPy; not on the processing path).

  psnr        peak signal-to-noise ratio of a uint8 B-mode image against a
              reference image (the MV image): 10 log10(255^2 / MSE).
  cyst_stats  for an anechoic cyst of a linear scan: contrast (dB) between the
              mean log-compressed level of a background ring and of the cyst
              interior, and the contrast-to-noise ratio of the envelope,
              |mu_out - mu_in| / sqrt(var_in + var_out).
"""
from __future__ import annotations

import numpy as np


def psnr(img, ref) -> float:
    a = np.asarray(img, np.float64)
    b = np.asarray(ref, np.float64)
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(255.0 ** 2 / mse)


def _line_coords(params: dict):
    xs = np.asarray(params["line_origin"], np.float64)[:, 0]
    zs = float(params["depth0"]) + np.arange(int(params["n_depth"])) * float(params["depth_step"])
    return np.meshgrid(xs, zs, indexing="ij")      # [n_lines, n_depth]


def cyst_stats(params: dict, env_lines, bm_lines, cyst, dyn_range_db: float = 60.0) -> dict:
    """cyst = (x, z, radius) in metres on a linear scan; env_lines float
    [n_lines, n_depth], bm_lines uint8 [n_lines, n_depth]."""
    X, Z = _line_coords(params)
    d = np.hypot(X - cyst[0], Z - cyst[1])
    r = cyst[2]
    inside = d < 0.7 * r
    ring = (d > 1.3 * r) & (d < 2.0 * r)
    env = np.asarray(env_lines, np.float64)
    bm = np.asarray(bm_lines, np.float64)
    mi, mo = env[inside].mean(), env[ring].mean()
    cnr = abs(mo - mi) / np.sqrt(env[inside].var() + env[ring].var())
    contrast = (bm[ring].mean() - bm[inside].mean()) * dyn_range_db / 255.0
    return {"contrast_db": float(contrast), "cnr": float(cnr), "n_inside": int(inside.sum()),
            "n_ring": int(ring.sum())}


def fwhm(profile, spacing: float) -> float:
    """Full width at half maximum (the -6 dB width of an envelope profile)
    around the profile's peak, with linear interpolation of the two half-level
    crossings; spacing is the sample distance."""
    y = np.asarray(profile, np.float64)
    k = int(np.argmax(y))
    half = y[k] / 2.0
    i = k
    while i > 0 and y[i - 1] > half:
        i -= 1
    left = (i - 1) + (half - y[i - 1]) / (y[i] - y[i - 1]) if i > 0 else 0.0
    j = k
    while j < len(y) - 1 and y[j + 1] > half:
        j += 1
    right = j + (y[j] - half) / (y[j] - y[j + 1]) if j < len(y) - 1 else float(len(y) - 1)
    return (right - left) * spacing


def point_fwhm(params: dict, env_lines, line: int, depth: int, search: int = 20) -> dict:
    """Lateral and axial -6 dB widths (metres) of a point target near (line,
    depth) in envelope lines of a linear scan: the peak within +-search
    samples, then its profile across lines and along depth."""
    env = np.asarray(env_lines, np.float64)
    L, N = env.shape
    i0, i1 = max(0, depth - search), min(N, depth + search + 1)
    l0, l1 = max(0, line - 3), min(L, line + 4)
    sub = env[l0:l1, i0:i1]
    pl, pi = np.unravel_index(int(np.argmax(sub)), sub.shape)
    pl, pi = pl + l0, pi + i0
    xs = np.asarray(params["line_origin"], np.float64)[:, 0]
    dx = float(np.mean(np.diff(xs))) if len(xs) > 1 else 1.0
    return {"lateral_m": fwhm(env[:, pi], dx), "axial_m": fwhm(env[pl, :], float(params["depth_step"])),
            "line": int(pl), "depth": int(pi)}
