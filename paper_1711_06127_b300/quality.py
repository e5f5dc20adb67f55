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
