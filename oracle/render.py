"""FP64 oracle of the headless volume renderer (test infrastructure only).

The paper shows rendered 3D volumes of the pipeline's output (Fig. 4b) and
names no rendering method; this is the textbook ray march of a scalar volume,
written out plainly:

  volume   uint8 [nz][ny][nx] on a grid: voxel (ix, iy, iz) at
           origin + (ix, iy, iz) * spacing (the scan-conversion grid)
  camera   orthographic: pixel (px, py) of a W x H image casts the ray
           o(px, py) = centre + (px - (W - 1)/2) * right + (py - (H - 1)/2) * down
           along the unit direction d, sampled at o + (t0 + k dt) d, k = 0 .. n_steps-1
  sample   trilinear interpolation in voxel coordinates; points outside
           [0, n - 1] on any axis read 0
  MIP      image = max over the ray's samples (0 if none)
  EA       front-to-back emission-absorption with a linear ramp transfer
           function: a_k = clamp((v_k - lo) / (hi - lo), 0, 1) * alpha,
           c_k = v_k / 255; C = sum_k T_k a_k c_k, T_{k+1} = T_k (1 - a_k),
           T_0 = 1 (no early termination)
"""
from __future__ import annotations

import numpy as np


def ray_points(camera: dict, W: int, H: int) -> np.ndarray:
    """Sample positions [H, W, n_steps, 3] of every pixel's ray."""
    c = np.asarray(camera["centre"], np.float64)
    r = np.asarray(camera["right"], np.float64)
    dn = np.asarray(camera["down"], np.float64)
    d = np.asarray(camera["dir"], np.float64)
    d = d / np.linalg.norm(d)
    px = np.arange(W) - (W - 1) / 2.0
    py = np.arange(H) - (H - 1) / 2.0
    t = float(camera["t0"]) + float(camera["dt"]) * np.arange(int(camera["n_steps"]))
    o = c + px[None, :, None] * r + py[:, None, None] * dn          # [H, W, 3]
    return o[:, :, None, :] + t[None, None, :, None] * d            # [H, W, S, 3]


def sample(vol: np.ndarray, grid: dict, pts: np.ndarray) -> np.ndarray:
    """Trilinear samples of vol (uint8 [nz][ny][nx]) at physical points pts
    [..., 3]; 0 outside the volume."""
    vol = np.asarray(vol, np.float64)
    nz, ny, nx = vol.shape
    org = np.asarray(grid["origin"], np.float64)
    sp = np.asarray(grid["spacing"], np.float64)
    u = (pts - org) / sp                                             # voxel coordinates (x, y, z)
    inside = np.all((u >= 0.0) & (u <= np.array([nx - 1, ny - 1, nz - 1], np.float64)), axis=-1)
    x, y, z = (np.clip(u[..., k], 0.0, n - 1) for k, n in enumerate((nx, ny, nz)))
    x0 = np.minimum(np.floor(x).astype(np.int64), max(nx - 2, 0))
    y0 = np.minimum(np.floor(y).astype(np.int64), max(ny - 2, 0))
    z0 = np.minimum(np.floor(z).astype(np.int64), max(nz - 2, 0))
    fx, fy, fz = x - x0, y - y0, z - z0
    x1, y1, z1 = np.minimum(x0 + 1, nx - 1), np.minimum(y0 + 1, ny - 1), np.minimum(z0 + 1, nz - 1)
    v = 0.0
    for zi, wz in ((z0, 1 - fz), (z1, fz)):
        for yi, wy in ((y0, 1 - fy), (y1, fy)):
            for xi, wx in ((x0, 1 - fx), (x1, fx)):
                v = v + wz * wy * wx * vol[zi, yi, xi]
    return np.where(inside, v, 0.0)


def render(vol, grid: dict, camera: dict, W: int, H: int, mode: str = "mip", lo: float = 0.0, hi: float = 255.0,
           alpha: float = 1.0) -> np.ndarray:
    """Image float [H, W]: MIP (values 0..255) or emission-absorption (0..1)."""
    v = sample(vol, grid, ray_points(camera, W, H))                  # [H, W, S]
    if mode == "mip":
        return v.max(axis=-1) if v.shape[-1] else np.zeros((H, W))
    a = np.clip((v - lo) / (hi - lo), 0.0, 1.0) * alpha
    c = v / 255.0
    out = np.zeros((H, W))
    T = np.ones((H, W))
    for k in range(v.shape[-1]):
        out += T * a[..., k] * c[..., k]
        T = T * (1.0 - a[..., k])
    return out
