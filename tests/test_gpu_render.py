"""GPU parity of the headless volume renderer (supra_render) against the
FP64 oracle on seeded volumes.  Tolerance: the sample positions are FP32
(~1e-5 voxel after hundreds of steps) and the trilinear blend FP32, so a
sample moves by at most ~1e-5 x 255 per voxel of gradient: max |gpu - oracle|
<= 1e-2 gray levels for MIP and 1e-4 for emission-absorption (0..1).  Rays
with a sample within 1e-3 voxel of a volume face are left out (FP32 and FP64
may place that sample on either side of the face)."""
import numpy as np
import pytest
import torch

import paper_1711_06127_b300 as supra
from oracle import render as orender

pytestmark = pytest.mark.gpu


def _volume(seed, shape=(40, 36, 44)):
    rng = np.random.default_rng(seed)
    v = rng.integers(0, 256, shape).astype(np.float64)
    # smooth a little so the trilinear field has structure at several scales
    for ax in range(3):
        v = (v + np.roll(v, 1, ax) + np.roll(v, -1, ax)) / 3.0
    return np.clip(np.round(v), 0, 255).astype(np.uint8)


GRID = {"n": (44, 36, 40), "origin": (-2.2e-3, -1.8e-3, 0.5e-3), "spacing": (1e-4, 1e-4, 1.2e-4)}


def _camera(seed, n_steps=120):
    rng = np.random.default_rng(seed)
    d = np.array([0.3, -0.2, 1.0]) + rng.normal(0, 0.05, 3)
    d /= np.linalg.norm(d)
    right = np.cross(d, [0.0, 1.0, 0.0])
    right = right / np.linalg.norm(right) * 0.9e-4
    down = np.cross(d, right)
    down = down / np.linalg.norm(down) * 0.9e-4
    centre = np.array([0.0, 0.0, 2.9e-3]) - 0.004 * d
    return {"centre": centre, "right": right, "down": down, "dir": d, "t0": 0.0, "dt": 0.6e-4, "n_steps": n_steps}


def _grazing(cam, W, H, grid):
    pts = orender.ray_points(cam, W, H)
    u = (pts - np.asarray(grid["origin"])) / np.asarray(grid["spacing"])
    n = np.asarray(grid["n"], np.float64) - 1
    near = np.zeros(pts.shape[:-1], bool)
    for k in range(3):
        others = np.ones(pts.shape[:-1], bool)
        for j in range(3):
            if j != k:
                others &= (u[..., j] >= -1e-3) & (u[..., j] <= n[j] + 1e-3)
        near |= others & ((np.abs(u[..., k]) < 1e-3) | (np.abs(u[..., k] - n[k]) < 1e-3))
    return near.any(axis=-1)


@pytest.mark.parametrize("mode,tol", [("mip", 1e-2), ("ea", 1e-4)])
def test_render_matches_oracle(mode, tol):
    vol = _volume(1)
    W, H = 70, 55
    cam = _camera(2)
    kw = dict(lo=60.0, hi=200.0, alpha=0.15) if mode == "ea" else {}
    got = supra.render(torch.as_tensor(vol).cuda(), GRID, cam, W, H, mode, **kw).cpu().numpy()
    ref = orender.render(vol, GRID, cam, W, H, mode, **kw)
    keep = ~_grazing(cam, W, H, GRID)
    assert keep.mean() > 0.9 and np.max(ref) > 0
    assert np.max(np.abs(got - ref)[keep]) <= tol


def test_render_rejects_bad_arguments():
    vol = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    g = {"n": (4, 4, 4), "origin": (0.0, 0.0, 0.0), "spacing": (1.0, 1.0, 1.0)}
    cam = {"centre": (1.5, 1.5, -1.0), "right": (1.0, 0, 0), "down": (0, 1.0, 0), "dir": (0, 0, 0.0), "t0": 0.0,
           "dt": 1.0, "n_steps": 4}
    with pytest.raises(supra.SupraError):
        supra.render(vol, g, cam, 4, 4)
    with pytest.raises(supra.SupraError):
        supra.render(vol, g, dict(cam, dir=(0, 0, 1.0)), 4, 4, "ea", lo=10.0, hi=10.0)
