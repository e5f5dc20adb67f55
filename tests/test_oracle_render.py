"""Pins of the volume-rendering oracle (textbook ray march; not in the
paper beyond its rendered volumes) and of the PSF width measure."""
import numpy as np
import pytest

from oracle import render
from paper_1711_06127_b300 import quality

GRID = {"origin": (0.0, 0.0, 0.0), "spacing": (1.0, 1.0, 1.0)}


def _axis_camera(W, H, n_steps, dt=1.0, t0=0.0, x0=0.0, y0=0.0):
    # rays along +z through voxel columns: pixel (px, py) -> x = x0 + px, y = y0 + py
    return {"centre": (x0 + (W - 1) / 2.0, y0 + (H - 1) / 2.0, -1.0), "right": (1.0, 0.0, 0.0),
            "down": (0.0, 1.0, 0.0), "dir": (0.0, 0.0, 1.0), "t0": 1.0 + t0, "dt": dt, "n_steps": n_steps}


def test_mip_along_voxel_columns_is_the_max_over_z():
    vol = np.random.default_rng(0).integers(0, 256, (9, 6, 7)).astype(np.uint8)
    img = render.render(vol, GRID, _axis_camera(7, 6, 9), 7, 6, "mip")
    np.testing.assert_array_equal(img, vol.max(axis=0).astype(np.float64))


def test_trilinear_sampling_is_exact_on_affine_data():
    z, y, x = np.meshgrid(np.arange(5), np.arange(6), np.arange(7), indexing="ij")
    vol = (3 + 2 * x + 5 * y + 7 * z).astype(np.uint8)
    pts = np.random.default_rng(1).uniform([0, 0, 0], [6, 5, 4], (50, 3))
    v = render.sample(vol, GRID, pts)
    np.testing.assert_allclose(v, 3 + 2 * pts[:, 0] + 5 * pts[:, 1] + 7 * pts[:, 2], rtol=1e-12)


def test_single_voxel_and_outside_points():
    vol = np.zeros((5, 5, 5), np.uint8)
    vol[2, 2, 2] = 200
    assert render.sample(vol, GRID, np.array([[2.0, 2.0, 2.0]]))[0] == 200.0
    assert render.sample(vol, GRID, np.array([[2.5, 2.0, 2.0]]))[0] == pytest.approx(100.0)
    assert render.sample(vol, GRID, np.array([[2.5, 2.5, 2.5]]))[0] == pytest.approx(25.0)
    assert render.sample(vol, GRID, np.array([[-0.01, 2.0, 2.0], [2.0, 4.01, 2.0]])).tolist() == [0.0, 0.0]
    # a ray that misses the volume renders 0 in both modes
    cam = _axis_camera(1, 1, 20, x0=10.0)
    assert render.render(vol, GRID, cam, 1, 1, "mip")[0, 0] == 0.0
    assert render.render(vol, GRID, cam, 1, 1, "ea")[0, 0] == 0.0


def test_emission_absorption_of_a_uniform_slab():
    # n samples of constant v inside: C = c (1 - (1 - a)^n), a = ramp(v) alpha, c = v / 255
    vol = np.full((10, 3, 3), 150, np.uint8)
    n, lo, hi, alpha = 8, 100.0, 200.0, 0.6
    img = render.render(vol, GRID, _axis_camera(3, 3, n, dt=1.0, t0=1.0), 3, 3, "ea", lo, hi, alpha)
    a = (150 - lo) / (hi - lo) * alpha
    np.testing.assert_allclose(img, 150 / 255 * (1 - (1 - a) ** n), rtol=1e-12)


def test_fwhm_of_gaussian_and_box_profiles():
    x = np.arange(-50, 51) * 0.1
    sig = 0.7
    g = 4.0 * np.exp(-x ** 2 / (2 * sig ** 2))
    assert quality.fwhm(g, 0.1) == pytest.approx(2 * np.sqrt(2 * np.log(2)) * sig, rel=2e-3)
    box = np.where(np.abs(x) <= 1.0, 1.0, 0.0)
    # linear interpolation between the last sample at 1 and the first at 0: half-level 0.05 beyond
    assert quality.fwhm(box, 0.1) == pytest.approx(2.1, rel=1e-9)
