"""Pins of the delay-and-sum oracle against closed forms, invariants and the
physics of the synthetic acquisition (receive beamforming, Sec. 1 step list;
Sec. 2 items 1-2)."""
import json
import os

import numpy as np
import pytest

import oracle
import phantom
from _setups import tiny, small_linear

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_single_element_at_line_origin_is_identity():
    # one element at the line origin, depth step c/(2 fs): the two-way delay of depth
    # sample i is exactly i samples, so the beamformer returns the record itself.
    p = tiny([[0, 0, 0]], n_samples=257)
    ch = np.random.default_rng(1).integers(-30000, 30000, (1, 1, 257)).astype(np.int16)
    rf = oracle.das(p, ch)
    np.testing.assert_allclose(rf[0], ch[0, 0].astype(np.float64), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "das_closed_form.json")))["cases"],
                         ids=lambda c: c["name"])
def test_pythagorean_arrivals(case):
    gold = json.load(open(os.path.join(GOLD, "das_closed_form.json")))
    p = tiny([case["elem_mm"]], [case["line_origin_mm"]], [case["line_dir"]], [case["tx_origin_mm"]],
             c=gold["c"], fs=gold["fs"], n_samples=400)
    i = int(round(case["depth_mm"] * 1e-3 / p["depth_step"]))
    ch = np.zeros((1, 1, 400), np.int16)
    ch[0, 0, case["arrival_sample"]] = 1
    rf = oracle.das(p, ch)
    assert rf[0, i] == pytest.approx(1.0, abs=1e-9)
    # neighbouring depths fall between samples: strictly between 0 and 1
    assert 0.0 < rf[0, i - 1] < 1.0 and 0.0 < rf[0, i + 1] < 1.0
    # shifting the record start by t0 moves the arrival by the same number of samples
    p2 = dict(p, t0=10 / gold["fs"])
    ch2 = np.zeros_like(ch)
    ch2[0, 0, case["arrival_sample"] - 10] = 1
    assert oracle.das(p2, ch2)[0, i] == pytest.approx(1.0, abs=1e-9)


def test_constant_records_beamform_to_the_constant():
    s = phantom.config1()
    p = s.params()
    ch = np.full((s.n_tx, s.n_el, s.n_samples), 1234, np.int16)
    rf = oracle.das(p, ch)
    # all interpolation points inside the record up to ~90% depth
    np.testing.assert_allclose(rf[:, : int(0.9 * s.n_depth)], 1234.0, rtol=0, atol=1e-9)


def test_fnumber_aperture_edge():
    # element 3 mm off a +z line, rect window, F = 1.5, minimum half width 0.3 mm:
    # it joins the aperture when z / (2 F) reaches 3 mm, i.e. at z = 9 mm (index 180).
    p = tiny([[0, 0, 0], [3, 0, 0]], fnumber=1.5, min_half_aperture=0.3e-3, n_samples=600)
    ch = np.zeros((1, 2, 600), np.int16)
    ch[0, 0, :] = 10
    ch[0, 1, :] = 40
    rf = oracle.das(p, ch)
    assert rf[0, 150] == pytest.approx(10.0) and rf[0, 178] == pytest.approx(10.0)
    assert rf[0, 182] == pytest.approx(25.0) and rf[0, 400] == pytest.approx(25.0)


@pytest.mark.parametrize("window,expect", [("hann", 4.0), ("hamming", (2 + 0.54 * 8) / 1.54), ("rect", 5.0)])
def test_window_weights(window, expect):
    # fixed half width 3 mm; elements at u = 0 and u = 1/2: Hann 1 and 1/2, Hamming 1 and 0.54
    p = tiny([[0, 0, 0], [1.5, 0, 0]], fnumber=1e6, min_half_aperture=3e-3, window=window)
    ch = np.zeros((1, 2, 400), np.int16)
    ch[0, 0, :] = 2
    ch[0, 1, :] = 8
    assert oracle.das(p, ch)[0, 100] == pytest.approx(expect, rel=1e-12)


def test_aperture_centre_clamped_to_array():
    # line 5 mm outside the array: centre clamps to the last element (x = 1.5 mm)
    p = tiny([[0, 0, 0], [1.5, 0, 0]], line_origin_mm=[[5, 0, 0]], fnumber=1e6, min_half_aperture=3e-3,
             window="hann")
    ch = np.zeros((1, 2, 400), np.int16)
    ch[0, 0, :] = 2
    ch[0, 1, :] = 8
    assert oracle.das(p, ch)[0, 150] == pytest.approx((0.5 * 2 + 8) / 1.5, rel=1e-12)


def test_record_end_zero_padding():
    p = tiny([[0, 0, 0]], n_samples=64, n_depth=70)
    ch = np.full((1, 1, 64), 7, np.int16)
    rf = oracle.das(p, ch)
    assert rf[0, 63] == pytest.approx(7.0)
    assert np.all(rf[0, 64:] == 0.0)


def test_linearity():
    s = small_linear()
    p = s.params()
    rng = np.random.default_rng(3)
    a = rng.integers(-1000, 1000, (s.n_tx, s.n_el, s.n_samples)).astype(np.int16)
    b = rng.integers(-1000, 1000, (s.n_tx, s.n_el, s.n_samples)).astype(np.int16)
    lhs = oracle.das(p, (3 * a.astype(np.int32) - 2 * b).astype(np.int16))
    rhs = 3 * oracle.das(p, a) - 2 * oracle.das(p, b)
    np.testing.assert_allclose(lhs, rhs, atol=1e-8)


def test_mirror_symmetry():
    # a symmetric probe and line set: mirroring x flips element and line order
    s = small_linear(n_el=16, n_lines=16)
    p = s.params()
    ch = np.random.default_rng(5).integers(-3000, 3000, (s.n_tx, s.n_el, s.n_samples)).astype(np.int16)
    rf = oracle.das(p, ch)
    rf_m = oracle.das(p, ch[::-1, ::-1, :].copy())
    np.testing.assert_allclose(rf_m, rf[::-1], atol=1e-8)


def test_point_scatterer_images_at_its_position():
    # a single bright point on the axis of a line: the envelope peaks on that line
    # at the sample of its two-way travel time
    s = small_linear(n_el=32, n_lines=32, n_samples=800)
    p = s.params()
    line = 11
    z = 12e-3
    pos = np.array([[s.line_origin[line, 0], 0.0, z]])
    ch = phantom.synth_channels(s, phantom.Phantom(pos, np.array([1.0])), seed=0, snr_db=None).numpy()
    env = oracle.envelope(p, oracle.das(p, ch))
    l, i = np.unravel_index(np.argmax(env), env.shape)
    assert l == line
    assert abs(i - round(2 * z * s.fs / s.c)) <= 1


def test_sampled_points_match_full_frame():
    s = small_linear()
    p = s.params()
    ch = phantom.random_channels(s, 9).numpy()
    rf = oracle.das(p, ch)
    rng = np.random.default_rng(0)
    lines = rng.integers(0, s.n_lines, 40)
    depths = rng.integers(0, s.n_depth, 40)
    got = oracle.das_points(p, lines, depths, [ch[s.line_tx[l]] for l in lines])
    np.testing.assert_array_equal(got, rf[lines, depths])


# ----------------------------------------------------------------------------- plane waves and compounding

def _plane_setup(n_el=16, n_lines=6, n_s=400, angles=(0.0,)):
    s = phantom.linear_setup(n_el, 0.3e-3, n_lines, n_s, fc=5e6, fs=40e6)
    p = s.params()
    th = np.deg2rad(np.asarray(angles, np.float64))
    p["tx_dir"] = np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], 1)
    # each plane wave passes the array's first (steering toward +x) or last element at time 0
    x0, x1 = p["elem_pos"][0, 0], p["elem_pos"][-1, 0]
    p["tx_origin"] = np.stack([np.where(th >= 0, x0, x1), np.zeros_like(th), np.zeros_like(th)], 1)
    p["line_tx"] = np.zeros(n_lines, np.int32)
    return s, p


def test_zero_degree_plane_wave_equals_the_line_origin_transmit():
    # straight-down lines from z = 0: the 0-degree plane wave arrives at depth r after r / c,
    # exactly as a spherical transmit from the line's own origin
    s, p = _plane_setup()
    ch = phantom.random_channels(s, 3).numpy()
    plane = oracle.das(p, ch[:1])
    q = dict(s.params(), tx_origin=np.asarray(s.line_origin), line_tx=np.arange(s.n_lines, dtype=np.int32))
    sph = oracle.das(q, np.repeat(ch[:1], s.n_lines, axis=0))
    np.testing.assert_allclose(plane, sph, rtol=1e-12, atol=1e-9)


def test_steered_plane_wave_pythagorean_arrival():
    # element and line at the origin, plane wave n = (3/5, 0, 4/5) through the origin: a point at
    # depth 5 mm is reached after 4 mm and heard after 5 mm more; fs / c = 10 samples per mm puts
    # the echo exactly on sample 90 (a spherical transmit from the origin would give sample 100)
    c, fs = 1540.0, 15.4e6
    p = dict(elem_pos=np.zeros((1, 3)), tx_origin=np.zeros((1, 3)), tx_dir=np.array([[0.6, 0.0, 0.8]]),
             line_origin=np.zeros((1, 3)), line_dir=np.array([[0.0, 0.0, 1.0]]), line_tx=np.zeros(1, np.int32),
             n_depth=201, depth0=0.0, depth_step=0.05e-3, c=c, fs=fs, t0=0.0, fnumber=1.0,
             min_half_aperture=1e-3, window="rect", n_samples=300)
    ch = np.zeros((1, 1, 300), np.int16)
    ch[0, 0, 90] = 1000
    rf = oracle.das(p, ch)[0]
    assert rf[100] == pytest.approx(1000.0, rel=1e-9)
    # a spherical transmit from the origin puts the same echo at 2 r = 9 mm: depth 4.5 mm (i = 90)
    spherical = oracle.das(dict(p, tx_dir=None), ch)[0]
    assert spherical[100] == 0.0 and spherical[90] == pytest.approx(1000.0, rel=1e-9)


def test_compounding_averages_the_transmits():
    s, p = _plane_setup(angles=(-6.0, 0.0, 6.0))
    ch = phantom.random_channels(s, 4).numpy()[:1]
    one = {a: oracle.das(dict(p, tx_dir=p["tx_dir"][a:a + 1], tx_origin=p["tx_origin"][a:a + 1]), ch)
           for a in range(3)}
    # identical transmits compound to the single-transmit image
    pc = dict(p, compound=1, tx_dir=np.repeat(p["tx_dir"][1:2], 3, 0), tx_origin=np.repeat(p["tx_origin"][1:2], 3, 0))
    np.testing.assert_allclose(oracle.das(pc, np.repeat(ch, 3, 0)), one[1], rtol=1e-12, atol=1e-9)
    # with the other transmits' records zero, the compound is that transmit's image / 3
    rec = np.zeros((3,) + ch.shape[1:], np.int16)
    rec[2] = ch[0]
    np.testing.assert_allclose(oracle.das(dict(p, compound=1), rec), one[2] / 3.0, rtol=1e-12, atol=1e-9)


def test_fp32_timing_variant_matches_the_oracle_within_single_precision():
    """oracle_das_f32 runs the oracle's loops in single precision (a CPU timing
    reference): its frame agrees with the FP64 oracle to single-precision rounding."""
    s = small_linear(32, 24, 700)
    ch = phantom.synth_channels(s, phantom.default_phantom(s, 11), 11).numpy()
    a = oracle.das(s.params(), ch)
    b = oracle.das_f32(s.params(), ch).astype(np.float64)
    assert np.abs(a - b).max() <= 5e-4 * np.abs(a).max()
