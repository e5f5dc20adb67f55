"""Pins of the envelope, log-compression and scan-conversion oracles (Sec. 1
steps "envelope detection", "log-compression", "scan conversion"; Sec. 2
items 3-5)."""
import math

import numpy as np
import pytest
import scipy.signal

import oracle
import phantom
from _setups import tiny


# ----------------------------------------------------------------------------- envelope

@pytest.mark.parametrize("K,cut,rate", [(63, 3.5e6, 40e6), (31, 2.5e6, 40e6), (63, 1.75e6, 20e6), (1, 1e6, 1e7)])
def test_fir_taps_match_scipy_firwin(K, cut, rate):
    # scipy's window-method design with a Blackman window and unit DC gain is the same filter
    ref = scipy.signal.firwin(K, cut, window="blackman", fs=rate) if K > 1 else np.array([1.0])
    np.testing.assert_allclose(oracle.fir_taps(K, cut, rate), ref, atol=1e-15)


def _p(fc=5e6, fs=40e6, K=63, n=1024):
    p = tiny([[0, 0, 0]], fs=fs, fc=fc, n_samples=n)
    p.update(fir_taps=K, fir_cutoff=fc / 2)
    return p


@pytest.mark.parametrize("fc,fs,phase", [(5e6, 40e6, 0.3), (7e6, 40e6, 1.1), (3.5e6, 20e6, -2.0)])
def test_pure_tone_envelope_is_its_amplitude(fc, fs, phase):
    p = _p(fc, fs)
    i = np.arange(1024)
    A = 1234.5
    rf = A * np.cos(2 * np.pi * fc * i / fs + phase)
    env = oracle.envelope(p, rf[None, :])[0]
    np.testing.assert_allclose(env[64:-64], A, rtol=1e-3)


def test_dc_is_rejected():
    p = _p()
    env = oracle.envelope(p, np.ones((1, 1024)))[0]
    assert np.max(env[64:-64]) < 1e-3


def test_gaussian_pulse_matches_hilbert_envelope():
    # the paper's offline PSF study takes the envelope with the Hilbert transform (Sec. 3.2)
    fc, fs = 5e6, 40e6
    p = _p(fc, fs)
    i = np.arange(1024)
    sig = 6.0 / fc / 2.3548 * fs   # 6-cycle FWHM: its band lies inside the low-pass
    x = 500 * np.exp(-((i - 512.3) ** 2) / (2 * sig ** 2)) * np.cos(2 * np.pi * fc * (i - 512.3) / fs)
    env = oracle.envelope(p, x[None, :])[0]
    hil = np.abs(scipy.signal.hilbert(x))
    core = slice(512 - 10, 512 + 10)
    np.testing.assert_allclose(env[core], hil[core], rtol=0, atol=0.01 * hil.max())
    assert np.argmax(env) == 512


def test_envelope_is_linear_in_amplitude_and_invariant_to_phase():
    p = _p()
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 1024))
    e1 = oracle.envelope(p, x)
    np.testing.assert_allclose(oracle.envelope(p, 3 * x), 3 * e1, rtol=1e-12)
    np.testing.assert_allclose(oracle.envelope(p, -x), e1, rtol=1e-12)


# ----------------------------------------------------------------------------- log compression

def test_logcompress_formula_points():
    D, ref = 60.0, 1000.0
    env = np.array([ref, ref * 10 ** (-D / 20), 0.0, 2 * ref, 1e-9, ref * 10 ** (-D / 20 * (1 - 100 / 255)),
                    ref * 10 ** (-D / 20 * (1 - 200.4 / 255)), ref * 10 ** (-D / 20 * (1 - 200.6 / 255))])
    got = oracle.logcompress(env, ref, D)
    assert list(got) == [255, 0, 0, 255, 0, 100, 200, 201]


def test_logcompress_monotone():
    env = np.geomspace(1e-3, 1e4, 5000)
    b = oracle.logcompress(env, 1000.0, 60.0).astype(int)
    assert np.all(np.diff(b) >= 0) and b[0] == 0 and b[-1] == 255


# ----------------------------------------------------------------------------- scan conversion

def _linear_p(n_lines=8, n_depth=40, pitch=0.3e-3):
    s = phantom.linear_setup(n_lines, pitch, n_lines, n_depth, fs=40e6)
    return s.params(), s


def test_linear_identity_grid():
    p, s = _linear_p()
    xs = s.line_origin[:, 0]
    p["grid"] = {"n": (len(xs), 1, s.n_depth), "origin": (xs[0], 0.0, 0.0),
                 "spacing": (xs[1] - xs[0], 1.0, s.depth_step)}
    bm = np.random.default_rng(1).integers(0, 256, (s.n_lines, s.n_depth)).astype(np.uint8)
    img = oracle.scanconvert(p, bm)[:, 0, :]
    np.testing.assert_array_equal(img, bm.T)


def test_linear_affine_is_exact_and_outside_is_zero():
    p, s = _linear_p()
    xs = s.line_origin[:, 0]
    l, i = np.meshgrid(np.arange(s.n_lines), np.arange(s.n_depth), indexing="ij")
    bm = (8 * l + 2 * i).astype(np.uint8)           # affine, max 8*7 + 2*39 = 134
    dx = xs[1] - xs[0]
    pts = np.array([[xs[0] + 1.5 * dx, 0, 10.25 * s.depth_step],   # u = 1.5, v = 10.25 -> 12 + 20.5 = 32.5 -> 33
                    [xs[0] + 6.25 * dx, 0, 3.0 * s.depth_step],    # 50 + 6 = 56
                    [xs[0] - 0.5 * dx, 0, 5 * s.depth_step],       # left of the first line -> 0
                    [xs[0] + 2 * dx, 0, (s.n_depth + 1) * s.depth_step]])  # beyond the last sample -> 0
    got = oracle.scanconvert(p, bm, pts)
    assert list(got) == [33, 56, 0, 0]


def test_linear_constant_inside_zero_outside():
    p, s = _linear_p()
    xs = s.line_origin[:, 0]
    p["grid"] = {"n": (30, 1, 50), "origin": (xs[0] - 0.5e-3, 0.0, 0.0),
                 "spacing": ((xs[-1] - xs[0] + 1e-3) / 29, 1.0, 1.2 * s.n_depth * s.depth_step / 49)}
    img = oracle.scanconvert(p, np.full((s.n_lines, s.n_depth), 77, np.uint8))[:, 0, :]
    pts = oracle.grid_points(p["grid"])[:, 0, :, :]
    inside = (pts[..., 0] >= xs[0]) & (pts[..., 0] <= xs[-1]) & (pts[..., 2] <= (s.n_depth - 1) * s.depth_step)
    assert np.all(img[inside] == 77) and np.all(img[~inside] == 0)


def test_sector_point_on_a_line():
    s = phantom.sector_setup(n_el=16, n_lines=9, half_angle_deg=40, n_samples=60)
    p = s.params()
    bm = np.random.default_rng(2).integers(1, 256, (s.n_lines, s.n_depth)).astype(np.uint8)
    th = np.deg2rad(np.linspace(-40, 40, 9))
    pts, want = [], []
    for l, i in [(0, 10), (4, 33), (8, 59), (2, 1)]:
        r = i * s.depth_step
        pts.append([r * math.sin(th[l]), 0, r * math.cos(th[l])])
        want.append(bm[l, i])
    r = 20 * s.depth_step
    pts.append([r * math.sin(np.deg2rad(45)), 0, r * math.cos(np.deg2rad(45))])   # outside the sector
    want.append(0)
    assert list(oracle.scanconvert(p, bm, np.array(pts))) == want


def test_sector_midway_between_lines_averages():
    s = phantom.sector_setup(n_el=16, n_lines=5, half_angle_deg=20, n_samples=60)
    p = s.params()
    bm = np.zeros((5, 60), np.uint8)
    bm[1, :] = 100
    bm[2, :] = 201
    th = np.deg2rad(np.linspace(-20, 20, 5))
    t = 0.5 * (th[1] + th[2])
    r = 30 * s.depth_step
    assert oracle.scanconvert(p, bm, np.array([[r * math.sin(t), 0, r * math.cos(t)]]))[0] == 151  # 150.5 -> 151


def test_pyramid_central_line_and_outside():
    s = phantom.pyramid_setup(4, 4, 0.3e-3, 5, 5, 30.0, 50, grid_n=None)
    p = s.params()
    bm = np.random.default_rng(3).integers(1, 256, (s.n_lines, s.n_depth)).astype(np.uint8)
    centre = 2 * 5 + 2
    r = 17 * s.depth_step
    # on the central line; behind the array; outside the +-30 deg pyramid; the apex itself
    # (z = 0 is never inside: the line angles are undefined there)
    pts = np.array([[0, 0, r], [0, 0, -r], [r, 0, 0.1 * r], [0, 0, 0]])
    got = oracle.scanconvert(p, bm, pts)
    assert list(got) == [bm[centre, 17], 0, 0, 0]
    # a corner line (ix = 4, iy = 0): direction normalize(tan 30, tan -30, 1)
    v = np.array([math.tan(math.radians(30)), math.tan(math.radians(-30)), 1.0])
    v /= np.linalg.norm(v)
    assert oracle.scanconvert(p, bm, (9 * s.depth_step * v)[None])[0] == bm[4, 9]


def test_pyramid_constant_volume():
    s = phantom.pyramid_setup(4, 4, 0.3e-3, 6, 6, 30.0, 40, grid_n=(20, 20, 20))
    p = s.params()
    vol = oracle.scanconvert(p, np.full((36, 40), 9, np.uint8))
    pts = oracle.grid_points(p["grid"])
    X, Y, Z = pts[..., 0], pts[..., 1], pts[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        inside = (Z > 0) & (np.abs(X) <= Z * math.tan(math.radians(30)) * (1 - 1e-6)) & \
                 (np.abs(Y) <= Z * math.tan(math.radians(30)) * (1 - 1e-6)) & \
                 (np.sqrt(X * X + Y * Y + Z * Z) <= 39 * s.depth_step * (1 - 1e-6))
    assert np.all(vol[inside] == 9)
    assert set(np.unique(vol[~inside])) <= {0, 9}
    assert vol.sum() > 0


# ----------------------------------------------------------------------------- frequency compounding

def _bank(K, step, fc=5e6, fs=40e6, taps=63):
    p = dict(c=1540.0, depth_step=1540.0 / (2 * fs), fc=fc, fir_taps=taps, fir_cutoff=fc / 2, n_bands=K,
             band_step=step)
    return p


def _response(p, f):
    # |H| of the low-pass at frequency offset f (direct DTFT of the taps)
    rate = oracle.depth_rate(p)
    h = oracle.fir_taps(int(p["fir_taps"]), float(p["fir_cutoff"]), rate)
    n = np.arange(len(h))
    return abs(np.sum(h * np.exp(-2j * np.pi * f / rate * n)))


def test_one_band_is_plain_iq_demodulation():
    p1 = _bank(1, 0.0)
    rf = np.random.default_rng(3).normal(size=(2, 500))
    a = oracle.envelope(p1, rf)
    b = oracle.envelope(dict(p1, n_bands=None, band_step=None), rf)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_allclose(oracle.band_centres(_bank(3, 1e6)), [4e6, 5e6, 6e6])


def test_bank_envelope_of_a_tone_is_the_mean_band_response():
    # a tone A cos(2 pi f0 t) through band k: steady-state envelope A |H(f0 - f_k)|
    # (the image at f0 + f_k lies far in the stop band); the bank averages them
    p = _bank(3, 1.5e6)
    rate = oracle.depth_rate(p)
    A, f0 = 3.0, 5.4e6
    n = np.arange(1200)
    rf = A * np.cos(2 * np.pi * f0 * n / rate + 0.3)
    env = oracle.envelope(p, rf[None])[0]
    want = A * np.mean([_response(p, f0 - fk) for fk in oracle.band_centres(p)])
    np.testing.assert_allclose(env[200:1000], want, rtol=2e-3)


def test_symmetric_bank_is_symmetric_about_fc():
    p = _bank(4, 1e6)
    rate = oracle.depth_rate(p)
    n = np.arange(900)
    lo = oracle.envelope(p, np.cos(2 * np.pi * (p["fc"] - 0.7e6) * n / rate)[None])[0]
    hi = oracle.envelope(p, np.cos(2 * np.pi * (p["fc"] + 0.7e6) * n / rate)[None])[0]
    np.testing.assert_allclose(lo[200:700], hi[200:700], rtol=2e-3)


def test_bank_widens_the_pass_band():
    # a tone 3 MHz above fc sits in the single band's transition (|H(3 MHz)| ~ 0.2 for 63 Blackman
    # taps at 40 MHz); a bank with 3 MHz steps centres its outer band on it: mean(|H|) ~ 0.4
    rate = oracle.depth_rate(_bank(1, 0.0))
    n = np.arange(900)
    rf = np.cos(2 * np.pi * 8e6 * n / rate)[None]
    one = oracle.envelope(_bank(1, 0.0), rf)[0, 200:700].mean()
    p3 = _bank(3, 3e6)
    bank = oracle.envelope(p3, rf)[0, 200:700].mean()
    assert one == pytest.approx(_response(_bank(1, 0.0), 3e6), rel=2e-3)
    assert bank == pytest.approx(np.mean([_response(p3, 8e6 - f) for f in oracle.band_centres(p3)]), rel=2e-3)
    assert bank > 1.9 * one
