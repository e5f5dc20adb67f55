"""FP64 CPU oracle of the SUPRA B-mode chain (arXiv:1711.06127).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / --impl reference legs of bench.py may import this package.  It
shares no code with the CUDA library (paper_1711_06127_b300) and never imports
it; both consume the same plain parameter dictionaries produced by the
`phantom` input generator.

The paper lists the pipeline steps (Sec. 1 step list; Sec. 2 method list
items 1-5; Table 1 columns Beamformer / Envelope / Log comp. / Scan conv.) but
states no formula for any of them, so every function here is the textbook
definition of the named step, written out plainly:

  das           receive delay-and-sum beamforming           (oracle.c, C + OpenMP)
  das_f32       the same loops in FP32: a CPU timing column beside the oracle, not an oracle
  fir_taps      windowed-sinc low-pass (Blackman), unit DC gain
  envelope      IQ demodulation: mix with exp(-j 2 pi fc t), low-pass, 2|iq|
  logcompress   20 log10(env/ref) mapped from [-D, 0] dB to [0, 255], half-up rounding
  scanconvert   inverse map of each grid point to (line, depth), bilinear (2D)
                / trilinear (3D) on the log-compressed lines, 0 outside

Readings taken where the paper is silent are stated in each docstring.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None

WINDOWS = {"rect": 0, "hann": 1, "hamming": 2}


class _Geom(ctypes.Structure):
    _fields_ = [
        ("n_el", ctypes.c_int32), ("elem", ctypes.POINTER(ctypes.c_double)),
        ("n_tx", ctypes.c_int32), ("tx_origin", ctypes.POINTER(ctypes.c_double)),
        ("n_lines", ctypes.c_int32), ("line_origin", ctypes.POINTER(ctypes.c_double)),
        ("line_dir", ctypes.POINTER(ctypes.c_double)), ("line_tx", ctypes.POINTER(ctypes.c_int32)),
        ("n_depth", ctypes.c_int32), ("depth0", ctypes.c_double), ("depth_step", ctypes.c_double),
        ("c", ctypes.c_double), ("fs", ctypes.c_double), ("t0", ctypes.c_double),
        ("fnumber", ctypes.c_double), ("min_half_aperture", ctypes.c_double),
        ("window", ctypes.c_int32), ("n_s", ctypes.c_int32),
        ("tx_dir", ctypes.POINTER(ctypes.c_double)), ("compound", ctypes.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        _lib.oracle_das.argtypes = [ctypes.POINTER(_Geom), ctypes.c_void_p, ctypes.c_void_p]
        _lib.oracle_das_f32.argtypes = [ctypes.POINTER(_Geom), ctypes.c_void_p, ctypes.c_void_p]
        _lib.oracle_das_points.argtypes = [ctypes.POINTER(_Geom), ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib.oracle_aperture.argtypes = [ctypes.POINTER(_Geom), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib.oracle_delayed_samples.argtypes = [ctypes.POINTER(_Geom), ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        _lib.oracle_delayed_samples.restype = ctypes.c_int32
    return _lib


class Geometry:
    """Holds the C geometry record and keeps its arrays alive."""

    def __init__(self, p: dict):
        self.elem = np.ascontiguousarray(p["elem_pos"], dtype=np.float64)
        self.tx = np.ascontiguousarray(p["tx_origin"], dtype=np.float64)
        self.lo = np.ascontiguousarray(p["line_origin"], dtype=np.float64)
        self.ld = np.ascontiguousarray(p["line_dir"], dtype=np.float64)
        self.lt = np.ascontiguousarray(p["line_tx"], dtype=np.int32)
        td = p.get("tx_dir")
        self.td = None if td is None else np.ascontiguousarray(td, dtype=np.float64).reshape(-1, 3)
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.g = _Geom(self.elem.shape[0], dp(self.elem), self.tx.shape[0], dp(self.tx), self.lo.shape[0],
                       dp(self.lo), dp(self.ld), self.lt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                       int(p["n_depth"]), float(p["depth0"]), float(p["depth_step"]), float(p["c"]),
                       float(p["fs"]), float(p.get("t0", 0.0)), float(p["fnumber"]),
                       float(p["min_half_aperture"]), WINDOWS[p["window"]], int(p["n_samples"]),
                       dp(self.td) if self.td is not None else None, int(p.get("compound", 0) or 0))

    @property
    def ref(self):
        return ctypes.byref(self.g)


# ----------------------------------------------------------------------------- delay-and-sum

def das(p: dict, ch) -> np.ndarray:
    """Receive delay-and-sum (Sec. 1 "receive beamforming"; Sec. 2 items 1-2).
    ch: int16 [n_tx, n_el, n_s] -> rf float64 [n_lines, n_depth].  See
    oracle.c for the definition and its readings."""
    ch = np.ascontiguousarray(np.asarray(ch), dtype=np.int16)
    g = Geometry(p)
    assert ch.shape == (g.tx.shape[0], g.elem.shape[0], int(p["n_samples"])), ch.shape
    rf = np.zeros((g.lo.shape[0], int(p["n_depth"])), dtype=np.float64)
    lib().oracle_das(g.ref, ch.ctypes.data, rf.ctypes.data)
    return rf


def das_f32(p: dict, ch) -> np.ndarray:
    """The delay-and-sum loops of `das` in single precision (oracle.c,
    oracle_das_f32): a CPU timing reference beside the FP64 oracle, not an
    oracle.  rf float32 [n_lines, n_depth]."""
    ch = np.ascontiguousarray(np.asarray(ch), dtype=np.int16)
    g = Geometry(p)
    assert ch.shape == (g.tx.shape[0], g.elem.shape[0], int(p["n_samples"])), ch.shape
    rf = np.zeros((g.lo.shape[0], int(p["n_depth"])), dtype=np.float32)
    lib().oracle_das_f32(g.ref, ch.ctypes.data, rf.ctypes.data)
    return rf


def das_points(p: dict, lines, depths, ch_tx_blocks) -> np.ndarray:
    """Delay-and-sum at selected (line, depth) points.  ch_tx_blocks[k] is the
    int16 [n_el, n_s] record block of the transmit event of lines[k]."""
    g = Geometry(p)
    lines = np.ascontiguousarray(lines, dtype=np.int32)
    depths = np.ascontiguousarray(depths, dtype=np.int32)
    blocks = [np.ascontiguousarray(b, dtype=np.int16) for b in ch_tx_blocks]
    ptrs = (ctypes.c_void_p * len(blocks))(*[b.ctypes.data for b in blocks])
    out = np.zeros(len(lines), dtype=np.float64)
    lib().oracle_das_points(g.ref, len(lines), lines.ctypes.data, depths.ctypes.data, ptrs, out.ctypes.data)
    return out


def aperture(p: dict, line: int, i: int):
    """(mask, weights, margin) of the receive aperture at (line, depth i)."""
    g = Geometry(p)
    n = g.elem.shape[0]
    mask = np.zeros(n, np.int32)
    w = np.zeros(n)
    m = np.zeros(n)
    lib().oracle_aperture(g.ref, int(line), int(i), mask.ctypes.data, w.ctypes.data, m.ctypes.data)
    return mask.astype(bool), w, m


def delayed_samples(p: dict, ch_tx, line: int, i: int):
    """Delayed, interpolated samples of the active elements at (line, i)."""
    g = Geometry(p)
    ch_tx = np.ascontiguousarray(ch_tx, dtype=np.int16)
    x = np.zeros(g.elem.shape[0])
    el = np.zeros(g.elem.shape[0], np.int32)
    m = lib().oracle_delayed_samples(g.ref, ch_tx.ctypes.data, int(line), int(i), x.ctypes.data, el.ctypes.data)
    return x[:m].copy(), el[:m].copy()


# ----------------------------------------------------------------------------- envelope

def depth_rate(p: dict) -> float:
    """Sample rate of the depth axis: one depth step is 2*depth_step/c of
    two-way travel time (equal to fs when depth_step = c / (2 fs))."""
    return float(p["c"]) / (2.0 * float(p["depth_step"]))


def fir_taps(n_taps: int, cutoff_hz: float, rate_hz: float) -> np.ndarray:
    """Low-pass FIR of the IQ demodulator (Sec. 2 item 3, "envelope detection
    by IQ-demodulation").  Reading: windowed sinc, Blackman window, odd
    length, centred, normalised to unit gain at DC."""
    assert n_taps % 2 == 1
    m = np.arange(n_taps) - (n_taps - 1) / 2.0
    fcn = cutoff_hz / rate_hz
    h = 2.0 * fcn * np.sinc(2.0 * fcn * m) * np.blackman(n_taps)
    return h / h.sum()


def band_centres(p: dict) -> np.ndarray:
    """Centre frequencies of the compounding bank (Sec. 2 item 3: envelope
    detection by IQ demodulation with frequency compounding through a bank of
    configurable bandpasses).  Reading: n_bands bands spaced band_step apart,
    symmetric about fc; n_bands = 1 is plain IQ demodulation at fc."""
    K = max(1, int(p.get("n_bands", 1) or 1))
    return float(p["fc"]) + (np.arange(K) - (K - 1) / 2.0) * float(p.get("band_step", 0.0) or 0.0)


def envelope(p: dict, rf: np.ndarray) -> np.ndarray:
    """IQ demodulation and envelope (Sec. 1 "envelope detection", Sec. 2
    item 3).  For each band centre f_k and each line: baseband
    b(i) = rf(i) exp(-j 2 pi f_k i / rate), low-pass with fir_taps (zero
    padding at the ends, output aligned with the input), band envelope
    2 |iq| so that a tone's envelope equals its amplitude; the compounded
    envelope is the mean of the band envelopes.  No decimation."""
    rf = np.asarray(rf, dtype=np.float64)
    rate = depth_rate(p)
    n_d = rf.shape[-1]
    h = fir_taps(int(p["fir_taps"]), float(p["fir_cutoff"]), rate)
    H = (len(h) - 1) // 2
    flat = rf.reshape(-1, n_d)
    out = np.zeros_like(flat)
    centres = band_centres(p)
    for f_k in centres:
        mix = np.exp(-2j * np.pi * f_k * np.arange(n_d) / rate)
        for k in range(flat.shape[0]):
            iq = np.convolve(flat[k] * mix, h, mode="full")[H:H + n_d]
            out[k] += 2.0 * np.abs(iq)
    return (out / len(centres)).reshape(rf.shape)


# ----------------------------------------------------------------------------- log compression

def logcompress(env: np.ndarray, ref: float, dyn_range_db: float) -> np.ndarray:
    """Log compression to a dynamic range of D dB (Sec. 1 "log-compression",
    Sec. 2 item 4): code = floor(255 (20 log10(env/ref) + D) / D + 1/2)
    clamped to [0, 255]; env <= 0 maps to 0.  Readings: explicit reference
    level ref, half-up rounding."""
    env = np.asarray(env, dtype=np.float64)
    D = float(dyn_range_db)
    with np.errstate(divide="ignore", invalid="ignore"):
        db = 20.0 * np.log10(env / float(ref))
        code = np.floor(255.0 * (db + D) / D + 0.5)
    code = np.where(env > 0, np.clip(code, 0, 255), 0)
    return code.astype(np.uint8)


# ----------------------------------------------------------------------------- scan conversion

INSIDE_EPS = 1e-3  # grid points within this many line/sample indices of the scanned region's edge count as inside


def scan_coordinates(p: dict, pts: np.ndarray):
    """Fractional (line_x, line_y, depth) indices of Cartesian points pts
    [..., 3] and an inside flag.  Scan conversion of Sec. 1 (lines "not
    necessarily parallel" interpolated onto an image with physical
    dimensions) and Sec. 2 item 5 (2D and 3D).

      linear : lines parallel to +z at evenly spaced x -> u = (x - x_0)/dx,
               depth index v = (z - z_0 - depth0) / depth_step
      sector : lines from a common apex at evenly spaced angles in the xz plane
               -> u from atan2(x, z), v from the distance to the apex
      pyramid: lines from a common apex along normalize(tan tx, tan ty, 1),
               tx and ty evenly spaced -> ux from atan(x/z), uy from atan(y/z)
    """
    lo = np.asarray(p["line_origin"], np.float64)
    ld = np.asarray(p["line_dir"], np.float64)
    n_d = int(p["n_depth"])
    d0, dr = float(p["depth0"]), float(p["depth_step"])
    kind = p["geometry"]
    nlx, nly = int(p["lines_x"]), int(p["lines_y"])
    X, Y, Z = pts[..., 0], pts[..., 1], pts[..., 2]
    if kind == "linear":
        x0, x1 = lo[0, 0], lo[-1, 0]
        ux = (X - x0) / ((x1 - x0) / (nlx - 1))
        uy = np.zeros_like(ux)
        v = (Z - lo[0, 2] - d0) / dr
        ok = np.ones(ux.shape, bool)
    elif kind == "sector":
        apex = lo[0]
        th = np.arctan2(ld[:, 0], ld[:, 2])
        rx, rz = X - apex[0], Z - apex[2]
        ux = (np.arctan2(rx, rz) - th[0]) / ((th[-1] - th[0]) / (nlx - 1))
        uy = np.zeros_like(ux)
        v = (np.hypot(rx, rz) - d0) / dr
        ok = np.ones(ux.shape, bool)
    elif kind == "pyramid":
        apex = lo[0]
        tx = np.arctan(ld[:nlx, 0] / ld[:nlx, 2])
        ty = np.arctan(ld[::nlx, 1][:nly] / ld[::nlx, 2][:nly])
        rx, ry, rz = X - apex[0], Y - apex[1], Z - apex[2]
        ok = rz > 0
        rzs = np.where(ok, rz, 1.0)
        ux = (np.arctan(rx / rzs) - tx[0]) / ((tx[-1] - tx[0]) / (nlx - 1))
        uy = (np.arctan(ry / rzs) - ty[0]) / ((ty[-1] - ty[0]) / (nly - 1))
        v = (np.sqrt(rx * rx + ry * ry + rz * rz) - d0) / dr
    else:
        raise ValueError(kind)
    e = INSIDE_EPS
    ok &= (ux >= -e) & (ux <= nlx - 1 + e) & (v >= -e) & (v <= n_d - 1 + e)
    if kind == "pyramid":
        ok &= (uy >= -e) & (uy <= nly - 1 + e)
    return ux, uy, v, ok


def _lerp_axis(u, n):
    """Clamp u to [0, n-1]; lower index and fraction of linear interpolation."""
    u = np.clip(u, 0.0, n - 1)
    i0 = np.minimum(np.floor(u).astype(np.int64), max(n - 2, 0))
    return i0, u - i0


def grid_points(grid: dict) -> np.ndarray:
    """Cartesian coordinates [nz, ny, nx, 3] of the output grid (x fastest)."""
    nx, ny, nz = grid["n"]
    ox, oy, oz = grid["origin"]
    sx, sy, sz = grid["spacing"]
    z, y, x = np.meshgrid(oz + sz * np.arange(nz), oy + sy * np.arange(ny), ox + sx * np.arange(nx), indexing="ij")
    return np.stack([x, y, z], axis=-1)


def scanconvert(p: dict, bm: np.ndarray, pts: np.ndarray | None = None) -> np.ndarray:
    """Scan conversion of log-compressed lines bm [n_lines, n_depth] (uint8)
    onto the grid (or onto explicit points pts [..., 3]).  Bilinear in
    (line, depth) for 2D, trilinear in (line_x, line_y, depth) for the
    pyramid; result floor(value + 1/2); 0 outside the scanned region.
    Readings: interpolation of the log-compressed values (the node order of
    Table 1), grid points within INSIDE_EPS index units of the region's edge
    are inside.  Output shape: grid [nz, ny, nx] (or pts.shape[:-1])."""
    if pts is None:
        pts = grid_points(p["grid"])
    nlx, nly, n_d = int(p["lines_x"]), int(p["lines_y"]), int(p["n_depth"])
    ux, uy, v, ok = scan_coordinates(p, pts)
    b = np.asarray(bm, dtype=np.float64).reshape(nly, nlx, n_d)
    ix, fx = _lerp_axis(ux, nlx)
    iv, fv = _lerp_axis(v, n_d)
    if p["geometry"] == "pyramid":
        iy, fy = _lerp_axis(uy, nly)
        val = 0.0
        for dy, wy in ((0, 1 - fy), (1, fy)):
            for dx, wx in ((0, 1 - fx), (1, fx)):
                for dv, wv in ((0, 1 - fv), (1, fv)):
                    yy = np.minimum(iy + dy, nly - 1)
                    xx = np.minimum(ix + dx, nlx - 1)
                    vv = np.minimum(iv + dv, n_d - 1)
                    val = val + wy * wx * wv * b[yy, xx, vv]
    else:
        val = 0.0
        for dx, wx in ((0, 1 - fx), (1, fx)):
            for dv, wv in ((0, 1 - fv), (1, fv)):
                xx = np.minimum(ix + dx, nlx - 1)
                vv = np.minimum(iv + dv, n_d - 1)
                val = val + wx * wv * b[0, xx, vv]
    out = np.where(ok, np.floor(val + 0.5), 0.0)
    return np.clip(out, 0, 255).astype(np.uint8)


# ----------------------------------------------------------------------------- whole chain

def bmode(p: dict, ch) -> np.ndarray:
    """The whole chain of Table 1 (beamformer -> envelope -> log compression
    -> scan conversion); without a grid the log-compressed lines are returned."""
    rf = das(p, ch)
    env = envelope(p, rf)
    bm = logcompress(env, p["log_ref"], p["dyn_range_db"])
    if p.get("grid") is None:
        return bm
    img = scanconvert(p, bm)
    return img[:, 0, :] if p["grid"]["n"][1] == 1 else img


# ----------------------------------------------------------------------------- minimum variance

def mv_weights(x: np.ndarray, L: int, loading: float | None = None):
    """Minimum-variance (Capon) weights of one pixel from its delayed samples x
    (active elements in element order): subapertures x_l = x[l : l + L],
    l = 0..K-1 with K = M - L + 1 (L clipped to M); R = (1/K) sum_l x_l x_l^T;
    diagonal loading relative to the mean eigenvalue,
    R + loading * (trace(R) / L) * I (default loading 0.01); steering vector 1
    (the data are already delayed); w = R^{-1} 1 / (1^T R^{-1} 1).  Not part of
    the paper: the spatially smoothed MV estimator the learned apodization is
    trained on.  Returns (w, xbar) with xbar = (1/K) sum_l x_l."""
    x = np.asarray(x, np.float64)
    M = len(x)
    L = min(int(L), M)
    K = M - L + 1
    X = np.stack([x[l:l + L] for l in range(K)])
    R = X.T @ X / K
    delta = 0.01 if loading is None else float(loading)
    tr = np.trace(R)
    if tr == 0.0:
        # all samples zero: R = 0 and the loading vanishes; the weights are the
        # infinite-loading limit (uniform) and the output is 0
        return np.full(L, 1.0 / L), X.mean(axis=0)
    R = R + delta * (tr / L) * np.eye(L)
    z = np.linalg.solve(R, np.ones(L))
    return z / z.sum(), X.mean(axis=0)


def mv_point(p: dict, ch_tx, line: int, i: int, L: int = 32, loading: float | None = None) -> float:
    """MV output y = w^T xbar at (line, depth i); fewer than two active
    elements fall back to the delay-and-sum value."""
    x, _ = delayed_samples(p, ch_tx, line, i)
    if len(x) < 2:
        return float(das_points(p, [line], [i], [ch_tx])[0])
    w, xbar = mv_weights(x, L, loading)
    return float(w @ xbar)


def mv(p: dict, ch, L: int = 32, loading: float | None = None, lines=None, depths=None) -> np.ndarray:
    """MV beamformed lines [n_lines, n_depth] (or the selected lines x depths)."""
    ch = np.asarray(ch)
    lines = range(len(p["line_tx"])) if lines is None else lines
    depths = range(int(p["n_depth"])) if depths is None else depths
    out = np.zeros((len(lines), len(depths)))
    for a, l in enumerate(lines):
        ch_tx = ch[int(p["line_tx"][l])]
        for b, i in enumerate(depths):
            out[a, b] = mv_point(p, ch_tx, l, i, L, loading)
    return out
