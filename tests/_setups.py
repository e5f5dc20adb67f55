"""Small parameter dictionaries shared by the tests (plain inputs, no method
arithmetic)."""
import numpy as np

import phantom


def tiny(elem_mm, line_origin_mm=((0, 0, 0),), line_dir=((0, 0, 1),), tx_origin_mm=None, line_tx=None,
         n_samples=400, n_depth=None, c=1540.0, fs=15.4e6, fnumber=1.0, min_half_aperture=50e-3,
         window="rect", t0=0.0, geometry="linear", lines_x=None, lines_y=1, fc=None, grid=None):
    elem = np.asarray(elem_mm, dtype=np.float64).reshape(-1, 3) * 1e-3
    lo = np.asarray(line_origin_mm, dtype=np.float64).reshape(-1, 3) * 1e-3
    ld = np.asarray(line_dir, dtype=np.float64).reshape(-1, 3)
    ld = ld / np.linalg.norm(ld, axis=1, keepdims=True)
    if tx_origin_mm is None:
        tx = lo.copy()
    else:
        tx = np.asarray(tx_origin_mm, dtype=np.float64).reshape(-1, 3) * 1e-3
    if line_tx is None:
        line_tx = np.arange(lo.shape[0]) if tx.shape[0] == lo.shape[0] else np.zeros(lo.shape[0])
    return dict(elem_pos=elem, tx_origin=tx, line_origin=lo, line_dir=ld,
                line_tx=np.asarray(line_tx, np.int32), n_depth=n_samples if n_depth is None else n_depth,
                depth0=0.0, depth_step=c / (2 * fs), geometry=geometry,
                lines_x=lo.shape[0] if lines_x is None else lines_x, lines_y=lines_y, c=c, fs=fs,
                fc=fs / 8 if fc is None else fc, fnumber=fnumber, min_half_aperture=min_half_aperture,
                window=window, n_samples=n_samples, t0=t0, fir_taps=31, fir_cutoff=(fs / 8 if fc is None else fc) / 2,
                dyn_range_db=60.0, log_ref=1000.0, grid=grid)


def small_linear(n_el=16, n_lines=12, n_samples=300, window="hann", seed=0, **kw):
    """A small linear-array acquisition that still spans several depth tiles."""
    s = phantom.linear_setup(n_el, 0.3e-3, n_lines, n_samples, fc=5e6, fs=40e6, focus=10e-3, fnumber=1.5,
                             window=window, **kw)
    return s
