"""Helpers of the GPU parity tests: tolerances and comparisons.

Tolerances (stated once, used everywhere):
  RF (beamformer output): max |gpu - oracle| / max |oracle| <= 1e-4
  envelope (same fp32 RF in): max |gpu - oracle| / max |oracle| <= 1e-5
  uint8 B-mode lines / images: every pixel within 1 gray level of the oracle
      and at least 99.9 % of pixels within 1 gray level after the whole chain
      (the fp32 chain moves values that sit near a rounding boundary).
"""
import numpy as np

RF_TOL = 1e-4
ENV_TOL = 1e-5
BM_FRAC = 0.999


def max_norm_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / (scale if scale > 0 else 1.0))


def gray_stats(got, ref):
    d = np.abs(np.asarray(got, np.int32) - np.asarray(ref, np.int32))
    return float(np.mean(d <= 1)), int(d.max()), float(np.mean(d == 0))


def assert_gray(got, ref, frac=BM_FRAC, what=""):
    within1, dmax, exact = gray_stats(got, ref)
    assert within1 >= frac, f"{what}: only {within1:.5f} within 1 gray level (max diff {dmax}, exact {exact:.5f})"
    return within1, dmax, exact
