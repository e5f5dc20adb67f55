"""Pins of the minimum-variance oracle (the exact MV beamformer the learned
apodization is trained against; not in the paper)."""
import numpy as np
import pytest

import oracle
import phantom


def test_single_element_subapertures_average():
    # L = 1: R is a scalar, w = 1, the output is the mean of the delayed samples
    x = np.random.default_rng(0).normal(size=17)
    w, xbar = oracle.mv_weights(x, 1)
    assert w[0] == pytest.approx(1.0) and float(w @ xbar) == pytest.approx(x.mean(), rel=1e-12)


@pytest.mark.parametrize("M,L", [(10, 4), (33, 32), (64, 32), (7, 7)])
def test_infinite_loading_is_trapezoid_average(M, L):
    # loading -> inf: w -> 1/L, y = (1/(L K)) sum_e c_e x_e, c_e = number of subapertures holding e
    x = np.random.default_rng(M).normal(size=M)
    w, xbar = oracle.mv_weights(x, L, loading=1e12)
    K = M - L + 1
    c = np.array([sum(1 for l in range(K) if l <= e < l + L) for e in range(M)])
    np.testing.assert_allclose(w, 1.0 / L, rtol=1e-9)
    assert float(w @ xbar) == pytest.approx(float(c @ x) / (L * K), rel=1e-9)


def test_constant_data_returns_the_constant_and_weights_are_distortionless():
    x = np.full(40, 3.25)
    w, xbar = oracle.mv_weights(x, 16)
    assert w.sum() == pytest.approx(1.0, rel=1e-12)
    assert float(w @ xbar) == pytest.approx(3.25, rel=1e-12)
    x = np.random.default_rng(1).normal(size=50)
    w, _ = oracle.mv_weights(x, 32)
    assert w.sum() == pytest.approx(1.0, rel=1e-12)


def test_two_by_two_closed_form():
    # M = L = 2, K = 1: R = x x^T + e (tr(R) / 2) I, inverse by the adjugate
    x0, x1, e = 3.0, -1.5, 0.01
    a, b, d = x0 * x0, x0 * x1, x1 * x1
    t = e * (a + d) / 2
    R = np.array([[a + t, b], [b, d + t]])
    det = R[0, 0] * R[1, 1] - R[0, 1] * R[1, 0]
    z = np.array([R[1, 1] - R[0, 1], R[0, 0] - R[1, 0]]) / det
    w_ref = z / z.sum()
    w, xbar = oracle.mv_weights(np.array([x0, x1]), 2, loading=e)
    np.testing.assert_allclose(w, w_ref, rtol=1e-12)
    assert float(w @ xbar) == pytest.approx(float(w_ref @ [x0, x1]), rel=1e-12)


def test_mv_suppresses_an_interferer_that_das_passes():
    # two plane-wave components across the aperture: the look direction (constant across
    # elements, already delayed) and an interferer with a linear phase; MV nulls the interferer
    M, L = 64, 16
    e = np.arange(M)
    look = 1.0
    interferer = 5.0 * np.cos(0.9 * e)
    w, xbar = oracle.mv_weights(look + interferer, L)
    y = float(w @ xbar)
    das = float(np.mean(look + interferer))
    assert abs(y - look) < 0.1 * abs(das - look) + 1e-3


def test_point_fallback_and_full_frame_agree():
    s = phantom.linear_setup(8, 0.3e-3, 4, 200, fc=5e6, fs=40e6)
    p = s.params()
    ch = phantom.random_channels(s, 2).numpy()
    full = oracle.mv(p, ch, L=4, lines=[1, 2], depths=range(0, 200, 17))
    for a, l in enumerate([1, 2]):
        for b, i in enumerate(range(0, 200, 17)):
            assert full[a, b] == pytest.approx(oracle.mv_point(p, ch[s.line_tx[l]], l, i, 4), rel=1e-12)
    # the first depths have a single active element: MV falls back to delay-and-sum there
    x, _ = oracle.delayed_samples(p, ch[1], 1, 0)
    if len(x) < 2:
        assert full[0, 0] == pytest.approx(oracle.das_points(p, [1], [0], [ch[1]])[0])


def test_all_zero_aperture_gives_uniform_weights_and_zero_output():
    # trace(R) = 0: no loading, singular R; the infinite-loading limit applies
    w, xbar = oracle.mv_weights(np.zeros(20), 8)
    np.testing.assert_array_equal(w, np.full(8, 1.0 / 8))
    assert float(w @ xbar) == 0.0
