"""Pins of the learned-apodization oracle (network, loss, gradient, Adam).
The network is not in the paper; every pin here follows from the definitions
(finite differences, softmax invariants, special cases that reduce to
delay-and-sum, Adam's closed form under a constant gradient)."""
import numpy as np
import pytest

import oracle
from oracle import apod
import phantom


def _inputs(seed, n, min_active=2):
    X, mask, norm, t = phantom.apod_random_batch(seed, n, min_active)
    return X.astype(np.float64) / norm[:, None], mask, t


def test_parameter_count_and_layout():
    assert apod.N_PARAMS == 20480 + 256
    p = phantom.apod_init(1, out_scale=1.0, bias_scale=0.1)
    d = apod.unpack(p)
    assert d["W1"].shape == (64, 128) and d["W3"].shape == (128, 64) and d["b3"].shape == (128,)
    np.testing.assert_array_equal(apod.pack(d), p.astype(np.float64))


def test_gradient_matches_central_differences():
    params = phantom.apod_init(3, out_scale=2.0, bias_scale=0.2).astype(np.float64)
    Xh, mask, t = _inputs(4, 6)
    loss, g = apod.loss_and_grad(params, Xh, mask, t)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(apod.N_PARAMS, 500, replace=False),
                          np.arange(8192, 8192 + 64), np.arange(12352, 12352 + 64), np.arange(20608, 20736)])
    h = 1e-6
    fd = np.empty(len(idx))
    for j, k in enumerate(idx):
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        fd[j] = (apod.loss_and_grad(pp, Xh, mask, t)[0] - apod.loss_and_grad(pm, Xh, mask, t)[0]) / (2 * h)
    scale = np.max(np.abs(g[idx]))
    assert scale > 0
    np.testing.assert_allclose(fd, g[idx], rtol=0, atol=1e-6 * scale + 1e-12)
    # every layer receives gradient
    d = apod.unpack(g)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert np.max(np.abs(d[name])) > 0, name


def test_softmax_weights_are_a_distribution_on_the_mask():
    params = phantom.apod_init(6, out_scale=3.0, bias_scale=0.5)
    Xh, mask, _ = _inputs(7, 20)
    mask[3] = False                      # an empty aperture: no weights, output 0
    Xh[3] = 0.0
    yh, w, _ = apod.forward(params, Xh, mask)
    assert np.all(w[~mask] == 0.0) and np.all(w >= 0.0)
    s = w.sum(axis=1)
    np.testing.assert_allclose(s[np.arange(20) != 3], 1.0, rtol=1e-12)
    assert s[3] == 0.0 and yh[3] == 0.0
    # the output is a convex combination of the masked inputs
    lo = np.where(mask, Xh, np.inf).min(axis=1)
    hi = np.where(mask, Xh, -np.inf).max(axis=1)
    k = np.arange(20) != 3
    assert np.all(yh[k] >= lo[k] - 1e-12) and np.all(yh[k] <= hi[k] + 1e-12)


def test_output_bias_gradient_sums_to_zero():
    # a constant shift of all logits leaves the softmax unchanged, so the
    # gradient of b3 sums to zero per pixel (a sign or term error breaks this)
    params = phantom.apod_init(8, out_scale=1.0, bias_scale=0.3)
    Xh, mask, t = _inputs(9, 10)
    _, g = apod.loss_and_grad(params, Xh, mask, t)
    gb3 = apod.unpack(g)["b3"]
    assert abs(gb3.sum()) <= 1e-12 * np.max(np.abs(gb3)) * 128


def test_single_active_element_has_no_gradient():
    params = phantom.apod_init(10, out_scale=1.0, bias_scale=0.3)
    Xh = np.zeros((1, 128))
    mask = np.zeros((1, 128), bool)
    Xh[0, 40], mask[0, 40] = -1.0, True
    yh, w, _ = apod.forward(params, Xh, mask)
    assert w[0, 40] == 1.0 and yh[0] == -1.0
    loss, g = apod.loss_and_grad(params, Xh, mask, np.array([0.25]))
    assert loss == pytest.approx(1.5625) and np.all(g == 0.0)


def test_invalid_pixels_do_not_contribute():
    params = phantom.apod_init(11, out_scale=1.0, bias_scale=0.1)
    Xh, mask, t = _inputs(12, 8)
    valid = np.array([1, 0, 1, 1, 0, 1, 1, 1], bool)
    l1, g1 = apod.loss_and_grad(params, Xh, mask, t, valid)
    l2, g2 = apod.loss_and_grad(params, Xh[valid], mask[valid], t[valid])
    assert l1 == pytest.approx(l2, rel=1e-12)
    np.testing.assert_allclose(g1, g2, rtol=1e-12, atol=1e-18)


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g, the bias-corrected moments are exactly g and
    # g^2 at every step, so each step moves by lr * g / (|g| + eps)
    p0 = np.array([0.5, -1.0, 2.0, 0.0])
    g = np.array([0.3, -2.0, 1e-9, 0.0])
    lr, eps = 1e-2, 1e-8
    p, m, v = p0.copy(), np.zeros(4), np.zeros(4)
    for s in range(1, 6):
        p, m, v = apod.adam(p, m, v, g, s, lr, eps=eps)
    np.testing.assert_allclose(p, p0 - 5 * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)


def test_zero_output_layer_is_rectangular_das():
    # W3 = 0, b3 = 0: uniform weights over the aperture, y = mean of the
    # delayed samples = delay-and-sum with a rectangular window
    s = phantom.linear_setup(16, 0.3e-3, 4, 300, fc=5e6, fs=40e6)
    p = dict(s.params(), window="rect")
    ch = phantom.random_channels(s, 21).numpy()
    params = phantom.apod_init(22)
    lines, depths = [0, 2, 3], list(range(0, 300, 13))
    y = apod.beamform(p, ch, params, lines, depths)
    ref = np.array([[oracle.das_points(p, [l], [i], [ch[s.line_tx[l]]])[0] for i in depths] for l in lines])
    np.testing.assert_allclose(y, ref, rtol=1e-9, atol=1e-9 * np.max(np.abs(ref)))


def test_round_bf16_special_values():
    one = 1.0
    ulp = 2.0 ** -7                       # spacing of BF16 values in [1, 2)
    vals = np.array([one, one + ulp, one + ulp / 2, one + 3 * ulp / 2, one + ulp / 2 + 2 ** -20, -2.5, 0.0,
                     3.0e38, 1e-40])
    want = np.array([one, one + ulp, one, one + 2 * ulp, one + ulp, -2.5, 0.0, 2.0 ** 128 * (1 - 2 ** -9), 0.0])
    got = apod.round_bf16(vals)
    np.testing.assert_array_equal(got[:6], want[:6])
    assert got[6] == 0.0
    # the largest finite float32 region rounds to a BF16 value within 2^-8 relative
    assert abs(got[7] - 3.0e38) <= 2 ** -8 * 3.0e38
    # BF16 keeps float32's exponent range: a subnormal stays within one subnormal step
    assert abs(got[8] - 1e-40) <= 2.0 ** -133


def test_bf16_mode_rounds_operands_only():
    # every rounded operand is BF16-representable, and the BF16 network stays
    # within a few BF16 ulps of the FP64 one
    params = phantom.apod_init(13, out_scale=1.0, bias_scale=0.1)
    Xh, mask, t = _inputs(14, 64)
    yh64, _, c64 = apod.forward(params, Xh, mask)
    yh16, _, c16 = apod.forward(params, Xh, mask, bf16=True)
    for h in (c16[2], c16[4]):
        np.testing.assert_array_equal(h, apod.round_bf16(h))
    assert np.max(np.abs(yh16 - yh64)) <= 5e-2 * np.max(np.abs(yh64))
    l64, g64 = apod.loss_and_grad(params, Xh, mask, t)
    l16, g16 = apod.loss_and_grad(params, Xh, mask, t, bf16=True)
    assert l16 == pytest.approx(l64, rel=5e-2)
    assert np.linalg.norm(g16 - g64) <= 0.1 * np.linalg.norm(g64)
    # with BF16-representable inputs and weights and bf16=False on both, the
    # modes agree on the first layer exactly (no rounding there)
    pr = apod.round_bf16(params)
    Xr = apod.round_bf16(Xh)
    _, _, ca = apod.forward(pr, Xr, mask)
    _, _, cb = apod.forward(pr, Xr, mask, bf16=True)
    np.testing.assert_array_equal(ca[1], cb[1])


def test_beamform_scales_with_the_records():
    # the network sees xh = x / ||x||: records scaled by two give the same weights (the
    # power-of-two scale leaves xh and its BF16 rounding unchanged) and twice the output
    s = phantom.linear_setup(24, 0.3e-3, 3, 300, fc=5e6, fs=40e6)
    p = s.params()
    ch = phantom.random_channels(s, 17, amplitude=4000).numpy()
    params = phantom.apod_init(18, out_scale=2.0, bias_scale=0.1)
    lines, depths = [0, 1, 2], list(range(0, 300, 7))
    for bf16 in (False, True):
        y1 = apod.beamform(p, ch, params, lines, depths, bf16=bf16)
        y2 = apod.beamform(p, 2 * ch, params, lines, depths, bf16=bf16)
        assert np.any(y1 != 0)
        np.testing.assert_array_equal(y2, 2 * y1)
