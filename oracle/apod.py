"""FP64 oracle of the learned apodization (test infrastructure only: imported by
the tests, the smoke check and the benchmark's CPU baseline, never by the
product path).

The paper has no learned beamformer; this is the per-pixel network that stands
in for the exact minimum-variance beamformer, written out plainly:

  x      delayed, interpolated samples of all n_el <= 128 elements at the pixel
         (delays and F-number aperture of the delay-and-sum step, Sec. 2 item 1;
         zero outside the aperture), mask = aperture membership
  xh     = x / ||x||                          (zero pixel: not a training pixel)
  h1     = relu(W1 xh + b1)                   W1: 64 x 128
  h2     = relu(W2 h1 + b2)                   W2: 64 x 64
  z      = W3 h2 + b3                         W3: 128 x 64
  w      = softmax of z over the masked elements (0 elsewhere)
  yh     = sum_e w_e xh_e,   beamformed value y = ||x|| yh = sum_e w_e x_e
  loss   = mean over training pixels of (yh - t)^2,  t = y_MV / ||x||

Parameters are one flat vector in the order W1, b1, W2, b2, W3, b3 (row-major
matrices, [out][in]); 20 480 weights and 256 biases.  Optimiser: Adam with bias
correction.

Precision.  The method's products are BF16 x BF16 with FP32 accumulation.
With bf16=True the oracle rounds every product operand to BF16 (round to
nearest even) exactly where the method defines one -- weights, the network
input xh, the layer inputs h1 and h2, and the output gradients dz, dz2, dz1 --
and keeps FP64 for everything else, so the ReLU decisions are taken on the same
values as the kernels take them.  Biases, softmax, loss and Adam are never
rounded.  With bf16=False (default) everything is FP64.  Two readings fix where
a rounding sits:
  * the network's input operand is the normalised xh = x / ||x|| rounded to
    BF16, in training and in inference alike (one network function);
  * the loss is a mean, i.e. a sum over pixels divided by their count n: the
    BF16 output-gradient operand of a pixel is the derivative of that pixel's
    squared error, 2 (yh - t) w (x - yh), and 1/n scales the FP32 sums, so no
    per-pixel operand depends on how many pixels share the minibatch.
"""
from __future__ import annotations

import numpy as np

from . import delayed_samples

N_IN, N_H1, N_H2 = 128, 64, 64
SHAPES = (("W1", (N_H1, N_IN)), ("b1", (N_H1,)), ("W2", (N_H2, N_H1)), ("b2", (N_H2,)),
          ("W3", (N_IN, N_H2)), ("b3", (N_IN,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def round_bf16(a) -> np.ndarray:
    """Nearest BFloat16 value (ties to even) of each element, as float64:
    the float32 value's top 16 bits after round-to-nearest-even."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _q(a, bf16: bool):
    return round_bf16(a) if bf16 else np.asarray(a, np.float64)


def unpack(params) -> dict:
    """Views of the flat parameter vector by name."""
    params = np.asarray(params, np.float64)
    assert params.shape == (N_PARAMS,)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = params[o:o + n].reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def features(p: dict, ch_tx, line: int, i: int):
    """(x[128], mask[128]) at (line, depth i): the delayed samples of the active
    elements at their element index, zero elsewhere."""
    xa, el = delayed_samples(p, ch_tx, line, i)
    x = np.zeros(N_IN)
    mask = np.zeros(N_IN, bool)
    x[el] = xa
    mask[el] = True
    return x, mask


def forward(params, X, mask, bf16: bool = False):
    """Network on a batch: X[B,128] normalised inputs xh, mask[B,128].
    Returns (yh[B], w[B,128], cache); yh = sum_e w_e X_e."""
    P = unpack(params)
    X = _q(X, bf16)
    mask = np.asarray(mask, bool)
    W1, W2, W3 = (_q(P[k], bf16) for k in ("W1", "W2", "W3"))
    z1 = X @ W1.T
    z1 = z1 + P["b1"]
    h1 = _q(np.maximum(z1, 0.0), bf16)
    z2 = h1 @ W2.T + P["b2"]
    h2 = _q(np.maximum(z2, 0.0), bf16)
    z = h2 @ W3.T + P["b3"]
    # masked softmax, shifted by the masked maximum
    zm = np.where(mask, z, -np.inf)
    zmax = np.max(zm, axis=1, keepdims=True)
    zmax = np.where(np.isfinite(zmax), zmax, 0.0)
    e = np.where(mask, np.exp(np.where(mask, z - zmax, 0.0)), 0.0)
    s = e.sum(axis=1, keepdims=True)
    w = np.divide(e, s, out=np.zeros_like(e), where=s > 0)
    yh = np.sum(w * X, axis=1)
    return yh, w, (X, z1, h1, z2, h2, w)


def loss_and_grad(params, X, mask, t, valid=None, bf16: bool = False):
    """Mean squared error over the valid pixels and its gradient with respect to
    the flat parameters (reverse-mode chain rule written out layer by layer).
    The per-pixel output gradients are formed unnormalised (2 (yh - t)) and the
    sums divided by the pixel count at the end."""
    P = unpack(params)
    t = np.asarray(t, np.float64)
    valid = np.ones(len(t), bool) if valid is None else np.asarray(valid, bool)
    n = int(valid.sum())
    yh, w, (X, z1, h1, z2, h2, _) = forward(params, X, mask, bf16)
    if n == 0:
        return 0.0, np.zeros(N_PARAMS)
    W2, W3 = _q(P["W2"], bf16), _q(P["W3"], bf16)
    r = np.where(valid, yh - t, 0.0)
    loss = float(np.sum(r * r) / n)
    dyh = 2.0 * r                                       # n * d loss / d yh
    # yh = sum_e w_e x_e, w = softmax(z):  d yh / d z_e = w_e (x_e - yh)
    dz = _q(w * (X - yh[:, None]) * dyh[:, None], bf16)
    g = {"W3": dz.T @ h2, "b3": dz.sum(axis=0)}
    dh2 = dz @ W3
    dz2 = _q(dh2 * (z2 > 0), bf16)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = _q(dh1 * (z1 > 0), bf16)
    g["W1"], g["b1"] = dz1.T @ X, dz1.sum(axis=0)
    return loss, pack(g) / n


def adam(params, m, v, grad, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1): m, v moving averages of the
    gradient and its square, bias-corrected by 1 - beta^step."""
    params, m, v, grad = (np.asarray(a, np.float64) for a in (params, m, v, grad))
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def batch(p: dict, ch, labels=None, lines=None, depths=None):
    """Training/evaluation arrays of selected pixels: (X normalised, mask, norm,
    t) with t = labels / norm (labels: [n_lines, n_depth], e.g. the MV output)."""
    ch = np.asarray(ch)
    lines = range(len(p["line_tx"])) if lines is None else lines
    depths = range(int(p["n_depth"])) if depths is None else depths
    xs, ms, ns, ts = [], [], [], []
    for l in lines:
        ch_tx = ch[int(p["line_tx"][l])]
        for i in depths:
            x, mk = features(p, ch_tx, l, i)
            nrm = float(np.sqrt(np.sum(x * x)))
            xs.append(x / nrm if nrm > 0 else x)
            ms.append(mk)
            ns.append(nrm)
            if labels is not None:
                ts.append(labels[l, i] / nrm if nrm > 0 else 0.0)
    return np.array(xs), np.array(ms), np.array(ns), (np.array(ts) if labels is not None else None)


def beamform(p: dict, ch, params, lines=None, depths=None, bf16: bool = False) -> np.ndarray:
    """Learned-apodization output y = ||x|| sum_e w_e xh_e = sum_e w_e x_e at
    the selected pixels, [len(lines), len(depths)].  With bf16=True the network
    input is xh rounded to BF16, as in training."""
    lines = list(range(len(p["line_tx"]))) if lines is None else list(lines)
    depths = list(range(int(p["n_depth"]))) if depths is None else list(depths)
    X, mask, norm, _ = batch(p, ch, None, lines, depths)
    yh, _, _ = forward(params, X, mask, bf16)
    return (yh * norm).reshape(len(lines), len(depths))
