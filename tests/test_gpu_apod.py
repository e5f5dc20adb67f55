"""GPU parity of the learned apodization (feature rows, forward, gradient,
Adam, fused inference) against the FP64 oracle, plus training behaviour.

Two comparisons per output.

1. Against the oracle's BF16 mode, which rounds the same operands as the
   method defines them (weights, the network input, the hidden activations,
   the output gradients) and computes the rest in FP64, so both sides take the
   same ReLU decisions: what remains is FP32 against FP64 accumulation and exp
   (~1e-6 relative) and the rare BF16 rounding tie that the two accumulations
   resolve differently (one BF16 ulp, 2^-8, on one operand element).  Outputs
   and gradients: max |gpu - oracle| <= 2e-3 of the largest magnitude.  The
   fused beamformer rounds the gathered samples before the 1/||x|| scale (the
   oracle rounds xh itself: the two placements differ by one rounding of the
   input, up to 2^-8 relative) and adds the gather's FP32 delay error (~1e-4 of
   ||x|| on white-noise records): 5e-3.
2. Element by element against the unrounded FP64 network.  BF16 rounding
   (unit roundoff u = 2^-9) perturbs each product of a sum by at most 2u
   relative per rounded stage; the forward output passes two rounded
   activations, a weight gradient at most five rounded stages (h1, h2, dz,
   dz2, dz1), so each term of a gradient sum moves by less than 6u = 3 * 2^-8
   of its magnitude, and a ReLU decision that flips near zero switches single
   terms.  The bound is therefore relative to the sum of the absolute values
   of the terms, S (its condition scale: the gradient of a minibatch with
   random targets is a near-cancelling sum, |g| ~ 1e-2 S), and a parameter
   block's gradient must satisfy max |g_gpu - g_64| <= 2^-6 max S (4 * 2^-8).
   The forward output is a convex combination of the inputs (no
   cancellation): max |y_gpu - y_64| <= 2^-7 of max |y_64|; the fused
   beamformer adds its gather error: 2^-6.
Adam: 1e-5 relative.  Bit equality where the same pixels are processed in the
same order.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import apod as oapod
import paper_1711_06127_b300 as supra
from paper_1711_06127_b300 import apod
import phantom
from _setups import small_linear

pytestmark = pytest.mark.gpu
TOL = 2e-3          # against the oracle's bf16 mode
TOL_INFER = 5e-3    # fused beamformer (adds the gather's FP32 delay error)
TOL_FP64_FWD = 2.0 ** -7     # against the unrounded FP64 network: forward output, of max |y|
TOL_FP64_INFER = 2.0 ** -6   # fused beamformer, of max |y|
TOL_FP64_GRAD = 2.0 ** -6    # gradients, of the block's condition scale max S


def _bf16(a):
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16)


def _rows(seed, n, min_active=2, zero_rows=()):
    """Random rows for both sides: feature rows bf16(x / ||x||) on the device,
    the same rounded values in FP64 for the oracle."""
    X, mask, norm, t = phantom.apod_random_batch(seed, n, min_active)
    for r in zero_rows:
        X[r], norm[r] = 0.0, 0.0
    xh = np.divide(X, norm[:, None], out=np.zeros_like(X), where=norm[:, None] > 0)
    feat = _bf16(xh)
    xh64 = feat.float().numpy().astype(np.float64)
    words = np.zeros((n, 4), np.uint32)
    for w in range(4):
        words[:, w] = (mask[:, 32 * w:32 * (w + 1)].astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1)
    dev = dict(feat=feat.cuda(), mask=torch.as_tensor(words.view(np.int32)).cuda(),
               norm=torch.as_tensor(norm.astype(np.float32)).cuda(),
               label=torch.as_tensor((t * norm).astype(np.float32)).cuda())
    return dev, xh64, mask, norm, t


def _params(seed, **kw):
    """Seeded parameters rounded to BF16-representable values, so that the GPU
    (which rounds its FP32 master weights to BF16 for the tensor cores) and the
    oracle use identical weights and take the same ReLU decisions."""
    return _bf16(phantom.apod_init(seed, **kw)).float().numpy()


def _data(dev):
    return apod.Dataset(dev["feat"], dev["mask"], dev["norm"], dev["label"])


def _max_rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-30))


def _grad_condition_scale(params, xh, mask, t, valid):
    """Per parameter block, the largest condition scale S of its gradient
    elements: the FP64 network's backward pass on absolute values (|terms| of
    every sum), with the residual's magnitude |yh - t| + sum_e w_e |xh_e| (so
    that a perturbation of the forward output counts), divided by the pixel
    count like the gradient."""
    P = oapod.unpack(params)
    yh, w, (X, z1, h1, z2, h2, _) = oapod.forward(params, xh, mask)
    n = int(np.sum(valid))
    R = np.where(valid, np.abs(yh - t) + np.sum(w * np.abs(X), axis=1), 0.0)
    dz = 2.0 * R[:, None] * w * (np.abs(X) + np.abs(yh)[:, None])
    S = {"W3": dz.T @ np.abs(h2), "b3": dz.sum(0)}
    dz2 = (dz @ np.abs(P["W3"])) * (z2 > 0)
    S["W2"], S["b2"] = dz2.T @ np.abs(h1), dz2.sum(0)
    dz1 = (dz2 @ np.abs(P["W2"])) * (z1 > 0)
    S["W1"], S["b1"] = dz1.T @ np.abs(X), dz1.sum(0)
    return {k: float(np.max(v)) / n for k, v in S.items()}


def test_features_match_the_oracle():
    s = small_linear(48, 6, 600)
    p = s.params()
    ch = phantom.random_channels(s, 31)
    plan = supra.Plan(**p)
    feat, mask, norm = plan.apod_features(ch.cuda())
    feat, mask, norm = feat.float().cpu().numpy(), mask.cpu().numpy().view(np.uint32), norm.cpu().numpy()
    checked = 0
    for l in range(s.n_lines):
        for i in range(0, s.n_depth, 23):
            x, m = oapod.features(p, ch.numpy()[s.line_tx[l]], l, i)
            _, _, margin = oracle.aperture(p, l, i)
            if np.min(np.abs(margin)) <= 1e-9:
                continue
            k = l * s.n_depth + i
            bits = np.array([(mask[k, e >> 5] >> (e & 31)) & 1 for e in range(128)], bool)
            np.testing.assert_array_equal(bits, m)
            nrm = np.sqrt(np.sum(x * x))
            assert norm[k] == pytest.approx(nrm, rel=1e-5, abs=1e-3)
            if nrm > 0:
                # BF16 rounding (2^-9 relative) plus the FP32 delay error: ~1e-5
                # samples times slopes of up to 16000 per sample on white-noise
                # records, ~1e-4 of ||x||
                np.testing.assert_allclose(feat[k], x / nrm, rtol=2 ** -8, atol=2e-4)
            checked += 1
    assert checked > 100


def test_forward_matches_the_oracle():
    params = _params(40, out_scale=2.0, bias_scale=0.1)
    dev, xh, mask, norm, _ = _rows(41, 1000, zero_rows=(5, 999))
    y = apod.forward(torch.as_tensor(params).cuda(), dev["feat"], dev["mask"], dev["norm"]).cpu().numpy()
    yh, _, _ = oapod.forward(params.astype(np.float64), xh, mask, bf16=True)
    ref = yh * norm
    assert y[5] == 0.0 and y[999] == 0.0
    assert _max_rel(y, ref) <= TOL
    yh64, _, _ = oapod.forward(params.astype(np.float64), xh, mask)
    err64 = _max_rel(y, yh64 * norm)
    assert err64 <= TOL_FP64_FWD, err64


@pytest.mark.parametrize("n", [1000, 148 * 128 * 2 + 77])
def test_gradient_matches_the_oracle(n):
    # n = 1000: one tile per CTA and a ragged last tile; the larger n makes every
    # CTA accumulate several tiles in tensor memory
    params = _params(50, out_scale=1.0, bias_scale=0.1)
    dev, xh, mask, norm, t = _rows(51, n, zero_rows=(0, 7))
    tr = apod.Trainer(params)
    grad, loss = tr.compute_grad(_data(dev))
    grad, loss = grad.cpu().numpy(), float(loss.item())
    valid = norm > 0
    ref_loss, ref = oapod.loss_and_grad(params.astype(np.float64), xh, mask, t, valid, bf16=True)
    assert loss == pytest.approx(ref_loss, rel=TOL)
    g, r = oapod.unpack(grad), oapod.unpack(ref)
    errs = {name: _max_rel(g[name], r[name]) for name in ("W1", "b1", "W2", "b2", "W3", "b3")}
    assert max(errs.values()) <= TOL, errs
    # element by element against the unrounded FP64 network, every block
    ref_loss64, ref64 = oapod.loss_and_grad(params.astype(np.float64), xh, mask, t, valid)
    assert loss == pytest.approx(ref_loss64, rel=TOL_FP64_FWD)
    S = _grad_condition_scale(params.astype(np.float64), xh, mask, t, valid)
    r64 = oapod.unpack(ref64)
    errs64 = {name: float(np.max(np.abs(g[name] - r64[name]))) / S[name] for name in S}
    assert max(errs64.values()) <= TOL_FP64_GRAD, errs64
    assert supra.device_status() == 0


def test_strided_minibatch_equals_the_gathered_rows_and_is_deterministic():
    params = phantom.apod_init(60, out_scale=1.0, bias_scale=0.1)
    dev, *_ = _rows(61, 5000)
    tr = apod.Trainer(params)
    g1 = tr.compute_grad(_data(dev), base=3, stride=7)[0].clone()
    g2 = tr.compute_grad(_data(dev), base=3, stride=7)[0].clone()
    sub = {k: v[3::7].contiguous() for k, v in dev.items()}
    g3 = tr.compute_grad(_data(sub))[0].clone()
    assert torch.equal(g1, g2) and torch.equal(g1, g3)


def test_adam_matches_the_oracle():
    rng = np.random.default_rng(70)
    p0 = rng.normal(0, 0.1, supra.APOD_PARAMS).astype(np.float32)
    tr = apod.Trainer(p0, lr=3e-3)
    p, m, v = p0.astype(np.float64), np.zeros(supra.APOD_PARAMS), np.zeros(supra.APOD_PARAMS)
    for step in range(1, 4):
        g = rng.normal(0, 1e-2, supra.APOD_PARAMS).astype(np.float32)
        tr.grad.copy_(torch.as_tensor(g))
        tr.apply()
        p, m, v = oapod.adam(p, m, v, g.astype(np.float64), step, 3e-3)
    np.testing.assert_allclose(tr.params.cpu().numpy(), p, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(tr.m.cpu().numpy(), m, rtol=1e-5, atol=1e-9)


def test_fused_training_step_equals_gradient_then_adam():
    # supra_apod_step (gradient, then the reduction and the Adam update in one kernel) against the
    # two separate calls (each checked against the oracle above), over three steps of strided minibatches
    params = phantom.apod_init(62, out_scale=1.0, bias_scale=0.1)
    dev, *_ = _rows(63, 3000)
    a, b = apod.Trainer(params, lr=2e-3), apod.Trainer(params, lr=2e-3)
    losses = torch.zeros(3, dtype=torch.float32, device="cuda")
    for k in range(3):
        ga, la = a.compute_grad(_data(dev), base=k, stride=3)
        la = la.clone()
        a.apply()
        b.step(_data(dev), base=k, stride=3, loss_out=losses[k : k + 1])
        torch.testing.assert_close(b.grad, ga, rtol=0, atol=0)
        assert losses[k].item() == la.item()
        torch.testing.assert_close(b.params, a.params, rtol=0, atol=0)
        torch.testing.assert_close(b.m, a.m, rtol=0, atol=0)
        torch.testing.assert_close(b.v, a.v, rtol=0, atol=0)
    assert b.step_count == 3
    with pytest.raises(ValueError):
        b.step(_data(dev), base=0, stride=1, n=4000)


def test_epoch_in_the_library_equals_the_steps_one_by_one():
    # supra_apod_epoch (the minibatch loop in the library) against supra_apod_step called per
    # minibatch in the same shuffled order: the same parameters, moments and losses, bit for bit
    params = phantom.apod_init(64, out_scale=1.0, bias_scale=0.1)
    dev, *_ = _rows(65, 4000)
    a, b = apod.Trainer(params, lr=2e-3), apod.Trainer(params, lr=2e-3)
    mean_loss = a.epoch(_data(dev), 5, seed=3)
    losses = torch.zeros(5, dtype=torch.float32, device="cuda")
    for j, k in enumerate(np.random.default_rng(3).permutation(5)):
        b.step(_data(dev), int(k), 5, loss_out=losses[j : j + 1])
    assert a.step_count == b.step_count == 5
    for name in ("params", "m", "v", "grad"):
        torch.testing.assert_close(getattr(a, name), getattr(b, name), rtol=0, atol=0)
    assert mean_loss == float(losses.mean())
    with pytest.raises(ValueError):
        a.epoch(_data(dev), 0, seed=1)


def test_epoch_of_row_blocks_equals_steps_on_the_gathered_blocks():
    # chunk = 128: minibatch b takes the 128-row blocks order[b], order[b] + 5, ... (the dataset's
    # last block is partial); each step equals a step on those rows gathered into one array
    params = phantom.apod_init(66, out_scale=1.0, bias_scale=0.1)
    dev, *_ = _rows(67, 3000)
    a, b = apod.Trainer(params, lr=2e-3), apod.Trainer(params, lr=2e-3)
    mean_loss = a.epoch(_data(dev), 5, seed=4, chunk=128)
    losses = torch.zeros(5, dtype=torch.float32, device="cuda")
    n_chunks = (3000 + 127) // 128
    for j, k in enumerate(np.random.default_rng(4).permutation(5)):
        rows = np.concatenate([np.arange(c * 128, min(c * 128 + 128, 3000)) for c in range(int(k), n_chunks, 5)])
        idx = torch.as_tensor(rows).cuda()
        sub = {name: v.index_select(0, idx).contiguous() for name, v in dev.items()}
        b.step(_data(sub), loss_out=losses[j : j + 1])
    for name in ("params", "m", "v", "grad"):
        torch.testing.assert_close(getattr(a, name), getattr(b, name), rtol=0, atol=0)
    assert mean_loss == float(losses.mean())
    with pytest.raises(ValueError):
        a.epoch(_data(dev), 25, seed=1, chunk=128)   # more minibatches than blocks


def test_fused_inference_matches_the_oracle():
    s = small_linear(64, 8, 700)
    p = s.params()
    ch = phantom.random_channels(s, 80)
    plan = supra.Plan(**p)
    params = _params(81, out_scale=2.0, bias_scale=0.1)
    got = plan.apod(ch.cuda(), torch.as_tensor(params).cuda()).cpu().numpy()
    lines, depths = list(range(8)), list(range(0, 700, 11))
    ref = oapod.beamform(p, ch.numpy(), params, lines, depths, bf16=True)
    ref64 = oapod.beamform(p, ch.numpy(), params, lines, depths)
    # no taper at the aperture edge: pixels with an element within 1e-9 m of the
    # edge (FP32 and FP64 may disagree on membership, which changes the
    # network's whole input) are left out
    keep = np.array([[np.min(np.abs(oracle.aperture(p, l, i)[2])) > 1e-9 for i in depths] for l in lines])
    assert keep.mean() > 0.9
    g = got[np.ix_(lines, depths)]
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(g - ref)[keep]) <= TOL_INFER * scale
    assert np.max(np.abs(g - ref64)[keep]) <= TOL_FP64_INFER * np.max(np.abs(ref64))
    assert supra.device_status() == 0


def test_fused_inference_is_deterministic():
    # several 128-depth tiles per CTA (64 lines x 16 tiles over two CTAs per SM), and lines near the
    # array's edges, whose aperture boxes sit at one end of a pixel row (the two warpgroups of a row
    # then exchange mask bits): repeated calls give the same bits
    s = small_linear(128, 64, 2048)
    ch = phantom.random_channels(s, 95).cuda()
    plan = supra.Plan(**s.params())
    params = torch.as_tensor(_params(96, out_scale=2.0, bias_scale=0.1)).cuda()
    outs = [plan.apod(ch, params) for _ in range(3)]
    assert all(torch.equal(outs[0], o) for o in outs[1:])
    assert torch.isfinite(outs[0]).all()
    assert supra.device_status() == 0


def test_zero_output_layer_is_rectangular_das_on_the_gpu():
    s = small_linear(40, 6, 500)
    p = s.params()
    ch = phantom.random_channels(s, 90).cuda()
    plan = supra.Plan(**p)
    rect = supra.Plan(**dict(p, window="rect"))
    got = plan.apod(ch, torch.as_tensor(phantom.apod_init(91)).cuda()).cpu().numpy()
    das = rect.beamform(ch).cpu().numpy()
    # uniform weights: the mean of the BF16-rounded samples (2^-9 relative each)
    assert _max_rel(got, das) <= 4e-3


def _training_data(s, seeds):
    frames = [phantom.synth_channels(s, phantom.make_phantom(s, sd, 1500, n_points=3), sd, device="cuda")
              for sd in seeds]
    return frames


def test_training_moves_the_output_toward_mv_and_resumes_from_a_checkpoint(tmp_path):
    s = phantom.linear_setup(64, 0.3e-3, 32, 1024, fc=5e6, fs=40e6)
    plan = supra.Plan(**s.params())
    train = apod.make_dataset(plan, _training_data(s, range(100, 106)), lambda pl, ch: pl.mv(ch, 16))
    evalf = _training_data(s, [200, 201])
    params0 = phantom.apod_init(7)

    def rel_err(params):
        e = d = 0.0
        for ch in evalf:
            y, ref = plan.apod(ch, params).cpu().numpy(), plan.mv(ch, 16).cpu().numpy()
            e += np.sum((y - ref) ** 2)
            d += np.sum(ref ** 2)
        return np.sqrt(e / d)

    das_err = 0.0
    for ch in evalf:
        y, ref = plan.beamform(ch).cpu().numpy(), plan.mv(ch, 16).cpu().numpy()
        das_err += np.sum((y - ref) ** 2) / np.sum(ref ** 2)
    das_err = np.sqrt(das_err / len(evalf))

    tr = apod.Trainer(params0, lr=2e-3)
    err0 = rel_err(tr.params)
    losses = [tr.epoch(train, 64, seed=e) for e in range(4)]
    ck = str(tmp_path / "apod.npz")
    tr.save(ck)
    tr.epoch(train, 64, seed=4)
    resumed = apod.Trainer(phantom.apod_init(999))
    resumed.load(ck)
    resumed.epoch(train, 64, seed=4)
    assert torch.equal(resumed.params, tr.params) and resumed.step_count == tr.step_count
    err = rel_err(tr.params)
    assert losses[-1] < losses[0]
    assert err < 0.9 * err0, (err, err0)
    assert err < das_err, (err, das_err)


def test_rejects_bad_arguments():
    s = phantom.config3(lines=8)   # 1024 elements: more than the network's 128 inputs
    plan = supra.Plan(**s.params())
    ch = torch.zeros(plan.ch_shape, dtype=torch.int16, device="cuda")
    with pytest.raises(supra.SupraError):
        plan.apod(ch, torch.zeros(supra.APOD_PARAMS, device="cuda"))
    dev, *_ = _rows(5, 64)
    tr = apod.Trainer(phantom.apod_init(1))
    lib = supra.load()
    # a feature pointer that is not 16-byte aligned
    rc = lib.supra_apod_forward(tr.params.data_ptr(), 8, 1, dev["feat"].data_ptr() + 2, dev["mask"].data_ptr(),
                                dev["norm"].data_ptr(), tr.grad.data_ptr(), None)
    assert rc == supra.EINVAL
    rc = lib.supra_apod_grad(tr.params.data_ptr(), 64, 1, dev["feat"].data_ptr(), dev["mask"].data_ptr(),
                             dev["norm"].data_ptr(), dev["label"].data_ptr(), tr.grad.data_ptr(), None,
                             tr.ws.data_ptr(), 16, None)
    assert rc == supra.EWORKSPACE
