"""GPU parity of the exact minimum-variance beamformer (supra_mv) against the
oracle.  MV has no taper at the aperture edge, so pixels with an element
within 1e-9 m of the edge (where fp32 and fp64 may disagree on membership) are
left out.  Tolerance: max |gpu - oracle| / max |oracle| <= 1e-3 (the loading
0.01 bounds the condition number by 1 + L/0.01 = 3201 for L = 32; FP32
Cholesky error ~ cond * 2^-24 * sqrt(L))."""
import numpy as np
import pytest
import torch

import oracle
import paper_1711_06127_b300 as supra
import phantom
from _setups import small_linear
from gpu_util import max_norm_err

pytestmark = pytest.mark.gpu
MV_TOL = 1e-3


def _edge_free(p, lines, depths):
    keep = np.ones((len(lines), len(depths)), bool)
    for a, l in enumerate(lines):
        for b, i in enumerate(depths):
            _, _, margin = oracle.aperture(p, l, i)
            keep[a, b] = np.min(np.abs(margin)) > 1e-9
    return keep


def _compare(p, ch, L, loading, lines, depths, tol=MV_TOL):
    plan = supra.Plan(**p)
    got = plan.mv(torch.as_tensor(ch).cuda(), L, loading).cpu().numpy()[np.ix_(lines, depths)]
    ref = oracle.mv(p, ch, L, loading, lines=lines, depths=depths)
    keep = _edge_free(p, lines, depths)
    assert keep.mean() > 0.9
    err = np.max(np.abs(got - ref)[keep]) / np.max(np.abs(ref))
    assert err <= tol, err
    return got, ref


def test_mv_small_frame_random_records():
    s = small_linear(24, 10, 400)
    p = s.params()
    ch = phantom.random_channels(s, 12).numpy()
    _compare(p, ch, 8, None, list(range(s.n_lines)), list(range(0, s.n_depth, 3)))


def test_mv_phantom_full_subaperture():
    s = phantom.linear_setup(64, 0.3e-3, 32, 1200, fc=7e6, fs=40e6)
    p = s.params()
    ch = phantom.synth_channels(s, phantom.make_phantom(s, 4, 800, n_points=3), 4).numpy()
    _compare(p, ch, 32, None, [3, 15, 16, 28], list(range(0, s.n_depth, 5)))


def test_mv_small_loading_uses_fp64():
    s = small_linear(32, 6, 500)
    p = s.params()
    ch = phantom.random_channels(s, 13).numpy()
    _compare(p, ch, 16, 1e-5, list(range(s.n_lines)), list(range(0, s.n_depth, 7)))


def test_mv_subaperture_one_is_rect_das_and_large_loading_is_trapezoid():
    s = small_linear(24, 8, 300)
    p = s.params()
    ch = torch.as_tensor(phantom.random_channels(s, 14)).cuda()
    plan = supra.Plan(**p)
    rect = supra.Plan(**dict(p, window="rect"))
    np.testing.assert_allclose(plan.mv(ch, 1, 0.01).cpu().numpy(), rect.beamform(ch).cpu().numpy(),
                               rtol=0, atol=2e-3 * float(ch.abs().max()))
    got = plan.mv(ch, 8, 1e6).cpu().numpy()
    ref = oracle.mv(p, ch.cpu().numpy(), 8, 1e6, lines=range(8), depths=range(0, 300, 4))
    assert max_norm_err(got[:, ::4], ref) <= MV_TOL


def test_mv_full_size_workload_sampled_lines():
    # the learned-apodization workload: 128 elements, 256 lines, 2048 samples, L = 32, loading 0.01
    s = phantom.config2()
    p = s.params()
    ch = phantom.synth_channels(s, phantom.default_phantom(s, 4000), 4000, device="cuda")
    plan = supra.Plan(**p)
    got = plan.mv(ch, 32).cpu().numpy()
    torch.cuda.synchronize()
    lines, depths = [0, 77, 128, 255], list(range(0, s.n_depth, 9))
    ref = oracle.mv(p, ch.cpu().numpy(), 32, None, lines=lines, depths=depths)
    keep = _edge_free(p, lines, depths)
    err = np.max(np.abs(got[np.ix_(lines, depths)] - ref)[keep]) / np.max(np.abs(ref))
    assert err <= MV_TOL, err
    assert supra.device_status() == 0


def test_mv_rejects_bad_arguments():
    s = small_linear(16, 4, 200)
    plan = supra.Plan(**s.params())
    ch = torch.zeros(plan.ch_shape, dtype=torch.int16, device="cuda")
    for L, lo in [(0, 0.01), (33, 0.01), (8, 0.0), (8, float("nan"))]:
        with pytest.raises(supra.SupraError):
            plan.mv(ch, L, lo)


def test_mv_all_zero_records_give_zero_without_a_device_error():
    s = small_linear(24, 6, 300)
    plan = supra.Plan(**s.params())
    supra.device_status()
    rf = plan.mv(torch.zeros(plan.ch_shape, dtype=torch.int16, device="cuda"), 8)
    assert torch.count_nonzero(rf).item() == 0
    assert supra.device_status() == 0
