"""The device-side input generator: records of a seed are the same bits on every
call (the echo sums use integer fixed point, whose sums do not depend on the
order the threads add in), and close to the FP64 host generator's."""
import numpy as np
import pytest
import torch

import phantom

pytestmark = pytest.mark.gpu


def test_device_synthesis_is_bit_reproducible():
    s = phantom.config2()
    ph = phantom.default_phantom(s, 21)
    a = phantom.synth_channels(s, ph, 21, device="cuda")
    b = phantom.synth_channels(s, ph, 21, device="cuda")
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    c = phantom.synth_channels(s, phantom.default_phantom(s, 22), 22, device="cuda")
    assert not torch.equal(a, c)


def test_device_synthesis_close_to_host():
    s = phantom.linear_setup(16, 0.3e-3, 8, 600, fc=5e6, fs=40e6)
    ph = phantom.make_phantom(s, 5, 300, n_points=2)
    # noise-free (the two generators draw different noise): FP32 echo times and phases on
    # the device against FP64 on the host, both scaled to a 16000 peak
    host = phantom.synth_channels(s, ph, 5, snr_db=None).numpy().astype(np.int64)
    dev = phantom.synth_channels(s, ph, 5, device="cuda", snr_db=None).cpu().numpy().astype(np.int64)
    d = np.abs(host - dev)
    assert d.max() <= 16, d.max()          # 1e-3 of the peak
    assert np.mean(d <= 1) > 0.99
