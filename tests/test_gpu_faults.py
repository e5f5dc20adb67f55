"""Failure detection on the device without a fault: every kernel's mbarrier waits
are bounded.  The self-test waits on an mbarrier that nothing completes, once with
a cycle budget and once on the abort-word path of the beamforming kernel's stage
consumers; both must give up, report SUPRA_ETIMEOUT through the device status
word, and leave the context usable (the chain still matches the oracle after)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1711_06127_b300 as supra
import phantom
from _setups import small_linear
from gpu_util import RF_TOL, max_norm_err

pytestmark = pytest.mark.gpu


def test_bounded_waits_time_out_and_the_context_stays_usable():
    assert supra.device_status(clear=True) == 0
    assert supra.selftest_bounded_wait(1 << 20) == (1, 1)
    assert supra.device_status(clear=True) == supra.ETIMEOUT
    assert supra.device_status() == 0   # cleared
    # the same context still beamforms correctly
    s = small_linear(16, 12, 300)
    ch = phantom.synth_channels(s, phantom.default_phantom(s, 7), 7).numpy()
    plan = supra.Plan(**s.params())
    rf = plan.beamform(torch.as_tensor(ch).cuda())
    torch.cuda.synchronize()
    ref = oracle.das(s.params(), ch)
    assert max_norm_err(rf.cpu().numpy().astype(np.float64), ref) <= RF_TOL
    assert supra.device_status() == 0
