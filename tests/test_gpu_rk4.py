"""GPU RK4 step against the oracle's RK4 with the oracle FMM as the rate."""
import numpy as np
import pytest

import workloads
from oracle import fmm as ofmm, rk4
from tests.gpu_util import dev, host3, rel

pytestmark = pytest.mark.gpu


def test_rk4_step_parity():
    from paper_1201_5430_gb300 import LHV
    x, w = workloads.ring(4000, 1)
    a, p, dt = 0.02, 8, 1e-3

    def rate(xx, ww):
        r = ofmm.fmm(xx.astype(np.float32), ww.astype(np.float32), p, leaf_max=32, a=a)
        return r.v, r.s

    x1, w1 = rk4.rk4_step(x, w, dt, rate)
    ctx = LHV(p=p, leaf_max=32, core_a=a, precision="fp32")
    x4, w4 = dev(x, "fp32"), dev(w, "fp32")
    ctx.step(x4, w4, dt)
    gx, gw = host3(x4), host3(w4)
    # the state is stored in FP32: |x| ~ 1 carries 6e-8 of rounding on a
    # displacement of ~1e-3, so the displacement is compared at 1e-4 and the
    # positions within a few units in the last place
    assert rel(gx - x, x1 - x) < 1e-4, rel(gx - x, x1 - x)
    assert np.abs(gx - x1).max() <= 4 * np.finfo(np.float32).eps * np.abs(x1).max()
    assert rel(gw - w, w1 - w) < 1e-4, rel(gw - w, w1 - w)


def test_step_host_matches_device():
    import torch
    from paper_1201_5430_gb300 import LHV
    x, w = workloads.ring(5000, 2)
    ctx = LHV(p=8, leaf_max=32, core_a=0.02)
    x4, w4 = dev(x, "fp32"), dev(w, "fp32")
    hx, hw = x4.cpu().clone(), w4.cpu().clone()
    ctx.step(x4, w4, 1e-3)
    ctx.step_host(hx, hw, 1e-3)
    # M2L and M2M accumulate with atomics, so two runs agree to rounding, not bitwise
    torch.testing.assert_close(hx, x4.cpu(), rtol=0, atol=4 * 2.0 ** -24 * float(x4.abs().max()))
    torch.testing.assert_close(hw, w4.cpu(), rtol=0, atol=4 * 2.0 ** -24 * float(w4.abs().max()))
