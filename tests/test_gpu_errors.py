"""Status codes of the C ABI on a GPU: bad arguments, non-finite input, empty input."""
import ctypes

import numpy as np
import pytest

import workloads
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def test_errors_and_recovery():
    import torch
    from paper_1201_5430_gb300 import LHV, LHVError
    from paper_1201_5430_gb300 import _lib
    ctx = LHV(p=6, leaf_max=16, core_a=0.01)
    lib = ctx.lib
    x, w = workloads.cube(500, 1)
    x4, w4 = dev(x, "fp32"), dev(w, "fp32")
    v4, s4 = torch.empty_like(x4), torch.empty_like(x4)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.lhv_evaluate_velocity_stretching(ctx.h, -1, p(x4), p(w4), p(v4), p(s4)) == _lib.LHV_EINVAL
    assert lib.lhv_evaluate_velocity_stretching(ctx.h, 500, None, p(w4), p(v4), p(s4)) == _lib.LHV_EINVAL
    mis = ctypes.c_void_p(x4.data_ptr() + 4)
    assert lib.lhv_evaluate_velocity_stretching(ctx.h, 499, mis, p(w4), p(v4), p(s4)) == _lib.LHV_EINVAL
    assert lib.lhv_evaluate_velocity_stretching_f64(ctx.h, 500, p(x4), p(w4), p(v4), p(s4)) == _lib.LHV_EINVAL
    assert lib.lhv_evaluate_velocity_stretching(ctx.h, 0, None, None, None, None) == 0
    bad = x4.clone()
    bad[17, 1] = float("nan")
    with pytest.raises(LHVError) as e:
        ctx.evaluate_velocity_stretching(bad, w4)
    assert e.value.status == _lib.LHV_ENONFINITE
    badw = w4.clone()
    badw[3, 0] = float("inf")
    with pytest.raises(LHVError):
        ctx.evaluate_velocity_stretching(x4, badw)
    v, s = ctx.evaluate_velocity_stretching(x4, w4)      # the context is still usable
    assert torch.isfinite(v).all() and torch.isfinite(s).all()
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_identical_points_and_single_element(prec):
    """All elements at one point: d = 0 gives v = 0, and s comes from the r = 0
    limit of the core alone; one element alone gives zero."""
    from paper_1201_5430_gb300 import LHV
    ctx = LHV(p=6, leaf_max=4, core_a=0.05, precision=prec)
    x = np.zeros((10, 3), np.float32) + np.float32(0.25)
    w = np.random.default_rng(0).normal(size=(10, 3)).astype(np.float32)
    v, s = ctx.evaluate_velocity_stretching(dev(x, prec), dev(w, prec))
    from oracle import direct
    v0, _, s0 = direct.direct(x, w, 0.05)
    if prec == "fp64":
        np.testing.assert_allclose(v[:, :3].cpu().numpy(), v0, atol=1e-12)
        np.testing.assert_allclose(s[:, :3].cpu().numpy(), s0, atol=1e-10)
    else:
        np.testing.assert_allclose(v[:, :3].cpu().numpy(), v0, atol=1e-6 * np.abs(s0).max())
        np.testing.assert_allclose(s[:, :3].cpu().numpy(), s0, rtol=1e-5, atol=1e-6 * np.abs(s0).max())
    v1, s1 = ctx.evaluate_velocity_stretching(dev(x[:1], prec), dev(w[:1], prec))
    assert float(v1.abs().max()) == 0.0 and float(s1.abs().max()) == 0.0
