"""Learned form plumbing: the feature rows against the oracle's, the choice of
p per level / leaf cap from the network's scores, and the fixed-p fallback when
the sampled direct-sum check fails."""
import numpy as np
import pytest
import torch

import workloads
from oracle import tree as T
from oracle.features import level_features
from tests.gpu_util import dev, host3, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["cube", "ring"])
def test_features_match_oracle(kind):
    from paper_1201_5430_gb300 import LHV
    if kind == "cube":
        x, w = workloads.cube(5000, 3)
        a, leaf = 0.01, 16
    else:
        x, w = workloads.ring(20000, 1)
        a, leaf = workloads.RING_CORE_A, 64
    ctx = LHV(p=8, leaf_max=leaf, core_a=a)
    got = ctx.selector_features(dev(x, "fp32"), dev(w, "fp32"), eps=1e-5).cpu().numpy()
    tr = T.build_tree(x, leaf_max=leaf, a=a, eps=1e-6)
    want = level_features(tr, w, 1e-5, a, 0.0)
    assert got.shape == want.shape
    assert np.abs(got - want).max() < 2e-6, np.abs(got - want).max(axis=0)


def _net(p_index, leaf_index):
    """A network whose scores are constant: all weights 0, biases pick the classes."""
    W = torch.zeros(10304, dtype=torch.bfloat16)
    b = torch.zeros(213, dtype=torch.float32)
    b[192 + p_index] = 5.0
    b[192 + 17 + leaf_index] = 5.0
    return W, b


def test_constant_network_reproduces_fixed_p():
    from paper_1201_5430_gb300 import LHV
    x, w = workloads.ring(30000, 2)
    a = workloads.RING_CORE_A
    x4, w4 = dev(x, "fp32"), dev(w, "fp32")
    ref = LHV(p=12, leaf_max=64, core_a=a)
    v0, s0 = ref.evaluate_velocity_stretching(x4, w4)
    ctx = LHV(p=6, leaf_max=16, core_a=a)
    ctx.set_selector(*_net(12 - 4, 2), eps=1e-2, check_every=1, check_samples=200)
    v, s = ctx.evaluate_velocity_stretching(x4, w4)
    st = ctx.stats()
    assert st["selector"]["leaf_max"] == 64 and st["selector"]["fallbacks"] == 0
    assert all(p == 12 for p in st["level_p"][2:])
    assert rel(host3(v), host3(v0)) < 1e-6 and rel(host3(s), host3(s0)) < 1e-6
    assert 0 <= st["selector"]["err_v"] < 1e-2


def test_failed_check_falls_back_to_fixed_p():
    from paper_1201_5430_gb300 import LHV
    x, w = workloads.ring(30000, 2)
    a = workloads.RING_CORE_A
    x4, w4 = dev(x, "fp32"), dev(w, "fp32")
    ref = LHV(p=12, leaf_max=64, core_a=a)
    v0, s0 = ref.evaluate_velocity_stretching(x4, w4)
    ctx = LHV(p=12, leaf_max=64, core_a=a)
    ctx.set_selector(*_net(0, 0), eps=1e-6, check_every=1, check_samples=300)   # p = 4 everywhere: too coarse
    v, s = ctx.evaluate_velocity_stretching(x4, w4)
    st = ctx.stats()
    assert st["selector"]["fallbacks"] == 1 and st["selector"]["checks"] == 1
    assert st["selector"]["err_v"] > 1e-6
    assert all(p == 12 for p in st["level_p"][2:])
    assert rel(host3(v), host3(v0)) < 1e-6 and rel(host3(s), host3(s0)) < 1e-6
    # a step through the selector: the fallback holds for its four stages
    xs, ws = x4.clone(), w4.clone()
    ctx.step(xs, ws, 1e-3)
    xr, wr = x4.clone(), w4.clone()
    ref.step(xr, wr, 1e-3)
    assert rel(host3(xs), host3(xr)) < 1e-7
    assert ctx.stats()["selector"]["fallbacks"] == 2


def test_check_schedule_and_off_switch():
    from paper_1201_5430_gb300 import LHV
    x, w = workloads.cube(8000, 1)
    x4, w4 = dev(x, "fp32"), dev(w, "fp32")
    ctx = LHV(p=8, leaf_max=32, core_a=0.01)
    ctx.set_selector(*_net(8, 1), eps=0.5, check_every=3, check_samples=100)
    for _ in range(7):
        ctx.evaluate_velocity_stretching(x4, w4)
    sel = ctx.stats()["selector"]
    assert sel["selections"] == 7 and sel["checks"] == 3  # selections 1, 4, 7
    ctx.set_selector(None)
    ctx.evaluate_velocity_stretching(x4, w4)
    assert all(p == 8 for p in ctx.stats()["level_p"][2:])
